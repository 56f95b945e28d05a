// Three-way (generalised) ACA of every admissible block (Algorithm 1) in one
// persistent launch.
//
// Each CTA claims blocks from an atomic queue counter (longest first) and runs
// Algorithm 1 on the block restricted to the unique frequencies:
//   face    partial-pivot ACA of the residual face at k_l (eps_face), with the
//           residual of earlier crosses subtracted row/column-wise;
//   recomp  Cholesky-QR of both ACA factors (float64, column-scaled Gram
//           matrices), one-sided Jacobi SVD of the r x r core R_U R_V^H,
//           truncation sigma_i < eps_face sigma_1 (Section 4, first remark);
//   pivot   argmax |H_l[i, j]| over the dense expansion of U' V'^H, tiled
//           through shared memory, ties to the smallest row-major index
//           (Section 4, last remark);
//   fiber   f_l[k] = (ENTRY(i_l, j_l, k) - sum_p H_p[i_l, j_l] f_p[k]) / H_l[i_l, j_l]
//           with the residual in float64;
//   norm    eq. (norm): ||C^(l)||^2 += 2 Re sum_d <H_l, H_d><f_l, f_d> + ||H_l||^2 ||f_l||^2,
//           face inner products through Gram products (U_d^H U_l)(V_l^H V_d);
//   stop    ||H_l|| ||f_l|| <= eps3 ||C^(l)|| -> rank l - 1; all frequencies
//           used -> rank l; else k_{l+1} = argmax over unused k of |f_l[k]|.
// Zero faces: up to three more frequencies are tested (last unique, middle,
// largest |s|) before a block is declared zero (Section 5.1 on DLP zero blocks).
//
// Precision: T = float (mixed) evaluates entries and face arithmetic in
// float32 and stores complex64 factors; T = double does everything in float64.
// Recompression, fiber residuals and norms are float64 in both.
//
// No CTA waits on another: the only inter-CTA communication is the atomic
// queue counter and the atomic pool allocator.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <numeric>
#include <vector>

#include "g3_device.cuh"

namespace g3 {

constexpr int KU_MAX = 256;   // largest unique-frequency count
constexpr int RF_MAX = 64;    // largest face rank cap

template <class T>
struct AcaArgs {
    GeomF gf;
    GeomD gd;
    SepView<T> sep;
    const double2* sd;
    int Ku, k_maxabs;
    const BlockRange* ranges;
    int n_far;
    const int* queue;
    int* queue_head;
    int single;              // >= 0: CTA 0 processes queue[single] only
    const int* k1;           // [n_far] first frequency per block, or null
    int Cmax, RF;
    double eps3, eps_face;
    int no_recompress;
    Cx<T>* pool;
    long long pool_cap;
    unsigned long long* pool_ctr;
    CrossRec* rec;
    int* r3;
    unsigned long long* counters;  // [0] entries [1] crosses computed [2] zero blocks [3] capped faces
    unsigned* status;
    char* ws;
    size_t ws_stride;
    int Mmax, Nmax;
};

template <class T>
struct Ws {
    Cx<T>* uw;            // [RF][Mmax]
    Cx<T>* vw;            // [RF][Nmax]
    Cx<T>* row;           // [Nmax]
    unsigned char* used;  // [Mmax]
    Cx<T>* pre;           // [Cmax * RF]
    Cx<double>* RU;       // [RF][RF]
    Cx<double>* RV;
    Cx<double>* TU;
    Cx<double>* TV;
    Cx<double>* fib;      // [Ku]
};

static inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

template <class T>
__host__ __device__ inline size_t ws_bytes(int RF, int Mmax, int Nmax, int Cmax, int Ku) {
    size_t b = 0;
    auto add = [&](size_t n) { b += (n + 255) & ~size_t(255); };
    add((size_t)RF * Mmax * sizeof(Cx<T>));
    add((size_t)RF * Nmax * sizeof(Cx<T>));
    add((size_t)Nmax * sizeof(Cx<T>));
    add((size_t)Mmax);
    add((size_t)Cmax * RF * sizeof(Cx<T>));
    for (int i = 0; i < 4; ++i) add((size_t)RF * RF * sizeof(Cx<double>));
    add((size_t)Ku * sizeof(Cx<double>));
    return b;
}

template <class T>
__device__ inline Ws<T> ws_carve(char* base, int RF, int Mmax, int Nmax, int Cmax, int Ku) {
    Ws<T> w;
    size_t o = 0;
    auto take = [&](size_t n) {
        char* p = base + o;
        o += (n + 255) & ~size_t(255);
        return p;
    };
    w.uw = (Cx<T>*)take((size_t)RF * Mmax * sizeof(Cx<T>));
    w.vw = (Cx<T>*)take((size_t)RF * Nmax * sizeof(Cx<T>));
    w.row = (Cx<T>*)take((size_t)Nmax * sizeof(Cx<T>));
    w.used = (unsigned char*)take((size_t)Mmax);
    w.pre = (Cx<T>*)take((size_t)Cmax * RF * sizeof(Cx<T>));
    w.RU = (Cx<double>*)take((size_t)RF * RF * sizeof(Cx<double>));
    w.RV = (Cx<double>*)take((size_t)RF * RF * sizeof(Cx<double>));
    w.TU = (Cx<double>*)take((size_t)RF * RF * sizeof(Cx<double>));
    w.TV = (Cx<double>*)take((size_t)RF * RF * sizeof(Cx<double>));
    w.fib = (Cx<double>*)take((size_t)Ku * sizeof(Cx<double>));
    return w;
}

// shared state of the block being processed
template <class T>
struct BlockSh {
    int M, N, rb, cb, blk;
    int ncross;
    int k;
    unsigned used_k[KU_MAX / 32];
    long long off[KU_MAX];
    int r[KU_MAX];
    int pre[KU_MAX + 1];
    Cx<T> fk[KU_MAX];
    Cx<double> hp[KU_MAX];   // H_p[i_l, j_l]
    Cx<double> ff[KU_MAX];   // <f_l, f_d>
    Cx<double> hh[KU_MAX];   // <H_l, H_d>
    Cx<double> gu[RF_MAX + 1];
    Cx<double> gv[RF_MAX + 1];
    double sig[RF_MAX];
    double dU[RF_MAX], dV[RF_MAX];
    int sel[RF_MAX];
    ArgMax am[32];
    double red[64];
    double norm2;
    double hself;            // ||H_l||^2
    double fself;            // ||f_l||^2
    Cx<double> hpiv;
    long long new_off;
    long long entries;
    int flag;
    int rot;
    int rnew;
    int ip, jp;
};

template <int NT>
__device__ __forceinline__ ArgMax block_argmax(ArgMax a, ArgMax* sh) {
    a = warp_argmax(a);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = a;
    __syncthreads();
    if (w == 0) {
        ArgMax b = (l < NT / 32) ? sh[l] : ArgMax{-1.0, LLONG_MAX};
        b = warp_argmax(b);
        if (l == 0) sh[0] = b;
    }
    __syncthreads();
    ArgMax r = sh[0];
    __syncthreads();
    return r;
}

// ---- entry access ----------------------------------------------------------------
template <int KER, class T>
__device__ __forceinline__ Cx<T> ent(const AcaArgs<T>& A, int gi, int gj, int k) {
    if constexpr (KER == G3_SEPARABLE) {
        Cx<T> acc{0, 0};
        for (int t = 0; t < A.sep.R; ++t) {
            Cx<T> a{A.sep.a[2 * ((size_t)t * A.sep.M + gi)], A.sep.a[2 * ((size_t)t * A.sep.M + gi) + 1]};
            Cx<T> b{A.sep.b[2 * ((size_t)t * A.sep.N + gj)], A.sep.b[2 * ((size_t)t * A.sep.N + gj) + 1]};
            Cx<T> c{A.sep.c[2 * ((size_t)t * A.sep.Ku + k)], A.sep.c[2 * ((size_t)t * A.sep.Ku + k) + 1]};
            cfma(acc, cmul(a, b), c);
        }
        return acc;
    } else {
        double2 s = A.sd[k];
        return colloc_entry<KER, T>(A.gf, A.gd, gi, gj, (T)s.x, (T)s.y, s.x, s.y);
    }
}

// pool views of cross p
template <class T>
__device__ __forceinline__ const Cx<T>* Up(const AcaArgs<T>& A, const BlockSh<T>& S, int p) {
    return A.pool + S.off[p];
}
template <class T>
__device__ __forceinline__ const Cx<T>* Vp(const AcaArgs<T>& A, const BlockSh<T>& S, int p) {
    return A.pool + S.off[p] + (long long)S.r[p] * S.M;
}
template <class T>
__device__ __forceinline__ const Cx<T>* Fp(const AcaArgs<T>& A, const BlockSh<T>& S, int p) {
    return A.pool + S.off[p] + (long long)S.r[p] * (S.M + S.N);
}

// ---- face ACA (partial pivoting) on the residual face at frequency kf -----------------
// Returns the rank m; columns 0..m-1 of uw / vw hold the crosses (S = U V^H).
template <int KER, class T, int NT>
__device__ int face_aca(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, int kf) {
    const int tid = threadIdx.x;
    const int M = S.M, N = S.N, nc = S.ncross;
    const int cap = min(min(M, N), A.RF);
    // f_p[kf] of earlier crosses
    for (int p = tid; p < nc; p += NT) S.fk[p] = Fp(A, S, p)[kf];
    for (int i = tid; i < M; i += NT) w.used[i] = 0;
    __syncthreads();
    double Sn2 = 0.0;
    int m = 0;
    int irow = 0;
    bool converged = false;
    while (m < cap) {
        int jp = -1;
        for (;;) {
            // residual row irow
            for (int p = 0; p < nc; ++p) {
                if (tid < S.r[p]) w.pre[S.pre[p] + tid] = cmul(S.fk[p], Up(A, S, p)[(long long)tid * M + irow]);
            }
            __syncthreads();
            ArgMax am{-1.0, LLONG_MAX};
            for (int j = tid; j < N; j += NT) {
                Cx<T> e = ent<KER, T>(A, S.rb + irow, S.cb + j, kf);
                for (int p = 0; p < nc; ++p) {
                    const Cx<T>* V = Vp(A, S, p);
                    const Cx<T>* pr = w.pre + S.pre[p];
                    const int rp = S.r[p];
                    Cx<T> acc{0, 0};
                    for (int t = 0; t < rp; ++t) cfmac(acc, pr[t], V[(long long)t * N + j]);
                    e.x -= acc.x;
                    e.y -= acc.y;
                }
                Cx<T> acc{0, 0};
                for (int t = 0; t < m; ++t) cfmac(acc, w.uw[(size_t)t * A.Mmax + irow], w.vw[(size_t)t * A.Nmax + j]);
                e.x -= acc.x;
                e.y -= acc.y;
                w.row[j] = e;
                am = amax_better(am, ArgMax{(double)cabs2(e), (long long)j});
            }
            if (tid == 0) S.entries += N;
            am = block_argmax<NT>(am, S.am);
            if (tid == 0) w.used[irow] = 1;
            if (am.v > 0.0) {
                jp = (int)am.i;
                break;
            }
            // zero residual row: next unused row in index order
            ArgMax un{-1.0, LLONG_MAX};
            for (int i = tid; i < M; i += NT)
                if (i != irow && !w.used[i]) un = amax_better(un, ArgMax{0.0, (long long)i});
            un = block_argmax<NT>(un, S.am);
            if (un.v < 0.0) {
                irow = -1;
                break;
            }
            irow = (int)un.i;
        }
        if (jp < 0) break;  // no row with a nonzero residual left
        const Cx<T> delta = w.row[jp];
        const T dn = (T)1 / cabs2(delta);
        Cx<T>* vm = w.vw + (size_t)m * A.Nmax;
        for (int j = tid; j < N; j += NT) {
            Cx<T> q = cmulc(w.row[j], delta);  // row * conj(delta) / |delta|^2 = row / delta
            vm[j] = Cx<T>{q.x * dn, -q.y * dn};  // conj(row / delta)
        }
        for (int p = 0; p < nc; ++p) {
            if (tid < S.r[p]) {
                Cx<T> v = Vp(A, S, p)[(long long)tid * N + jp];
                w.pre[S.pre[p] + tid] = cmul(S.fk[p], cconj(v));
            }
        }
        __syncthreads();
        // residual column jp
        Cx<T>* um = w.uw + (size_t)m * A.Mmax;
        for (int i = tid; i < M; i += NT) {
            Cx<T> e = ent<KER, T>(A, S.rb + i, S.cb + jp, kf);
            for (int p = 0; p < nc; ++p) {
                const Cx<T>* U = Up(A, S, p);
                const Cx<T>* pr = w.pre + S.pre[p];
                const int rp = S.r[p];
                Cx<T> acc{0, 0};
                for (int t = 0; t < rp; ++t) cfma(acc, U[(long long)t * M + i], pr[t]);
                e.x -= acc.x;
                e.y -= acc.y;
            }
            Cx<T> acc{0, 0};
            for (int t = 0; t < m; ++t) cfmac(acc, w.uw[(size_t)t * A.Mmax + i], w.vw[(size_t)t * A.Nmax + jp]);
            e.x -= acc.x;
            e.y -= acc.y;
            um[i] = e;
        }
        if (tid == 0) S.entries += M;
        __syncthreads();
        // recursive Frobenius norm of the face approximant:
        // ||S_m||^2 = ||S_{m-1}||^2 + 2 Re sum_t (u_t^H u_m)(v_m^H v_t) + ||u_m||^2 ||v_m||^2
        const int wid = tid >> 5, lane = tid & 31;
        for (int t = wid; t <= m; t += NT / 32) {
            const Cx<T>* ut = w.uw + (size_t)t * A.Mmax;
            const Cx<T>* vt = w.vw + (size_t)t * A.Nmax;
            Cx<double> gu{0, 0}, gv{0, 0};
            for (int i = lane; i < M; i += 32) {
                Cx<T> a = cmulc(um[i], ut[i]);  // conj(u_t) u_m
                gu.x += a.x;
                gu.y += a.y;
            }
            for (int j = lane; j < N; j += 32) {
                Cx<T> a = cmulc(vt[j], vm[j]);  // conj(v_m) v_t
                gv.x += a.x;
                gv.y += a.y;
            }
            gu.x = warp_sum(gu.x);
            gu.y = warp_sum(gu.y);
            gv.x = warp_sum(gv.x);
            gv.y = warp_sum(gv.y);
            if (lane == 0) {
                S.gu[t] = gu;
                S.gv[t] = gv;
            }
        }
        __syncthreads();
        double cross = 0.0;
        for (int t = 0; t < m; ++t) cross += 2.0 * (S.gu[t].x * S.gv[t].x - S.gu[t].y * S.gv[t].y);
        const double nu2 = S.gu[m].x, nv2 = S.gv[m].x;
        Sn2 += cross + nu2 * nv2;
        ++m;
        __syncthreads();
        if (sqrt(nu2 * nv2) <= A.eps_face * sqrt(fmax(Sn2, 0.0))) {
            converged = true;
            break;
        }
        // next row: argmax over unused rows of |u_m|
        ArgMax nx{-1.0, LLONG_MAX};
        for (int i = tid; i < M; i += NT)
            if (!w.used[i]) nx = amax_better(nx, ArgMax{(double)cabs2(um[i]), (long long)i});
        nx = block_argmax<NT>(nx, S.am);
        if (nx.v < 0.0) break;
        irow = (int)nx.i;
    }
    if (!converged && m == A.RF && m < min(M, N)) {
        if (tid == 0) {
            atomicOr(A.status, ST_FACE_CAPPED);
            atomicAdd(&A.counters[3], 1ull);
        }
    }
    __syncthreads();
    return m;
}

// ---- recompression: Cholesky-QR + one-sided Jacobi SVD ---------------------------------
// Input uw, vw (r columns).  Output: the rank r' and the transforms
// T_U (r x r'), T_V (r x r') in shared memory (row-major, stride RF) such that
// U' = uw T_U, V' = vw T_V, U' V'^H = uw vw^H truncated.  Returns r' or -1 if
// Cholesky broke down (caller keeps the raw factors).
template <class T, int NT>
__device__ int recompress(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, int r, Cx<double>* shB,
                          Cx<double>* shJ) {
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int M = S.M, N = S.N, RF = A.RF;
    // Gram matrices (upper triangles): G[a][b] = sum conj(x_a) x_b
    const int npair = r * (r + 1) / 2;
    for (int it = wid; it < 2 * npair; it += NT / 32) {
        const bool isU = it < npair;
        int q = isU ? it : it - npair;
        int a = 0;
        while (q >= r - a) {
            q -= r - a;
            ++a;
        }
        const int b = a + q;
        const Cx<T>* xa = isU ? w.uw + (size_t)a * A.Mmax : w.vw + (size_t)a * A.Nmax;
        const Cx<T>* xb = isU ? w.uw + (size_t)b * A.Mmax : w.vw + (size_t)b * A.Nmax;
        const int L = isU ? M : N;
        Cx<double> g{0, 0};
        for (int i = lane; i < L; i += 32) {
            Cx<double> va = ccast<double>(xa[i]), vb = ccast<double>(xb[i]);
            g.x += va.x * vb.x + va.y * vb.y;
            g.y += va.x * vb.y - va.y * vb.x;
        }
        g.x = warp_sum(g.x);
        g.y = warp_sum(g.y);
        if (lane == 0) (isU ? w.RU : w.RV)[a * RF + b] = g;
    }
    if (tid == 0) S.flag = 0;
    __syncthreads();
    // column scaling and upper Cholesky of the scaled Gram matrices: warp 0 -> U, warp 1 -> V
    if (wid < 2) {
        Cx<double>* R = wid == 0 ? w.RU : w.RV;
        double* dsc = wid == 0 ? S.dU : S.dV;
        for (int a = lane; a < r; a += 32) dsc[a] = 1.0 / sqrt(fmax(R[a * RF + a].x, 1e-300));
        __syncwarp();
        for (int a = lane; a < r; a += 32)
            for (int b = a; b < r; ++b) {
                double s = dsc[a] * dsc[b];
                R[a * RF + b].x *= s;
                R[a * RF + b].y *= s;
            }
        __syncwarp();
        for (int k = 0; k < r; ++k) {
            double dkk = R[k * RF + k].x;
            for (int i = 0; i < k; ++i) dkk -= R[i * RF + k].x * R[i * RF + k].x + R[i * RF + k].y * R[i * RF + k].y;
            bool bad = !(dkk > 1e-24);
            if (bad) {
                if (lane == 0) atomicOr(&S.flag, 1);
                break;
            }
            double rkk = sqrt(dkk);
            for (int j = k + 1 + lane; j < r; j += 32) {
                Cx<double> acc = R[k * RF + j];
                for (int i = 0; i < k; ++i) {
                    Cx<double> rik = R[i * RF + k], rij = R[i * RF + j];
                    acc.x -= rik.x * rij.x + rik.y * rij.y;  // conj(R[i][k]) R[i][j]
                    acc.y -= rik.x * rij.y - rik.y * rij.x;
                }
                R[k * RF + j] = Cx<double>{acc.x / rkk, acc.y / rkk};
            }
            __syncwarp();
            if (lane == 0) R[k * RF + k] = Cx<double>{rkk, 0.0};
            __syncwarp();
        }
    }
    __syncthreads();
    if (S.flag) return -1;
    // core C = R_U R_V^H with R_U = Rhat_U diag(1/dU): C[a][b] = sum_{c >= max(a,b)}
    //   RhatU[a][c] conj(RhatV[b][c]) / (dU[c] dV[c]); stored column-major in shB, J = I
    for (int e = tid; e < r * r; e += NT) {
        const int a = e % r, b = e / r;
        Cx<double> acc{0, 0};
        for (int c = max(a, b); c < r; ++c) {
            Cx<double> x = w.RU[a * RF + c], y = w.RV[b * RF + c];
            double s = 1.0 / (S.dU[c] * S.dV[c]);
            acc.x += (x.x * y.x + x.y * y.y) * s;
            acc.y += (x.y * y.x - x.x * y.y) * s;
        }
        shB[b * RF + a] = acc;
        shJ[b * RF + a] = Cx<double>{a == b ? 1.0 : 0.0, 0.0};
    }
    __syncthreads();
    // one-sided Jacobi (Hestenes) on the columns of C, round-robin pair schedule
    const int n = (r + 1) & ~1;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (tid == 0) S.rot = 0;
        __syncthreads();
        for (int rho = 0; rho < n - 1; ++rho) {
            for (int pi = wid; pi < n / 2; pi += NT / 32) {
                int p, q;
                if (pi == 0) {
                    p = rho;
                    q = n - 1;
                } else {
                    p = (rho + pi) % (n - 1);
                    q = (rho - pi + (n - 1)) % (n - 1);
                }
                if (p >= r || q >= r) continue;
                Cx<double>* bp = shB + p * RF;
                Cx<double>* bq = shB + q * RF;
                double al = 0, be = 0;
                Cx<double> ga{0, 0};
                for (int i = lane; i < r; i += 32) {
                    Cx<double> x = bp[i], y = bq[i];
                    al += x.x * x.x + x.y * x.y;
                    be += y.x * y.x + y.y * y.y;
                    ga.x += x.x * y.x + x.y * y.y;
                    ga.y += x.x * y.y - x.y * y.x;
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga.x = warp_sum(ga.x);
                ga.y = warp_sum(ga.y);
                double ag = sqrt(ga.x * ga.x + ga.y * ga.y);
                if (ag > 1e-15 * sqrt(al * be) && ag > 1e-300) {
                    double zeta = (be - al) / (2.0 * ag);
                    double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    Cx<double> ph{ga.x / ag, ga.y / ag};  // e^{i phi}
                    Cx<double>* jp_ = shJ + p * RF;
                    Cx<double>* jq_ = shJ + q * RF;
                    for (int i = lane; i < r; i += 32) {
                        Cx<double> x = bp[i], y = bq[i];
                        // x' = c x - s e^{-i phi} y ; y' = s e^{i phi} x + c y
                        Cx<double> ey = cmulc(y, ph), ex = cmul(x, ph);
                        bp[i] = Cx<double>{c * x.x - s * ey.x, c * x.y - s * ey.y};
                        bq[i] = Cx<double>{s * ex.x + c * y.x, s * ex.y + c * y.y};
                        x = jp_[i];
                        y = jq_[i];
                        ey = cmulc(y, ph);
                        ex = cmul(x, ph);
                        jp_[i] = Cx<double>{c * x.x - s * ey.x, c * x.y - s * ey.y};
                        jq_[i] = Cx<double>{s * ex.x + c * y.x, s * ex.y + c * y.y};
                    }
                    if (lane == 0) atomicAdd(&S.rot, 1);
                }
            }
            __syncthreads();
        }
        const int rot = S.rot;
        __syncthreads();
        if (rot == 0) break;
        if (sweep == 29 && tid == 0) atomicOr(A.status, ST_JACOBI_NOCONV);
    }
    // singular values, sort descending, truncation sigma < eps_face * sigma_max
    for (int a = tid; a < r; a += NT) {
        double s2 = 0;
        for (int i = 0; i < r; ++i) s2 += cabs2(shB[a * RF + i]);
        S.sig[a] = sqrt(s2);
    }
    __syncthreads();
    double smax = 0;
    for (int a = 0; a < r; ++a) smax = fmax(smax, S.sig[a]);
    for (int a = tid; a < r; a += NT) {
        int rank = 0;
        for (int b = 0; b < r; ++b)
            if (S.sig[b] > S.sig[a] || (S.sig[b] == S.sig[a] && b < a)) ++rank;
        bool keep = S.sig[a] > 0.0 && S.sig[a] >= A.eps_face * smax;
        S.sel[rank] = keep ? a : -1;
    }
    __syncthreads();
    int rn = 0;
    while (rn < r && S.sel[rn] >= 0) ++rn;
    // T_U = diag(dU) RhatU^{-1} B[:, sel] ;  T_V = diag(dV) RhatV^{-1} J[:, sel]   (back substitution)
    for (int item = tid; item < 2 * rn; item += NT) {
        const bool isU = item < rn;
        const int b = isU ? item : item - rn;
        const Cx<double>* R = isU ? w.RU : w.RV;
        const Cx<double>* rhs = (isU ? shB : shJ) + S.sel[b] * RF;
        const double* dsc = isU ? S.dU : S.dV;
        Cx<double>* Tm = isU ? w.TU : w.TV;
        for (int a = r - 1; a >= 0; --a) {
            Cx<double> acc = rhs[a];
            for (int c = a + 1; c < r; ++c) {
                Cx<double> z = Tm[c * RF + b];  // z[c] (unscaled, stored temporarily)
                Cx<double> rr = R[a * RF + c];
                acc.x -= rr.x * z.x - rr.y * z.y;
                acc.y -= rr.x * z.y + rr.y * z.x;
            }
            double rd = R[a * RF + a].x;
            Tm[a * RF + b] = Cx<double>{acc.x / rd, acc.y / rd};
        }
        for (int a = 0; a < r; ++a) {
            Tm[a * RF + b].x *= dsc[a];
            Tm[a * RF + b].y *= dsc[a];
        }
    }
    __syncthreads();
    // move T_U, T_V into shared memory (the Jacobi buffers are free now)
    for (int e = tid; e < r * rn; e += NT) {
        const int a = e / rn, b = e % rn;
        shB[a * RF + b] = w.TU[a * RF + b];
        shJ[a * RF + b] = w.TV[a * RF + b];
    }
    __syncthreads();
    return rn;
}

// ---- the persistent kernel ---------------------------------------------------------
template <int KER, class T, int NT>
__global__ void __launch_bounds__(NT) k_aca3(AcaArgs<T> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockSh<T> S;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int RF = A.RF;
    Cx<double>* shB = reinterpret_cast<Cx<double>*>(smem_raw);
    Cx<double>* shJ = shB + RF * RF;
    const Ws<T> w = ws_carve<T>(A.ws + (size_t)blockIdx.x * A.ws_stride, RF, A.Mmax, A.Nmax, A.Cmax, A.Ku);
    __shared__ int s_q;
    for (int iter = 0;; ++iter) {
        if (tid == 0) {
            if (A.single >= 0)
                s_q = (iter == 0 && blockIdx.x == 0) ? A.single : -1;
            else {
                int q = atomicAdd(A.queue_head, 1);
                s_q = q < A.n_far ? q : -1;
            }
        }
        __syncthreads();
        const int qi = s_q;
        __syncthreads();
        if (qi < 0) break;
        const int blk = A.queue[qi];
        if (tid == 0) {
            BlockRange br = A.ranges[blk];
            S.rb = br.rb;
            S.cb = br.cb;
            S.M = br.re - br.rb;
            S.N = br.ce - br.cb;
            S.blk = blk;
            S.ncross = 0;
            S.pre[0] = 0;
            S.norm2 = 0.0;
            S.entries = 0;
            S.k = A.k1 ? A.k1[blk] : 0;
            for (int i = 0; i < KU_MAX / 32; ++i) S.used_k[i] = 0u;
        }
        __syncthreads();
        const int M = S.M, N = S.N, Ku = A.Ku;
        bool zero_block = false;
        int computed = 0;
        bool overflow = false;
        if (M > A.Mmax || N > A.Nmax) {  // cannot happen: workspace is sized from the block list
            if (tid == 0) atomicOr(A.status, ST_BAD_INDEX);
            overflow = true;
        }
        while (!overflow) {
            // ---------------- face at S.k ----------------
            int kf = S.k;
            int r = face_aca<KER, T, NT>(A, w, S, kf);
            if (tid == 0) S.used_k[kf >> 5] |= 1u << (kf & 31);
            __syncthreads();
            if (r == 0) {
                // zero face: test up to three more unused frequencies
                int cand[3] = {Ku - 1, Ku / 2, A.k_maxabs};
                bool found = false;
                int tested = 0;
                for (int c = 0; c < 3 && !found; ++c) {
                    int kk = cand[c];
                    bool dup = false;
                    for (int d = 0; d < c; ++d) dup |= (cand[d] == kk);
                    if (dup || (S.used_k[kk >> 5] >> (kk & 31)) & 1u) continue;
                    ++tested;
                    __syncthreads();
                    if (tid == 0) S.used_k[kk >> 5] |= 1u << (kk & 31);
                    __syncthreads();
                    r = face_aca<KER, T, NT>(A, w, S, kk);
                    if (r > 0) {
                        found = true;
                        kf = kk;
                    }
                }
                if (!found) {
                    zero_block = (S.ncross == 0);
                    break;
                }
                if (tid == 0) S.k = kf;
                __syncthreads();
            }
            ++computed;
            // ---------------- recompression ----------------
            int rn = -1;
            if (!A.no_recompress) {
                rn = recompress<T, NT>(A, w, S, r, shB, shJ);
                if (rn < 0 && tid == 0) atomicOr(A.status, ST_CHOL_FALLBACK);
            }
            const bool raw = rn < 0;
            if (raw) rn = r;
            // allocate U', V', f in the pool
            if (tid == 0) {
                long long need = (long long)rn * (M + N) + Ku;
                unsigned long long o = atomicAdd(A.pool_ctr, (unsigned long long)need);
                if ((long long)o + need > A.pool_cap) {
                    atomicOr(A.status, ST_POOL_OVERFLOW);
                    S.new_off = -1;
                } else {
                    S.new_off = (long long)o;
                }
                S.rnew = rn;
            }
            __syncthreads();
            if (S.new_off < 0) {
                overflow = true;
                break;
            }
            const long long off = S.new_off;
            Cx<T>* Un = A.pool + off;
            Cx<T>* Vn = A.pool + off + (long long)rn * M;
            Cx<T>* Fn = A.pool + off + (long long)rn * (M + N);
            if (raw) {
                for (int e = tid; e < rn * M; e += NT) Un[e] = w.uw[(size_t)(e / M) * A.Mmax + e % M];
                for (int e = tid; e < rn * N; e += NT) Vn[e] = w.vw[(size_t)(e / N) * A.Nmax + e % N];
            } else {
                for (int i = tid; i < M; i += NT) {
                    for (int b = 0; b < rn; ++b) {
                        Cx<double> acc{0, 0};
                        for (int a = 0; a < r; ++a) cfma(acc, ccast<double>(w.uw[(size_t)a * A.Mmax + i]), shB[a * RF + b]);
                        Un[(long long)b * M + i] = ccast<T>(acc);
                    }
                }
                for (int j = tid; j < N; j += NT) {
                    for (int b = 0; b < rn; ++b) {
                        Cx<double> acc{0, 0};
                        for (int a = 0; a < r; ++a) cfma(acc, ccast<double>(w.vw[(size_t)a * A.Nmax + j]), shJ[a * RF + b]);
                        Vn[(long long)b * N + j] = ccast<T>(acc);
                    }
                }
            }
            __syncthreads();
            // ---------------- pivot: argmax |U' V'^H| ----------------
            {
                constexpr int TM = sizeof(T) == 4 ? 64 : 32;
                constexpr int TN = TM;
                constexpr int RM = TM * TN / NT >= 16 ? 4 : 2;  // micro-tile edge
                constexpr int TX = TN / RM;                     // threads along j
                Cx<T>* tu = reinterpret_cast<Cx<T>*>(smem_raw);  // [rn][TM]
                Cx<T>* tv = tu + (size_t)RF * TM;                // [rn][TN]
                const int tx = tid % TX, ty = tid / TX;
                ArgMax best{-1.0, LLONG_MAX};
                for (int i0 = 0; i0 < M; i0 += TM) {
                    for (int j0 = 0; j0 < N; j0 += TN) {
                        for (int e = tid; e < rn * TM; e += NT) {
                            int b = e / TM, ii = e % TM;
                            tu[b * TM + ii] = (i0 + ii < M) ? Un[(long long)b * M + i0 + ii] : Cx<T>{0, 0};
                        }
                        for (int e = tid; e < rn * TN; e += NT) {
                            int b = e / TN, jj = e % TN;
                            tv[b * TN + jj] = (j0 + jj < N) ? Vn[(long long)b * N + j0 + jj] : Cx<T>{0, 0};
                        }
                        __syncthreads();
                        if (ty * RM < TM) {
                            Cx<T> acc[RM][RM];
#pragma unroll
                            for (int a = 0; a < RM; ++a)
#pragma unroll
                                for (int c = 0; c < RM; ++c) acc[a][c] = Cx<T>{0, 0};
                            for (int b = 0; b < rn; ++b) {
                                Cx<T> uu[RM], vv[RM];
#pragma unroll
                                for (int a = 0; a < RM; ++a) uu[a] = tu[b * TM + ty * RM + a];
#pragma unroll
                                for (int c = 0; c < RM; ++c) vv[c] = tv[b * TN + tx * RM + c];
#pragma unroll
                                for (int a = 0; a < RM; ++a)
#pragma unroll
                                    for (int c = 0; c < RM; ++c) cfmac(acc[a][c], uu[a], vv[c]);
                            }
#pragma unroll
                            for (int a = 0; a < RM; ++a)
#pragma unroll
                                for (int c = 0; c < RM; ++c) {
                                    int gi = i0 + ty * RM + a, gj = j0 + tx * RM + c;
                                    if (gi < M && gj < N)
                                        best = amax_better(best, ArgMax{(double)cabs2(acc[a][c]), (long long)gi * N + gj});
                                }
                        }
                        __syncthreads();
                    }
                }
                best = block_argmax<NT>(best, S.am);
                if (tid == 0) {
                    S.ip = (int)(best.i / N);
                    S.jp = (int)(best.i % N);
                    Cx<double> h{0, 0};
                    for (int b = 0; b < rn; ++b)
                        cfmac(h, ccast<double>(Un[(long long)b * M + S.ip]), ccast<double>(Vn[(long long)b * N + S.jp]));
                    S.hpiv = h;
                }
            }
            __syncthreads();
            if (S.hpiv.x == 0.0 && S.hpiv.y == 0.0) break;  // vanishing face: nothing to divide by
            // H_p[i_l, j_l] of earlier crosses (float64)
            for (int p = tid; p < S.ncross; p += NT) {
                const Cx<T>* U = Up(A, S, p);
                const Cx<T>* V = Vp(A, S, p);
                Cx<double> h{0, 0};
                for (int t = 0; t < S.r[p]; ++t)
                    cfmac(h, ccast<double>(U[(long long)t * M + S.ip]), ccast<double>(V[(long long)t * N + S.jp]));
                S.hp[p] = h;
            }
            __syncthreads();
            // ---------------- fiber (float64 residual) ----------------
            const int ip = S.ip, jp = S.jp, nc = S.ncross;
            const Cx<double> hpiv = S.hpiv;
            for (int k = tid; k < Ku; k += NT) {
                Cx<double> e = ccast<double>(ent<KER, T>(A, S.rb + ip, S.cb + jp, k));
                for (int p = 0; p < nc; ++p) {
                    Cx<double> fp = ccast<double>(Fp(A, S, p)[k]);
                    Cx<double> hf = cmul(S.hp[p], fp);
                    e.x -= hf.x;
                    e.y -= hf.y;
                }
                Cx<double> fv = cdiv(e, hpiv);
                w.fib[k] = fv;
                Fn[k] = ccast<T>(fv);
            }
            if (tid == 0) S.entries += Ku;
            __syncthreads();
            // ---------------- eq. (norm) ----------------
            // <f_l, f_d> and ||f_l||^2
            for (int d = wid; d <= nc; d += NT / 32) {
                Cx<double> acc{0, 0};
                if (d < nc) {
                    const Cx<T>* fd = Fp(A, S, d);
                    for (int k = lane; k < Ku; k += 32) cfmac(acc, w.fib[k], ccast<double>(fd[k]));
                } else {
                    for (int k = lane; k < Ku; k += 32) acc.x += cabs2(w.fib[k]);
                }
                acc.x = warp_sum(acc.x);
                acc.y = warp_sum(acc.y);
                if (lane == 0) {
                    if (d < nc) S.ff[d] = acc;
                    else S.fself = acc.x;
                }
            }
            for (int d = tid; d < nc; d += NT) S.hh[d] = Cx<double>{0, 0};
            if (tid == 0) S.hself = 0.0;
            __syncthreads();
            // <H_l, H_d> = sum_{a,b} (U_d^H U_l)[a][b] (V_l^H V_d)[b][a]; d = nc gives ||H_l||^2
            {
                long long total = 0;
                for (int d = 0; d <= nc; ++d) total += (long long)(d < nc ? S.r[d] : rn) * rn;
                for (long long it = wid; it < total; it += NT / 32) {
                    long long q = it;
                    int d = 0;
                    while (true) {
                        long long sz = (long long)(d < nc ? S.r[d] : rn) * rn;
                        if (q < sz) break;
                        q -= sz;
                        ++d;
                    }
                    const int a = (int)(q / rn), b = (int)(q % rn);
                    const Cx<T>* Ud = d < nc ? Up(A, S, d) : Un;
                    const Cx<T>* Vd = d < nc ? Vp(A, S, d) : Vn;
                    const Cx<T>* ua = Ud + (long long)a * M;
                    const Cx<T>* ub = Un + (long long)b * M;
                    const Cx<T>* va = Vd + (long long)a * N;
                    const Cx<T>* vb = Vn + (long long)b * N;
                    Cx<T> gu{0, 0}, gv{0, 0};
                    for (int i = lane; i < M; i += 32) cfmac(gu, ub[i], ua[i]);  // conj(U_d[a]) U_l[b]
                    for (int j = lane; j < N; j += 32) cfmac(gv, va[j], vb[j]);  // conj(V_l[b]) V_d[a]
                    double gux = warp_sum((double)gu.x), guy = warp_sum((double)gu.y);
                    double gvx = warp_sum((double)gv.x), gvy = warp_sum((double)gv.y);
                    if (lane == 0) {
                        double px = gux * gvx - guy * gvy, py = gux * gvy + guy * gvx;
                        if (d < nc) {
                            atomicAdd(&S.hh[d].x, px);
                            atomicAdd(&S.hh[d].y, py);
                        } else {
                            atomicAdd(&S.hself, px);
                        }
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                double add = 0.0;
                for (int d = 0; d < nc; ++d) add += 2.0 * (S.hh[d].x * S.ff[d].x - S.hh[d].y * S.ff[d].y);
                double own = S.hself * S.fself;
                S.norm2 += add + own;
                bool stop = sqrt(fmax(own, 0.0)) <= A.eps3 * sqrt(fmax(S.norm2, 0.0));
                S.flag = 0;
                if (!stop) {
                    CrossRec cr;
                    cr.off = off;
                    cr.r = rn;
                    cr.ip = ip;
                    cr.jp = jp;
                    cr.kp = S.k;
                    A.rec[(size_t)blk * A.Cmax + nc] = cr;
                    S.off[nc] = off;
                    S.r[nc] = rn;
                    S.pre[nc + 1] = S.pre[nc] + rn;
                    S.ncross = nc + 1;
                    bool all_used = true;
                    for (int k = 0; k < Ku; ++k) all_used &= (S.used_k[k >> 5] >> (k & 31)) & 1u;
                    if (S.ncross >= A.Cmax || all_used) S.flag = 1;
                } else {
                    S.flag = 1;
                }
            }
            __syncthreads();
            if (S.flag) break;
            // next frequency: argmax over unused k of |f_l[k]|
            ArgMax nk{-1.0, LLONG_MAX};
            for (int k = tid; k < Ku; k += NT)
                if (!((S.used_k[k >> 5] >> (k & 31)) & 1u)) nk = amax_better(nk, ArgMax{cabs2(w.fib[k]), (long long)k});
            nk = block_argmax<NT>(nk, S.am);
            if (tid == 0) S.k = (int)nk.i;
            __syncthreads();
        }
        if (tid == 0) {
            A.r3[blk] = S.ncross;
            atomicAdd(&A.counters[0], (unsigned long long)S.entries);
            atomicAdd(&A.counters[1], (unsigned long long)computed);
            if (zero_block) atomicAdd(&A.counters[2], 1ull);
        }
        __syncthreads();
    }
}

// ============================================================================
// host driver
// ============================================================================

template <int KER, class T, int NT>
static g3_status launch_aca_t(g3_ctx* ctx, AcaArgs<T>& A, int grid, size_t smem) {
    auto kfn = k_aca3<KER, T, NT>;
    G3_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kfn<<<grid, NT, smem, ctx->stream>>>(A);
    ctx->count(KER == G3_SEPARABLE ? "k_aca3_separable" : "k_aca3");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

template <int KER, class T, int NT>
static int occupancy(size_t smem) {
    int nb = 0;
    auto kfn = k_aca3<KER, T, NT>;
    cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, NT, smem) != cudaSuccess) nb = 1;
    return std::max(nb, 1);
}

template <class T>
static g3_status run_aca_t(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_factors* fa, int kernel,
                           double eps3, const g3_opts& o, const void* sep_a, const void* sep_b, const void* sep_c,
                           int sep_R) {
    const bool sep = kernel == G3_SEPARABLE;
    const int Ku = fa->Ku;
    const int RF = o.face_rank_max > 0 ? std::min(o.face_rank_max, RF_MAX) : 48;
    // block list (far order) and queue
    std::vector<BlockRange> ranges;
    if (sep) {
        ranges.push_back(BlockRange{0, fa->M_sep, 0, fa->N_sep});
    } else {
        for (int b : t->far_index) {
            const int32_t* r = &t->blocks[5 * (size_t)b];
            ranges.push_back(BlockRange{r[0], r[1], r[2], r[3]});
        }
    }
    const int n_far = (int)ranges.size();
    fa->n_far = n_far;
    fa->ranges = ranges;
    fa->Cmax = Ku;
    fa->r3.assign(n_far, 0);
    if (n_far == 0) return G3_OK;
    int Mmax = 0, Nmax = 0;
    long long sumMN = 0;
    for (auto& r : ranges) {
        Mmax = std::max(Mmax, r.re - r.rb);
        Nmax = std::max(Nmax, r.ce - r.cb);
        sumMN += (r.re - r.rb) + (r.ce - r.cb);
    }
    std::vector<int> queue(n_far);
    std::iota(queue.begin(), queue.end(), 0);
    const int order = o.order_by_cost;  // 0 given -> default on
    if (order >= 0) {
        std::vector<double> cost(n_far);
        for (int i = 0; i < n_far; ++i) {
            double mm = ranges[i].re - ranges[i].rb, nn = ranges[i].ce - ranges[i].cb;
            cost[i] = o.cost ? (double)o.cost[i] : mm * nn;
        }
        std::stable_sort(queue.begin(), queue.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    }
    DevBuf d_ranges, d_queue, d_head, d_k1, d_counters, d_ctr;
    G3_CUDA(d_ranges.alloc(n_far * sizeof(BlockRange)));
    G3_CUDA(d_queue.alloc(n_far * sizeof(int)));
    G3_CUDA(d_head.alloc(sizeof(int)));
    G3_CUDA(d_counters.alloc(8 * sizeof(unsigned long long)));
    G3_CUDA(d_ctr.alloc(sizeof(unsigned long long)));
    G3_CUDA(cudaMemcpyAsync(d_ranges.p, ranges.data(), n_far * sizeof(BlockRange), cudaMemcpyHostToDevice, ctx->stream));
    G3_CUDA(cudaMemcpyAsync(d_queue.p, queue.data(), n_far * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    if (o.k1) {
        for (int i = 0; i < n_far; ++i)
            if (o.k1[i] < 0 || o.k1[i] >= Ku) return fail(G3_EINVAL, "opts->k1[%d] = %d outside [0, %d)", i, o.k1[i], Ku);
        G3_CUDA(d_k1.alloc(n_far * sizeof(int)));
        G3_CUDA(cudaMemcpyAsync(d_k1.p, o.k1, n_far * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    }
    // separable inputs (converted to T)
    DevBuf d_sa, d_sb, d_sc;
    SepView<T> sv{};
    if (sep) {
        auto up = [&](DevBuf& d, const void* src, size_t n) -> g3_status {
            std::vector<T> tmp(2 * n);
            const double* s = (const double*)src;
            for (size_t i = 0; i < 2 * n; ++i) tmp[i] = (T)s[i];
            G3_CUDA(d.alloc(tmp.size() * sizeof(T)));
            G3_CUDA(cudaMemcpy(d.p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
            return G3_OK;
        };
        g3_status st;
        if ((st = up(d_sa, sep_a, (size_t)sep_R * fa->M_sep)) != G3_OK) return st;
        if ((st = up(d_sb, sep_b, (size_t)sep_R * fa->N_sep)) != G3_OK) return st;
        if ((st = up(d_sc, sep_c, (size_t)sep_R * Ku)) != G3_OK) return st;
        sv = SepView<T>{sep_R, fa->M_sep, fa->N_sep, Ku, d_sa.as<T>(), d_sb.as<T>(), d_sc.as<T>()};
    }
    constexpr int NT = 256;
    // dynamic shared memory: Jacobi matrices (2 RF^2 complex double), reused for
    // the pivot-search tiles (2 RF TM complex T, TM = 64 float / 32 double)
    const size_t tile_bytes = 2 * (size_t)RF * (sizeof(T) == 4 ? 64 : 32) * sizeof(Cx<T>);
    const size_t smem = std::max(2 * (size_t)RF * RF * sizeof(Cx<double>), tile_bytes);
    int per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : 0;
    if (per_sm == 0) {
        if (kernel == G3_SLP) per_sm = occupancy<G3_SLP, T, NT>(smem);
        else if (kernel == G3_DLP) per_sm = occupancy<G3_DLP, T, NT>(smem);
        else per_sm = occupancy<G3_SEPARABLE, T, NT>(smem);
    }
    int grid = o.unbatched ? 1 : std::min(n_far, ctx->n_sm * per_sm);
    const size_t stride = al256(ws_bytes<T>(RF, Mmax, Nmax, Ku, Ku));
    DevBuf d_ws;
    G3_CUDA(d_ws.alloc(stride * grid));
    G3_CUDA(fa->d_rec.alloc((size_t)n_far * Ku * sizeof(CrossRec)));
    G3_CUDA(fa->d_r3.alloc((size_t)n_far * sizeof(int)));
    // factor pool: initial estimate, regrown on overflow
    double pf = o.pool_factor > 0 ? o.pool_factor : 1.0;
    long long cap = (long long)(pf * (double)(sumMN * 16 * 12 + (long long)n_far * Ku * 16));
    cap = std::max(cap, (long long)1 << 16);
    int regrows = 0;
    cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1];
    float ms_total = 0;
    for (;;) {
        G3_CUDA(fa->pool.alloc((size_t)cap * sizeof(Cx<T>)));
        fa->pool_cap = cap;
        G3_CUDA(cudaMemsetAsync(d_head.p, 0, sizeof(int), ctx->stream));
        G3_CUDA(cudaMemsetAsync(d_counters.p, 0, 8 * sizeof(unsigned long long), ctx->stream));
        G3_CUDA(cudaMemsetAsync(d_ctr.p, 0, sizeof(unsigned long long), ctx->stream));
        G3_CUDA(cudaMemsetAsync(ctx->status.p, 0, sizeof(unsigned), ctx->stream));
        AcaArgs<T> A{};
        A.gf = t ? t->gf : GeomF{};
        A.gd = t ? t->gd : GeomD{};
        A.sep = sv;
        A.sd = f ? f->d_sd.as<double2>() : nullptr;
        A.Ku = Ku;
        A.k_maxabs = f ? f->k_maxabs : Ku - 1;
        A.ranges = d_ranges.as<BlockRange>();
        A.n_far = n_far;
        A.queue = d_queue.as<int>();
        A.queue_head = d_head.as<int>();
        A.single = -1;
        A.k1 = o.k1 ? d_k1.as<int>() : nullptr;
        A.Cmax = Ku;
        A.RF = RF;
        A.eps3 = eps3;
        A.eps_face = eps3 / 100.0;
        A.no_recompress = o.no_recompress;
        A.pool = fa->pool.as<Cx<T>>();
        A.pool_cap = cap;
        A.pool_ctr = d_ctr.as<unsigned long long>();
        A.rec = fa->d_rec.as<CrossRec>();
        A.r3 = fa->d_r3.as<int>();
        A.counters = d_counters.as<unsigned long long>();
        A.status = ctx->status.as<unsigned>();
        A.ws = d_ws.as<char>();
        A.ws_stride = stride;
        A.Mmax = Mmax;
        A.Nmax = Nmax;
        G3_CUDA(cudaEventRecord(e0, ctx->stream));
        g3_status st = G3_OK;
        const int launches = o.unbatched ? n_far : 1;
        for (int l = 0; l < launches && st == G3_OK; ++l) {
            if (o.unbatched) A.single = l;
            if (kernel == G3_SLP) st = launch_aca_t<G3_SLP, T, NT>(ctx, A, grid, smem);
            else if (kernel == G3_DLP) st = launch_aca_t<G3_DLP, T, NT>(ctx, A, grid, smem);
            else st = launch_aca_t<G3_SEPARABLE, T, NT>(ctx, A, grid, smem);
        }
        if (st != G3_OK) return st;
        G3_CUDA(cudaEventRecord(e1, ctx->stream));
        unsigned status = 0;
        unsigned long long ctr = 0;
        G3_CUDA(cudaMemcpyAsync(&status, ctx->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaMemcpyAsync(&ctr, d_ctr.p, sizeof(ctr), cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
        float ms = 0;
        G3_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms_total += ms;
        if (status & ST_POOL_OVERFLOW) {
            if (++regrows > 6) return fail(G3_EOVERFLOW, "aca3_compress: factor pool overflow after %d regrows", regrows);
            cap = std::max(cap * 2, (long long)(ctr * 5 / 4));
            continue;
        }
        unsigned long long cnt[8];
        G3_CUDA(cudaMemcpy(cnt, d_counters.p, sizeof(cnt), cudaMemcpyDeviceToHost));
        fa->r3.resize(n_far);
        G3_CUDA(cudaMemcpy(fa->r3.data(), fa->d_r3.p, n_far * sizeof(int), cudaMemcpyDeviceToHost));
        fa->rec.resize((size_t)n_far * Ku);
        G3_CUDA(cudaMemcpy(fa->rec.data(), fa->d_rec.p, fa->rec.size() * sizeof(CrossRec), cudaMemcpyDeviceToHost));
        g3_stats& S = fa->stats;
        S = g3_stats{};
        S.n_far = n_far;
        S.entries = (int64_t)cnt[0];
        S.crosses_computed = (int64_t)cnt[1];
        S.zero_blocks = (int32_t)cnt[2];
        S.capped_faces = (int32_t)cnt[3];
        S.pool_regrows = regrows;
        S.status_bits = (int32_t)status;
        S.ms = ms_total;
        for (int b = 0; b < n_far; ++b) {
            const int M = ranges[b].re - ranges[b].rb, N = ranges[b].ce - ranges[b].cb;
            S.crosses += fa->r3[b];
            S.r3_max = std::max(S.r3_max, fa->r3[b]);
            S.dense_bytes += (int64_t)M * N * Ku * (int64_t)sizeof(Cx<T>);
            for (int p = 0; p < fa->r3[b]; ++p) {
                const CrossRec& c = fa->rec[(size_t)b * Ku + p];
                S.face_rank_sum += c.r;
                S.face_rank_max = std::max(S.face_rank_max, c.r);
                S.factor_bytes += ((int64_t)c.r * (M + N) + Ku) * (int64_t)sizeof(Cx<T>);
            }
        }
        return G3_OK;
    }
}

g3_status run_aca(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_factors* fa, int kernel, int scheme,
                  double eps3, const g3_opts& o, const void* sep_a, const void* sep_b, const void* sep_c, int sep_R) {
    if (scheme != G3_COLLOC7 && kernel != G3_SEPARABLE)
        return fail(G3_EUNSUPPORTED, "aca3_compress: only G3_COLLOC7 is implemented");
    if (fa->Ku > KU_MAX) return fail(G3_EINVAL, "aca3_compress: %d unique frequencies exceed %d", fa->Ku, KU_MAX);
    if (fa->prec == G3_MIXED) return run_aca_t<float>(ctx, t, f, fa, kernel, eps3, o, sep_a, sep_b, sep_c, sep_R);
    return run_aca_t<double>(ctx, t, f, fa, kernel, eps3, o, sep_a, sep_b, sep_c, sep_R);
}

}  // namespace g3
