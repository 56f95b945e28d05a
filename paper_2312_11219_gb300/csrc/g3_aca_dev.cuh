#pragma once
// Three-way (generalised) ACA of every admissible block (Algorithm 1) in one
// persistent launch.
//
// Each CTA claims blocks from an atomic queue counter (longest first) and runs
// Algorithm 1 on the block restricted to the unique frequencies:
//   face    partial-pivot ACA of the residual face at k_l (eps_face), with the
//           residual of earlier crosses subtracted row/column-wise;
//   recomp  Cholesky-QR of both ACA factors (float64 Cholesky of column-scaled
//           Gram matrices), then the r x r core R_U R_V^H is factored: float64
//           (T = double) by a one-sided Jacobi SVD truncated at
//           sigma_i < eps_face sigma_1, float32 (T = float) by a column-pivoted
//           QR stopped when the largest remaining column norm falls below the
//           same threshold (Section 4, second implementation remark);
//   pivot   argmax |H_l[i, j]| over the dense expansion of U' V'^H, tiled
//           through shared memory, ties to the smallest row-major index
//           (Section 4, last remark), or optionally (single layer) the
//           row of eq. (index) from the factors and the largest entry of
//           that row;
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
// In both, the fiber residuals, the Cholesky factors of the recompression,
// the sums over crosses of eq. (norm) and ||C^(l)|| are float64; with
// T = float the Gram products, the core factorisation and the back
// substitution of the recompression are float32.
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
constexpr int SAMPLES = 32;   // sample entries of the convergence checks
constexpr int NPH = 10;       // per-block diagnostics: 7 phases, steps, start, end
constexpr int NSUB = 12;      // sub-step cycle counters (diagnostics)
// rows staged per pass of the eq. (norm) Gram products
template <class T>
constexpr int NORM_RC = sizeof(T) == 4 ? 64 : 32;

// sub-step timing by thread 0: adds the cycles since *t0 to slot i
template <class T>
__device__ __forceinline__ void sublap(T& S, int i, long long& t0) {
    if (threadIdx.x == 0) {
        const long long t = clock64();
        S.sub[i] += t - t0;
        t0 = t;
    }
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int RF_MAX = 64;    // largest face rank cap

// geometry and frequencies of one mesh of a batched compression
struct GeoDesc {
    GeomF gf;
    GeomD gd;
    const double2* sd;
    const float2* sf;
    int Ku, k_maxabs;
};

template <class T>
struct AcaArgs {
    const GeoDesc* geos;     // batched compression: per-mesh data (null: gf ... k_maxabs below)
    const int* bgeo;         // [n_far] mesh of each block
    GeomF gf;
    GeomD gd;
    SepView<T> sep;
    const double2* sd;
    const float2* sf;        // the unique frequencies rounded once to float32
    int Ku, k_maxabs;
    const BlockRange* ranges;
    int n_far;
    const int* queue;
    int* queue_head;
    int single;              // >= 0: CTA 0 processes queue[single] only
    const int* k1;           // [n_far] first frequency per block, or null
    int Cmax, RF;
    int dense_max;           // blocks with M N <= dense_max use exact dense faces
    int sample_check;        // confirm each stop on fixed sample entries
    int pivot_index;         // single layer: pivot of low-rank faces by eq. (index)
    double eps3, eps_face;
    double face_floor;       // absolute floor factor of the face tests (0 = none)
    double trunc_floor;      // absolute floor factor of the recompression truncation (0 = none)
    int no_recompress;
    Cx<T>* pool;
    long long pool_cap;
    unsigned long long* pool_ctr;
    int* spill;              // [n_far] blocks that found the pool full
    int* spill_n;
    int spill_cap;
    CrossRec* rec;
    int* r3;
    long long* blk_cycles;   // [n_far][NPH] SM cycles per phase spent on each block, its face ACA
                             // steps, and its start and end time (global timer, ns)
    unsigned long long* counters;  // [0] entries [1] crosses computed [2] zero blocks [3] capped faces
                                   // [8..14] clock cycles per phase (thread 0 of each CTA)
    unsigned* status;
    char* ws;
    size_t ws_stride;
    int Mmax, Nmax;
    int drf_max;             // float32 low-rank faces of blocks with M N <= drf_max are evaluated
                             // densely into a working buffer before their ACA (0 = never)
    size_t drf_off;          // byte offset of that buffer in each CTA's workspace slice
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
    long long* colU;      // [Cmax * RF] flattened column tables (when they exceed shared memory)
    long long* colV;
    short* colP;
    Cx<double>* hs;       // [SAMPLES][Cmax] H_p at the stop-check samples
    double* rk;           // [Ku] sampled residual per frequency
    Cx<T>* dres;          // [drf_max] dense residual working face (row-major, ld N), or null
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
    add((size_t)(Cmax + 1) * RF * sizeof(Cx<T>));
    for (int i = 0; i < 4; ++i) add((size_t)RF * RF * sizeof(Cx<double>));
    add((size_t)Ku * sizeof(Cx<double>));
    add((size_t)Cmax * RF * sizeof(long long));
    add((size_t)Cmax * RF * sizeof(long long));
    add((size_t)Cmax * RF * sizeof(short));
    add((size_t)32 * Cmax * sizeof(Cx<double>));
    add((size_t)Ku * sizeof(double));
    return b;
}

template <class T>
__device__ inline Ws<T> ws_carve(char* base, int RF, int Mmax, int Nmax, int Cmax, int Ku, size_t drf_off = 0) {
    Ws<T> w;
    w.dres = drf_off ? reinterpret_cast<Cx<T>*>(base + drf_off) : nullptr;
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
    w.pre = (Cx<T>*)take((size_t)(Cmax + 1) * RF * sizeof(Cx<T>));
    w.RU = (Cx<double>*)take((size_t)RF * RF * sizeof(Cx<double>));
    w.RV = (Cx<double>*)take((size_t)RF * RF * sizeof(Cx<double>));
    w.TU = (Cx<double>*)take((size_t)RF * RF * sizeof(Cx<double>));
    w.TV = (Cx<double>*)take((size_t)RF * RF * sizeof(Cx<double>));
    w.fib = (Cx<double>*)take((size_t)Ku * sizeof(Cx<double>));
    w.colU = (long long*)take((size_t)Cmax * RF * sizeof(long long));
    w.colV = (long long*)take((size_t)Cmax * RF * sizeof(long long));
    w.colP = (short*)take((size_t)Cmax * RF * sizeof(short));
    w.hs = (Cx<double>*)take((size_t)32 * Cmax * sizeof(Cx<double>));
    w.rk = (double*)take((size_t)Ku * sizeof(double));
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
    double rdU[RF_MAX], rdV[RF_MAX];  // 1 / diagonal of the Cholesky factors
    T cnV[RF_MAX];                    // column norms of V' (pivot of eq. (index))
    T tdU[RF_MAX], tdV[RF_MAX];       // dU, dV and rdU, rdV in the working precision
    T trdU[RF_MAX], trdV[RF_MAX];
    double fsn2;             // ||S_m||_F^2 of the face approximant (recursive)
    int fconv;               // face test passed (written by warp 0)
    int fbs;                 // sample of the largest residual
    int sel[RF_MAX];
    int piv;                 // pivoted QR of the core: pivot column of the step
    float rkk;               // and its norm
    ArgMaxT<T> am[32];
    double red[64];
    double norm2;
    double red2[2];          // sampled residual / data norms of the stop check
    double samp[SAMPLES];    // |residual|^2 of the face approximant at the samples
    int stop;
    double hself;            // ||H_l||^2
    double fself;            // ||f_l||^2
    Cx<double> hpiv;
    long long new_off;
    long long entries;
    int raw;              // face ACA steps of the block (ranks before recompression)
    long long sub[NSUB];  // SM cycles of sub-steps (thread 0): recompression Gram, Cholesky,
                          // core, Jacobi, rest; face table, rows, columns, norm, samples
    int flag;
    int rot;
    int rnew;
    int ip, jp;
};

// sh: NT / 32 + 1 slots; the result goes to its own slot, so two barriers
// suffice (the next call writes the per-warp slots only after every thread
// has passed this call's second barrier, and the result slot only after its
// own first one)
template <int NT, class V>
__device__ __forceinline__ ArgMaxT<V> block_argmax(ArgMaxT<V> a, ArgMaxT<V>* sh) {
    a = warp_argmax(a);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = a;
    __syncthreads();
    if (w == 0) {
        ArgMaxT<V> b = (l < NT / 32) ? sh[l] : amax_none<V>();
        b = warp_argmax(b);
        if (l == 0) sh[NT / 32] = b;
    }
    __syncthreads();
    return sh[NT / 32];
}

template <class T>
__device__ __forceinline__ T tiny_norm2();
template <>
__device__ __forceinline__ float tiny_norm2<float>() { return 1.1754944e-38f; }
template <>
__device__ __forceinline__ double tiny_norm2<double>() { return 2.2250738585072014e-308; }

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
    } else if constexpr (KER == G3_GAL_SLP) {
        // admissible blocks never hold pairs with a common vertex
        if constexpr (sizeof(T) == 4) {
            const float2 s = A.sf[k];
            return gal_regular<T>(A.gf, A.gd, gi, gj, s.x, s.y);
        } else {
            const double2 s = A.sd[k];
            return gal_regular<T>(A.gf, A.gd, gi, gj, s.x, s.y);
        }
    } else if constexpr (KER == G3_GAL_P1D || KER == G3_GAL_P1KP) {
        // linear elements, element-local functions: regular pairs only (as above)
        if constexpr (sizeof(T) == 4) {
            const float2 s = A.sf[k];
            return p1_entry<KER, T>(A.gf, A.gd, gi, gj, s.x, s.y);
        } else {
            const double2 s = A.sd[k];
            return p1_entry<KER, T>(A.gf, A.gd, gi, gj, s.x, s.y);
        }
    } else {
        if constexpr (sizeof(T) == 4) {
            const float2 s = A.sf[k];
            return colloc_entry<KER, T>(A.gf, A.gd, gi, gj, s.x, s.y);
        } else {
            const double2 s = A.sd[k];
            return colloc_entry<KER, T>(A.gf, A.gd, gi, gj, s.x, s.y);
        }
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

// ---- one quadrature point of a collocation entry --------------------------------------
template <int KER, class G, class T>
__device__ __forceinline__ Cx<T> colloc_q(const G& g, int i, int j, int q, T sre, T sim) {
    T d[3];
    cdiff(g, i, j, d);
    T rx = d[0] - qoff(g, q, 0, j), ry = d[1] - qoff(g, q, 1, j), rz = d[2] - qoff(g, q, 2, j);
    T r2 = rx * rx + ry * ry + rz * rz;
    T ri = krsqrt(r2);
    T r = r2 * ri;
    T wq = qwt(g, q, j) * (T)G3_INV4PI;
    T amp;
    if (KER == G3_DLP) {
        T pd = d[0] * nrm(g, 0, j) + d[1] * nrm(g, 1, j) + d[2] * nrm(g, 2, j);
        amp = wq * pd * ri * ri * ri;
    } else {
        amp = wq * ri;
    }
    T m = amp * kexp(-sre * r);
    T sn, cs;
    ksincos(sim * r, &sn, &cs);
    if (KER == G3_DLP) {
        T fr = (T)1 + sre * r, fi = sim * r;
        return {m * (fr * cs + fi * sn), m * (fi * cs - fr * sn)};
    }
    return {m * cs, -m * sn};
}

// part `part` of a gang of G threads evaluating ENTRY(gi, gj, k): the
// quadrature points (terms) are dealt round-robin to the parts, so that no
// part idles while another evaluates the whole entry.  The gang sum is the
// entry (admissible blocks hold no self entries).
template <int KER, class T>
__device__ __forceinline__ Cx<T> ent_part(const AcaArgs<T>& A, int gi, int gj, int k, int part, int G) {
    if constexpr (KER == G3_SEPARABLE || KER == G3_GAL_P1D || KER == G3_GAL_P1KP) {
        return part == 0 ? ent<KER, T>(A, gi, gj, k) : Cx<T>{0, 0};
    } else if constexpr (KER == G3_GAL_SLP) {
        // 16 terms dealt round-robin to the gang's parts
        Cx<T> acc{0, 0};
        T sre, sim;
        if constexpr (sizeof(T) == 4) {
            const float2 s = A.sf[k];
            sre = s.x;
            sim = s.y;
        } else {
            const double2 s = A.sd[k];
            sre = s.x;
            sim = s.y;
        }
        for (int t = part; t < 16; t += G) {
            Cx<T> v;
            if constexpr (sizeof(T) == 4)
                v = gal_q(A.gf, gi, gj, t, sre, sim);
            else
                v = gal_q(A.gd, gi, gj, t, sre, sim);
            acc.x += v.x;
            acc.y += v.y;
        }
        return acc;
    } else {
        // the 7 quadrature points dealt round-robin to the gang's parts
        if (G == 1) return ent<KER, T>(A, gi, gj, k);
        T sre, sim;
        if constexpr (sizeof(T) == 4) {
            const float2 s = A.sf[k];
            sre = s.x;
            sim = s.y;
        } else {
            const double2 s = A.sd[k];
            sre = s.x;
            sim = s.y;
        }
        Cx<T> acc{0, 0};
        for (int q = part; q < 7; q += G) {
            Cx<T> v;
            if constexpr (sizeof(T) == 4)
                v = colloc_q<KER>(A.gf, gi, gj, q, sre, sim);
            else
                v = colloc_q<KER>(A.gd, gi, gj, q, sre, sim);
            acc.x += v.x;
            acc.y += v.y;
        }
        return acc;
    }
}

template <class T>
__device__ __forceinline__ Cx<T> shfl_xor_c(Cx<T> v, int o) {
    return Cx<T>{__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}

// gang size: the largest power of two <= 32 with L * G <= 2 NT (at most two
// passes over the line; a serial-work model that allowed more passes with
// larger gangs measured slower)
template <int NT>
__device__ __forceinline__ int gang_size(int L) {
    int G = 1;
    while (G < 32 && L * (G * 2) <= 2 * NT) G *= 2;
    return G;
}

// Per-face tables of the earlier crosses' columns, flattened over (p, t):
//   colU[c] / colV[c]  pool offsets of U_p[:, t] / V_p[:, t],  colP[c] = p,
// and the coefficient vector of the line being evaluated (coef[c], then the
// current face's m coefficients).  In shared memory when they fit, else in
// the workspace.
constexpr int TABMAX = 1024;    // flattened columns kept in shared memory
constexpr int ROWMAX = 1024;    // row buffer length kept in shared memory

template <class T>
struct FaceTab {
    const long long* colU;
    const long long* colV;
    const short* colP;
    Cx<T>* coef;
    Cx<T>* row;
    int ncol;   // sum of the earlier crosses' ranks
};

template <class T>
__host__ __device__ constexpr size_t facetab_smem_bytes() {
    return 2 * TABMAX * sizeof(long long) + TABMAX * sizeof(short) + (TABMAX + RF_MAX) * sizeof(Cx<T>) +
           ROWMAX * sizeof(Cx<T>) + 64;
}

template <class T, int NT>
__device__ FaceTab<T> facetab_build(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, unsigned char* arena) {
    FaceTab<T> F;
    const int nc = S.ncross;
    F.ncol = S.pre[nc];
    const bool sm = F.ncol <= TABMAX;
    unsigned char* p = arena;
    long long* cu = sm ? reinterpret_cast<long long*>(p) : w.colU;
    p += TABMAX * sizeof(long long);
    long long* cv = sm ? reinterpret_cast<long long*>(p) : w.colV;
    p += TABMAX * sizeof(long long);
    short* cp = sm ? reinterpret_cast<short*>(p) : w.colP;
    p += TABMAX * sizeof(short);
    p = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    F.coef = sm ? reinterpret_cast<Cx<T>*>(p) : w.pre;
    p += (TABMAX + RF_MAX) * sizeof(Cx<T>);
    F.row = S.N <= ROWMAX ? reinterpret_cast<Cx<T>*>(p) : w.row;
    for (int c = threadIdx.x; c < F.ncol; c += NT) {
        int q = 0;
        while (S.pre[q + 1] <= c) ++q;
        const int t = c - S.pre[q];
        cu[c] = S.off[q] + (long long)t * S.M;
        cv[c] = S.off[q] + (long long)S.r[q] * S.M + (long long)t * S.N;
        cp[c] = (short)q;
    }
    F.colU = cu;
    F.colV = cv;
    F.colP = cp;
    return F;
}

// coefficients of a row (f_p[kf] U_p[t][fix], then u_t[fix] of the current face)
// or of a column (f_p[kf] conj(V_p[t][fix]), then conj(v_t[fix]))
template <class T, int NT, bool ROW>
__device__ void line_coeffs(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, const FaceTab<T>& F, int fix,
                            int m) {
    for (int c = threadIdx.x; c < F.ncol + m; c += NT) {
        if (c < F.ncol) {
            const Cx<T> fk = S.fk[F.colP[c]];
            F.coef[c] = ROW ? cmul(fk, A.pool[F.colU[c] + fix]) : cmul(fk, cconj(A.pool[F.colV[c] + fix]));
        } else {
            const int t = c - F.ncol;
            F.coef[c] = ROW ? w.uw[(size_t)t * A.Mmax + fix] : cconj(w.vw[(size_t)t * A.Nmax + fix]);
        }
    }
}

// Residual of one row (ROW: fixed row `fix`, all columns) or one column (!ROW:
// fixed column `fix`, all rows) of the face at kf:
//   ENTRY - sum_p f_p[kf] (U_p V_p^H) - sum_{t<m} u_t v_t^H
//   ROW:  out[j] = ENTRY(fix, j) - sum_c coef[c] conj(X_c[j]),  X_c = V_p[:, t] | v_t
//   !ROW: out[i] = ENTRY(i, fix) - sum_c X_c[i] coef[c],        X_c = U_p[:, t] | u_t
// G threads per output element share the sum (sixteen loads in flight, four
// independent partial sums) and the quadrature points.  Returns the
// block-wide argmax of |out|^2 (ROW: over all columns; !ROW: over the rows
// not yet used).
constexpr int LIF = 16;  // loads in flight per thread in the residual lines' sums

template <int KER, class T, int NT, bool ROW>
__device__ ArgMaxT<T> residual_line(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, const FaceTab<T>& F,
                                    int fix, int kf, int m, Cx<T>* out, const Cx<T>* D) {
    const int tid = threadIdx.x;
    const int M = S.M, N = S.N;
    const int L = ROW ? N : M;
    const int G = gang_size<NT>(L);
    const int per = NT / G;
    const int part = tid % G;
    const long long* col = ROW ? F.colV : F.colU;
    const Cx<T>* cur = ROW ? w.vw : w.uw;
    const size_t ldc = ROW ? A.Nmax : A.Mmax;
    const int nt = F.ncol;
    ArgMaxT<T> am = amax_none<T>();
    for (int base = 0; base < L; base += per) {
        const int v = base + tid / G;
        Cx<T> acc{0, 0};
        if (v < L) {
            if (D) {
                // the dense residual working face holds ENTRY minus the earlier crosses
                if (part == 0) acc = ldcx(D + (ROW ? (size_t)fix * N + v : (size_t)v * N + fix));
            } else {
                const int gi = S.rb + (ROW ? fix : v), gj = S.cb + (ROW ? v : fix);
                const long long te = tid == 0 ? clock64() : 0;
                acc = ent_part<KER, T>(A, gi, gj, kf, part, G);
                if (tid == 0) S.sub[10] += clock64() - te;
            }
            Cx<T> s0{0, 0}, s1{0, 0}, s2{0, 0}, s3{0, 0};
            int c = part;
            // LIF loads in flight per thread (the sums wait on memory, not on arithmetic)
            for (; c + (LIF - 1) * G < nt; c += LIF * G) {
                Cx<T> x[LIF];
#pragma unroll
                for (int u = 0; u < LIF; ++u) x[u] = ldcx(A.pool + col[c + u * G] + v);
#pragma unroll
                for (int u = 0; u < LIF; ++u) {
                    Cx<T>& acc_u = (u & 3) == 0 ? s0 : (u & 3) == 1 ? s1 : (u & 3) == 2 ? s2 : s3;
                    if (ROW) cfmac(acc_u, F.coef[c + u * G], x[u]);
                    else cfma(acc_u, x[u], F.coef[c + u * G]);
                }
            }
            for (; c + 7 * G < nt; c += 8 * G) {
                Cx<T> x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = ldcx(A.pool + col[c + u * G] + v);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    Cx<T>& acc_u = (u & 3) == 0 ? s0 : (u & 3) == 1 ? s1 : (u & 3) == 2 ? s2 : s3;
                    if (ROW) cfmac(acc_u, F.coef[c + u * G], x[u]);
                    else cfma(acc_u, x[u], F.coef[c + u * G]);
                }
            }
            for (; c + 3 * G < nt; c += 4 * G) {
                const Cx<T> x0 = ldcx(A.pool + col[c] + v), x1 = ldcx(A.pool + col[c + G] + v);
                const Cx<T> x2 = ldcx(A.pool + col[c + 2 * G] + v), x3 = ldcx(A.pool + col[c + 3 * G] + v);
                if (ROW) {
                    cfmac(s0, F.coef[c], x0);
                    cfmac(s1, F.coef[c + G], x1);
                    cfmac(s2, F.coef[c + 2 * G], x2);
                    cfmac(s3, F.coef[c + 3 * G], x3);
                } else {
                    cfma(s0, x0, F.coef[c]);
                    cfma(s1, x1, F.coef[c + G]);
                    cfma(s2, x2, F.coef[c + 2 * G]);
                    cfma(s3, x3, F.coef[c + 3 * G]);
                }
            }
            for (; c < nt; c += G) {
                const Cx<T> x0 = ldcx(A.pool + col[c] + v);
                if (ROW) cfmac(s0, F.coef[c], x0);
                else cfma(s0, x0, F.coef[c]);
            }
            int t = part;
            for (; t + G < m; t += 2 * G) {
                const Cx<T> x0 = ldcx(cur + (size_t)t * ldc + v), x1 = ldcx(cur + (size_t)(t + G) * ldc + v);
                if (ROW) {
                    cfmac(s1, F.coef[nt + t], x0);
                    cfmac(s2, F.coef[nt + t + G], x1);
                } else {
                    cfma(s1, x0, F.coef[nt + t]);
                    cfma(s2, x1, F.coef[nt + t + G]);
                }
            }
            for (; t < m; t += G) {
                const Cx<T> x0 = ldcx(cur + (size_t)t * ldc + v);
                if (ROW) cfmac(s3, F.coef[nt + t], x0);
                else cfma(s3, x0, F.coef[nt + t]);
            }
            acc.x -= (s0.x + s1.x) + (s2.x + s3.x);
            acc.y -= (s0.y + s1.y) + (s2.y + s3.y);
        }
        for (int o = G >> 1; o > 0; o >>= 1) {
            Cx<T> y = shfl_xor_c(acc, o);
            acc.x += y.x;
            acc.y += y.y;
        }
        if (part == 0 && v < L) {
            out[v] = acc;
            if (ROW || !w.used[v]) am = amax_better(am, ArgMaxT<T>{cabs2(acc), v});
        }
    }
    if (tid == 0) S.entries += L;
    return block_argmax<NT>(am, S.am);
}

// ---- sampled residual of the face approximant ------------------------------------------
// R_s = ENTRY(i_s, j_s, kf) - sum_p f_p[kf] H_p[i_s, j_s] - sum_{t<m} u_t[i_s] conj(v_t[j_s])
// at the 32 sample positions; one warp per sample, lanes over the flattened
// columns of the earlier crosses.  Writes |R_s|^2 to S.samp.
template <int KER, class T, int NT>
__device__ void face_samples(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, const FaceTab<T>& F, int kf,
                             int m, const Cx<T>* D) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int M = S.M, N = S.N;
    for (int sm = wid; sm < SAMPLES; sm += NT / 32) {
        const int i = (2 * sm + 1) * M / (2 * SAMPLES), j = (2 * ((11 * sm) % SAMPLES) + 1) * N / (2 * SAMPLES);
        Cx<T> acc{0, 0};
        for (int c = lane; c < F.ncol; c += 32) {
            const Cx<T> h = cmulc(A.pool[F.colU[c] + i], A.pool[F.colV[c] + j]);
            cfma(acc, S.fk[F.colP[c]], h);
        }
        for (int t = lane; t < m; t += 32) cfmac(acc, w.uw[(size_t)t * A.Mmax + i], w.vw[(size_t)t * A.Nmax + j]);
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        if (lane == 0) {
            const Cx<T> e = D ? D[(size_t)i * N + j] : ent<KER, T>(A, S.rb + i, S.cb + j, kf);
            S.samp[sm] = cabs2d(Cx<T>{e.x - acc.x, e.y - acc.y});
        }
    }
    if (threadIdx.x == 0) S.entries += SAMPLES;
    __syncthreads();
}

// ---- dense residual working face ------------------------------------------------------
// D[i][j] = ENTRY(i, j, kf) - sum_p f_p[kf] (U_p V_p^H)[i, j]  (row-major, ld N) for all
// i < M, j < N, in one parallel pass before the face ACA: the ACA then reads its rows
// and columns from D and sums only the current face's crosses.  The partial-pivot
// ACA takes the same rows and columns as with on-demand lines; only the order of
// the float32 sums over the earlier crosses differs.  Tiles of 64 x (NT / 4)
// outputs; the earlier crosses' columns (scaled by f_p[kf]) staged DRF_KC at a
// time in shared memory.  The sum over them is a dense complex product, on the
// tensor cores at 256 threads (the TF32 three-term split, float32 accuracy),
// else on the CUDA cores (a 4 x 4 micro-tile per thread).  Float32 only.
constexpr int DRF_KC = 16;     // columns per staged chunk, CUDA-core path
constexpr int DRF_KC_TC = 16;  // columns per staged chunk, tensor-core path (256 threads, two buffers)
// shared-memory staging of the dense residual face, placed after the face's
// column tables (the coefficient and row buffers that follow them are not in
// use while the dense face is formed)
template <class T>
constexpr size_t drf_stage_offset() {
    return (2 * TABMAX * sizeof(long long) + TABMAX * sizeof(short) + 255) & ~size_t(255);
}
template <class T, int NT>
constexpr size_t drf_stage_bytes() {
    return (size_t)(NT == 256 ? 2 * DRF_KC_TC : DRF_KC) * (64 + NT / 4) * sizeof(Cx<T>);
}

template <int KER, class T, int NT>
__device__ void face_dense_residual(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, const FaceTab<T>& F,
                                    int kf, unsigned char* arena) {
    static_assert(sizeof(T) == 4, "dense residual faces are a float32 path");
    constexpr int TI = 64, TJ = NT / 4, TXN = TJ / 4;
    const int tid = threadIdx.x;
    const int M = S.M, N = S.N, nc = F.ncol;
    const int tx = tid % TXN, ty = tid / TXN;  // ty < 16
    Cx<T>* su = reinterpret_cast<Cx<T>*>(arena + drf_stage_offset<T>());  // [DRF_KC][TI]
    Cx<T>* sv = su + DRF_KC * TI;                                          // [DRF_KC][TJ]
    Cx<T>* D = w.dres;
    // the entries, one thread per entry (consecutive threads take consecutive
    // columns); linear elements: one thread per element pair, whose nine local
    // entries share the pair's quadrature points
    const int MN = M * N;
    long long te = clock64();
    if constexpr (KER == G3_GAL_P1D || KER == G3_GAL_P1KP) {
        const float2 s = A.sf[kf];
        const int Me = M / 3, Ne = N / 3;
        for (int e = tid; e < Me * Ne; e += NT) {
            const int pe = e / Ne, qe = e - pe * Ne;
            T r[16], m[16], gz[16], cab[9], nn;
            p1_pair_setup<KER>(A.gf, S.rb / 3 + pe, S.cb / 3 + qe, r, m, gz, cab, nn);
            Cx<T> v[9];
            p1_pair_eval<KER, T>(r, m, gz, cab, nn, s.x, s.y, v);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) D[(size_t)(3 * pe + a) * N + 3 * qe + b] = v[a * 3 + b];
        }
    } else {
        for (int e = tid; e < MN; e += NT) {
            const int i = e / N, j = e - i * N;
            D[e] = ent<KER, T>(A, S.rb + i, S.cb + j, kf);
        }
    }
    __syncthreads();
    sublap(S, 10, te);  // the residual lines evaluate no entries when this runs
    if constexpr (NT == 256) {
        // tensor cores: per 64 x 64 tile, warp w takes rows 16 (w % 4) and columns
        // 32 (w / 4) (four 16 x 8 output tiles); sum_c u_ic conj(v_jc) as the real
        // products Re = ur vr + ui vi, Im = ui vr - ur vi (mma_tf32x3 each)
        const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
        const int rw = (warp & 3) * 16, cw = (warp >> 2) * 32;
        constexpr int KC = DRF_KC_TC;
        // two staging buffers of KC columns each, filled by cp.async (8 bytes per
        // element, zero-filled outside the face and past the last column) while the
        // tensor cores work on the other; f_p[kf] is applied to the A fragments
        Cx<T>* bu[2] = {su, su + KC * (TI + TJ)};
        auto issue = [&](int buf, int i0, int j0, int c0) {
            Cx<T>* du = bu[buf];
            Cx<T>* dv = du + KC * TI;
            for (int e = tid; e < KC * TI; e += NT) {
                const int kk = e / TI, ii = e - kk * TI, c = c0 + kk;
                const bool in = c < nc && i0 + ii < M;
                cp_async8(du + e, in ? A.pool + F.colU[c] + i0 + ii : A.pool, in);
            }
            for (int e = tid; e < KC * TJ; e += NT) {
                const int kk = e / TJ, jj = e - kk * TJ, c = c0 + kk;
                const bool in = c < nc && j0 + jj < N;
                cp_async8(dv + e, in ? A.pool + F.colV[c] + j0 + jj : A.pool, in);
            }
            cp_async_commit();
        };
        for (int i0 = 0; i0 < M; i0 += TI) {
            for (int j0 = 0; j0 < N; j0 += TJ) {
                float are[4][4], aim[4][4];
#pragma unroll
                for (int n8 = 0; n8 < 4; ++n8)
#pragma unroll
                    for (int q = 0; q < 4; ++q) are[n8][q] = aim[n8][q] = 0.f;
                __syncthreads();  // the previous tile's buffers are consumed
                if (nc > 0) issue(0, i0, j0, 0);
                for (int c0 = 0, b = 0; c0 < nc; c0 += KC, b ^= 1) {
                    if (c0 + KC < nc) {
                        issue(b ^ 1, i0, j0, c0 + KC);
                        cp_async_wait<1>();
                    } else {
                        cp_async_wait<0>();
                    }
                    __syncthreads();  // chunk c0 is in buffer b for every thread
                    const Cx<T>* cu = bu[b];
                    const Cx<T>* cv = cu + KC * TI;
#pragma unroll
                    for (int ks = 0; ks < KC; ks += 8) {
                        // A fragment (row i, column c): (g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4)
                        unsigned urh[4], url[4], uih[4], uil[4], nrh[4], nrl[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c = c0 + ks + t + (q >> 1) * 4;
                            const Cx<T> u = c < nc ? cmul(S.fk[F.colP[c]], cu[(ks + t + (q >> 1) * 4) * TI + rw + g + (q & 1) * 8])
                                                   : Cx<T>{0, 0};
                            const Tf32Pair pr = tf32_split(u.x), pi = tf32_split(u.y);
                            urh[q] = pr.hi;
                            url[q] = pr.lo;
                            uih[q] = pi.hi;
                            uil[q] = pi.lo;
                        }
                        tf32_neg4(urh, nrh);
                        tf32_neg4(url, nrl);
#pragma unroll
                        for (int n8 = 0; n8 < 4; ++n8) {
                            // B fragment (row c, column j): (t, g), (t + 4, g)
                            unsigned vrh[2], vrl[2], vih[2], vil[2];
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                const Cx<T> v = cv[(ks + t + q * 4) * TJ + cw + n8 * 8 + g];
                                const Tf32Pair pr = tf32_split(v.x), pi = tf32_split(v.y);
                                vrh[q] = pr.hi;
                                vrl[q] = pr.lo;
                                vih[q] = pi.hi;
                                vil[q] = pi.lo;
                            }
                            mma_tf32x3(are[n8], urh, url, vrh, vrl);
                            mma_tf32x3(are[n8], uih, uil, vih, vil);
                            mma_tf32x3(aim[n8], uih, uil, vrh, vrl);
                            mma_tf32x3(aim[n8], nrh, nrl, vih, vil);
                        }
                    }
                    __syncthreads();  // buffer b is consumed before the next chunk refills it
                }
                // C fragment (row, column): (g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1)
#pragma unroll
                for (int n8 = 0; n8 < 4; ++n8)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int gi = i0 + rw + g + (q >> 1) * 8, gj = j0 + cw + n8 * 8 + 2 * t + (q & 1);
                        if (gi < M && gj < N) {
                            Cx<T>* dp = D + (size_t)gi * N + gj;
                            const Cx<T> e = *dp;
                            *dp = Cx<T>{e.x - are[n8][q], e.y - aim[n8][q]};
                        }
                    }
            }
        }
        if (tid == 0) atomicAdd(&A.counters[7], (unsigned long long)M * N);
        __syncthreads();
        return;
    }
    for (int i0 = 0; i0 < M; i0 += TI) {
        for (int j0 = 0; j0 < N; j0 += TJ) {
            Cx<T> acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int gi = i0 + ty * 4 + a, gj = j0 + tx * 4 + b;
                    acc[a][b] = (gi < M && gj < N) ? ldcx(D + (size_t)gi * N + gj) : Cx<T>{0, 0};
                }
            for (int c0 = 0; c0 < nc; c0 += DRF_KC) {
                __syncthreads();  // the previous chunk is consumed
                for (int e = tid; e < DRF_KC * TI; e += NT) {
                    const int kk = e / TI, ii = e - kk * TI, c = c0 + kk;
                    su[e] = (c < nc && i0 + ii < M) ? cmul(S.fk[F.colP[c]], ldcx(A.pool + F.colU[c] + i0 + ii))
                                                    : Cx<T>{0, 0};
                }
                for (int e = tid; e < DRF_KC * TJ; e += NT) {
                    const int kk = e / TJ, jj = e - kk * TJ, c = c0 + kk;
                    sv[e] = (c < nc && j0 + jj < N) ? ldcx(A.pool + F.colV[c] + j0 + jj) : Cx<T>{0, 0};
                }
                __syncthreads();
#pragma unroll 4
                for (int kk = 0; kk < DRF_KC; ++kk) {
                    Cx<T> u[4], v[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) u[a] = su[kk * TI + ty * 4 + a];
#pragma unroll
                    for (int b = 0; b < 4; ++b) v[b] = sv[kk * TJ + tx * 4 + b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            // acc -= u conj(v)
                            acc[a][b].x -= u[a].x * v[b].x + u[a].y * v[b].y;
                            acc[a][b].y -= u[a].y * v[b].x - u[a].x * v[b].y;
                        }
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int gi = i0 + ty * 4 + a, gj = j0 + tx * 4 + b;
                    if (gi < M && gj < N) D[(size_t)gi * N + gj] = acc[a][b];
                }
        }
    }
    if (tid == 0) atomicAdd(&A.counters[7], (unsigned long long)M * N);
    __syncthreads();
}

// ---- face ACA (partial pivoting) on the residual face at frequency kf -----------------
// Returns the rank m; columns 0..m-1 of uw / vw hold the crosses (S = U V^H).
template <int KER, class T, int NT>
__device__ int face_aca(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, int kf, unsigned char* arena) {
    const int tid = threadIdx.x;
    const int M = S.M, N = S.N, nc = S.ncross;
    const int cap = min(min(M, N), A.RF);
    if (kf < 0 || kf >= A.Ku) {  // cannot happen: every caller passes a checked index
        if (tid == 0) atomicOr(A.status, ST_BAD_INDEX);
        return 0;
    }
    // f_p[kf] of earlier crosses, the column tables, used-row flags
    for (int p = tid; p < nc; p += NT) S.fk[p] = Fp(A, S, p)[kf];
    long long tf = clock64();
    FaceTab<T> F = facetab_build<T, NT>(A, w, S, arena);
    for (int i = tid; i < M; i += NT) w.used[i] = 0;
    __syncthreads();
    // dense residual working face (float32, blocks up to drf_max entries): ENTRY
    // minus the earlier crosses evaluated for the whole face at once; the lines
    // below then subtract only the current face's crosses
    const Cx<T>* D = nullptr;
    if constexpr (sizeof(T) == 4 && KER != G3_SEPARABLE) {
        if (w.dres && (long long)M * N <= A.drf_max) {
            face_dense_residual<KER, T, NT>(A, w, S, F, kf, arena);
            D = w.dres;
            F.ncol = 0;
            sublap(S, 11, tf);
        }
    }
    if (tid == 0) S.fsn2 = 0.0;
    int m = 0;
    int irow = 0;
    bool converged = false;
    // absolute floor of the face tests (float32 entries only): a residual face
    // far below the block's typical face, face_floor ||C^(l-1)||_F / sqrt(Ku),
    // is resolved to that level rather than relative to its own norm, which
    // the entries' rounding noise would never let the test reach
    const double floor2 = A.face_floor * A.face_floor * S.norm2 / (double)A.Ku;
    while (m < cap) {
        int jp = -1;
        for (;;) {
            sublap(S, 5, tf);
            line_coeffs<T, NT, true>(A, w, S, F, irow, m);
            __syncthreads();
            ArgMaxT<T> am = residual_line<KER, T, NT, true>(A, w, S, F, irow, kf, m, F.row, D);
            if (tid == 0) w.used[irow] = 1;
            // a row counts as nonzero when |delta|^2 is a normal number of the
            // working precision (below that the entries are far under any tolerance)
            if (am.v > tiny_norm2<T>()) {
                jp = am.i;
                break;
            }
            // zero residual row: next unused row in index order
            ArgMaxT<T> un = amax_none<T>();
            for (int i = tid; i < M; i += NT)
                if (i != irow && !w.used[i]) un = amax_better(un, ArgMaxT<T>{(T)0, i});
            un = block_argmax<NT>(un, S.am);
            if (un.v < 0.0) {
                irow = -1;
                break;
            }
            irow = un.i;
        }
        if (jp < 0) break;  // no row with a nonzero residual left
        // v = conj(row / delta) with delta scaled to magnitude ~1 first, so that a
        // tiny pivot of a strongly damped face cannot overflow 1 / |delta|^2
        // (|row[j]| <= |delta| since delta is the row's largest entry)
        const Cx<T> delta = F.row[jp];
        const T sc = (T)1 / fmax(fabs(delta.x), fabs(delta.y));
        const Cx<T> ds{delta.x * sc, delta.y * sc};
        const T dn = (T)1 / cabs2(ds);
        Cx<T>* vm = w.vw + (size_t)m * A.Nmax;
        for (int j = tid; j < N; j += NT) {
            const Cx<T> rj = F.row[j];
            const Cx<T> q = cmulc(Cx<T>{rj.x * sc, rj.y * sc}, ds);  // (row / s) conj(delta / s)
            vm[j] = Cx<T>{q.x * dn, -q.y * dn};                      // conj(row / delta)
        }
        line_coeffs<T, NT, false>(A, w, S, F, jp, m);
        __syncthreads();
        // residual column jp = u_m; the argmax over unused rows of |u_m| is the next row
        Cx<T>* um = w.uw + (size_t)m * A.Mmax;
        sublap(S, 6, tf);
        ArgMaxT<T> nx = residual_line<KER, T, NT, false>(A, w, S, F, jp, kf, m, um, D);
        sublap(S, 7, tf);
        // recursive Frobenius norm of the face approximant:
        // ||S_m||^2 = ||S_{m-1}||^2 + 2 Re sum_t (u_t^H u_m)(v_m^H v_t) + ||u_m||^2 ||v_m||^2
        const int wid = tid >> 5, lane = tid & 31;
        for (int t = wid; t <= m; t += NT / 32) {
            const Cx<T>* ut = w.uw + (size_t)t * A.Mmax;
            const Cx<T>* vt = w.vw + (size_t)t * A.Nmax;
            Cx<T> gu{0, 0}, gv{0, 0};
            // both sums in one loop, unrolled: their loads are in flight together
            const int L = max(M, N);
#pragma unroll 4
            for (int i = lane; i < L; i += 32) {
                if (i < M) cfmac(gu, ldcx(um + i), ldcx(ut + i));  // conj(u_t) u_m
                if (i < N) cfmac(gv, ldcx(vt + i), ldcx(vm + i));  // conj(v_m) v_t
            }
            const T gux = warp_sum(gu.x), guy = warp_sum(gu.y);
            const T gvx = warp_sum(gv.x), gvy = warp_sum(gv.y);
            if (lane == 0) {
                S.gu[t] = Cx<double>{(double)gux, (double)guy};
                S.gv[t] = Cx<double>{(double)gvx, (double)gvy};
            }
        }
        __syncthreads();
        // the float64 scalars of the test on warp 0 only (float64 runs at a
        // small fraction of the float32 rate on this part)
        if (wid == 0) {
            double cross = 0.0;
            for (int t = lane; t < m; t += 32) cross += 2.0 * (S.gu[t].x * S.gv[t].x - S.gu[t].y * S.gv[t].y);
            cross = warp_sum(cross);
            if (lane == 0) {
                const double nu2 = S.gu[m].x, nv2 = S.gv[m].x;
                const double sn2 = S.fsn2 + cross + nu2 * nv2;
                S.fsn2 = sn2;
                S.fconv = nu2 * nv2 <= fmax(A.eps_face * A.eps_face * fmax(sn2, 0.0), floor2);
            }
        }
        ++m;
        __syncthreads();
        sublap(S, 8, tf);
        if (S.fconv) {
            if (!A.sample_check) {
                converged = true;
                break;
            }
            // confirm on the sample entries: partial pivoting can miss a block
            // of the face that no visited row or column reaches
            face_samples<KER, T, NT>(A, w, S, F, kf, m, D);
            sublap(S, 9, tf);
            static_assert(SAMPLES == 32, "one sample per lane");
            if (wid == 0) {
                const double sv = S.samp[lane];
                const double tot = warp_sum(sv);
                ArgMaxT<T> b{(T)sv, lane};
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ArgMaxT<T> y{__shfl_xor_sync(0xffffffffu, b.v, o), __shfl_xor_sync(0xffffffffu, b.i, o)};
                    b = amax_better(b, y);
                }
                if (lane == 0) {
                    S.fconv = (double)M * (double)N / SAMPLES * tot <=
                              fmax(A.eps_face * A.eps_face * fmax(S.fsn2, 0.0), floor2);
                    S.fbs = b.i;
                }
            }
            __syncthreads();
            if (S.fconv) {
                converged = true;
                break;
            }
            if (tid == 0) atomicAdd(&A.counters[5], 1ull);
            irow = (2 * S.fbs + 1) * M / (2 * SAMPLES);
            __syncthreads();  // S.fbs is rewritten by the next test
            continue;
        }
        if (nx.v < 0) break;  // every row used
        irow = nx.i;
    }
    if (tid == 0) S.raw += m;
    if (!converged && m == A.RF && m < min(M, N)) {
        if (tid == 0) {
            atomicOr(A.status, ST_FACE_CAPPED);
            atomicAdd(&A.counters[3], 1ull);
        }
    }
    __syncthreads();
    return m;
}

// ---- tiled Gram of the face factors: G[a][b] = sum_i conj(X_a[i]) X_b[i], a <= b < r ----
// Products and the sum over a 32-row chunk in the working precision T, the sum
// over chunks in float64.  sh: >= 33 * r complex T.
template <class T, int NT>
__device__ void gram_upper(const Cx<T>* X, size_t ld, int L, int r, Cx<double>* G, int RF, Cx<T>* sh) {
    constexpr int QMAX = (RF_MAX * (RF_MAX + 1) / 2 + NT - 1) / NT;
    const int tid = threadIdx.x;
    const int npair = r * (r + 1) / 2;
    int pa[QMAX], pb[QMAX];
    Cx<double> acc[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
        int p = tid + q * NT;
        acc[q] = Cx<double>{0, 0};
        pa[q] = -1;
        pb[q] = 0;
        if (p < npair) {
            int a = 0;
            while (p >= r - a) {
                p -= r - a;
                ++a;
            }
            pa[q] = a;
            pb[q] = a + p;
        }
    }
    for (int i0 = 0; i0 < L; i0 += 32) {
        for (int e = tid; e < r * 32; e += NT) {
            const int c = e >> 5, ii = e & 31;
            sh[c * 33 + ii] = (i0 + ii < L) ? ldcx(X + (size_t)c * ld + i0 + ii) : Cx<T>{0, 0};
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
            if (pa[q] < 0) continue;
            const Cx<T>* xa = sh + pa[q] * 33;
            const Cx<T>* xb = sh + pb[q] * 33;
            Cx<T> s{0, 0};
#pragma unroll 8
            for (int ii = 0; ii < 32; ++ii) cfmac(s, xb[ii], xa[ii]);  // conj(x_a) x_b
            acc[q].x += (double)s.x;
            acc[q].y += (double)s.y;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < QMAX; ++q)
        if (pa[q] >= 0) G[pa[q] * RF + pb[q]] = acc[q];
}

// 1 / sqrt(x) in float64 for the Cholesky pivots of the column-scaled Gram
// matrices (x in (1e-24, 1], inside the float32 range): a float32 estimate
// refined by one Newton-Raphson step for the inverse square root,
// y <- y (3 - x y^2) / 2, which squares its relative error (~1e-7 -> ~1e-14)
// at the cost of a few float64 operations.
__device__ __forceinline__ double rsqrt_pivot(double x) {
    const double y = (double)rsqrtf((float)x);
    return y * (1.5 - 0.5 * x * y * y);
}

// ---- recompression: Cholesky-QR + one-sided Jacobi SVD ---------------------------------
// Input uw, vw (r columns).  Output: the rank r' and the transforms T_U, T_V
// (r x r', complex T, row-major with stride *ldT) such that U' = uw T_U,
// V' = vw T_V.  For any invertible triangular R used consistently,
// uw T_U T_V^H vw^H = uw vw^H before truncation, so the Gram matrices may be
// formed in the working precision; the r x r algebra is float64.
//
// The four r x r float64 matrices (R_U, R_V, B = C J, J) live in shared memory
// (stride RS) when r <= RS, else in the global workspace (stride RF).  The
// back substitution runs in place on the selected columns of B and J.
// Returns r' or -1 (Cholesky breakdown or a non-finite SVD: the caller keeps
// the raw factors).
constexpr int RS = 32;

template <class T>
__device__ __forceinline__ T jacobi_tol();
template <>
__device__ __forceinline__ float jacobi_tol<float>() { return 1e-3f; }
template <>
__device__ __forceinline__ double jacobi_tol<double>() { return 1e-12; }

// One-sided Jacobi SVD (Hestenes) of the r x r core C (columns of B, J = I on
// entry): B <- C J with orthogonal columns, J unitary; singular values = column
// norms of B; sel[] lists the kept columns in descending order.  Returns the
// kept rank or -1 (non-finite).
template <class T, int NT>
__device__ int jacobi_core(const AcaArgs<T>& A, BlockSh<T>& S, Cx<T>* shB, Cx<T>* shJ, int ld, int r) {
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    // one-sided Jacobi (Hestenes) on the columns of C, round-robin pair schedule;
    // a pair is rotated while |<c_p, c_q>| > tol ||c_p|| ||c_q||.  Column norms
    // are recomputed at each sweep start and updated after every rotation
    // (||c_p'||^2 = ||c_p||^2 - t |g|, ||c_q'||^2 = ||c_q||^2 + t |g|).
    const int n = (r + 1) & ~1;
    const T tol = jacobi_tol<T>();
    T* cn = reinterpret_cast<T*>(S.sig);  // column norms (S.sig is free until the SVD finishes)
    for (int sweep = 0; sweep < 16; ++sweep) {
        if (tid == 0) S.rot = 0;
        for (int a = wid; a < r; a += NT / 32) {
            T s2 = 0;
            for (int i = lane; i < r; i += 32) s2 += cabs2(shB[a * ld + i]);
            s2 = warp_sum(s2);
            if (lane == 0) cn[a] = s2;
        }
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
                Cx<T>* bp = shB + p * ld;
                Cx<T>* bq = shB + q * ld;
                const T al = cn[p], be = cn[q];
                Cx<T> ga{0, 0};
                for (int i = lane; i < r; i += 32) {
                    Cx<T> x = bp[i], y = bq[i];
                    ga.x += x.x * y.x + x.y * y.y;
                    ga.y += x.x * y.y - x.y * y.x;
                }
                ga.x = warp_sum(ga.x);
                ga.y = warp_sum(ga.y);
                T ag = sqrt(ga.x * ga.x + ga.y * ga.y);
                if (ag > tol * sqrt(al * be) && ag > (T)1e-30) {
                    T zeta = (be - al) / ((T)2 * ag);
                    T t = (zeta >= 0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
                    T c = (T)1 / sqrt((T)1 + t * t), s = c * t;
                    Cx<T> ph{ga.x / ag, ga.y / ag};  // e^{i phi}
                    Cx<T>* jp_ = shJ + p * ld;
                    Cx<T>* jq_ = shJ + q * ld;
                    for (int i = lane; i < r; i += 32) {
                        Cx<T> x = bp[i], y = bq[i];
                        // x' = c x - s e^{-i phi} y ; y' = s e^{i phi} x + c y
                        Cx<T> ey = cmulc(y, ph), ex = cmul(x, ph);
                        bp[i] = Cx<T>{c * x.x - s * ey.x, c * x.y - s * ey.y};
                        bq[i] = Cx<T>{s * ex.x + c * y.x, s * ex.y + c * y.y};
                        x = jp_[i];
                        y = jq_[i];
                        ey = cmulc(y, ph);
                        ex = cmul(x, ph);
                        jp_[i] = Cx<T>{c * x.x - s * ey.x, c * x.y - s * ey.y};
                        jq_[i] = Cx<T>{s * ex.x + c * y.x, s * ex.y + c * y.y};
                    }
                    if (lane == 0) {
                        atomicAdd(&S.rot, 1);
                        cn[p] = al - t * ag;
                        cn[q] = be + t * ag;
                    }
                }
            }
            __syncthreads();
        }
        const int rot = S.rot;
        __syncthreads();
        if (rot == 0) break;
        if (sweep == 15 && tid == 0) atomicOr(A.status, ST_JACOBI_NOCONV);
    }

    // singular values, sort descending, truncation sigma < eps_face * sigma_max
    for (int a = tid; a < r; a += NT) {
        double s2 = 0;
        for (int i = 0; i < r; ++i) s2 += cabs2d(shB[a * ld + i]);
        S.sig[a] = sqrt(s2);
    }
    __syncthreads();
    double smax = 0;
    bool finite = true;
    for (int a = 0; a < r; ++a) {
        smax = fmax(smax, S.sig[a]);
        finite &= (bool)isfinite(S.sig[a]);
    }
    if (!finite || !(smax > 0.0)) return -1;
    // (float32 entries: also below the face tests' absolute floor, keeping sigma_1)
    const double sfloor = A.trunc_floor * sqrt(S.norm2 / (double)A.Ku);
    for (int a = tid; a < r; a += NT) {
        int rank = 0;
        for (int b = 0; b < r; ++b)
            if (S.sig[b] > S.sig[a] || (S.sig[b] == S.sig[a] && b < a)) ++rank;
        bool keep = S.sig[a] > 0.0 && S.sig[a] >= A.eps_face * smax && (rank == 0 || S.sig[a] >= sfloor);
        S.sel[rank] = keep ? a : -1;
    }
    __syncthreads();
    int rn = 0;
    while (rn < r && S.sel[rn] >= 0) ++rn;
    return rn;
}

// Column-pivoted QR of the r x r core C (columns of B) by modified
// Gram-Schmidt (see the caller).  On return B[:, sel[k]] = q_k and
// J[:, sel[k]] = (Pi R^H)[:, k] in the original column order, k < rank.
template <class T, int NT>
__device__ int cpqr_core(const AcaArgs<T>& A, BlockSh<T>& S, Cx<T>* shB, Cx<T>* shJ, int ld, int r) {
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    constexpr int NW = NT / 32;
    T* cn = reinterpret_cast<T*>(S.sig);     // squared column norms, -1 once used
    for (int c = wid; c < r; c += NW) {
        T s2 = 0;
        for (int i = lane; i < r; i += 32) s2 += cabs2(shB[c * ld + i]);
        s2 = warp_sum(s2);
        if (lane == 0) cn[c] = s2;
    }
    for (int e = tid; e < r * r; e += NT) shJ[(e / r) * ld + (e % r)] = Cx<T>{0, 0};
    __syncthreads();
    const double sfloor = A.trunc_floor * sqrt(S.norm2 / (double)A.Ku);
    float r00 = 0.f;
    int k = 0;
    for (; k < r; ++k) {
        if (wid == 0) {
            ArgMaxT<T> best = amax_none<T>();
            for (int c = lane; c < r; c += 32)
                if (cn[c] >= (T)0) best = amax_better(best, ArgMaxT<T>{cn[c], c});
            best = warp_argmax(best);
            const int pv = best.i;
            T s2 = 0;
            if (best.v >= (T)0 && pv >= 0 && pv < r)
                for (int i = lane; i < r; i += 32) s2 += cabs2(shB[pv * ld + i]);
            s2 = warp_sum(s2);
            if (lane == 0) {
                S.piv = (best.v >= (T)0 && pv >= 0 && pv < r) ? pv : -1;
                S.rkk = sqrt(s2);
                if (S.piv >= 0) cn[pv] = (T)-1;
            }
        }
        __syncthreads();
        const int pv = S.piv;
        const float rkk = S.rkk;
        if (k == 0) r00 = rkk;
        if (pv < 0 || !(rkk > 0.f) || !isfinite(rkk) || rkk < (float)A.eps_face * r00 ||
            (k > 0 && (double)rkk < sfloor))
            break;
        const T inv = (T)1 / (T)rkk;
        const Cx<T>* q = shB + pv * ld;
        if (tid == 0) {
            S.sel[k] = pv;
            shJ[pv * ld + pv] = Cx<T>{(T)rkk, (T)0};
        }
        for (int j = wid; j < r; j += NW) {
            if (!(cn[j] >= (T)0)) continue;  // used (or the pivot)
            Cx<T>* cj = shB + j * ld;
            Cx<T> g{0, 0};
            for (int i = lane; i < r; i += 32) cfmac(g, cj[i], q[i]);  // conj(q) c_j, q unscaled
            g.x = warp_sum(g.x) * inv;
            g.y = warp_sum(g.y) * inv;
            for (int i = lane; i < r; i += 32) {
                const Cx<T> qi{q[i].x * inv, q[i].y * inv};
                cj[i].x -= qi.x * g.x - qi.y * g.y;
                cj[i].y -= qi.x * g.y + qi.y * g.x;
            }
            if (lane == 0) {
                shJ[pv * ld + j] = Cx<T>{g.x, -g.y};  // conj(R[k][j])
                cn[j] = fmax(cn[j] - cabs2(g), (T)0);
            }
        }
        __syncthreads();
    }
    // scale the pivot columns to q (their norms rkk sit on J's diagonal)
    for (int e = tid; e < k * r; e += NT) {
        const int b = e / r, i = e - b * r;
        const int pv = S.sel[b];
        const T inv = (T)1 / shJ[pv * ld + pv].x;
        shB[pv * ld + i].x *= inv;
        shB[pv * ld + i].y *= inv;
    }
    __syncthreads();
    return k;
}

template <class T, int NT>
__device__ int recompress(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, int r, Cx<double>* smem,
                          const Cx<T>** tUo, const Cx<T>** tVo, int* ldTo) {
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int M = S.M, N = S.N;
    const bool small = r <= RS;
    const int ld = small ? RS : A.RF;
    Cx<double>* RU = small ? smem : w.RU;
    Cx<double>* RV = small ? smem + RS * RS : w.RV;
    // B = C J and J in the working precision T (the Jacobi sweeps dominate the
    // r x r work; float64 is rate-limited on this part)
    Cx<T>* shB = small ? reinterpret_cast<Cx<T>*>(smem + 2 * RS * RS) : reinterpret_cast<Cx<T>*>(w.TU);
    Cx<T>* shJ = shB + (small ? RS * RS : A.RF * A.RF);
    // Gram staging after R_U, R_V
    Cx<T>* stage = reinterpret_cast<Cx<T>*>(smem + 2 * RS * RS);
    long long tc = clock64();
    gram_upper<T, NT>(w.uw, A.Mmax, M, r, RU, ld, stage);
    gram_upper<T, NT>(w.vw, A.Nmax, N, r, RV, ld, stage);
    if (tid == 0) S.flag = 0;
    __syncthreads();
    sublap(S, 0, tc);
    // column scaling and upper Cholesky of the scaled Gram matrices (float64),
    // both matrices at once by all threads, right-looking: step k scales row k
    // by 1 / sqrt(R[k][k]) and then updates the trailing block
    // R[i][j] -= conj(R[k][i]) R[k][j] (k < i <= j)
    for (int e = tid; e < 2 * r; e += NT) {
        const int mtx = e / r, a = e - mtx * r;
        const Cx<double>* R = mtx == 0 ? RU : RV;
        (mtx == 0 ? S.dU : S.dV)[a] = rsqrt(fmax(R[a * ld + a].x, 1e-300));
    }
    __syncthreads();
    for (int e = tid; e < 2 * r * r; e += NT) {
        const int mtx = e / (r * r), q = e - mtx * r * r, a = q / r, b = q - a * r;
        if (b < a) continue;
        Cx<double>* R = mtx == 0 ? RU : RV;
        const double* dsc = mtx == 0 ? S.dU : S.dV;
        const double sc = dsc[a] * dsc[b];
        R[a * ld + b].x *= sc;
        R[a * ld + b].y *= sc;
    }
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        const int tail = r - k - 1;
        // row k of both matrices (the diagonal itself is written after the sync)
        for (int e = tid; e < 2 * tail; e += NT) {
            const int mtx = e / tail, j = k + 1 + (e - mtx * tail);
            Cx<double>* R = mtx == 0 ? RU : RV;
            const double dkk = R[k * ld + k].x;
            if (!(dkk > 1e-24)) {
                S.flag = 1;
                continue;
            }
            const double irkk = rsqrt_pivot(dkk);
            R[k * ld + j].x *= irkk;
            R[k * ld + j].y *= irkk;
        }
        if (tid < 2 && !(((tid == 0 ? RU : RV)[k * ld + k].x) > 1e-24)) S.flag = 1;
        __syncthreads();
        // trailing update and the diagonal entry of step k
        for (int e = tid; e < 2 * tail * tail; e += NT) {
            const int mtx = e / (tail * tail), q = e - mtx * tail * tail;
            const int i = k + 1 + q / tail, j = k + 1 + (q - (q / tail) * tail);
            if (j < i) continue;
            Cx<double>* R = mtx == 0 ? RU : RV;
            const Cx<double> rki = R[k * ld + i], rkj = R[k * ld + j];
            R[i * ld + j].x -= rki.x * rkj.x + rki.y * rkj.y;  // conj(R[k][i]) R[k][j]
            R[i * ld + j].y -= rki.x * rkj.y - rki.y * rkj.x;
        }
        if (tid < 2) {
            Cx<double>* R = tid == 0 ? RU : RV;
            const double dkk = R[k * ld + k].x;
            const double irkk = dkk > 1e-24 ? rsqrt_pivot(dkk) : 0.0;
            R[k * ld + k] = Cx<double>{dkk * irkk, 0.0};  // sqrt(dkk)
            (tid == 0 ? S.rdU : S.rdV)[k] = irkk;          // its reciprocal
        }
        __syncthreads();
    }
    sublap(S, 1, tc);
    if (S.flag) return -1;
    // working-precision copies of Rhat_U, Rhat_V (upper triangles) and of the
    // scalings for the back substitution (float32: after the two r x r float64
    // matrices and B, J in shared memory, or in the workspace's T_V block)
    Cx<T>* RUf = small ? reinterpret_cast<Cx<T>*>(smem + 2 * RS * RS) + 2 * RS * RS : reinterpret_cast<Cx<T>*>(w.TV);
    Cx<T>* RVf = RUf + (small ? RS * RS : A.RF * A.RF);
    if constexpr (sizeof(T) == 4) {
        for (int e = tid; e < 2 * r * r; e += NT) {
            const int mtx = e / (r * r), q = e - mtx * r * r, a = q / r, c = q - a * r;
            if (c < a) continue;
            (mtx == 0 ? RUf : RVf)[a * ld + c] = ccast<T>((mtx == 0 ? RU : RV)[a * ld + c]);
        }
        for (int e = tid; e < 2 * r; e += NT) {
            const int a = e < r ? e : e - r;
            if (e < r) {
                S.tdU[a] = (T)S.dU[a];
                S.trdU[a] = (T)S.rdU[a];
            } else {
                S.tdV[a] = (T)S.dV[a];
                S.trdV[a] = (T)S.rdV[a];
            }
        }
    }
    // core C = R_U R_V^H with R_U = Rhat_U diag(1/dU): C[a][b] = sum_{c >= max(a,b)}
    //   RhatU[a][c] conj(RhatV[b][c]) / (dU[c] dV[c]); stored column-major in B, J = I
    double* isc = S.sig;  // 1 / (dU[c] dV[c]); S.sig is free until the core is factored
    for (int c = tid; c < r; c += NT) isc[c] = 1.0 / (S.dU[c] * S.dV[c]);
    __syncthreads();
    for (int e = tid; e < r * r; e += NT) {
        const int a = e % r, b = e / r;
        Cx<double> acc{0, 0};
        for (int c = max(a, b); c < r; ++c) {
            Cx<double> x = RU[a * ld + c], y = RV[b * ld + c];
            const double s = isc[c];
            acc.x += (x.x * y.x + x.y * y.y) * s;
            acc.y += (x.y * y.x - x.x * y.y) * s;
        }
        shB[b * ld + a] = ccast<T>(acc);
        shJ[b * ld + a] = Cx<T>{(T)(a == b ? 1 : 0), (T)0};
    }
    __syncthreads();
    sublap(S, 2, tc);
    int rn = 0;
    if constexpr (sizeof(T) == 4) {
        // float32: column-pivoted QR of C by modified Gram-Schmidt, C Pi = Q R,
        // stopped when the largest remaining column norm falls below the
        // truncation threshold; dropping the remaining columns removes exactly
        // their norms (||R_22||_F), as truncating the SVD removes its dropped
        // singular values.  Step k (two barriers): warp 0 picks the unused
        // column of largest (downdated) norm and recomputes its norm exactly;
        // then every other unused column j is orthogonalised against it by a
        // warp (g = q^H c_j, c_j -= q g) and J[:, pivot][j] = conj(g), which
        // builds Pi R^H column by column.  The pivot columns are scaled to q
        // at the end; sel[k] = pivot of step k.
        rn = cpqr_core<T, NT>(A, S, shB, shJ, ld, r);
        if (rn < 0) return -1;
    } else {
        rn = jacobi_core<T, NT>(A, S, shB, shJ, ld, r);
        if (rn < 0) return -1;
    }
    sublap(S, 3, tc);
    // T_U[:, b] = diag(dU) RhatU^{-1} B[:, sel[b]],  T_V[:, b] = diag(dV) RhatV^{-1} J[:, sel[b]]
    // in place on the selected columns.  float32: in the working precision (the
    // columns of B and J are held in it already, so the solve's forward error
    // is of the order cond(Rhat) u either way); float64: in float64.
    if constexpr (sizeof(T) == 4) {
        for (int item = tid; item < 2 * rn; item += NT) {
            const bool isU = item < rn;
            const int b = isU ? item : item - rn;
            const Cx<T>* R = isU ? RUf : RVf;
            Cx<T>* z = (isU ? shB : shJ) + S.sel[b] * ld;
            const T* dsc = isU ? S.tdU : S.tdV;
            const T* rdg = isU ? S.trdU : S.trdV;
            for (int a = r - 1; a >= 0; --a) {
                Cx<T> acc = z[a];
                for (int c = a + 1; c < r; ++c) {
                    const Cx<T> rr = R[a * ld + c], zc = z[c];
                    acc.x -= rr.x * zc.x - rr.y * zc.y;
                    acc.y -= rr.x * zc.y + rr.y * zc.x;
                }
                const T rd = rdg[a];
                z[a] = Cx<T>{acc.x * rd, acc.y * rd};
            }
            for (int a = 0; a < r; ++a) {
                z[a].x *= dsc[a];
                z[a].y *= dsc[a];
            }
        }
    } else
    for (int item = tid; item < 2 * rn; item += NT) {
        const bool isU = item < rn;
        const int b = isU ? item : item - rn;
        const Cx<double>* R = isU ? RU : RV;
        Cx<T>* z = (isU ? shB : shJ) + S.sel[b] * ld;
        const double* dsc = isU ? S.dU : S.dV;
        const double* rdg = isU ? S.rdU : S.rdV;
        for (int a = r - 1; a >= 0; --a) {
            Cx<double> acc = ccast<double>(z[a]);
            for (int c = a + 1; c < r; ++c) {
                Cx<double> rr = R[a * ld + c];
                Cx<double> zc = ccast<double>(z[c]);
                acc.x -= rr.x * zc.x - rr.y * zc.y;
                acc.y -= rr.x * zc.y + rr.y * zc.x;
            }
            const double rd = rdg[a];
            z[a] = Cx<T>{(T)(acc.x * rd), (T)(acc.y * rd)};
        }
        for (int a = 0; a < r; ++a) {
            z[a].x *= (T)dsc[a];
            z[a].y *= (T)dsc[a];
        }
    }
    __syncthreads();
    // compact T_U, T_V (row-major r x r', complex T) into the R_U / R_V storage (dead now)
    Cx<T>* tU = reinterpret_cast<Cx<T>*>(RU);
    Cx<T>* tV = reinterpret_cast<Cx<T>*>(RV);
    for (int e = tid; e < r * rn; e += NT) {
        const int a = e / rn, b = e % rn;
        tU[a * ld + b] = shB[S.sel[b] * ld + a];
        tV[a * ld + b] = shJ[S.sel[b] * ld + a];
    }
    __syncthreads();
    sublap(S, 4, tc);
    *tUo = tU;
    *tVo = tV;
    *ldTo = ld;
    return rn;
}

// ---- eq. (norm) inner products ------------------------------------------------------------
// hh[d] = <H_l, H_d>_F = sum_{a in cross d, b} (U_d^H U_l)[a][b] conj((V_d^H V_l)[a][b]) for the
// earlier crosses d < nc, and hself = ||H_l||_F^2 (a over the columns of cross l).
// Tiled: 32 columns of [U_1 .. U_nc U_l] at a time against all rn columns of U_l,
// over NORM_RC-row chunks staged in shared memory; the products per (column,
// b) go to a shared buffer and one warp per cross sums its own (sh: >=
// (NORM_RC + 1) (32 + RF) + 32 RF complex T).  With recompressed factors one of
// U, V has orthonormal columns, so the products have the scale of the face
// values and are formed in the working precision; the sums over crosses are
// float64.
template <class T, int NT>
__device__ void norm_grams(const AcaArgs<T>& A, BlockSh<T>& S, const Cx<T>* Un, const Cx<T>* Vn, int rn,
                           Cx<T>* sh) {
    constexpr int QMAX = (32 * RF_MAX + NT - 1) / NT;
    constexpr int RC = NORM_RC<T>;  // rows staged per pass (fewer barriers per column chunk)
    const int tid = threadIdx.x;
    const int M = S.M, N = S.N, nc = S.ncross;
    const int na = S.pre[nc] + rn;
    Cx<T>* sa = sh;                  // [32][RC + 1]
    Cx<T>* sb = sh + 32 * (RC + 1);  // [rn][RC + 1]
    // column starts of the chunk's 32 columns, U then V (after sb and the
    // combine buffer pr)
    const Cx<T>** cbase = reinterpret_cast<const Cx<T>**>(sb + rn * (RC + 1) + 32 * rn);
    for (int a0 = 0; a0 < na; a0 += 32) {
        const int acnt = min(32, na - a0);
        Cx<T> zu[QMAX], zv[QMAX];
#pragma unroll
        for (int q = 0; q < QMAX; ++q) zu[q] = zv[q] = Cx<T>{0, 0};
        if (tid < acnt) {
            const int col = a0 + tid;
            if (col < S.pre[nc]) {
                int d = 0;
                while (S.pre[d + 1] <= col) ++d;
                const int t = col - S.pre[d];
                cbase[tid] = A.pool + S.off[d] + (long long)t * M;
                cbase[32 + tid] = A.pool + S.off[d] + (long long)S.r[d] * M + (long long)t * N;
            } else {
                const int t = col - S.pre[nc];
                cbase[tid] = Un + (long long)t * M;
                cbase[32 + tid] = Vn + (long long)t * N;
            }
        }
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {  // 0: U (rows M), 1: V (rows N)
            const int L = pass == 0 ? M : N;
            const Cx<T>* const* cb = cbase + 32 * pass;
            for (int i0 = 0; i0 < L; i0 += RC) {
                // staging: eight independent loads in flight per thread
                const int na_e = acnt * RC, nb_e = rn * RC;
                for (int e0 = 0; e0 < na_e + nb_e; e0 += 8 * NT) {
                    Cx<T> x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int e = e0 + tid + u * NT;
                        x[u] = Cx<T>{0, 0};
                        if (e < na_e) {
                            const int c = e / RC, ii = e - c * RC;
                            if (i0 + ii < L) x[u] = ldcx(cb[c] + i0 + ii);
                        } else if (e < na_e + nb_e) {
                            const int b = (e - na_e) / RC, ii = (e - na_e) - b * RC;
                            const Cx<T>* base = pass == 0 ? Un + (long long)b * M : Vn + (long long)b * N;
                            if (i0 + ii < L) x[u] = ldcx(base + i0 + ii);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int e = e0 + tid + u * NT;
                        if (e < na_e) {
                            const int c = e / RC, ii = e - c * RC;
                            sa[c * (RC + 1) + ii] = x[u];
                        } else if (e < na_e + nb_e) {
                            const int b = (e - na_e) / RC, ii = (e - na_e) - b * RC;
                            sb[b * (RC + 1) + ii] = x[u];
                        }
                    }
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < QMAX; ++q) {
                    const int o = tid + q * NT;
                    if (o >= acnt * rn) break;
                    const int al = o / rn, b = o % rn;
                    const Cx<T>* xa = sa + al * (RC + 1);
                    const Cx<T>* xb = sb + b * (RC + 1);
                    Cx<T> s{0, 0};
#pragma unroll 8
                    for (int ii = 0; ii < RC; ++ii) cfmac(s, xb[ii], xa[ii]);
                    if (pass == 0) {
                        zu[q].x += s.x;
                        zu[q].y += s.y;
                    } else {
                        zv[q].x += s.x;
                        zv[q].y += s.y;
                    }
                }
                __syncthreads();
            }
        }
        // combine: contribution zu conj(zv) to the cross that owns column a
        Cx<T>* pr = sb + rn * (RC + 1);  // [acnt][rn]
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
            const int o = tid + q * NT;
            if (o >= acnt * rn) break;
            pr[o] = Cx<T>{zu[q].x * zv[q].x + zu[q].y * zv[q].y, zu[q].y * zv[q].x - zu[q].x * zv[q].y};
        }
        __syncthreads();
        // owners of the chunk's columns: crosses d_lo.. (d = nc: the new cross)
        int d_lo = 0;
        while (d_lo < nc && S.pre[d_lo + 1] <= a0) ++d_lo;
        for (int d = d_lo + (tid >> 5); d <= nc; d += NT / 32) {
            const int lane = tid & 31;
            const int c_lo = max(a0, S.pre[d]);
            const int c_hi = min(a0 + acnt, d < nc ? S.pre[d + 1] : na);
            if (c_lo >= c_hi) continue;
            T sx = 0, sy = 0;
            for (int e = lane; e < (c_hi - c_lo) * rn; e += 32) {
                const Cx<T> v = pr[(c_lo - a0) * rn + e];
                sx += v.x;
                sy += v.y;
            }
            sx = warp_sum(sx);
            sy = warp_sum(sy);
            if (lane == 0) {
                if (d < nc) {
                    S.hh[d].x += (double)sx;
                    S.hh[d].y += (double)sy;
                } else {
                    S.hself += (double)sx;
                }
            }
        }
        __syncthreads();
    }
}

// ---- confirmed stop --------------------------------------------------------------------
// Algorithm 1's test measures only the newest cross.  When it passes, the
// residual of the approximant with crosses 0..ncl-1 (the newest one included,
// staged in S.off / S.r) is evaluated at 32 fixed sample entries over all
// frequencies: rows (2s+1) M / 64, columns (2 (11 s mod 32) + 1) N / 64.
// Returns true when ||R_samples||_F <= eps3 ||A_samples||_F; otherwise w.rk[k]
// holds the sampled residual energy per frequency.

template <class T>
__device__ __forceinline__ const Cx<T>* f_of(const AcaArgs<T>& A, const BlockSh<T>& S, int p) {
    const long long span = S.r[p] < 0 ? (long long)S.M * S.N : (long long)S.r[p] * (S.M + S.N);
    return A.pool + S.off[p] + span;
}

template <int KER, class T, int NT>
__device__ __noinline__ bool confirm_stop(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, int ncl) {
    const int tid = threadIdx.x, Ku = A.Ku;
    const int M = S.M, N = S.N;
    // H_p at the samples and the residuals in the working precision (values
    // of the face's scale); the squared norms summed in float64
    Cx<T>* hs = reinterpret_cast<Cx<T>*>(w.hs);
    for (int e = tid; e < SAMPLES * ncl; e += NT) {
        const int sm = e / ncl, p = e % ncl;
        const int i = (2 * sm + 1) * M / (2 * SAMPLES), j = (2 * ((11 * sm) % SAMPLES) + 1) * N / (2 * SAMPLES);
        Cx<T> h{0, 0};
        if (S.r[p] < 0) {
            h = A.pool[S.off[p] + i + (long long)j * M];
        } else {
            const Cx<T>* U = A.pool + S.off[p];
            const Cx<T>* V = U + (long long)S.r[p] * M;
            for (int t = 0; t < S.r[p]; ++t) cfmac(h, U[(long long)t * M + i], V[(long long)t * N + j]);
        }
        hs[sm * A.Cmax + p] = h;
    }
    if (tid == 0) {
        S.red2[0] = 0.0;
        S.red2[1] = 0.0;
        S.entries += (long long)SAMPLES * Ku;
    }
    __syncthreads();
    double rr_t = 0.0, aa_t = 0.0;
    for (int k = tid; k < Ku; k += NT) {
        double rr = 0.0, aa = 0.0;
        for (int sm = 0; sm < SAMPLES; ++sm) {
            const int i = (2 * sm + 1) * M / (2 * SAMPLES), j = (2 * ((11 * sm) % SAMPLES) + 1) * N / (2 * SAMPLES);
            const Cx<T> a = ent<KER, T>(A, S.rb + i, S.cb + j, k);
            Cx<T> r = a;
            for (int p = 0; p < ncl; ++p) {
                const Cx<T> c = cmul(hs[sm * A.Cmax + p], f_of(A, S, p)[k]);
                r.x -= c.x;
                r.y -= c.y;
            }
            rr += cabs2d(r);
            aa += cabs2d(a);
        }
        w.rk[k] = rr;
        rr_t += rr;
        aa_t += aa;
    }
    rr_t = warp_sum(rr_t);
    aa_t = warp_sum(aa_t);
    if ((tid & 31) == 0) {
        atomicAdd(&S.red2[0], rr_t);
        atomicAdd(&S.red2[1], aa_t);
    }
    __syncthreads();
    const bool ok = S.red2[0] <= A.eps3 * A.eps3 * S.red2[1];
    __syncthreads();
    return ok;
}

// ---- dense-face blocks ---------------------------------------------------------------
// Algorithm 1 with the exact residual face (no low-rank approximation in the
// face, the paper's "No Lwr" variant) for blocks with M N <= dense_max.  A
// cross is stored as H (M x N, column-major) followed by f (Ku) and recorded
// with r = -1.  Per cross: one parallel pass over the M N face entries (the
// residual of earlier crosses is nc multiply-adds per entry), a block argmax
// for the pivot, the fiber, and eq. (norm) through dense inner products.
template <int KER, class T, int NT>
__device__ void dense_block(const AcaArgs<T>& A, const Ws<T>& w, BlockSh<T>& S, bool& zero_block, int& computed,
                            bool& overflow, long long* ph, long long& tclk) {
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int M = S.M, N = S.N, MN = M * N, Ku = A.Ku, blk = S.blk;
    auto lap = [&](int i) {
        if (tid == 0) {
            long long tn = clock64();
            ph[i] += tn - tclk;
            tclk = tn;
        }
    };
    for (;;) {
        const int nc = S.ncross;
        if (tid == 0) {
            const long long need = (long long)MN + Ku;
            unsigned long long o = atomicAdd(A.pool_ctr, (unsigned long long)need);
            if ((long long)o + need > A.pool_cap) {
                atomicOr(A.status, ST_POOL_OVERFLOW);
                S.new_off = -1;
            } else {
                S.new_off = (long long)o;
            }
        }
        __syncthreads();
        if (S.new_off < 0) {
            overflow = true;
            return;
        }
        const long long off = S.new_off;
        Cx<T>* Hn = A.pool + off;
        Cx<T>* Fn = Hn + MN;
        // ---- face: exact residual at S.k, else up to three more frequencies ----
        int cand[4] = {S.k, Ku - 1, Ku / 2, A.k_maxabs};
        ArgMaxT<T> am = amax_none<T>();
        int kf = -1;
        for (int c = 0; c < 4; ++c) {
            const int kk = cand[c];
            bool skip = false;
            for (int d = 1; d < c; ++d) skip |= (cand[d] == kk);
            if (c > 0) skip |= ((S.used_k[kk >> 5] >> (kk & 31)) & 1u) != 0;
            if (skip) continue;
            for (int p = tid; p < nc; p += NT) S.fk[p] = (A.pool + S.off[p] + MN)[kk];
            __syncthreads();
            ArgMaxT<T> a = amax_none<T>();
            for (int e = tid; e < MN; e += NT) {
                const int i = e % M, j = e / M;
                Cx<T> v = ent<KER, T>(A, S.rb + i, S.cb + j, kk);
                for (int p = 0; p < nc; ++p) {
                    const Cx<T> h = A.pool[S.off[p] + e];
                    const Cx<T> x = cmul(S.fk[p], h);
                    v.x -= x.x;
                    v.y -= x.y;
                }
                Hn[e] = v;
                a = amax_better(a, ArgMaxT<T>{cabs2(v), i * N + j});
            }
            a = block_argmax<NT>(a, S.am);
            if (tid == 0) {
                S.entries += MN;
                S.used_k[kk >> 5] |= 1u << (kk & 31);
            }
            __syncthreads();
            if (a.v > tiny_norm2<T>()) {
                am = a;
                kf = kk;
                break;
            }
            if (c == 0 && nc > 0) {
                // a vanishing residual face after the first cross: nothing left at
                // this frequency; test the others only to confirm a zero block
            }
        }
        lap(0);
        if (kf < 0) {
            zero_block = (nc == 0);
            return;
        }
        if (tid == 0) S.k = kf;
        ++computed;
        const int ip = am.i / N, jp = am.i % N;
        const int ep = ip + jp * M;
        const Cx<double> hpiv = ccast<double>(Hn[ep]);
        for (int p = tid; p < nc; p += NT) S.hp[p] = ccast<double>(A.pool[S.off[p] + ep]);
        __syncthreads();
        lap(3);
        // ---- fiber (float64 residual) ----
        for (int k = tid; k < Ku; k += NT) {
            Cx<double> e = ccast<double>(ent<KER, T>(A, S.rb + ip, S.cb + jp, k));
            for (int p = 0; p < nc; ++p) {
                Cx<double> hf = cmul(S.hp[p], ccast<double>((A.pool + S.off[p] + MN)[k]));
                e.x -= hf.x;
                e.y -= hf.y;
            }
            Cx<double> fv = cdiv(e, hpiv);
            w.fib[k] = fv;
            Fn[k] = ccast<T>(fv);
        }
        if (tid == 0) S.entries += Ku;
        __syncthreads();
        lap(4);
        // ---- eq. (norm) with dense faces ----
        for (int d = wid; d <= nc; d += NT / 32) {
            Cx<double> ff{0, 0};
            Cx<T> hh{0, 0};
            if (d < nc) {
                const Cx<T>* fd = A.pool + S.off[d] + MN;
                for (int k = lane; k < Ku; k += 32) cfmac(ff, w.fib[k], ccast<double>(fd[k]));
                const Cx<T>* Hd = A.pool + S.off[d];
                for (int e = lane; e < MN; e += 32) cfmac(hh, Hn[e], Hd[e]);
            } else {
                for (int k = lane; k < Ku; k += 32) ff.x += cabs2(w.fib[k]);
                for (int e = lane; e < MN; e += 32) hh.x += cabs2(Hn[e]);
            }
            ff.x = warp_sum(ff.x);
            ff.y = warp_sum(ff.y);
            const T hx = warp_sum(hh.x), hy = warp_sum(hh.y);
            if (lane == 0) {
                if (d < nc) {
                    S.ff[d] = ff;
                    S.hh[d] = Cx<double>{(double)hx, (double)hy};
                } else {
                    S.fself = ff.x;
                    S.hself = (double)hx;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            double add = 0.0;
            for (int d = 0; d < nc; ++d) add += 2.0 * (S.hh[d].x * S.ff[d].x - S.hh[d].y * S.ff[d].y);
            double own = S.hself * S.fself;
            S.norm2 += add + own;
            S.stop = sqrt(fmax(own, 0.0)) <= A.eps3 * sqrt(fmax(S.norm2, 0.0));
            bool all_used = true;
            for (int k = 0; k < Ku; ++k) all_used &= (S.used_k[k >> 5] >> (k & 31)) & 1u;
            S.flag = all_used;
            S.off[nc] = off;  // staged for the stop check
            S.r[nc] = -1;
        }
        __syncthreads();
        bool from_samples = false;
        if (S.stop && A.sample_check && !S.flag) {
            from_samples = !confirm_stop<KER, T, NT>(A, w, S, nc + 1);
                if (from_samples && threadIdx.x == 0) atomicAdd(&A.counters[6], 1ull);
        }
        if (tid == 0) {
            const bool stop = S.stop && !from_samples;
            S.flag = 0;
            if (!stop) {
                CrossRec cr;
                cr.off = off;
                cr.r = -1;
                cr.ip = ip;
                cr.jp = jp;
                cr.kp = S.k;
                A.rec[(size_t)blk * A.Cmax + nc] = cr;
                S.off[nc] = off;
                S.r[nc] = -1;
                S.ncross = nc + 1;
                bool all_used = true;
                for (int k = 0; k < Ku; ++k) all_used &= (S.used_k[k >> 5] >> (k & 31)) & 1u;
                if (S.ncross >= A.Cmax || all_used) S.flag = 1;
            } else {
                S.flag = 1;
            }
        }
        __syncthreads();
        lap(5);
        if (S.flag) return;
        ArgMaxT<T> nk = amax_none<T>();
        for (int k = tid; k < Ku; k += NT)
            if (!((S.used_k[k >> 5] >> (k & 31)) & 1u))
                nk = amax_better(nk, ArgMaxT<T>{(T)(from_samples ? w.rk[k] : cabs2(w.fib[k])), k});
        nk = block_argmax<NT>(nk, S.am);
        if (nk.v < 0 || nk.i < 0 || nk.i >= Ku) return;
        if (tid == 0) S.k = nk.i;
        __syncthreads();
        lap(6);
    }
}

// ---- the persistent kernel ---------------------------------------------------------
// DENSE selects the block class this launch serves (dense faces or low-rank
// faces); the two classes run as two persistent launches with their own queues.
// resident CTAs per SM the register allocation is sized for: 128 registers
// a thread at 128 threads (4 CTAs), 256 (2 CTAs) and 512 (1 CTA); 384
// threads keep 2 CTAs (80 registers a thread, 24 warps per SM)
template <int NT>
constexpr int aca_min_ctas() { return NT <= 128 ? 4 : (NT <= 384 ? 2 : 1); }

template <int KER, class T, int NT, bool DENSE>
__global__ void __launch_bounds__(NT, aca_min_ctas<NT>()) k_aca3(const AcaArgs<T> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockSh<T> S;
    // the arguments of the block being processed: P, with the geometry and
    // frequencies of the block's own mesh in a batched compression
    __shared__ AcaArgs<T> Ash;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int RF = P.RF;
    Cx<double>* shB = reinterpret_cast<Cx<double>*>(smem_raw);  // arena base
    const Ws<T> w = ws_carve<T>(P.ws + (size_t)blockIdx.x * P.ws_stride, RF, P.Mmax, P.Nmax, P.Cmax, P.Ku,
                                P.drf_max > 0 ? P.drf_off : 0);
    __shared__ int s_q;
    for (int iter = 0;; ++iter) {
        if (tid == 0) {
            if (P.single >= 0)
                s_q = (iter == 0 && blockIdx.x == 0) ? P.single : -1;
            else {
                int q = atomicAdd(P.queue_head, 1);
                s_q = q < P.n_far ? q : -1;
            }
        }
        __syncthreads();
        const int qi = s_q;
        __syncthreads();
        if (qi < 0) break;
        const int blk = P.queue[qi];
        if (tid == 0) {
            Ash = P;
            if (P.geos) {
                const GeoDesc g = P.geos[P.bgeo[blk]];
                Ash.gf = g.gf;
                Ash.gd = g.gd;
                Ash.sd = g.sd;
                Ash.sf = g.sf;
                Ash.Ku = g.Ku;
                Ash.k_maxabs = g.k_maxabs;
            }
        }
        __syncthreads();
        const AcaArgs<T>& A = Ash;
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
            S.raw = 0;
            for (int i = 0; i < NSUB; ++i) S.sub[i] = 0;
            S.k = A.k1 ? A.k1[blk] : 0;
            for (int i = 0; i < KU_MAX / 32; ++i) S.used_k[i] = 0u;
        }
        __syncthreads();
        const int M = S.M, N = S.N, Ku = A.Ku;
        const unsigned long long t_start = globaltimer_ns();
        // phase cycle counters: face, recompress, formation, pivot, fiber, norm, next-k
        long long ph[7] = {0, 0, 0, 0, 0, 0, 0};
        long long tclk = clock64();
        auto lap = [&](int i) {
            if (tid == 0) {
                long long tn = clock64();
                ph[i] += tn - tclk;
                tclk = tn;
            }
        };
        bool zero_block = false;
        int computed = 0;
        bool overflow = false, spilled = false;
        if (M > A.Mmax || N > A.Nmax) {  // cannot happen: workspace is sized from the block list
            if (tid == 0) atomicOr(A.status, ST_BAD_INDEX);
            overflow = true;
        }
        if (DENSE) {
            if (!overflow) dense_block<KER, T, NT>(A, w, S, zero_block, computed, spilled, ph, tclk);
            overflow = true;  // the low-rank loop below is not for this launch
        }
        while (!overflow) {
            // ---------------- face at S.k ----------------
            int kf = S.k;
            int r = face_aca<KER, T, NT>(A, w, S, kf, smem_raw);
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
                    r = face_aca<KER, T, NT>(A, w, S, kk, smem_raw);
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
            lap(0);
            // ---------------- recompression ----------------
            int rn = -1;
            const Cx<T>* tU = nullptr;
            const Cx<T>* tV = nullptr;
            int ldT = 0;
            if (!A.no_recompress) {
                rn = recompress<T, NT>(A, w, S, r, shB, &tU, &tV, &ldT);
                if (rn < 0 && tid == 0) {
                    atomicOr(A.status, ST_CHOL_FALLBACK);
                    atomicAdd(&A.counters[4], 1ull);
                }
            }
            const bool raw = rn < 0;
            if (raw) rn = r;
            lap(1);
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
                overflow = spilled = true;
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
                // U' = uw T_U, V' = vw T_V in the working precision, 8 output columns per pass
                for (int e = tid; e < (M + N) * ((rn + 7) / 8); e += NT) {
                    const int row = e % (M + N), b0 = (e / (M + N)) * 8;
                    const bool isU = row < M;
                    const int i = isU ? row : row - M;
                    const Cx<T>* src = isU ? w.uw + i : w.vw + i;
                    const size_t ld = isU ? A.Mmax : A.Nmax;
                    const Cx<T>* Tm = isU ? tU : tV;
                    Cx<T> acc[8];
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) acc[bb] = Cx<T>{0, 0};
                    for (int a = 0; a < r; ++a) {
                        const Cx<T> u = src[(size_t)a * ld];
#pragma unroll
                        for (int bb = 0; bb < 8; ++bb) cfma(acc[bb], u, Tm[a * ldT + min(b0 + bb, rn - 1)]);
                    }
                    Cx<T>* dst = isU ? Un + i : Vn + i;
                    const long long L = isU ? M : N;
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb)
                        if (b0 + bb < rn) dst[(long long)(b0 + bb) * L] = acc[bb];
                }
            }
            __syncthreads();
            lap(2);
            // ---------------- pivot: argmax |U' V'^H| ----------------
            if (KER != G3_DLP && A.pivot_index) {
                // the estimate of eq. (index) (Section 4, last remark): the row
                // i = argmax_i sum_b |U'[i, b]| ||V'[:, b]|| (for U' = U Sigma and
                // orthonormal V' the paper's sum_k |u_ik sigma_k|, a bound on the
                // entries of row i), then the column found in that row: j =
                // argmax_j |(U' V'^H)[i, j]|, O((M + N) r) instead of the dense
                // expansion's O(M N r); ties to the smallest index.  The double
                // layer keeps the dense expansion, as the paper does.
                for (int b = wid; b < rn; b += NT / 32) {
                    const Cx<T>* col = Vn + (long long)b * N;
                    T s2 = 0;
                    for (int i = lane; i < N; i += 32) s2 += cabs2(ldcx(col + i));
                    s2 = warp_sum(s2);
                    if (lane == 0) S.cnV[b] = sqrt(s2);
                }
                __syncthreads();
                ArgMaxT<T> bi = amax_none<T>();
                for (int i = tid; i < M; i += NT) {
                    T sc = 0;
                    for (int b = 0; b < rn; ++b) sc += sqrt(cabs2(ldcx(Un + (long long)b * M + i))) * S.cnV[b];
                    bi = amax_better(bi, ArgMaxT<T>{sc, i});
                }
                bi = block_argmax<NT>(bi, S.am);
                const int ir = (bi.v >= 0 && bi.i >= 0 && bi.i < M) ? bi.i : 0;
                // row ir of the face: U'[ir, :] (r values, one broadcast load each)
                for (int b = tid; b < rn; b += NT) S.fk[b] = Un[(long long)b * M + ir];
                __syncthreads();
                ArgMaxT<T> bj = amax_none<T>();
                for (int j = tid; j < N; j += NT) {
                    Cx<T> h{0, 0};
                    for (int b = 0; b < rn; ++b) cfmac(h, S.fk[b], ldcx(Vn + (long long)b * N + j));
                    bj = amax_better(bj, ArgMaxT<T>{cabs2(h), j});
                }
                bj = block_argmax<NT>(bj, S.am);
                if (tid == 0) {
                    if (bi.v < 0 || bj.v < 0 || bi.i < 0 || bi.i >= M || bj.i < 0 || bj.i >= N) {
                        S.ip = 0;
                        S.jp = 0;
                        S.hpiv = Cx<double>{0.0, 0.0};
                    } else {
                        S.ip = bi.i;
                        S.jp = bj.i;
                        Cx<T> hw{0, 0};
                        for (int b = 0; b < rn; ++b) cfmac(hw, Un[(long long)b * M + S.ip], Vn[(long long)b * N + S.jp]);
                        Cx<double> h = ccast<double>(hw);
                        if (!isfinite(h.x) || !isfinite(h.y)) h = Cx<double>{0.0, 0.0};
                        S.hpiv = h;
                    }
                }
            } else {
                constexpr int TM = sizeof(T) == 4 ? 64 : 32;
                constexpr int TN = TM;
                constexpr int RM = TM * TN / NT >= 16 ? 4 : 2;  // micro-tile edge
                constexpr int TX = TN / RM;                     // micro-tiles along j
                constexpr int NMT = (TM / RM) * TX;             // micro-tiles per tile
                Cx<T>* tu = reinterpret_cast<Cx<T>*>(smem_raw);  // [rn][TM]
                Cx<T>* tv = tu + (size_t)RF * TM;                // [rn][TN]
                ArgMaxT<T> best = amax_none<T>();
                for (int i0 = 0; i0 < M; i0 += TM) {
                    for (int j0 = 0; j0 < N; j0 += TN) {
                        for (int e = tid; e < rn * TM; e += NT) {
                            int b = e / TM, ii = e % TM;
                            tu[b * TM + ii] = (i0 + ii < M) ? ldcx(Un + (long long)b * M + i0 + ii) : Cx<T>{0, 0};
                        }
                        for (int e = tid; e < rn * TN; e += NT) {
                            int b = e / TN, jj = e % TN;
                            tv[b * TN + jj] = (j0 + jj < N) ? ldcx(Vn + (long long)b * N + j0 + jj) : Cx<T>{0, 0};
                        }
                        __syncthreads();
                        for (int mt = tid; mt < NMT; mt += NT) {
                            const int tx = mt % TX, ty = mt / TX;
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
                                        best = amax_better(best, ArgMaxT<T>{cabs2(acc[a][c]), gi * N + gj});
                                }
                        }
                        __syncthreads();
                    }
                }
                best = block_argmax<NT>(best, S.am);
                if (tid == 0) {
                    // no finite candidate (a non-finite face): report a vanishing pivot
                    if (best.v < 0 || best.i < 0 || best.i >= M * N) {
                        S.ip = 0;
                        S.jp = 0;
                        S.hpiv = Cx<double>{0.0, 0.0};
                        if (best.v >= 0) atomicOr(A.status, ST_BAD_INDEX);
                    } else {
                        S.ip = (int)(best.i / N);
                        S.jp = (int)(best.i % N);
                        Cx<T> hw{0, 0};
                        for (int b = 0; b < rn; ++b) cfmac(hw, Un[(long long)b * M + S.ip], Vn[(long long)b * N + S.jp]);
                        Cx<double> h = ccast<double>(hw);
                        if (!isfinite(h.x) || !isfinite(h.y)) h = Cx<double>{0.0, 0.0};
                        S.hpiv = h;
                    }
                }
            }
            __syncthreads();
            lap(3);
            if (S.hpiv.x == 0.0 && S.hpiv.y == 0.0) break;  // vanishing face: nothing to divide by
            // H_p[i_l, j_l] of earlier crosses (values of the face's scale: working precision)
            for (int p = tid; p < S.ncross; p += NT) {
                const Cx<T>* U = Up(A, S, p);
                const Cx<T>* V = Vp(A, S, p);
                Cx<T> h{0, 0};
                for (int t = 0; t < S.r[p]; ++t) cfmac(h, U[(long long)t * M + S.ip], V[(long long)t * N + S.jp]);
                S.hp[p] = ccast<double>(h);
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
            lap(4);
            // ---------------- eq. (norm) ----------------
            // <f_l, f_d> and ||f_l||^2
            // (the fibers are normalised by their pivot entry: working precision)
            for (int d = wid; d <= nc; d += NT / 32) {
                Cx<T> acc{0, 0};
                if (d < nc) {
                    const Cx<T>* fd = Fp(A, S, d);
                    for (int k = lane; k < Ku; k += 32) cfmac(acc, Fn[k], fd[k]);
                } else {
                    for (int k = lane; k < Ku; k += 32) acc.x += cabs2(Fn[k]);
                }
                acc.x = warp_sum(acc.x);
                acc.y = warp_sum(acc.y);
                if (lane == 0) {
                    if (d < nc) S.ff[d] = ccast<double>(acc);
                    else S.fself = (double)acc.x;
                }
            }
            for (int d = tid; d < nc; d += NT) S.hh[d] = Cx<double>{0, 0};
            if (tid == 0) S.hself = 0.0;
            __syncthreads();
            // <H_l, H_d> and ||H_l||^2 through tiled Gram products
            norm_grams<T, NT>(A, S, Un, Vn, rn, reinterpret_cast<Cx<T>*>(smem_raw));
            if (tid == 0) {
                double add = 0.0;
                for (int d = 0; d < nc; ++d) add += 2.0 * (S.hh[d].x * S.ff[d].x - S.hh[d].y * S.ff[d].y);
                double own = S.hself * S.fself;
                S.norm2 += add + own;
                S.stop = sqrt(fmax(own, 0.0)) <= A.eps3 * sqrt(fmax(S.norm2, 0.0));
                bool all_used = true;
                for (int k = 0; k < Ku; ++k) all_used &= (S.used_k[k >> 5] >> (k & 31)) & 1u;
                S.flag = all_used;
                S.off[nc] = off;  // staged for the stop check
                S.r[nc] = rn;
            }
            __syncthreads();
            bool from_samples = false;
            if (S.stop && A.sample_check && !S.flag) {
                from_samples = !confirm_stop<KER, T, NT>(A, w, S, nc + 1);
                if (from_samples && threadIdx.x == 0) atomicAdd(&A.counters[6], 1ull);
            }
            if (tid == 0) {
                const bool stop = S.stop && !from_samples;
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
            lap(5);
            if (S.flag) break;
            // next frequency: argmax over unused k of |f_l[k]|
            ArgMaxT<T> nk = amax_none<T>();
            for (int k = tid; k < Ku; k += NT)
                if (!((S.used_k[k >> 5] >> (k & 31)) & 1u))
                    nk = amax_better(nk, ArgMaxT<T>{from_samples ? (T)w.rk[k] : cabs2(Fn[k]), k});
            nk = block_argmax<NT>(nk, S.am);
            if (nk.v < 0 || nk.i < 0 || nk.i >= Ku) break;  // no finite candidate left
            if (tid == 0) S.k = nk.i;
            __syncthreads();
            lap(6);
        }
        if (tid == 0) {
            // a block that found the pool full goes to the spill queue and is
            // rerun from its start with a fresh pool segment
            A.r3[blk] = spilled ? 0 : S.ncross;
            if (spilled) {
                const int q = atomicAdd(A.spill_n, 1);
                if (q < A.spill_cap) A.spill[q] = blk;
            }
            for (int i = 0; i < 7; ++i) A.blk_cycles[(size_t)blk * NPH + i] += ph[i];
            A.blk_cycles[(size_t)blk * NPH + 7] += S.raw;
            A.blk_cycles[(size_t)blk * NPH + 8] = (long long)t_start;
            A.blk_cycles[(size_t)blk * NPH + 9] = (long long)globaltimer_ns();
            atomicAdd(&A.counters[0], (unsigned long long)S.entries);
            atomicAdd(&A.counters[1], (unsigned long long)computed);
            if (zero_block && !spilled) atomicAdd(&A.counters[2], 1ull);
            for (int i = 0; i < 7; ++i) atomicAdd(&A.counters[8 + i], (unsigned long long)ph[i]);
            for (int i = 0; i < NSUB; ++i) atomicAdd(&A.counters[16 + i], (unsigned long long)S.sub[i]);
        }
        __syncthreads();
    }
}

// ============================================================================
// Three-way ACA of the H-matrix as a whole (Section 4, first implementation
// remark): all admissible blocks share the frequency sequence k_l and one
// fiber per cross; the pivot is the largest entry of the whole face and the
// stopping test sums eq. (norm) over the blocks.  The host runs the loop
// over crosses; per cross:
//   k_aca3_face   one CTA per block (persistent queue): the block's residual
//                 face at k_l (face ACA with the shared fibers of the earlier
//                 crosses, already copied into each block's cross slots),
//                 recompression, U' and V' in the pool, the block's largest
//                 face entry (dense expansion), and the block's terms of
//                 eq. (norm): <H_l^b, H_d^b> for d < l and ||H_l^b||^2;
//   k_whole_fiber the shared fiber at the global pivot (block b*, i, j):
//                 f_l[k] = (ENTRY - sum_p H_p^b*[i, j] f_p[k]) / H_l^b*[i, j],
//                 and <f_l, f_d>, ||f_l||^2;
//   k_whole_norm  copies f_l into every block's slot of cross l and adds the
//                 blocks' eq. (norm) terms (per block and in total).
// ============================================================================

struct WholeCand {
    double v;   // |H_l^b[i, j]|^2 of the block's largest entry (-1: zero face)
    int i, j;
};

template <int KER, class T, int NT>
__global__ void __launch_bounds__(NT, aca_min_ctas<NT>()) k_aca3_face(const AcaArgs<T> P, int kf, int nc,
                                                                      const double* __restrict__ normb,
                                                                      WholeCand* __restrict__ cand,
                                                                      Cx<double>* __restrict__ hh_out,
                                                                      double* __restrict__ hself_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockSh<T> S;
    __shared__ int s_q;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const AcaArgs<T>& A = P;
    const int RF = A.RF;
    Cx<double>* shB = reinterpret_cast<Cx<double>*>(smem_raw);
    const Ws<T> w = ws_carve<T>(A.ws + (size_t)blockIdx.x * A.ws_stride, RF, A.Mmax, A.Nmax, A.Cmax, A.Ku);
    for (;;) {
        if (tid == 0) {
            const int q = atomicAdd(A.queue_head, 1);
            s_q = q < A.n_far ? q : -1;
        }
        __syncthreads();
        const int qi = s_q;
        __syncthreads();
        if (qi < 0) break;
        const int blk = A.queue[qi];
        if (tid == 0) {
            const BlockRange br = A.ranges[blk];
            S.rb = br.rb;
            S.cb = br.cb;
            S.M = br.re - br.rb;
            S.N = br.ce - br.cb;
            S.blk = blk;
            S.ncross = nc;
            S.pre[0] = 0;
            for (int p = 0; p < nc; ++p) {
                const CrossRec cr = A.rec[(size_t)blk * A.Cmax + p];
                S.off[p] = cr.off;
                S.r[p] = cr.r;
                S.pre[p + 1] = S.pre[p] + cr.r;
            }
            S.norm2 = normb[blk];
            S.entries = 0;
            S.raw = 0;
            for (int i = 0; i < NSUB; ++i) S.sub[i] = 0;
            S.k = kf;
        }
        __syncthreads();
        const int M = S.M, N = S.N;
        bool ok = M <= A.Mmax && N <= A.Nmax;
        int r = ok ? face_aca<KER, T, NT>(A, w, S, kf, smem_raw) : 0;
        int rn = 0;
        const Cx<T>* tU = nullptr;
        const Cx<T>* tV = nullptr;
        int ldT = 0;
        bool raw = false;
        if (r > 0) {
            rn = A.no_recompress ? -1 : recompress<T, NT>(A, w, S, r, shB, &tU, &tV, &ldT);
            raw = rn < 0;
            if (raw) rn = r;
        }
        // the cross slot: U' (M x rn), V' (N x rn), then the shared fiber (Ku)
        if (tid == 0) {
            const long long need = (long long)rn * (M + N) + A.Ku;
            const unsigned long long o = atomicAdd(A.pool_ctr, (unsigned long long)need);
            if ((long long)o + need > A.pool_cap) {
                atomicOr(A.status, ST_POOL_OVERFLOW);
                S.new_off = -1;
            } else {
                S.new_off = (long long)o;
            }
        }
        __syncthreads();
        const long long off = S.new_off;
        if (off < 0) {
            if (tid == 0) {
                cand[blk] = WholeCand{-1.0, 0, 0};
                A.rec[(size_t)blk * A.Cmax + nc] = CrossRec{-1, 0, 0, 0, kf};  // no slot (overflow status set)
            }
            for (int d = tid; d < nc; d += NT) hh_out[(size_t)blk * A.Cmax + d] = Cx<double>{0, 0};
            if (tid == 0) hself_out[blk] = 0.0;
            __syncthreads();
            continue;
        }
        Cx<T>* Un = A.pool + off;
        Cx<T>* Vn = A.pool + off + (long long)rn * M;
        if (rn > 0) {
            if (raw) {
                for (int e = tid; e < rn * M; e += NT) Un[e] = w.uw[(size_t)(e / M) * A.Mmax + e % M];
                for (int e = tid; e < rn * N; e += NT) Vn[e] = w.vw[(size_t)(e / N) * A.Nmax + e % N];
            } else {
                for (int e = tid; e < (M + N) * rn; e += NT) {
                    const int row = e % (M + N), b = e / (M + N);
                    const bool isU = row < M;
                    const int i = isU ? row : row - M;
                    const Cx<T>* src = isU ? w.uw + i : w.vw + i;
                    const size_t ld = isU ? A.Mmax : A.Nmax;
                    const Cx<T>* Tm = isU ? tU : tV;
                    Cx<T> acc{0, 0};
                    for (int a = 0; a < r; ++a) cfma(acc, src[(size_t)a * ld], Tm[a * ldT + b]);
                    (isU ? Un + i : Vn + i)[(long long)b * (isU ? M : N)] = acc;
                }
            }
        }
        __syncthreads();
        // the block's largest face entry: dense expansion of U' V'^H, one
        // entry per thread and pass (ties to the smallest row-major index)
        ArgMaxT<T> best = amax_none<T>();
        if (rn > 0)
            for (long long e = tid; e < (long long)M * N; e += NT) {
                const int i = (int)(e / N), j = (int)(e - (long long)i * N);
                Cx<T> h{0, 0};
                for (int b = 0; b < rn; ++b) cfmac(h, ldcx(Un + (long long)b * M + i), ldcx(Vn + (long long)b * N + j));
                best = amax_better(best, ArgMaxT<T>{cabs2(h), (int)e});
            }
        best = block_argmax<NT>(best, S.am);
        // eq. (norm) terms of the block: <H_l^b, H_d^b> (d < nc) and ||H_l^b||^2
        for (int d = tid; d < nc; d += NT) S.hh[d] = Cx<double>{0, 0};
        if (tid == 0) S.hself = 0.0;
        __syncthreads();
        if (rn > 0) norm_grams<T, NT>(A, S, Un, Vn, rn, reinterpret_cast<Cx<T>*>(smem_raw));
        __syncthreads();
        for (int d = tid; d < nc; d += NT) hh_out[(size_t)blk * A.Cmax + d] = S.hh[d];
        if (tid == 0) {
            hself_out[blk] = S.hself;
            const bool have = rn > 0 && best.v >= 0 && best.i >= 0 && best.i < M * N;
            cand[blk] = have ? WholeCand{(double)best.v, best.i / N, best.i % N} : WholeCand{-1.0, 0, 0};
            A.rec[(size_t)blk * A.Cmax + nc] = CrossRec{off, rn, have ? best.i / N : 0, have ? best.i % N : 0, kf};
            A.r3[blk] = nc + 1;
            atomicAdd(&A.counters[0], (unsigned long long)S.entries);
        }
        __syncthreads();
    }
}

// the shared fiber of cross nc at the pivot (block pb, local i, j): one CTA
template <int KER, class T, int NT>
__global__ void __launch_bounds__(NT) k_whole_fiber(const AcaArgs<T> A, int pb, int pi, int pj, int nc,
                                                    Cx<double>* __restrict__ fib,   // [Cmax][Ku] shared fibers
                                                    Cx<double>* __restrict__ ff,    // [Cmax]: <f_nc, f_d>, then ||f||^2
                                                    double* __restrict__ scal) {    // [0] ||f||^2 [1] |H_pivot|^2
    __shared__ Cx<double> hp[KU_MAX];
    __shared__ Cx<double> hpiv;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const BlockRange br = A.ranges[pb];
    const int M = br.re - br.rb, N = br.ce - br.cb;
    // H_p^pb[i, j] for the earlier crosses and the new one
    for (int p = tid; p <= nc; p += NT) {
        const CrossRec cr = A.rec[(size_t)pb * A.Cmax + p];
        const Cx<T>* U = A.pool + cr.off;
        const Cx<T>* V = U + (long long)cr.r * M;
        Cx<T> h{0, 0};
        for (int t = 0; t < cr.r; ++t) cfmac(h, U[(long long)t * M + pi], V[(long long)t * N + pj]);
        if (p < nc) hp[p] = ccast<double>(h);
        else hpiv = ccast<double>(h);
    }
    __syncthreads();
    const Cx<double> hv = hpiv;
    const double h2 = hv.x * hv.x + hv.y * hv.y;
    Cx<double>* fn = fib + (size_t)nc * A.Ku;
    for (int k = tid; k < A.Ku; k += NT) {
        Cx<double> e = ccast<double>(ent<KER, T>(A, br.rb + pi, br.cb + pj, k));
        for (int p = 0; p < nc; ++p) {
            const Cx<double> hf = cmul(hp[p], fib[(size_t)p * A.Ku + k]);
            e.x -= hf.x;
            e.y -= hf.y;
        }
        fn[k] = h2 > 0 ? cdiv(e, hv) : Cx<double>{0, 0};
    }
    __syncthreads();
    // <f_nc, f_d> = sum_k f_nc[k] conj(f_d[k]) for d < nc, and ||f_nc||^2
    for (int d = wid; d <= nc; d += NT / 32) {
        const Cx<double>* fd = fib + (size_t)d * A.Ku;
        Cx<double> acc{0, 0};
        for (int k = lane; k < A.Ku; k += 32) cfmac(acc, fn[k], fd[k]);
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        if (lane == 0) ff[d] = acc;
    }
    if (tid == 0) scal[1] = h2;
    __syncthreads();
    if (tid == 0) scal[0] = ff[nc].x;
    if (tid == 0 && threadIdx.x == 0) atomicAdd(&A.counters[0], (unsigned long long)A.Ku);
}

// copy the shared fiber of cross nc into every block's slot; add the blocks'
// eq. (norm) terms: per block 2 Re sum_d <H_nc^b, H_d^b><f_nc, f_d> + ||H_nc^b||^2 ||f||^2
// (into normb), in total (tot[0]) and sum_b ||H_nc^b||^2 (tot[1])
template <class T>
__global__ void k_whole_norm(const AcaArgs<T> A, int nc, const Cx<double>* __restrict__ fib,
                             const Cx<double>* __restrict__ ff, const Cx<double>* __restrict__ hh,
                             const double* __restrict__ hself, double* __restrict__ normb,
                             double* __restrict__ tot) {
    const int blk = blockIdx.x;
    const BlockRange br = A.ranges[blk];
    const int M = br.re - br.rb, N = br.ce - br.cb;
    const CrossRec cr = A.rec[(size_t)blk * A.Cmax + nc];
    const Cx<double>* fn = fib + (size_t)nc * A.Ku;
    if (cr.off >= 0) {
        Cx<T>* fs = A.pool + cr.off + (long long)cr.r * (M + N);
        for (int k = threadIdx.x; k < A.Ku; k += blockDim.x) fs[k] = ccast<T>(fn[k]);
    }
    double add = 0.0;
    for (int d = threadIdx.x; d < nc; d += blockDim.x) {
        const Cx<double> a = hh[(size_t)blk * A.Cmax + d], b = ff[d];
        add += 2.0 * (a.x * b.x - a.y * b.y);
    }
    add = warp_sum(add);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = add;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += part[q];
        const double own = hself[blk] * ff[nc].x;
        normb[blk] += s + own;
        atomicAdd(&tot[0], s + own);
        atomicAdd(&tot[1], hself[blk]);
    }
}

template <int KER, class T>
g3_status launch_whole_t(g3_ctx* ctx, AcaArgs<T>& A, int grid, size_t smem, int kf, int nc, const double* normb,
                         WholeCand* cand, Cx<double>* hh, double* hself) {
    constexpr int NT = 256;
    auto kfn = k_aca3_face<KER, T, NT>;
    G3_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kfn<<<grid, NT, smem, ctx->stream>>>(A, kf, nc, normb, cand, hh, hself);
    ctx->count("k_aca3_face");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

template <int KER, class T>
g3_status launch_whole_fiber_t(g3_ctx* ctx, AcaArgs<T>& A, int pb, int pi, int pj, int nc, Cx<double>* fib,
                               Cx<double>* ff, double* scal, int n_far, const Cx<double>* hh, const double* hself,
                               double* normb, double* tot) {
    k_whole_fiber<KER, T, 256><<<1, 256, 0, ctx->stream>>>(A, pb, pi, pj, nc, fib, ff, scal);
    ctx->count("k_whole_fiber");
    G3_CUDA(cudaGetLastError());
    k_whole_norm<T><<<n_far, 128, 0, ctx->stream>>>(A, nc, fib, ff, hh, hself, normb, tot);
    ctx->count("k_whole_norm");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

// ============================================================================
// launch helpers (instantiated once per kernel kind, in g3_aca_slp.cu,
// g3_aca_dlp.cu and g3_aca_sep.cu, so that the kinds compile in parallel)
// ============================================================================

template <int KER, class T, int NT, bool DENSE>
g3_status launch_aca_t(g3_ctx* ctx, AcaArgs<T>& A, int grid, size_t smem) {
    auto kfn = k_aca3<KER, T, NT, DENSE>;
    G3_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kfn<<<grid, NT, smem, ctx->stream>>>(A);
    ctx->count(KER == G3_SEPARABLE   ? (DENSE ? "k_aca3_dense_separable" : "k_aca3_separable")
               : KER == G3_GAL_SLP ? (DENSE ? "k_aca3_dense_galerkin" : "k_aca3_galerkin")
               : KER == G3_GAL_P1D ? (DENSE ? "k_aca3_dense_hypersingular" : "k_aca3_hypersingular")
               : KER == G3_GAL_P1KP ? (DENSE ? "k_aca3_dense_adjoint_dlp" : "k_aca3_adjoint_dlp")
                                   : (DENSE ? "k_aca3_dense" : "k_aca3"));
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

template <int KER, class T, int NT, bool DENSE>
int occupancy(size_t smem) {
    int nb = 0;
    auto kfn = k_aca3<KER, T, NT, DENSE>;
    cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, NT, smem) != cudaSuccess) nb = 1;
    return std::max(nb, 1);
}

}  // namespace g3
