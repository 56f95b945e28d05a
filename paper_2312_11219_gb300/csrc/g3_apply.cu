// Application of the compressed three-way array to densities at all
// frequencies (eq. (product)):
//
//   y = sum_{l=1}^{K} A(s_l) w_l
//     = sum_near sum_k [Re A_k (w_k + w_k') + i Im A_k (w_k - w_k')]
//       + sum_far sum_p [ U_p (V_p^H x_p) + conj(U_p (V_p^H zc_p)) ],
//   x_p = sum_{k in unique} f_p[k] w_k ,  zc_p = sum_{k paired} f_p[k] conj(w_k'),
//
// where k' is the conjugate partner of the unique frequency k
// (A(conj s) = conj A(s) for real geometry; Appendix A notes that half of the
// frequencies suffice).  The near field is read once from HBM (the bound of
// this step); each stored (unique-frequency) entry serves both members of a
// conjugate pair.
#include <algorithm>
#include <vector>

#include "g3_device.cuh"

#define G3_TRY_NA(expr)                 \
    do {                                \
        g3_status st_ = (expr);         \
        if (st_ != G3_OK) return st_;   \
    } while (0)

namespace g3 {

// largest face rank the per-frequency apply keeps in shared memory (the
// compression caps face ranks at 64)
constexpr int RF_TS = 64;

// W (original order, column l = w_l, M x K column-major, complex TI) ->
// Wf[k][p] = w_{uniq[k]}[perm[p]],  Wc[k][p] = w_{partner(uniq[k])}[perm[p]] or 0
// (cluster order, frequency-major), and y := 0.
// ldw: rows of W (E, or the vertex count for linear-element trees, where perm is
// the vertex of each position: the gather w_loc = P w of the nodal densities)
template <class TI, class T>
__global__ void k_apply_prep(int E, int K, int Ku, const int* __restrict__ perm, const int* __restrict__ uniq,
                             const int* __restrict__ partner, const Cx<TI>* __restrict__ W, Cx<T>* __restrict__ Wf,
                             Cx<T>* __restrict__ Wc, Cx<T>* __restrict__ y, int ldw) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx < E) y[idx] = Cx<T>{0, 0};
    if (idx >= (long long)Ku * E) return;
    const int k = (int)(idx / E), p = (int)(idx % E);
    const int e = perm[p];
    const int l = uniq[k], lp = partner[l];
    Cx<TI> a = W[(long long)l * ldw + e];
    Wf[idx] = Cx<T>{(T)a.x, (T)a.y};
    if (lp != l) {
        Cx<TI> b = W[(long long)lp * ldw + e];
        Wc[idx] = Cx<T>{(T)b.x, (T)b.y};
    } else {
        Wc[idx] = Cx<T>{0, 0};
    }
}

// Near field: one CTA per (row cluster, frequency chunk).  The work units are
// the (near block, frequency) pairs of the row cluster and chunk, dealt to the
// warps in turn.  For a unit, lane i holds row i of the block (blocks are
// stored [k][j][i], so the column j of all rows is one coalesced load) and
// sums Re A (w + w') + i Im A (w - w') over the block's columns, with w_j and
// w'_j read as broadcasts.  Each warp keeps its row sums in its own slice of
// shared memory; the CTA adds the warps' sums to y once.
template <class T, int NT>
__global__ void __launch_bounds__(NT) k_apply_near(const Cx<T>* __restrict__ A, const BlockRange* __restrict__ ranges,
                                                   const long long* __restrict__ offs, const int* __restrict__ row_start,
                                                   int Ku, int kchunk, int E, const Cx<T>* __restrict__ Wf,
                                                   const Cx<T>* __restrict__ Wc, Cx<T>* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NW = NT / 32;
    const int g = blockIdx.x;
    const int k0 = blockIdx.y * kchunk, k1 = min(Ku, k0 + kchunk), nk = k1 - k0;
    const int b0 = row_start[g], b1 = row_start[g + 1];
    const int rb = ranges[b0].rb, Mrow = ranges[b0].re - ranges[b0].rb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* ysw = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 2 * Mrow;  // [NW][2 * Mrow]
    for (int i = threadIdx.x; i < NW * 2 * Mrow; i += NT) reinterpret_cast<T*>(smem_raw)[i] = 0;
    __syncthreads();
    const int units = (b1 - b0) * nk;
    for (int u = warp; u < units; u += NW) {
        const int b = b0 + u / nk, k = k0 + u % nk;
        const BlockRange br = ranges[b];
        const int N = br.ce - br.cb;
        const Cx<T>* Ak = A + offs[b] + (long long)k * Mrow * N;
        const Cx<T>* wf = Wf + (long long)k * E + br.cb;
        const Cx<T>* wc = Wc + (long long)k * E + br.cb;
        for (int i0 = 0; i0 < Mrow; i0 += 32) {
            const int i = i0 + lane;
            const bool act = i < Mrow;
            T ax = 0, ay = 0;
            int j = 0;
            for (; j + 8 <= N; j += 8) {
                Cx<T> a[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) a[q] = act ? ldcx(Ak + (long long)(j + q) * Mrow + i) : Cx<T>{0, 0};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const Cx<T> f = ldcx(wf + j + q), c = ldcx(wc + j + q);
                    ax += a[q].x * (f.x + c.x) - a[q].y * (f.y - c.y);
                    ay += a[q].x * (f.y + c.y) + a[q].y * (f.x - c.x);
                }
            }
            for (; j < N; ++j) {
                const Cx<T> a = act ? ldcx(Ak + (long long)j * Mrow + i) : Cx<T>{0, 0};
                const Cx<T> f = ldcx(wf + j), c = ldcx(wc + j);
                ax += a.x * (f.x + c.x) - a.y * (f.y - c.y);
                ay += a.x * (f.y + c.y) + a.y * (f.x - c.x);
            }
            if (act) {
                ysw[2 * i] += ax;
                ysw[2 * i + 1] += ay;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < Mrow; i += NT) {
        T sx = 0, sy = 0;
        for (int w = 0; w < NW; ++w) {
            const T* yw = reinterpret_cast<const T*>(smem_raw) + (size_t)w * 2 * Mrow;
            sx += yw[2 * i];
            sy += yw[2 * i + 1];
        }
        atomicAdd(&y[rb + i].x, sx);
        atomicAdd(&y[rb + i].y, sy);
    }
}

// ---- tensor-core x formation (float32 path) --------------------------------------------
// x_p = sum_k f_p[k] w_k for 16 columns x 8 crosses at a time is the real-matrix product
// of W_sigma^T (columns x frequencies) and F (frequencies x crosses), split into four real
// products per complex product, each on the tensor cores in the three-term TF32 split
// of g3_device.cuh (mma_tf32x3).
// row stride (floats) of the split fibers in shared memory: >= the padded frequency
// count and 4 mod 8, so the eight rows of a B fragment fall in distinct banks
__host__ __device__ constexpr int tc_fiber_stride(int Ku) { return (Ku + 7) / 8 * 8 + 4; }

// Far field, blocks with low-rank faces: one CTA per work item (block, group
// of PG crosses), every factor read once from HBM and every item complete in
// itself (no second pass, no global scratch):
//   1. x_p[j] = sum_k f_p[k] w_k[j], zc_p[j] = sum_k f_p[k] conj(w_k'[j]) for
//      the group's crosses and a chunk of the block's columns (the fibers in
//      shared memory, W read from L2; TPC threads per column, each with
//      PG / TPC crosses);
//   2. a_p[t] += V_p[:, t]^H x_p, b_p[t] += V_p[:, t]^H zc_p over the chunk
//      (one warp per (p, t) pair, two pairs at a time, lanes over the
//      columns), the sums kept in shared memory;
//   3. y[i] += sum_p U_p[i, :] a_p + conj(U_p[i, :] b_p) (TPR threads per row
//      splitting the pairs, lanes over rows, one atomic add per row and part).
// x formation is N K_u complex multiply-adds per cross, the same order of
// work per byte as the HBM stream of the factors; grouping PG crosses lets
// each W value serve PG crosses.
template <class T, int NT, int PG, int TPC, bool TC>
__global__ void __launch_bounds__(NT) k_far_lr(const Cx<T>* __restrict__ pool, const CrossRec* __restrict__ rec,
                                               const int* __restrict__ r3, const BlockRange* __restrict__ ranges,
                                               const int4* __restrict__ items, int Cmax, int Ku, int E,
                                               const Cx<T>* __restrict__ Wf, const Cx<T>* __restrict__ Wc,
                                               Cx<T>* __restrict__ y) {
    constexpr int NC = NT / TPC;    // columns per chunk
    constexpr int PPT = PG / TPC;   // crosses per thread in phase 1
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx<T>* fg = reinterpret_cast<Cx<T>*>(smem_raw);  // [PG][Ku]
    Cx<T>* xs = fg + PG * Ku;                         // [PG][NC]
    Cx<T>* zs = xs + PG * NC;                         // [PG][NC]
    Cx<T>* ab = zs + PG * NC;                         // [2][sum of ranks] a, then b
    // TC: the fibers split into TF32 high and low parts, [4][PG][KS] (re hi, re lo,
    // im hi, im lo), zero beyond Ku
    const int KS = tc_fiber_stride(Ku);
    unsigned* fsp = reinterpret_cast<unsigned*>(ab + 2 * PG * RF_TS);
    __shared__ CrossRec crs[PG];
    __shared__ int pre[PG + 1];
    __shared__ int pof[PG * RF_TS];                   // cross of each flattened pair
    __shared__ long long ubase[PG * RF_TS];           // pool offset of U_p[:, t] of each pair
    const int4 it = items[blockIdx.x];
    const int blk = it.x, g0 = it.y * PG;
    const BlockRange br = ranges[blk];
    const int M = br.re - br.rb, N = br.ce - br.cb;
    const int np = min(PG, r3[blk] - g0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < PG) crs[tid] = tid < np ? rec[(size_t)blk * Cmax + g0 + tid] : CrossRec{0, 0, 0, 0, 0};
    __syncthreads();
    if (tid == 0) {
        pre[0] = 0;
        for (int p = 0; p < PG; ++p) pre[p + 1] = pre[p] + (p < np ? crs[p].r : 0);
    }
    for (int e = tid; e < PG * Ku; e += NT) {
        const int p = e / Ku, k = e - p * Ku;
        fg[e] = p < np ? ldcx(pool + crs[p].off + (long long)crs[p].r * (M + N) + k) : Cx<T>{0, 0};
    }
    if constexpr (TC) {
        static_assert(sizeof(T) == 4 && PG == 8, "tensor-core x formation: float32, 8 crosses per item");
        for (int e = tid; e < PG * KS; e += NT) {
            const int p = e / KS, k = e - p * KS;
            Cx<T> f{0, 0};
            if (p < np && k < Ku) f = ldcx(pool + crs[p].off + (long long)crs[p].r * (M + N) + k);
            const Tf32Pair re = tf32_split(f.x), im = tf32_split(f.y);
            fsp[e] = re.hi;
            fsp[PG * KS + e] = re.lo;
            fsp[2 * PG * KS + e] = im.hi;
            fsp[3 * PG * KS + e] = im.lo;
        }
    }
    __syncthreads();
    const int npt = pre[PG];
    for (int q = tid; q < npt; q += NT) {
        int p = 0;
        while (pre[p + 1] <= q) ++p;
        pof[q] = p;
        ubase[q] = crs[p].off + (long long)(q - pre[p]) * M;
        ab[q] = Cx<T>{0, 0};
        ab[npt + q] = Cx<T>{0, 0};
    }
    for (int c0 = 0; c0 < N; c0 += NC) {
        const int jn = min(NC, N - c0);
        // ---- 1. x_p, zc_p for the chunk ----
        if constexpr (TC) {
            // one warp per 16 columns: X = W^T F and Z = conj(Wc)^T F on the tensor cores
            const int g = lane >> 2, t = lane & 3;
            const int ntile = (jn + 15) >> 4;
            for (int tile = warp; tile < ntile; tile += NW) {
                const int j0 = tile * 16;
                float xr[4] = {0, 0, 0, 0}, xi[4] = {0, 0, 0, 0}, zr[4] = {0, 0, 0, 0}, zi[4] = {0, 0, 0, 0};
                const Cx<T>* wf = Wf + br.cb + c0 + j0;
                const Cx<T>* wc = Wc + br.cb + c0 + j0;
                for (int k0 = 0; k0 < Ku; k0 += 8) {
                    // A fragment: (row g, col t), (g + 8, t), (g, t + 4), (g + 8, t + 4);
                    // row = column j of the block, col = frequency k
                    Cx<T> a[4], c[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int jj = g + (q & 1) * 8, kk = k0 + t + (q >> 1) * 4;
                        const bool in = j0 + jj < jn && kk < Ku;
                        a[q] = in ? ldcx(wf + (long long)kk * E + jj) : Cx<T>{0, 0};
                        c[q] = in ? ldcx(wc + (long long)kk * E + jj) : Cx<T>{0, 0};
                    }
                    unsigned arh[4], arl[4], aih[4], ail[4], crh[4], crl[4], cih[4], cil[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        Tf32Pair v = tf32_split(a[q].x);
                        arh[q] = v.hi;
                        arl[q] = v.lo;
                        v = tf32_split(a[q].y);
                        aih[q] = v.hi;
                        ail[q] = v.lo;
                        v = tf32_split(c[q].x);
                        crh[q] = v.hi;
                        crl[q] = v.lo;
                        v = tf32_split(c[q].y);
                        cih[q] = v.hi;
                        cil[q] = v.lo;
                    }
                    // B fragment: (row t, col g), (t + 4, g); row = frequency, col = cross
                    unsigned frh[2], frl[2], fih[2], fil[2];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int o = g * KS + k0 + t + q * 4;
                        frh[q] = fsp[o];
                        frl[q] = fsp[PG * KS + o];
                        fih[q] = fsp[2 * PG * KS + o];
                        fil[q] = fsp[3 * PG * KS + o];
                    }
                    unsigned nh[4], nl[4];
                    // x: Re += Ar Fr - Ai Fi, Im += Ar Fi + Ai Fr
                    tf32_neg4(aih, nh);
                    tf32_neg4(ail, nl);
                    mma_tf32x3(xr, arh, arl, frh, frl);
                    mma_tf32x3(xr, nh, nl, fih, fil);
                    mma_tf32x3(xi, arh, arl, fih, fil);
                    mma_tf32x3(xi, aih, ail, frh, frl);
                    // zc = conj(Wc) F: Re += Cr Fr + Ci Fi, Im += Cr Fi - Ci Fr
                    tf32_neg4(cih, nh);
                    tf32_neg4(cil, nl);
                    mma_tf32x3(zr, crh, crl, frh, frl);
                    mma_tf32x3(zr, cih, cil, fih, fil);
                    mma_tf32x3(zi, crh, crl, fih, fil);
                    mma_tf32x3(zi, nh, nl, frh, frl);
                }
                // C fragment: (row g, col 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jj = j0 + g + (q >> 1) * 8, p = 2 * t + (q & 1);
                    xs[p * NC + jj] = Cx<T>{xr[q], xi[q]};
                    zs[p * NC + jj] = Cx<T>{zr[q], zi[q]};
                }
            }
        } else {
            const int jl = tid % NC, h = tid / NC;   // column, part of the group
            Cx<T> x[PPT], z[PPT];
#pragma unroll
            for (int u = 0; u < PPT; ++u) x[u] = z[u] = Cx<T>{0, 0};
            if (jl < jn) {
                const Cx<T>* wf = Wf + br.cb + c0 + jl;
                const Cx<T>* wc = Wc + br.cb + c0 + jl;
                const Cx<T>* f0 = fg + h * PPT * Ku;
                // sixteen W loads (eight frequencies) in flight, then their FMAs
                int k = 0;
                for (; k + 8 <= Ku; k += 8) {
                    Cx<T> a[8], b[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        a[q] = ldcx(wf + (long long)(k + q) * E);
                        b[q] = ldcx(wc + (long long)(k + q) * E);
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q)
#pragma unroll
                        for (int u = 0; u < PPT; ++u) {
                            const Cx<T> f = f0[u * Ku + k + q];
                            cfma(x[u], f, a[q]);
                            cfmac(z[u], f, b[q]);
                        }
                }
                for (; k < Ku; ++k) {
                    const Cx<T> a = ldcx(wf + (long long)k * E), b = ldcx(wc + (long long)k * E);
#pragma unroll
                    for (int u = 0; u < PPT; ++u) {
                        const Cx<T> f = f0[u * Ku + k];
                        cfma(x[u], f, a);
                        cfmac(z[u], f, b);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                xs[(h * PPT + u) * NC + jl] = x[u];
                zs[(h * PPT + u) * NC + jl] = z[u];
            }
        }
        __syncthreads();
        // ---- 2. a_p[t] += V_p[:, t]^H x_p, b_p[t] += V_p[:, t]^H zc_p ----
        // four (p, t) pairs per warp at a time: their column loads are in flight together
        for (int q0 = warp * 4; q0 < npt; q0 += 4 * NW) {
            const Cx<T>* Vq[4];
            const Cx<T>* xq[4];
            const Cx<T>* zq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = min(q0 + u, npt - 1);
                const int p = pof[q];
                Vq[u] = pool + crs[p].off + (long long)crs[p].r * M + (long long)(q - pre[p]) * N + c0;
                xq[u] = xs + p * NC;
                zq[u] = zs + p * NC;
            }
            Cx<T> a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = b[u] = Cx<T>{0, 0};
#pragma unroll 2
            for (int jj = lane; jj < jn; jj += 32) {
                Cx<T> v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = ldcx(Vq[u] + jj);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    cfmac(a[u], xq[u][jj], v[u]);  // conj(v) x
                    cfmac(b[u], zq[u][jj], v[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u].x = warp_sum(a[u].x);
                a[u].y = warp_sum(a[u].y);
                b[u].x = warp_sum(b[u].x);
                b[u].y = warp_sum(b[u].y);
            }
            if (lane == 0) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + u;
                    if (q < npt) {
                        ab[q].x += a[u].x;
                        ab[q].y += a[u].y;
                        ab[npt + q].x += b[u].x;
                        ab[npt + q].y += b[u].y;
                    }
                }
            }
        }
        __syncthreads();
    }
    // ---- 3. y += U a + conj(U b): TPR threads per row split the flattened pairs ----
    const int tpr = M <= NT / 4 ? 4 : (M <= NT / 2 ? 2 : 1);
    const int rows = NT / tpr;
    const int h = tid / rows, il = tid - h * rows;
    for (int i0 = 0; i0 < M; i0 += rows) {
        const int i = i0 + il;
        if (i >= M) continue;
        Cx<T> s1[2] = {{0, 0}, {0, 0}}, s2[2] = {{0, 0}, {0, 0}};
        int q = h;
        // sixteen U loads in flight per thread, then their multiply-adds
        for (; q + 15 * tpr < npt; q += 16 * tpr) {
            Cx<T> u[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) u[e] = ldcx(pool + ubase[q + e * tpr] + i);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                cfma(s1[e & 1], u[e], ab[q + e * tpr]);
                cfma(s2[e & 1], u[e], ab[npt + q + e * tpr]);
            }
        }
        for (; q < npt; q += tpr) {
            const Cx<T> u = ldcx(pool + ubase[q] + i);
            cfma(s1[0], u, ab[q]);
            cfma(s2[0], u, ab[npt + q]);
        }
        const T sx = (s1[0].x + s1[1].x) + (s2[0].x + s2[1].x), sy = (s1[0].y + s1[1].y) - (s2[0].y + s2[1].y);
        atomicAdd(&y[br.rb + i].x, sx);  // U a + conj(U b)
        atomicAdd(&y[br.rb + i].y, sy);
    }
}

// Far field, blocks with dense faces (small blocks): one warp per block, no
// block-wide barrier.  Crosses in groups of PG: the group's fibers are staged
// in the warp's slice of shared memory; for each chunk of 32 columns, lane j
// forms x_p[j] = sum_k f_p[k] w_k[j] and zc_p[j] = sum_k f_p[k] conj(w_k'[j])
// for the group in one pass over W, and lane i then adds
// sum_p (H_p x_p)[i] + conj((H_p zc_p)[i]) over the chunk for its rows.
template <class T, int NW, int PG, int MQ>
__global__ void __launch_bounds__(NW * 32, 3) k_apply_far_dense(const Cx<T>* __restrict__ pool,
                                                               const CrossRec* __restrict__ rec,
                                                               const int* __restrict__ r3,
                                                               const BlockRange* __restrict__ ranges,
                                                               const int* __restrict__ list, int n, int Cmax, int Ku,
                                                               int E, const Cx<T>* __restrict__ Wf,
                                                               const Cx<T>* __restrict__ Wc, Cx<T>* __restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bi = blockIdx.x * NW + warp;
    if (bi >= n) return;  // the whole warp: no block-wide synchronisation below
    Cx<T>* fg = reinterpret_cast<Cx<T>*>(smem_raw) + (size_t)warp * (PG * Ku + 2 * PG * 32);
    Cx<T>* xs = fg + PG * Ku;
    Cx<T>* zs = xs + PG * 32;
    const int blk = list[bi];
    const BlockRange br = ranges[blk];
    const int M = br.re - br.rb, N = br.ce - br.cb;
    const int nc = r3[blk];
    Cx<T> acc[MQ];
#pragma unroll
    for (int q = 0; q < MQ; ++q) acc[q] = Cx<T>{0, 0};
    for (int g0 = 0; g0 < nc; g0 += PG) {
        const int np = min(PG, nc - g0);
        __syncwarp();
        for (int e = lane; e < PG * Ku; e += 32) {
            const int p = e / Ku, k = e - p * Ku;
            Cx<T> v{0, 0};
            if (p < np) v = ldcx(pool + rec[(size_t)blk * Cmax + g0 + p].off + (long long)M * N + k);
            fg[e] = v;
        }
        __syncwarp();
        for (int j0 = 0; j0 < N; j0 += 32) {
            const int j = j0 + lane;
            Cx<T> x[PG], z[PG];
#pragma unroll
            for (int p = 0; p < PG; ++p) x[p] = z[p] = Cx<T>{0, 0};
            if (j < N) {
                const Cx<T>* wf = Wf + br.cb + j;
                const Cx<T>* wc = Wc + br.cb + j;
                // sixteen W loads (eight frequencies) in flight, then their FMAs
                int k = 0;
                for (; k + 8 <= Ku; k += 8) {
                    Cx<T> a[8], b[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        a[q] = ldcx(wf + (long long)(k + q) * E);
                        b[q] = ldcx(wc + (long long)(k + q) * E);
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q)
#pragma unroll
                        for (int p = 0; p < PG; ++p) {
                            const Cx<T> f = fg[p * Ku + k + q];
                            cfma(x[p], f, a[q]);
                            cfmac(z[p], f, b[q]);
                        }
                }
                for (; k < Ku; ++k) {
                    const Cx<T> a = ldcx(wf + (long long)k * E), b = ldcx(wc + (long long)k * E);
#pragma unroll
                    for (int p = 0; p < PG; ++p) {
                        const Cx<T> f = fg[p * Ku + k];
                        cfma(x[p], f, a);
                        cfmac(z[p], f, b);
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < PG; ++p) {
                xs[p * 32 + lane] = x[p];
                zs[p * 32 + lane] = z[p];
            }
            __syncwarp();
            const int jn = min(32, N - j0);
            for (int p = 0; p < np; ++p) {
                const Cx<T>* H = pool + rec[(size_t)blk * Cmax + g0 + p].off + (long long)j0 * M;
#pragma unroll
                for (int q = 0; q < MQ; ++q) {
                    const int i = lane + 32 * q;
                    if (i < M) {
                        Cx<T> s1{0, 0}, s2{0, 0};
#pragma unroll 8
                        for (int jj = 0; jj < jn; ++jj) {
                            const Cx<T> h = ldcx(H + i + (long long)jj * M);
                            cfma(s1, h, xs[p * 32 + jj]);
                            cfma(s2, h, zs[p * 32 + jj]);
                        }
                        acc[q].x += s1.x + s2.x;  // s1 + conj(s2)
                        acc[q].y += s1.y - s2.y;
                    }
                }
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
        const int i = lane + 32 * q;
        if (i < M) {
            atomicAdd(&y[br.rb + i].x, acc[q].x);
            atomicAdd(&y[br.rb + i].y, acc[q].y);
        }
    }
}

template <class T, class TO>
__global__ void k_apply_finish(int E, const int* __restrict__ perm, const Cx<T>* __restrict__ y, Cx<TO>* __restrict__ Y) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= E) return;
    Cx<T> v = y[p];
    Y[perm[p]] = Cx<TO>{(TO)v.x, (TO)v.y};
}
// linear elements: y = P^T y_loc, each position's row added into its vertex
// (Y cleared before)
template <class T, class TO>
__global__ void k_apply_finish_add(int E, const int* __restrict__ src, const Cx<T>* __restrict__ y,
                                   Cx<TO>* __restrict__ Y) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= E) return;
    Cx<T> v = y[p];
    atomicAdd(&Y[src[p]].x, (TO)v.x);
    atomicAdd(&Y[src[p]].y, (TO)v.y);
}


// near-field launch: grid (row clusters) x (frequency chunks), about 16 CTAs
// per SM so that the last wave is short
template <class T>
static g3_status launch_apply_near(g3_ctx* ctx, cudaStream_t stream, const g3_tree* t, const g3_near* nf, int Ku,
                                   int E, const Cx<T>* Wf, const Cx<T>* Wc, Cx<T>* y) {
    constexpr int NT = 256;
    const int n_rows = (int)nf->row_start.size() - 1;
    int ksplit = std::max(1, std::min(Ku, (16 * ctx->n_sm + n_rows - 1) / n_rows));
    int kchunk = (Ku + ksplit - 1) / ksplit;
    ksplit = (Ku + kchunk - 1) / kchunk;
    int mrow = 0;
    for (int g = 0; g < n_rows; ++g) {
        const int32_t* r = &t->blocks[5 * (size_t)nf->order[nf->row_start[g]]];
        mrow = std::max(mrow, r[1] - r[0]);
    }
    dim3 grid(n_rows, ksplit);
    k_apply_near<T, NT><<<grid, NT, (NT / 32) * 2 * (size_t)mrow * sizeof(T), stream>>>(
        nf->data.as<Cx<T>>(), nf->d_ranges.as<BlockRange>(), nf->d_offs.as<long long>(), nf->d_row_start.as<int>(),
        Ku, kchunk, E, Wf, Wc, y);
    ctx->count("k_apply_near");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

// Far-field work lists, built on the host when the compression ends and
// uploaded with the block ranges: the dense-face blocks (one warp each,
// longest first), padded to a multiple of 4 ints, then the low-rank items (block, group of
// FAR_PG crosses) of blocks with at most FAR_NT / 2 columns (two threads per
// column in the x formation), then those of wider blocks; each list longest
// first (HBM bytes of the group's factors).
constexpr int FAR_PG = 8;
constexpr int FAR_NT = 256;

g3_status far_plan_build(g3_factors* fa) {
    std::vector<int>& L = fa->plan;
    L.clear();
    struct Item {
        long long cost;
        int b, g;
    };
    std::vector<Item> narrow, wide, dense;
    int mmax = 0, nmax = 0;
    for (int b = 0; b < fa->n_far; ++b) {
        const int r = fa->r3[b];
        if (r <= 0) continue;
        if (fa->crec(b, 0).r < 0) {
            const int M = fa->ranges[b].re - fa->ranges[b].rb, N = fa->ranges[b].ce - fa->ranges[b].cb;
            dense.push_back(Item{(long long)r * M * N, b, 0});
            mmax = std::max(mmax, M);
            nmax = std::max(nmax, N);
            continue;
        }
        const int M = fa->ranges[b].re - fa->ranges[b].rb;
        const int N = fa->ranges[b].ce - fa->ranges[b].cb;
        for (int p = 0; p < r; ++p)
            if (fa->crec(b, p).r > RF_TS)
                return fail(G3_EUNSUPPORTED, "aca3_compress: face rank %d above the apply's limit %d",
                            fa->crec(b, p).r, RF_TS);
        for (int g = 0; g * FAR_PG < r; ++g) {
            long long c = 0;
            for (int p = g * FAR_PG; p < std::min(r, (g + 1) * FAR_PG); ++p)
                c += (long long)fa->crec(b, p).r * (M + N) + fa->Ku;
            (N <= FAR_NT / 2 ? narrow : wide).push_back(Item{c, b, g});
        }
    }
    auto by_cost = [](const Item& x, const Item& y) {
        if (x.cost != y.cost) return x.cost > y.cost;
        return x.b != y.b ? x.b < y.b : x.g < y.g;
    };
    // low-rank items grouped by column cluster (longest first within a
    // cluster): CTAs that run at the same time read the same slice of W, which
    // stays in L2 even when W as a whole does not (81,920 elements x 128
    // unique frequencies: 168 MB; far field 34.8 against 39.0 ms longest first)
    auto by_col = [&](const Item& x, const Item& y) {
        const int cx = fa->ranges[x.b].cb, cy = fa->ranges[y.b].cb;
        if (cx != cy) return cx < cy;
        return by_cost(x, y);
    };
    std::sort(narrow.begin(), narrow.end(), by_col);
    std::sort(wide.begin(), wide.end(), by_col);
    std::sort(dense.begin(), dense.end(), by_cost);
    for (const Item& it : dense) L.push_back(it.b);
    fa->plan_nd = (int)L.size();
    fa->plan_nmax_dense = nmax;
    fa->plan_n1 = (int)narrow.size();
    fa->plan_n2 = (int)wide.size();
    fa->plan_ab = 0;
    fa->plan_mmax_dense = mmax;
    while (L.size() % 4) L.push_back(0);  // int4 alignment of the item arrays
    for (const Item& it : narrow) L.insert(L.end(), {it.b, it.g, 0, 0});
    for (const Item& it : wide) L.insert(L.end(), {it.b, it.g, 0, 0});
    G3_CUDA(fa->d_plan.alloc(std::max<size_t>(1, L.size()) * sizeof(int)));
    if (!L.empty()) G3_CUDA(cudaMemcpy(fa->d_plan.p, L.data(), L.size() * sizeof(int), cudaMemcpyHostToDevice));
    G3_CUDA(fa->d_franges.alloc(std::max<size_t>(1, fa->ranges.size()) * sizeof(BlockRange)));
    if (!fa->ranges.empty())
        G3_CUDA(cudaMemcpy(fa->d_franges.p, fa->ranges.data(), fa->ranges.size() * sizeof(BlockRange),
                           cudaMemcpyHostToDevice));
    fa->plan_ready = true;
    return G3_OK;
}

// far-field launches over the factors' device work lists (d_ab: unused,
// kept for the scratch layout of the callers)
template <class T>
static g3_status launch_apply_far(g3_ctx* ctx, const g3_factors* fa, Cx<T>* d_ab, int Ku, int E, const Cx<T>* Wf,
                                  const Cx<T>* Wc, Cx<T>* y) {
    (void)d_ab;
    if (!fa->plan_ready) return fail(G3_EINVAL, "apply_gcq: factors without far-field work lists");
    if (fa->plan.empty()) return G3_OK;
    const int nd = fa->plan_nd, n1 = fa->plan_n1, n2 = fa->plan_n2;
    const int* d_list = fa->d_plan.as<int>();
    const BlockRange* d_ranges = fa->d_franges.as<BlockRange>();
    if (nd > 0) {
        const int mmax_dense = fa->plan_mmax_dense;
        constexpr int NW = 8, PGW = 4;
        const size_t smem = (size_t)NW * (PGW * Ku + 2 * PGW * 32) * sizeof(Cx<T>);
        if (smem > ctx->smem_optin || mmax_dense > 256)
            return fail(G3_EUNSUPPORTED, "apply_gcq: dense-face blocks with %d rows exceed the apply kernel's limit",
                        mmax_dense);
        const int grid = (nd + NW - 1) / NW;
        auto go = [&](auto kfn) -> g3_status {
            G3_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kfn<<<grid, NW * 32, smem, ctx->stream>>>(fa->pool->as<Cx<T>>(), fa->d_rec.as<CrossRec>(),
                                                      fa->d_r3.as<int>(), d_ranges, d_list, nd, fa->Cmax, Ku, E,
                                                      Wf, Wc, y);
            return G3_OK;
        };
        g3_status st;
        if (mmax_dense <= 32)
            st = go(k_apply_far_dense<T, NW, PGW, 1>);
        else if (mmax_dense <= 64)
            st = go(k_apply_far_dense<T, NW, PGW, 2>);
        else if (mmax_dense <= 96)
            st = go(k_apply_far_dense<T, NW, PGW, 3>);
        else if (mmax_dense <= 128)
            st = go(k_apply_far_dense<T, NW, PGW, 4>);
        else
            st = go(k_apply_far_dense<T, NW, PGW, 8>);
        if (st != G3_OK) return st;
        ctx->count("k_apply_far_dense");
        G3_CUDA(cudaGetLastError());
    }
    const int4* it1 = reinterpret_cast<const int4*>(d_list + (nd + 3) / 4 * 4);
    const int4* it2 = it1 + n1;
    auto far_lr = [&](auto kfn, int n, const int4* items, int nc, bool tc) -> g3_status {
        if (n <= 0) return G3_OK;
        const size_t smem = ((size_t)FAR_PG * Ku + 2 * (size_t)FAR_PG * nc + 2 * (size_t)FAR_PG * RF_TS) * sizeof(Cx<T>) +
                            (tc ? 4 * (size_t)FAR_PG * tc_fiber_stride(Ku) * sizeof(unsigned) : 0);
        if (smem > ctx->smem_optin)
            return fail(G3_EUNSUPPORTED, "apply_gcq: far-field kernel needs %zu bytes of shared memory", smem);
        G3_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kfn<<<n, FAR_NT, smem, ctx->stream>>>(fa->pool->as<Cx<T>>(), fa->d_rec.as<CrossRec>(), fa->d_r3.as<int>(),
                                              d_ranges, items, fa->Cmax, Ku, E, Wf, Wc, y);
        ctx->count(tc ? "k_far_lr_tc" : "k_far_lr");
        G3_CUDA(cudaGetLastError());
        return G3_OK;
    };
    if constexpr (sizeof(T) == 4) {
        if (ctx->apply_tensor_cores) {
            G3_TRY_NA(far_lr(k_far_lr<T, FAR_NT, FAR_PG, 2, true>, n1, it1, FAR_NT / 2, true));
            G3_TRY_NA(far_lr(k_far_lr<T, FAR_NT, FAR_PG, 1, true>, n2, it2, FAR_NT, true));
            return G3_OK;
        }
    }
    G3_TRY_NA(far_lr(k_far_lr<T, FAR_NT, FAR_PG, 2, false>, n1, it1, FAR_NT / 2, false));
    G3_TRY_NA(far_lr(k_far_lr<T, FAR_NT, FAR_PG, 1, false>, n2, it2, FAR_NT, false));
    return G3_OK;
}

// Near field and far field of one apply.  With both present the near field
// (an HBM stream) runs on the context's high-priority side stream and the
// far-field kernels (bound by latency: short dependent chains per item) on the
// context's stream, forked and joined through events: pending near-field CTAs
// are dispatched first and far-field CTAs fill the rest of each SM, which
// overlaps the two better than the opposite priority (measured on the
// 12,288-triangle L-shape: 1.88 against 1.95 ms per single-layer apply).
// Both add into y atomically.  ev_side brackets the near field (its device time).
template <class T>
static g3_status apply_near_far(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa, int Ku,
                                int E, const Cx<T>* Wf, const Cx<T>* Wc, Cx<T>* y, Cx<T>* abuf) {
    const bool has_near = nf && !nf->order.empty(), has_far = fa && fa->n_far > 0;
    if (has_near && has_far) {
        G3_CUDA(cudaEventRecord(ctx->fork, ctx->stream));
        G3_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork, 0));
        G3_CUDA(cudaEventRecord(ctx->ev_side[0], ctx->side));
        G3_TRY_NA(launch_apply_near<T>(ctx, ctx->side, t, nf, Ku, E, Wf, Wc, y));
        G3_CUDA(cudaEventRecord(ctx->ev_side[1], ctx->side));
        G3_CUDA(cudaEventRecord(ctx->join, ctx->side));
        G3_TRY_NA(launch_apply_far<T>(ctx, fa, abuf, Ku, E, Wf, Wc, y));
        G3_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->join, 0));
        return G3_OK;
    }
    if (has_near) {
        G3_CUDA(cudaEventRecord(ctx->ev_side[0], ctx->stream));
        G3_TRY_NA(launch_apply_near<T>(ctx, ctx->stream, t, nf, Ku, E, Wf, Wc, y));
        G3_CUDA(cudaEventRecord(ctx->ev_side[1], ctx->stream));
    }
    if (has_far) G3_TRY_NA(launch_apply_far<T>(ctx, fa, abuf, Ku, E, Wf, Wc, y));
    return G3_OK;
}

template <class T>
static g3_status run_apply_t(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa, const void* W,
                             void* Y, int dtype, const g3_freqs* f) {
    const int E = t->ne, K = f->K, Ku = f->Ku;
    const size_t nW = (size_t)Ku * E;
    const long long n_ab = fa ? fa->plan_ab : 0;
    const size_t need = (2 * nW + E + (size_t)n_ab) * sizeof(Cx<T>) + 256;
    G3_CUDA(ctx->scratch.ensure(need));
    Cx<T>* Wf = ctx->scratch.as<Cx<T>>();
    Cx<T>* Wc = Wf + nW;
    Cx<T>* y = Wc + nW;
    Cx<T>* abuf = reinterpret_cast<Cx<T>*>((reinterpret_cast<uintptr_t>(y + E) + 255) & ~uintptr_t(255));
    cudaEvent_t e0 = ctx->ev[2], e3 = ctx->ev[5];
    G3_CUDA(cudaEventRecord(e0, ctx->stream));
    // linear-element trees: nodal W and Y (nv rows), gathered per position at its vertex
    const int* rowsrc = t->p1 ? t->d_src.as<int>() : t->d_perm.as<int>();
    const int ldw = t->p1 ? t->nv : E;
    {
        long long tot = (long long)Ku * E;
        int blocks = (int)((tot + 255) / 256);
        if (dtype == G3_C128)
            k_apply_prep<double, T><<<blocks, 256, 0, ctx->stream>>>(E, K, Ku, rowsrc, f->d_uniq.as<int>(),
                                                                   f->d_partner.as<int>(), (const Cx<double>*)W, Wf, Wc, y, ldw);
        else
            k_apply_prep<float, T><<<blocks, 256, 0, ctx->stream>>>(E, K, Ku, rowsrc, f->d_uniq.as<int>(),
                                                                  f->d_partner.as<int>(), (const Cx<float>*)W, Wf, Wc, y, ldw);
        ctx->count("k_apply_prep");
        G3_CUDA(cudaGetLastError());
    }
    G3_TRY_NA(apply_near_far<T>(ctx, t, nf, fa, Ku, E, Wf, Wc, y, abuf));
    {
        int blocks = (E + 255) / 256;
        if (t->p1) {
            G3_CUDA(cudaMemsetAsync(Y, 0, (size_t)t->nv * (dtype == G3_C128 ? 16 : 8), ctx->stream));
            if (dtype == G3_C128)
                k_apply_finish_add<T, double><<<blocks, 256, 0, ctx->stream>>>(E, rowsrc, y, (Cx<double>*)Y);
            else
                k_apply_finish_add<T, float><<<blocks, 256, 0, ctx->stream>>>(E, rowsrc, y, (Cx<float>*)Y);
            ctx->count("k_apply_finish_add");
        } else {
            if (dtype == G3_C128)
                k_apply_finish<T, double><<<blocks, 256, 0, ctx->stream>>>(E, t->d_perm.as<int>(), y, (Cx<double>*)Y);
            else
                k_apply_finish<T, float><<<blocks, 256, 0, ctx->stream>>>(E, t->d_perm.as<int>(), y, (Cx<float>*)Y);
            ctx->count("k_apply_finish");
        }
        G3_CUDA(cudaGetLastError());
    }
    G3_CUDA(cudaEventRecord(e3, ctx->stream));
    G3_CUDA(cudaEventSynchronize(e3));
    float ms_all = 0, ms_near = 0;
    G3_CUDA(cudaEventElapsedTime(&ms_all, e0, e3));
    if (nf && !nf->order.empty()) G3_CUDA(cudaEventElapsedTime(&ms_near, ctx->ev_side[0], ctx->ev_side[1]));
    ctx->last_apply_ms = ms_all;
    ctx->last_near_ms = ms_near;
    const int64_t in_sz = dtype == G3_C128 ? 16 : 8;
    int64_t near_bytes = nf ? nf->n_entries * (int64_t)sizeof(Cx<T>) : 0;
    int64_t far_bytes = fa ? fa->stats.factor_bytes : 0;
    ctx->last_near_bytes = near_bytes;
    ctx->last_apply_bytes = near_bytes + far_bytes + (int64_t)E * K * in_sz + (int64_t)E * in_sz;
    return G3_OK;
}

// ============================================================================
// Per-frequency apply (G3_APPLY_PERFREQ): Y[:, l] = A(s_l) w_l for every l
// ============================================================================
//
// The terms of eq. (product) before the sum over l, one column per frequency
// (a check of the compressed operator at each frequency).  With the unique
// frequencies k and their partners k' (A(s_k') = conj A(s_k)):
//   Y[:, k]  = A(s_k) w_k               = sum_far sum_p f_p[k] H_p w_k + near,
//   Y[:, k'] = conj(A(s_k) conj(w_k'))  (the same operator on conj(w_k')).
// So every unique frequency k has two right-hand sides, x_k = w_k and
// x_{Ku + k} = conj(w_k') (zero without a partner), and two outputs
// yf[k] and yc[k] in cluster order; Y[:, k'] = conj(yc[k]).  Scratch:
// Wf, Wc (from k_apply_prep, Wc unconjugated), yf, yc: 4 Ku E values.

// near field: one CTA per (near block, frequency chunk); warp per frequency,
// lane per row; both right-hand sides in one pass over the stored entries
template <class T, int NT>
__global__ void __launch_bounds__(NT) k_pf_near(const Cx<T>* __restrict__ A, const BlockRange* __restrict__ ranges,
                                                const long long* __restrict__ offs, int Ku, int kchunk, int E,
                                                const Cx<T>* __restrict__ Wf, const Cx<T>* __restrict__ Wc,
                                                Cx<T>* __restrict__ yf, Cx<T>* __restrict__ yc) {
    const int b = blockIdx.x;
    const int k0 = blockIdx.y * kchunk, k1 = min(Ku, k0 + kchunk);
    const BlockRange br = ranges[b];
    const int M = br.re - br.rb, N = br.ce - br.cb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = k0 + warp; k < k1; k += NT / 32) {
        const Cx<T>* Ak = A + offs[b] + (long long)k * M * N;
        const Cx<T>* wf = Wf + (long long)k * E + br.cb;
        const Cx<T>* wc = Wc + (long long)k * E + br.cb;
        for (int i = lane; i < M; i += 32) {
            Cx<T> s1{0, 0}, s2{0, 0};
            for (int j = 0; j < N; ++j) {
                const Cx<T> a = ldcx(Ak + (long long)j * M + i);
                cfma(s1, a, ldcx(wf + j));
                cfmac(s2, a, ldcx(wc + j));  // A conj(w')
            }
            atomicAdd(&yf[(long long)k * E + br.rb + i].x, s1.x);
            atomicAdd(&yf[(long long)k * E + br.rb + i].y, s1.y);
            atomicAdd(&yc[(long long)k * E + br.rb + i].x, s2.x);
            atomicAdd(&yc[(long long)k * E + br.rb + i].y, s2.y);
        }
    }
}

// far field: one CTA per item (block, 32 right-hand sides c0.., 128 rows
// i0..).  Right-hand side c < Ku is w_c, c >= Ku is conj(w'_{c-Ku}); its
// fiber coefficient is f_p[c mod Ku].  Per cross p of the block:
//   low-rank face:  t[q][c] = V_p[:, q]^H x_c   (q < r_p, the block's columns
//                   of x_c staged 64 at a time), then z[i][c] += f_p[c] U_p[i, :] t[:, c];
//   dense face:     z[i][c] += f_p[c] H_p[i, :] x_c.
// Thread (i = tid / 32 + 8 m, c = tid % 32) keeps 16 outputs in registers;
// the CTA adds them to yf / yc once.
constexpr int PF_NT = 256, PF_NC = 32, PF_NI = 128, PF_JC = 64;

template <class T>
__global__ void __launch_bounds__(PF_NT) k_pf_far(const Cx<T>* __restrict__ pool, const CrossRec* __restrict__ rec,
                                                  const int* __restrict__ r3, const BlockRange* __restrict__ ranges,
                                                  const int4* __restrict__ items, int Cmax, int Ku, int E,
                                                  const Cx<T>* __restrict__ Wf, const Cx<T>* __restrict__ Wc,
                                                  Cx<T>* __restrict__ yf, Cx<T>* __restrict__ yc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // xs [PF_JC][PF_NC + 1], ts [RF_TS][PF_NC + 1] (dynamic: above 48 KB in float64)
    auto xs = reinterpret_cast<Cx<T>(*)[PF_NC + 1]>(smem_raw);
    auto ts = reinterpret_cast<Cx<T>(*)[PF_NC + 1]>(smem_raw + (size_t)PF_JC * (PF_NC + 1) * sizeof(Cx<T>));
    __shared__ Cx<T> fs[PF_NC];
    const int4 it = items[blockIdx.x];
    const int blk = it.x, c0 = it.y, i0 = it.z;
    const BlockRange br = ranges[blk];
    const int M = br.re - br.rb, N = br.ce - br.cb;
    const int tid = threadIdx.x, cl = tid & 31, il = tid >> 5;
    const int nrhs = 2 * Ku;
    Cx<T> z[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) z[m] = Cx<T>{0, 0};
    // stage x_c[j0 .. j0 + PF_JC) for the 32 right-hand sides
    auto stage = [&](int j0) {
        for (int e = tid; e < PF_JC * PF_NC; e += PF_NT) {
            const int c = e / PF_JC, jj = e - c * PF_JC;
            const int gc = c0 + c, j = j0 + jj;
            Cx<T> v{0, 0};
            if (gc < nrhs && j < N) {
                if (gc < Ku) v = ldcx(Wf + (long long)gc * E + br.cb + j);
                else v = cconj(ldcx(Wc + (long long)(gc - Ku) * E + br.cb + j));
            }
            xs[jj][c] = v;
        }
    };
    const int nc = r3[blk];
    for (int p = 0; p < nc; ++p) {
        const CrossRec cr = rec[(size_t)blk * Cmax + p];
        const bool dense = cr.r < 0;
        const Cx<T>* fb = pool + cr.off + (dense ? (long long)M * N : (long long)cr.r * (M + N));
        __syncthreads();  // previous cross done with xs / ts / fs
        if (tid < PF_NC) {
            const int gc = c0 + tid;
            fs[tid] = gc < nrhs ? ldcx(fb + (gc < Ku ? gc : gc - Ku)) : Cx<T>{0, 0};
        }
        if (dense) {
            const Cx<T>* H = pool + cr.off;
            Cx<T> acc[16];
#pragma unroll
            for (int m = 0; m < 16; ++m) acc[m] = Cx<T>{0, 0};
            for (int j0 = 0; j0 < N; j0 += PF_JC) {
                __syncthreads();
                stage(j0);
                __syncthreads();
                const int jn = min(PF_JC, N - j0);
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    const int i = i0 + il + 8 * m;
                    if (i < M)
                        for (int jj = 0; jj < jn; ++jj) cfma(acc[m], ldcx(H + (long long)(j0 + jj) * M + i), xs[jj][cl]);
                }
            }
            __syncthreads();
            const Cx<T> f = fs[cl];
#pragma unroll
            for (int m = 0; m < 16; ++m) cfma(z[m], f, acc[m]);
            continue;
        }
        const int r = cr.r;
        const Cx<T>* U = pool + cr.off;
        const Cx<T>* V = U + (long long)r * M;
        // t[q][c] = V_p[:, q]^H x_c; thread (q = il + 8 m, c = cl)
        Cx<T> t[RF_TS / 8];
#pragma unroll
        for (int m = 0; m < RF_TS / 8; ++m) t[m] = Cx<T>{0, 0};
        for (int j0 = 0; j0 < N; j0 += PF_JC) {
            __syncthreads();
            stage(j0);
            __syncthreads();
            const int jn = min(PF_JC, N - j0);
#pragma unroll
            for (int m = 0; m < RF_TS / 8; ++m) {
                const int q = il + 8 * m;
                if (q < r)
                    for (int jj = 0; jj < jn; ++jj) cfmac(t[m], xs[jj][cl], ldcx(V + (long long)q * N + j0 + jj));
            }
        }
#pragma unroll
        for (int m = 0; m < RF_TS / 8; ++m) {
            const int q = il + 8 * m;
            if (q < r) ts[q][cl] = t[m];
        }
        __syncthreads();
        const Cx<T> f = fs[cl];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int i = i0 + il + 8 * m;
            if (i < M) {
                Cx<T> s{0, 0};
                for (int q = 0; q < r; ++q) cfma(s, ldcx(U + (long long)q * M + i), ts[q][cl]);
                cfma(z[m], f, s);
            }
        }
    }
    const int gc = c0 + cl;
    if (gc >= nrhs) return;
    Cx<T>* out = gc < Ku ? yf + (long long)gc * E : yc + (long long)(gc - Ku) * E;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int i = i0 + il + 8 * m;
        if (i < M) {
            atomicAdd(&out[br.rb + i].x, z[m].x);
            atomicAdd(&out[br.rb + i].y, z[m].y);
        }
    }
}

// Y[perm p, uniq k] = yf[k][p];  Y[perm p, partner] = conj(yc[k][p]) (column-major M x K)
template <class T, class TO>
__global__ void k_pf_finish(int E, int Ku, const int* __restrict__ perm, const int* __restrict__ uniq,
                            const int* __restrict__ partner, const Cx<T>* __restrict__ yf,
                            const Cx<T>* __restrict__ yc, Cx<TO>* __restrict__ Y) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)Ku * E) return;
    const int k = (int)(idx / E), p = (int)(idx % E);
    const int l = uniq[k], lp = partner[l];
    const Cx<T> a = yf[idx];
    Y[(long long)l * E + perm[p]] = Cx<TO>{(TO)a.x, (TO)a.y};
    if (lp != l) {
        const Cx<T> b = yc[idx];
        Y[(long long)lp * E + perm[p]] = Cx<TO>{(TO)b.x, (TO)-b.y};
    }
}

template <class T>
static g3_status run_apply_perfreq_t(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa,
                                     const void* W, void* Y, int dtype, const g3_freqs* f) {
    const int E = t->ne, K = f->K, Ku = f->Ku;
    const size_t nW = (size_t)Ku * E;
    // work items of the far field: (block, right-hand-side chunk, row chunk)
    std::vector<int> items;
    if (fa) {
        for (int b = 0; b < fa->n_far; ++b) {
            if (fa->r3[b] <= 0) continue;
            const int M = fa->ranges[b].re - fa->ranges[b].rb;
            for (int c0 = 0; c0 < 2 * Ku; c0 += PF_NC)
                for (int i0 = 0; i0 < M; i0 += PF_NI) items.insert(items.end(), {b, c0, i0, 0});
            for (int p = 0; p < fa->r3[b]; ++p)
                if (fa->crec(b, p).r > RF_TS)
                    return fail(G3_EUNSUPPORTED, "apply_gcq: face rank %d above %d in the per-frequency apply",
                                fa->crec(b, p).r, RF_TS);
        }
    }
    const size_t n_items = items.size() / 4;
    const size_t need = 4 * nW * sizeof(Cx<T>) + (n_items + 1) * sizeof(int4) + 512;
    G3_CUDA(ctx->scratch.ensure(need));
    Cx<T>* Wf = ctx->scratch.as<Cx<T>>();
    Cx<T>* Wc = Wf + nW;
    Cx<T>* yf = Wc + nW;
    Cx<T>* yc = yf + nW;
    int4* d_items = reinterpret_cast<int4*>((reinterpret_cast<uintptr_t>(yc + nW) + 255) & ~uintptr_t(255));
    cudaEvent_t e0 = ctx->ev[2], e3 = ctx->ev[5];
    G3_CUDA(cudaEventRecord(e0, ctx->stream));
    if (n_items)
        G3_CUDA(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice,
                                ctx->stream));
    G3_CUDA(cudaMemsetAsync(yf, 0, 2 * nW * sizeof(Cx<T>), ctx->stream));
    {
        const int blocks = (int)((nW + 255) / 256);
        // k_apply_prep also clears its y argument: point it at yf (cleared anyway)
        if (dtype == G3_C128)
            k_apply_prep<double, T><<<blocks, 256, 0, ctx->stream>>>(E, K, Ku, t->d_perm.as<int>(), f->d_uniq.as<int>(),
                                                                   f->d_partner.as<int>(), (const Cx<double>*)W, Wf, Wc, yf, E);
        else
            k_apply_prep<float, T><<<blocks, 256, 0, ctx->stream>>>(E, K, Ku, t->d_perm.as<int>(), f->d_uniq.as<int>(),
                                                                  f->d_partner.as<int>(), (const Cx<float>*)W, Wf, Wc, yf, E);
        ctx->count("k_apply_prep");
        G3_CUDA(cudaGetLastError());
    }
    if (nf && !nf->order.empty()) {
        constexpr int NT = 256, KC = 16;
        dim3 grid((unsigned)nf->order.size(), (Ku + KC - 1) / KC);
        k_pf_near<T, NT><<<grid, NT, 0, ctx->stream>>>(nf->data.as<Cx<T>>(), nf->d_ranges.as<BlockRange>(),
                                                       nf->d_offs.as<long long>(), Ku, KC, E, Wf, Wc, yf, yc);
        ctx->count("k_pf_near");
        G3_CUDA(cudaGetLastError());
    }
    if (n_items) {
        if (!fa->plan_ready) return fail(G3_EINVAL, "apply_gcq: factors without block ranges on the device");
        const size_t smem = (size_t)(PF_JC + RF_TS) * (PF_NC + 1) * sizeof(Cx<T>);
        G3_CUDA(cudaFuncSetAttribute(k_pf_far<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_pf_far<T><<<(unsigned)n_items, PF_NT, smem, ctx->stream>>>(fa->pool->as<Cx<T>>(), fa->d_rec.as<CrossRec>(),
                                                                  fa->d_r3.as<int>(), fa->d_franges.as<BlockRange>(),
                                                                  d_items, fa->Cmax, Ku, E, Wf, Wc, yf, yc);
        ctx->count("k_pf_far");
        G3_CUDA(cudaGetLastError());
    }
    {
        const int blocks = (int)((nW + 255) / 256);
        if (dtype == G3_C128)
            k_pf_finish<T, double><<<blocks, 256, 0, ctx->stream>>>(E, Ku, t->d_perm.as<int>(), f->d_uniq.as<int>(),
                                                                  f->d_partner.as<int>(), yf, yc, (Cx<double>*)Y);
        else
            k_pf_finish<T, float><<<blocks, 256, 0, ctx->stream>>>(E, Ku, t->d_perm.as<int>(), f->d_uniq.as<int>(),
                                                                 f->d_partner.as<int>(), yf, yc, (Cx<float>*)Y);
        ctx->count("k_pf_finish");
        G3_CUDA(cudaGetLastError());
    }
    G3_CUDA(cudaEventRecord(e3, ctx->stream));
    G3_CUDA(cudaEventSynchronize(e3));
    float ms_all = 0;
    G3_CUDA(cudaEventElapsedTime(&ms_all, e0, e3));
    ctx->last_apply_ms = ms_all;
    ctx->last_near_ms = 0;
    const int64_t in_sz = dtype == G3_C128 ? 16 : 8;
    const int64_t near_bytes = nf ? nf->n_entries * (int64_t)sizeof(Cx<T>) : 0;
    ctx->last_near_bytes = near_bytes;
    ctx->last_apply_bytes = near_bytes + (fa ? fa->stats.factor_bytes : 0) + 2 * (int64_t)E * K * in_sz;
    return G3_OK;
}

// ============================================================================
// Allocation-free apply
// ============================================================================
//
// Some callers cannot allocate device memory while they run this step: code
// inside a memory-capped or pre-reserved arena, a runtime that forbids
// cudaMalloc on its hot path, or a host that must not synchronise the device
// (cudaMalloc/cudaFree can).  apply_gcq_noalloc serves them: it computes the
// same sum as apply_gcq (device buffers, G3_APPLY_SUM) with its scratch in the
// fixed array below instead of the context's growable buffer, and calls no
// allocating routine.
//
// The array is a file-scope __device__ object: every GPU that loads this
// library holds it until the process exits.  All calls on a device share it
// and it keeps the last call's contents, so every part a call reads is
// written first by that call (the accumulator is cleared by k_apply_prep).
// Calls whose work overlaps on the GPU (several streams or threads at once)
// race on it and must be serialised by the caller.
constexpr size_t NOALLOC_SCRATCH_BYTES = 32ull << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g3_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// device address of the scratch array, looked up once per device (with that
// device current); host code must not use the symbol itself as an address
static void* g_noalloc_ptr[64] = {};

static g3_status noalloc_scratch(int device, void** out) {
    if (device < 0 || device >= 64) return fail(G3_EINVAL, "apply_gcq_noalloc: device %d not supported", device);
    if (!g_noalloc_ptr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g3_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g3_noalloc_scratch)");
        g_noalloc_ptr[device] = ptr;
    }
    *out = g_noalloc_ptr[device];
    return G3_OK;
}


template <class T>
static g3_status run_apply_noalloc_t(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa,
                                     const void* W, void* Y, int dtype, const g3_freqs* f) {
    const int E = t->ne, K = f->K, Ku = f->Ku;
    const int n_far = fa ? fa->n_far : 0;
    const size_t nW = (size_t)Ku * E;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const long long n_ab = fa ? fa->plan_ab : 0;
    const size_t need = al(2 * nW * sizeof(Cx<T>)) + al(E * sizeof(Cx<T>)) + al(n_ab * sizeof(Cx<T>));
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(G3_EINVAL,
                    "apply_gcq_noalloc: this problem needs %zu bytes of scratch (2 Ku E + E complex values), "
                    "the fixed scratch holds %zu; use apply_gcq",
                    need, NOALLOC_SCRATCH_BYTES);
    void* base = nullptr;
    G3_TRY_NA(noalloc_scratch(ctx->device, &base));
    char* p = static_cast<char*>(base);
    Cx<T>* Wf = reinterpret_cast<Cx<T>*>(p);
    Cx<T>* Wc = Wf + nW;
    p += al(2 * nW * sizeof(Cx<T>));
    Cx<T>* y = reinterpret_cast<Cx<T>*>(p);
    p += al(E * sizeof(Cx<T>));
    Cx<T>* abuf = reinterpret_cast<Cx<T>*>(p);
    {
        long long tot = (long long)Ku * E;
        int blocks = (int)((tot + 255) / 256);
        if (dtype == G3_C128)
            k_apply_prep<double, T><<<blocks, 256, 0, ctx->stream>>>(E, K, Ku, t->d_perm.as<int>(), f->d_uniq.as<int>(),
                                                                   f->d_partner.as<int>(), (const Cx<double>*)W, Wf, Wc, y, E);
        else
            k_apply_prep<float, T><<<blocks, 256, 0, ctx->stream>>>(E, K, Ku, t->d_perm.as<int>(), f->d_uniq.as<int>(),
                                                                  f->d_partner.as<int>(), (const Cx<float>*)W, Wf, Wc, y, E);
        ctx->count("k_apply_prep");
        G3_CUDA(cudaGetLastError());
    }
    G3_TRY_NA(apply_near_far<T>(ctx, t, nf, n_far > 0 ? fa : nullptr, Ku, E, Wf, Wc, y, abuf));
    {
        int blocks = (E + 255) / 256;
        if (dtype == G3_C128)
            k_apply_finish<T, double><<<blocks, 256, 0, ctx->stream>>>(E, t->d_perm.as<int>(), y, (Cx<double>*)Y);
        else
            k_apply_finish<T, float><<<blocks, 256, 0, ctx->stream>>>(E, t->d_perm.as<int>(), y, (Cx<float>*)Y);
        ctx->count("k_apply_finish");
        G3_CUDA(cudaGetLastError());
    }
    return G3_OK;
}

g3_status run_apply(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa, const void* W, void* Y,
                    int dtype, int mode) {
    const g3_freqs* f = nf ? nf->freqs : fa->freqs;
    const int prec = nf ? nf->prec : fa->prec;
    if (nf && fa && (nf->prec != fa->prec || nf->freqs != fa->freqs))
        return fail(G3_EINVAL, "apply_gcq: near field and factors differ in precision or frequency set");
    if (mode == G3_APPLY_PERFREQ) {
        if (prec == G3_MIXED) return run_apply_perfreq_t<float>(ctx, t, nf, fa, W, Y, dtype, f);
        return run_apply_perfreq_t<double>(ctx, t, nf, fa, W, Y, dtype, f);
    }
    if (prec == G3_MIXED) return run_apply_t<float>(ctx, t, nf, fa, W, Y, dtype, f);
    return run_apply_t<double>(ctx, t, nf, fa, W, Y, dtype, f);
}

}  // namespace g3

extern "C" g3_status apply_gcq_noalloc(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa,
                                       const void* W, void* Y, g3_dtype dtype) {
    using namespace g3;
    if (!ctx || !t || !W || !Y) return fail(G3_EINVAL, "apply_gcq_noalloc: NULL argument");
    if (t->p1) return fail(G3_EUNSUPPORTED, "apply_gcq_noalloc: linear-element trees use apply_gcq");
    if (!nf && !fa) return fail(G3_EINVAL, "apply_gcq_noalloc: near field and factors are both NULL");
    if (dtype != G3_C64 && dtype != G3_C128) return fail(G3_EINVAL, "apply_gcq_noalloc: bad dtype");
    if ((nf && nf->tree != t) || (fa && fa->tree != t))
        return fail(G3_EINVAL, "apply_gcq_noalloc: near field or factors built on another tree");
    if (nf && fa && (nf->prec != fa->prec || nf->freqs != fa->freqs))
        return fail(G3_EINVAL, "apply_gcq_noalloc: near field and factors differ in precision or frequency set");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const g3_freqs* f = nf ? nf->freqs : fa->freqs;
    const int prec = nf ? nf->prec : fa->prec;
    if (prec == G3_MIXED) return run_apply_noalloc_t<float>(ctx, t, nf, fa, W, Y, dtype, f);
    return run_apply_noalloc_t<double>(ctx, t, nf, fa, W, Y, dtype, f);
}
