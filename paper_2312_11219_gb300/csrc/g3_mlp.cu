// Block rank / first-frequency predictor: a 12 -> 64 -> 64 -> 2 ReLU network
// trained and evaluated on the GPU.
//
// Not part of the paper's method.  The three-way ACA (Algorithm 1) decides
// every block's rank by its own stopping test; the predictor only supplies
// scheduling information before the compression starts:
//   y0 = log2(1 + r3)   -> factor-pool size and the longest-first queue order
//   y1 = k* / K_u       -> the first frequency k1 of the block (Section 3.2
//                          starts at an arbitrary frequency; k* is the
//                          frequency of the largest pivot entry of the block)
//
// Numerics: weights are kept in float32 (master copy, Adam state) and used in
// bfloat16 (rounded to nearest even when loaded into shared memory); inputs
// are standardised in float32, (x - mean) * inv_std, and rounded to bfloat16;
// activations, accumulation, gradients and the Adam update are float32.
//
// Parameter layout (5,122 floats): W1 [64][12], b1 [64], W2 [64][64], b2 [64],
// W3 [2][64], b3 [2], row-major (output index first).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "g3_device.cuh"
#include "g3_internal.h"

namespace g3 {

namespace {

constexpr int NF = G3_MLP_NF, HID = 64, NO = 2;
constexpr int OW1 = 0, OB1 = OW1 + HID * NF, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + NO * HID, NP = OB3 + NO;
static_assert(NP == G3_MLP_NP, "parameter count");
constexpr int CH = 32;   // samples per chunk
constexpr int MT = 256;  // threads per CTA
constexpr int PPT = (NP + MT - 1) / MT;  // parameters owned per thread in the gradient kernel

// shared-memory layout (floats)
constexpr int S_W1T = 0;                    // [12][64]  W1 transposed
constexpr int S_B1 = S_W1T + NF * HID;      // [64]
constexpr int S_W2 = S_B1 + HID;            // [64][64]  W2[u][v]
constexpr int S_W2T = S_W2 + HID * HID;     // [64][64]  W2[u][v] at [v][u]
constexpr int S_B2 = S_W2T + HID * HID;     // [64]
constexpr int S_W3 = S_B2 + HID;            // [2][64]
constexpr int S_B3 = S_W3 + NO * HID;       // [2] (+2 pad)
constexpr int S_X = S_B3 + 4;               // [32][12]
constexpr int S_A1 = S_X + CH * NF;         // [32][64]
constexpr int S_A2 = S_A1 + CH * HID;       // [32][64]
constexpr int S_D2 = S_A2 + CH * HID;       // [32][64]  dL/dz2
constexpr int S_D1 = S_D2 + CH * HID;       // [32][64]  dL/dz1
constexpr int S_Y = S_D1 + CH * HID;        // [32][2]
constexpr int S_DY = S_Y + CH * NO;         // [32][2]
constexpr int S_RED = S_DY + CH * NO;       // [32] loss partials
constexpr int S_TOTAL = S_RED + 32;
constexpr size_t SMEM_BYTES = S_TOTAL * sizeof(float);

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// weights (bfloat16-rounded) into shared memory
__device__ void load_weights(const float* __restrict__ P, float* sh) {
    for (int p = threadIdx.x; p < NP; p += MT) {
        const float w = bf16r(P[p]);
        if (p < OB1) {
            const int u = p / NF, c = p % NF;
            sh[S_W1T + c * HID + u] = w;
        } else if (p < OW2) {
            sh[S_B1 + (p - OB1)] = w;
        } else if (p < OB2) {
            const int q = p - OW2, u = q / HID, v = q % HID;
            sh[S_W2 + q] = w;
            sh[S_W2T + v * HID + u] = w;
        } else if (p < OW3) {
            sh[S_B2 + (p - OB2)] = w;
        } else if (p < OB3) {
            sh[S_W3 + (p - OW3)] = w;
        } else {
            sh[S_B3 + (p - OB3)] = w;
        }
    }
}

// standardised, bfloat16-rounded inputs of one chunk; samples >= n are zero
__device__ void load_chunk(const float* __restrict__ X, long long s0, long long n, const float* __restrict__ mean,
                           const float* __restrict__ inv_std, float* sh) {
    for (int e = threadIdx.x; e < CH * NF; e += MT) {
        const int s = e / NF, c = e % NF;
        const long long g = s0 + s;
        float x = 0.f;
        if (g < n) {
            const float d = __fsub_rn(X[g * NF + c], mean[c]);
            x = bf16r(__fmul_rn(d, inv_std[c]));
        }
        sh[S_X + e] = x;
    }
}

// forward pass of one chunk: a1, a2 (post-ReLU) and y
__device__ void forward_chunk(float* sh) {
    const int t = threadIdx.x, u = t & (HID - 1), s0 = t >> 6;
    for (int s = s0; s < CH; s += MT / HID) {
        float z = sh[S_B1 + u];
#pragma unroll
        for (int c = 0; c < NF; ++c) z = fmaf(sh[S_W1T + c * HID + u], sh[S_X + s * NF + c], z);
        sh[S_A1 + s * HID + u] = fmaxf(z, 0.f);
    }
    __syncthreads();
    for (int s = s0; s < CH; s += MT / HID) {
        float z = sh[S_B2 + u];
#pragma unroll 16
        for (int v = 0; v < HID; ++v) z = fmaf(sh[S_W2T + v * HID + u], sh[S_A1 + s * HID + v], z);
        sh[S_A2 + s * HID + u] = fmaxf(z, 0.f);
    }
    __syncthreads();
    if (t < CH * NO) {
        const int s = t >> 1, o = t & 1;
        float z = sh[S_B3 + o];
#pragma unroll 16
        for (int v = 0; v < HID; ++v) z = fmaf(sh[S_W3 + o * HID + v], sh[S_A2 + s * HID + v], z);
        sh[S_Y + s * NO + o] = z;
    }
    __syncthreads();
}

// inference: out[n][2]
__global__ void __launch_bounds__(MT) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ mean,
                                                      const float* __restrict__ inv_std, const float* __restrict__ X,
                                                      long long n, float* __restrict__ out) {
    extern __shared__ float sh[];
    load_weights(P, sh);
    for (long long s0 = (long long)blockIdx.x * CH; s0 < n; s0 += (long long)gridDim.x * CH) {
        __syncthreads();
        load_chunk(X, s0, n, mean, inv_std, sh);
        __syncthreads();
        forward_chunk(sh);
        const int t = threadIdx.x;
        if (t < CH * NO && s0 + (t >> 1) < n) out[s0 * NO + t] = sh[S_Y + t];
    }
}

// loss 0.5 / n_scale * sum (y - t)^2 and its gradient over the samples
// [0, n), accumulated per CTA over chunks blockIdx.x, blockIdx.x + gridDim.x, ...
// Partials: part[blockIdx.x][NP], lpart[blockIdx.x].
__global__ void __launch_bounds__(MT) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ mean,
                                                   const float* __restrict__ inv_std, const float* __restrict__ X,
                                                   const float* __restrict__ Y, long long n, float inv_n,
                                                   float* __restrict__ part, float* __restrict__ lpart) {
    extern __shared__ float sh[];
    const int t = threadIdx.x;
    load_weights(P, sh);
    float g[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) g[j] = 0.f;
    float lacc = 0.f;
    for (long long s0 = (long long)blockIdx.x * CH; s0 < n; s0 += (long long)gridDim.x * CH) {
        __syncthreads();
        load_chunk(X, s0, n, mean, inv_std, sh);
        __syncthreads();
        forward_chunk(sh);
        // output error dL/dy = (y - t) / n_scale (zero for padding samples)
        if (t < CH * NO) {
            const int s = t >> 1;
            const long long gi = s0 + s;
            float dy = 0.f, l = 0.f;
            if (gi < n) {
                const float e = sh[S_Y + t] - Y[gi * NO + (t & 1)];
                dy = e * inv_n;
                l = 0.5f * e * e;
            }
            sh[S_DY + t] = dy;
            l += __shfl_xor_sync(0xffffffffu, l, 1);
            if ((t & 1) == 0) sh[S_RED + s] = l;
        }
        __syncthreads();
        if (t == 0) {
            float l = 0.f;
            for (int s = 0; s < CH; ++s) l += sh[S_RED + s];
            lacc += l * inv_n;
        }
        // dL/dz2 = (W3^T dy) * [z2 > 0]
        {
            const int u = t & (HID - 1);
            for (int s = t >> 6; s < CH; s += MT / HID) {
                const float da = sh[S_W3 + u] * sh[S_DY + s * NO] + sh[S_W3 + HID + u] * sh[S_DY + s * NO + 1];
                sh[S_D2 + s * HID + u] = sh[S_A2 + s * HID + u] > 0.f ? da : 0.f;
            }
        }
        __syncthreads();
        // dL/dz1 = (W2^T dz2) * [z1 > 0]
        {
            const int v = t & (HID - 1);
            for (int s = t >> 6; s < CH; s += MT / HID) {
                float da = 0.f;
#pragma unroll 16
                for (int u = 0; u < HID; ++u) da = fmaf(sh[S_W2 + u * HID + v], sh[S_D2 + s * HID + u], da);
                sh[S_D1 + s * HID + v] = sh[S_A1 + s * HID + v] > 0.f ? da : 0.f;
            }
        }
        __syncthreads();
        // parameter gradients of this chunk (sample order 0..31), added to the
        // per-thread accumulators
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int p = t + j * MT;
            float a = 0.f;
            if (p >= NP) {
            } else if (p < OB1) {
                const int u = p / NF, c = p % NF;
                for (int s = 0; s < CH; ++s) a = fmaf(sh[S_D1 + s * HID + u], sh[S_X + s * NF + c], a);
            } else if (p < OW2) {
                const int u = p - OB1;
                for (int s = 0; s < CH; ++s) a += sh[S_D1 + s * HID + u];
            } else if (p < OB2) {
                const int q = p - OW2, u = q / HID, v = q % HID;
                for (int s = 0; s < CH; ++s) a = fmaf(sh[S_D2 + s * HID + u], sh[S_A1 + s * HID + v], a);
            } else if (p < OW3) {
                const int u = p - OB2;
                for (int s = 0; s < CH; ++s) a += sh[S_D2 + s * HID + u];
            } else if (p < OB3) {
                const int q = p - OW3, o = q / HID, v = q % HID;
                for (int s = 0; s < CH; ++s) a = fmaf(sh[S_DY + s * NO + o], sh[S_A2 + s * HID + v], a);
            } else {
                const int o = p - OB3;
                for (int s = 0; s < CH; ++s) a += sh[S_DY + s * NO + o];
            }
            g[j] += a;
        }
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const int p = t + j * MT;
        if (p < NP) part[(size_t)blockIdx.x * NP + p] = g[j];
    }
    if (t == 0) lpart[blockIdx.x] = lacc;
}

// Sum of the per-CTA partials in CTA order; optionally the Adam update
// (Kingma & Ba 2015, Algorithm 1) of the float32 master weights:
//   t <- t + 1, m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
//   theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
// t = *t_dev + local + 1; the loss of the step goes to loss[*t_dev + local - t0].
__global__ void __launch_bounds__(MT) k_mlp_reduce(const float* __restrict__ part, const float* __restrict__ lpart,
                                                     int nparts, float* __restrict__ grad_out, float* __restrict__ P,
                                                     float* __restrict__ m, float* __restrict__ v,
                                                     const long long* __restrict__ t_dev, int local, long long t0,
                                                     float lr, float b1, float b2, float eps, float* __restrict__ loss) {
    const int p = blockIdx.x * MT + threadIdx.x;
    const long long step = (t_dev ? *t_dev : 0) + local;
    if (p < NP) {
        float g = 0.f;
        for (int c = 0; c < nparts; ++c) g += part[(size_t)c * NP + p];
        if (grad_out) grad_out[p] = g;
        if (m) {
            const double tt = (double)(step + 1);
            const float bc1 = (float)(1.0 - pow((double)b1, tt));
            const float bc2 = (float)(1.0 - pow((double)b2, tt));
            const float mm = b1 * m[p] + (1.f - b1) * g;
            const float vv = b2 * v[p] + (1.f - b2) * g * g;
            m[p] = mm;
            v[p] = vv;
            P[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        float l = 0.f;
        for (int c = 0; c < nparts; ++c) l += lpart[c];
        loss[step - t0] = l;
    }
}

__global__ void k_mlp_tick(long long* t_dev, int steps) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *t_dev += steps;
}

// --------------------------------------------------------------------------
// block features (warp per admissible block), float64 reductions
__device__ __forceinline__ double wmin(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ double wmax(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

struct ClusterStats {
    double lo[3], hi[3], A, nA[3], cA[3];
};

__device__ ClusterStats cluster_stats(const GeomD& gd, int b, int e) {
    const int lane = threadIdx.x & 31, E = gd.E;
    ClusterStats c;
    for (int d = 0; d < 3; ++d) {
        c.lo[d] = INFINITY;
        c.hi[d] = -INFINITY;
        c.nA[d] = 0.0;
        c.cA[d] = 0.0;
    }
    c.A = 0.0;
    for (int i = b + lane; i < e; i += 32) {
        double a = 0.0;
        for (int q = 0; q < 7; ++q) a += gd.w[(size_t)q * E + i];
        c.A += a;
        for (int d = 0; d < 3; ++d) {
            for (int vi = 0; vi < 3; ++vi) {
                const double x = gd.v[(size_t)(vi * 3 + d) * E + i];
                c.lo[d] = fmin(c.lo[d], x);
                c.hi[d] = fmax(c.hi[d], x);
            }
            c.nA[d] += a * gd.n[(size_t)d * E + i];
            c.cA[d] += a * gd.c[(size_t)d * E + i];
        }
    }
    c.A = warp_sum(c.A);
    for (int d = 0; d < 3; ++d) {
        c.lo[d] = wmin(c.lo[d]);
        c.hi[d] = wmax(c.hi[d]);
        c.nA[d] = warp_sum(c.nA[d]);
        c.cA[d] = warp_sum(c.cA[d]) / c.A;
    }
    return c;
}

__global__ void __launch_bounds__(256) k_mlp_features(GeomD gd, const BlockRange* __restrict__ far, int n_far,
                                                        const double2* __restrict__ sd, int Ku, int kernel,
                                                        double eps3, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= n_far) return;
    // frequency extremes of the unique set
    double smax = 0.0, srmin = INFINITY, simax = 0.0;
    for (int k = lane; k < Ku; k += 32) {
        const double2 s = sd[k];
        smax = fmax(smax, sqrt(s.x * s.x + s.y * s.y));
        srmin = fmin(srmin, s.x);
        simax = fmax(simax, fabs(s.y));
    }
    smax = wmax(smax);
    srmin = wmin(srmin);
    simax = wmax(simax);
    const BlockRange r = far[b];
    const ClusterStats ct = cluster_stats(gd, r.rb, r.re);
    const ClusterStats cs = cluster_stats(gd, r.cb, r.ce);
    if (lane != 0) return;
    double dt2 = 0.0, ds2 = 0.0, dist2 = 0.0, nt = 0.0, ns = 0.0, ntns = 0.0, dc2 = 0.0, dcn = 0.0;
    for (int d = 0; d < 3; ++d) {
        dt2 += (ct.hi[d] - ct.lo[d]) * (ct.hi[d] - ct.lo[d]);
        ds2 += (cs.hi[d] - cs.lo[d]) * (cs.hi[d] - cs.lo[d]);
        const double g = fmax(0.0, fmax(cs.lo[d] - ct.hi[d], ct.lo[d] - cs.hi[d]));
        dist2 += g * g;
        nt += ct.nA[d] * ct.nA[d];
        ns += cs.nA[d] * cs.nA[d];
        ntns += ct.nA[d] * cs.nA[d];
        const double dc = cs.cA[d] - ct.cA[d];
        dc2 += dc * dc;
        dcn += dc * ct.nA[d];
    }
    const double dist = sqrt(dist2), diam_t = sqrt(dt2), diam_s = sqrt(ds2);
    const double tiny = 1e-300;
    float* o = out + (size_t)b * NF;
    o[0] = (float)log2((double)(r.re - r.rb));
    o[1] = (float)log2((double)(r.ce - r.cb));
    o[2] = (float)log2(fmax(diam_t / dist, tiny));
    o[3] = (float)log2(fmax(diam_s / dist, tiny));
    o[4] = (float)log2(fmax(dist * smax, tiny));
    o[5] = (float)log2(fmax(dist * srmin, tiny));
    o[6] = (float)log2(1.0 + fmax(diam_t, diam_s) * simax / (2.0 * M_PI));
    o[7] = (float)log2((double)Ku);
    o[8] = (float)(-log10(eps3));
    o[9] = (float)kernel;
    o[10] = (float)(fabs(ntns) / (ct.A * cs.A));
    o[11] = (nt > 0.0 && dc2 > 0.0) ? (float)(fabs(dcn) / sqrt(nt * dc2)) : 1.0f;
}

// training labels from a compression: y0 = log2(1 + r3), y1 = k* / K_u with
// k* = argmax_k |f_1[k]| (first fiber, ties to the smallest k; 0 if r3 = 0)
template <class T>
__global__ void __launch_bounds__(256) k_mlp_labels(const CrossRec* __restrict__ rec, const int* __restrict__ r3,
                                                      const BlockRange* __restrict__ ranges,
                                                      const Cx<T>* __restrict__ pool, int n_far, int Ku,
                                                      int Cmax, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= n_far) return;
    const int r = r3[b];
    int kstar = 0;
    if (r > 0) {
        const CrossRec c = rec[(size_t)b * Cmax];
        const BlockRange br = ranges[b];
        const long long M = br.re - br.rb, N = br.ce - br.cb;
        const Cx<T>* f = pool + c.off + (c.r < 0 ? M * N : (long long)c.r * (M + N));
        ArgMaxT<T> best = amax_none<T>();
        for (int k = lane; k < Ku; k += 32) best = amax_better(best, ArgMaxT<T>{cabs2(f[k]), k});
        best = warp_argmax(best);
        kstar = (best.i >= 0 && best.i < Ku) ? best.i : 0;
    }
    if (lane == 0) {
        out[(size_t)b * 2] = (float)log2(1.0 + (double)r);
        out[(size_t)b * 2 + 1] = (float)((double)kstar / (double)Ku);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

static cudaError_t mlp_smem_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
}

g3_status mlp_forward_dev(g3_ctx* ctx, const g3_mlp* net, const float* d_x, long long n, float* d_out) {
    if (n <= 0) return G3_OK;
    G3_CUDA(mlp_smem_attr());
    const long long chunks = (n + CH - 1) / CH;
    const int grid = (int)std::min<long long>(chunks, (long long)ctx->n_sm * 4);
    k_mlp_forward<<<grid, MT, SMEM_BYTES, ctx->stream>>>(net->d_params.as<float>(), net->d_mean.as<float>(),
                                                          net->d_inv_std.as<float>(), d_x, n, d_out);
    ctx->count("k_mlp_forward");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

g3_status mlp_features_dev(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, int kernel, double eps3, float* d_out) {
    const int n_far = (int)t->far_index.size();
    if (n_far == 0) return G3_OK;
    std::vector<BlockRange> rg(n_far);
    for (int i = 0; i < n_far; ++i) {
        const int32_t* r = &t->blocks[5 * (size_t)t->far_index[i]];
        rg[i] = BlockRange{r[0], r[1], r[2], r[3]};
    }
    DevBuf d_far;
    G3_CUDA(d_far.alloc(n_far * sizeof(BlockRange)));
    G3_CUDA(cudaMemcpy(d_far.p, rg.data(), n_far * sizeof(BlockRange), cudaMemcpyHostToDevice));
    const int grid = (n_far + 7) / 8;
    k_mlp_features<<<grid, 256, 0, ctx->stream>>>(t->gd, d_far.as<BlockRange>(), n_far, f->d_sd.as<double2>(),
                                                   f->Ku, kernel, eps3, d_out);
    ctx->count("k_mlp_features");
    G3_CUDA(cudaGetLastError());
    G3_CUDA(cudaStreamSynchronize(ctx->stream));  // d_far is released on return
    return G3_OK;
}

g3_status mlp_labels_dev(g3_ctx* ctx, const g3_factors* fa, const BlockRange* d_ranges, float* d_out) {
    if (fa->n_far == 0) return G3_OK;
    const int grid = (fa->n_far + 7) / 8;
    if (fa->prec == G3_MIXED)
        k_mlp_labels<float><<<grid, 256, 0, ctx->stream>>>(fa->d_rec.as<CrossRec>(), fa->d_r3.as<int>(), d_ranges,
                                                            fa->pool->as<Cx<float>>(), fa->n_far, fa->Ku, fa->Cmax, d_out);
    else
        k_mlp_labels<double><<<grid, 256, 0, ctx->stream>>>(fa->d_rec.as<CrossRec>(), fa->d_r3.as<int>(), d_ranges,
                                                             fa->pool->as<Cx<double>>(), fa->n_far, fa->Ku, fa->Cmax, d_out);
    ctx->count("k_mlp_labels");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

// gradient (and loss) over n samples at the current master weights
g3_status mlp_grad_dev(g3_ctx* ctx, const g3_mlp* net, const float* d_x, const float* d_y, long long n,
                       float* d_grad, float* d_loss) {
    G3_CUDA(mlp_smem_attr());
    const long long chunks = (n + CH - 1) / CH;
    const int grid = (int)std::max<long long>(1, std::min<long long>(chunks, (long long)ctx->n_sm * 2));
    DevBuf part, lpart;
    G3_CUDA(part.alloc((size_t)grid * NP * sizeof(float)));
    G3_CUDA(lpart.alloc((size_t)grid * sizeof(float)));
    k_mlp_grad<<<grid, MT, SMEM_BYTES, ctx->stream>>>(net->d_params.as<float>(), net->d_mean.as<float>(),
                                                       net->d_inv_std.as<float>(), d_x, d_y, n, 1.0f / (float)n,
                                                       part.as<float>(), lpart.as<float>());
    ctx->count("k_mlp_grad");
    G3_CUDA(cudaGetLastError());
    k_mlp_reduce<<<(NP + MT - 1) / MT, MT, 0, ctx->stream>>>(part.as<float>(), lpart.as<float>(), grid, d_grad,
                                                               nullptr, nullptr, nullptr, nullptr, 0, 0, 0.f, 0.f,
                                                               0.f, 0.f, d_loss);
    ctx->count("k_mlp_reduce");
    G3_CUDA(cudaGetLastError());
    G3_CUDA(cudaStreamSynchronize(ctx->stream));
    return G3_OK;
}

// `epochs` passes of minibatch Adam over the n samples (batches are the
// consecutive slices [b B, (b + 1) B); the last one may be shorter)
g3_status mlp_fit_dev(g3_ctx* ctx, g3_mlp* net, const float* d_x, const float* d_y, long long n, int epochs,
                      int batch, double lr, double b1, double b2, double eps, int use_graph, float* d_loss) {
    if (n <= 0 || epochs <= 0) return G3_OK;
    G3_CUDA(mlp_smem_attr());
    const long long nb = (n + batch - 1) / batch;
    const long long max_chunks = (std::min<long long>(batch, n) + CH - 1) / CH;
    const int gmax = (int)std::max<long long>(1, std::min<long long>(max_chunks, (long long)ctx->n_sm * 2));
    DevBuf part, lpart;
    G3_CUDA(part.alloc((size_t)gmax * NP * sizeof(float)));
    G3_CUDA(lpart.alloc((size_t)gmax * sizeof(float)));
    const long long t0 = net->t;
    auto enqueue_epoch = [&](cudaStream_t st) -> g3_status {
        for (long long b = 0; b < nb; ++b) {
            const long long s0 = b * batch, bs = std::min<long long>(batch, n - s0);
            const long long chunks = (bs + CH - 1) / CH;
            const int grid = (int)std::max<long long>(1, std::min<long long>(chunks, gmax));
            k_mlp_grad<<<grid, MT, SMEM_BYTES, st>>>(net->d_params.as<float>(), net->d_mean.as<float>(),
                                                      net->d_inv_std.as<float>(), d_x + s0 * NF, d_y + s0 * NO, bs,
                                                      1.0f / (float)bs, part.as<float>(), lpart.as<float>());
            k_mlp_reduce<<<(NP + MT - 1) / MT, MT, 0, st>>>(part.as<float>(), lpart.as<float>(), grid, nullptr,
                                                           net->d_params.as<float>(), net->d_m.as<float>(),
                                                           net->d_v.as<float>(), net->d_t.as<long long>(), (int)b, t0,
                                                           (float)lr, (float)b1, (float)b2, (float)eps, d_loss);
        }
        k_mlp_tick<<<1, 32, 0, st>>>(net->d_t.as<long long>(), (int)nb);
        return cudaGetLastError() == cudaSuccess ? G3_OK : G3_ECUDA;
    };
    if (use_graph) {
        // the epoch is captured on a private stream (the context's stream may
        // be the legacy default stream, which cannot be captured) and replayed
        // on the context's stream
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cap = nullptr;
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
        G3_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        g3_status st = G3_ECUDA;
        if (ce == cudaSuccess) {
            st = enqueue_epoch(cap);
            ce = cudaStreamEndCapture(cap, &graph);
        }
        cudaStreamDestroy(cap);
        if (st != G3_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(G3_ECUDA, "mlp fit: graph capture failed (%s)", cudaGetErrorString(ce));
        }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(ce, "mlp fit: cudaGraphInstantiate");
        }
        for (int e = 0; e < epochs; ++e) {
            const cudaError_t le = cudaGraphLaunch(exec, ctx->stream);
            if (le != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(graph);
                return fail(G3_ECUDA, "mlp fit: graph launch: %s", cudaGetErrorString(le));
            }
        }
        ctx->count("k_mlp_grad", (int64_t)epochs * nb);
        ctx->count("k_mlp_reduce", (int64_t)epochs * nb);
        ctx->count("k_mlp_tick", epochs);
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
    } else {
        for (int e = 0; e < epochs; ++e) {
            const g3_status st = enqueue_epoch(ctx->stream);
            if (st != G3_OK) return fail(G3_ECUDA, "mlp fit: launch failed");
        }
        ctx->count("k_mlp_grad", (int64_t)epochs * nb);
        ctx->count("k_mlp_reduce", (int64_t)epochs * nb);
        ctx->count("k_mlp_tick", epochs);
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    net->t += (long long)epochs * nb;
    return G3_OK;
}

// He-uniform initial weights: W ~ U(-sqrt(6 / fan_in), sqrt(6 / fan_in)),
// biases 0, drawn from splitmix64 (Steele, Lea & Flood 2014) with 53-bit
// uniforms
void mlp_init_params(uint64_t seed, float* P) {
    uint64_t x = seed;
    auto next = [&]() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto fill = [&](int off, int n, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int i = 0; i < n; ++i) {
            const double u = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
            P[off + i] = (float)((2.0 * u - 1.0) * a);
        }
    };
    std::memset(P, 0, NP * sizeof(float));
    fill(OW1, HID * NF, NF);
    fill(OW2, HID * HID, HID);
    fill(OW3, NO * HID, HID);
}

}  // namespace g3
