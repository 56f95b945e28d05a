// Throughput micro-benchmarks of the arithmetic pipes the entry generation
// runs on (special-function unit and FP32/FP64 fused multiply-add), used for
// the ALU roofline of the compression.  Each thread runs 8 independent
// dependency chains of one instruction; the result is folded into a sink so
// that nothing is eliminated.
#include "g3_device.cuh"

namespace g3 {

enum { PK_FFMA = 0, PK_RSQRT = 1, PK_EX2 = 2, PK_SIN = 3, PK_COS = 4, PK_DFMA = 5 };

__device__ __forceinline__ float ptx_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ptx_rsqrt(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ptx_sin(float x) {
    float y;
    asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ptx_cos(float x) {
    float y;
    asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KIND>
__global__ void k_peak(int iters, float seed, float* sink) {
    float v[8];
    double d[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        v[c] = seed + 0.001f * (threadIdx.x + c);
        d[c] = (double)v[c];
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (KIND == PK_FFMA) v[c] = fmaf(v[c], 0.999999f, 1e-7f);
            if (KIND == PK_RSQRT) v[c] = ptx_rsqrt(v[c]);
            if (KIND == PK_EX2) v[c] = ptx_ex2(v[c]) - 1.0f;   // stays in a bounded range
            if (KIND == PK_SIN) v[c] = ptx_sin(v[c]);
            if (KIND == PK_COS) v[c] = ptx_cos(v[c]);
            if (KIND == PK_DFMA) d[c] = fma(d[c], 0.9999999999, 1e-12);
        }
    }
    float acc = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc += v[c] + (float)d[c];
    if (acc == 12345.678f) sink[threadIdx.x] = acc;  // practically never taken
}

g3_status run_peak(g3_ctx* ctx, int kind, double* ops_per_s, double* ms_out) {
    DevBuf sink;
    G3_CUDA(sink.alloc(1024 * sizeof(float)));
    const int threads = 256, blocks = ctx->n_sm * 8;
    const int iters = kind == PK_DFMA ? 512 : (kind == PK_FFMA ? 16384 : 4096);
    auto launch = [&](int it) {
        switch (kind) {
            case PK_FFMA: k_peak<PK_FFMA><<<blocks, threads, 0, ctx->stream>>>(it, 0.5f, sink.as<float>()); break;
            case PK_RSQRT: k_peak<PK_RSQRT><<<blocks, threads, 0, ctx->stream>>>(it, 0.5f, sink.as<float>()); break;
            case PK_EX2: k_peak<PK_EX2><<<blocks, threads, 0, ctx->stream>>>(it, 0.5f, sink.as<float>()); break;
            case PK_SIN: k_peak<PK_SIN><<<blocks, threads, 0, ctx->stream>>>(it, 0.5f, sink.as<float>()); break;
            case PK_COS: k_peak<PK_COS><<<blocks, threads, 0, ctx->stream>>>(it, 0.5f, sink.as<float>()); break;
            default: k_peak<PK_DFMA><<<blocks, threads, 0, ctx->stream>>>(it, 0.5f, sink.as<float>()); break;
        }
    };
    launch(iters / 8);  // warm-up
    G3_CUDA(cudaGetLastError());
    G3_CUDA(cudaEventRecord(ctx->ev[0], ctx->stream));
    launch(iters);
    G3_CUDA(cudaEventRecord(ctx->ev[1], ctx->stream));
    G3_CUDA(cudaEventSynchronize(ctx->ev[1]));
    G3_CUDA(cudaGetLastError());
    ctx->count("k_peak", 2);
    float ms = 0;
    G3_CUDA(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
    const double ops = (double)blocks * threads * 8.0 * iters;  // one FMA counts as one op
    *ops_per_s = ops / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return G3_OK;
}

}  // namespace g3
