// The gCQ time-stepping consumer of the apply: the history update of
// eq. (gCQ_xn) and the weight vectors of eq. (gcq_formula), for the
// implicit-Euler reading of the gCQ (one stage, A = b = 1; the contour of
// Appendix A with q = dt_max / dt_min).  Per element i and frequency l:
//
//   x_{n-1}(s_l) = (x_{n-2}(s_l) + dt_{n-1} theta_{n-1}) / (1 - dt_{n-1} s_l)
//   W[:, l]      = w_l x_{n-1}(s_l) / (1 - dt_n s_l),
//
// where w_l is the weight of the paper's contour integral in eq.
// (conv_discrete).  That integral gives +V((dt_n A)^{-1}) theta_n from the
// pole of (1 - dt_n s)^{-1}, so it runs clockwise around the poles; the
// frequency set's weights omega_l are normalised counterclockwise
// (sum_l omega_l / (s_l - a) = 1 for a inside), hence w_l = -omega_l.
// apply_gcq on W then gives the history sum of eq. (gcq_formula).
//
// One elementwise pass over X (read and written) and W (written): an HBM
// stream.  Grid (column chunks, frequencies): each CTA forms its
// frequency's two coefficients once in float64.
#include <algorithm>
#include <cmath>

#include "g3_device.cuh"

namespace g3 {

template <class T>
__global__ void k_gcq_history(int M, const double2* __restrict__ s, const double2* __restrict__ om, double dt_prev,
                              double dt_next, Cx<T>* __restrict__ X, const Cx<T>* __restrict__ theta,
                              Cx<T>* __restrict__ W) {
    __shared__ Cx<T> coef[2];
    const int l = blockIdx.y;
    if (threadIdx.x == 0) {
        const double2 sl = s[l], wl = om[l];
        // a = 1 / (1 - dt_prev s),  c = -omega / (1 - dt_next s)
        const Cx<double> d1{1.0 - dt_prev * sl.x, -dt_prev * sl.y};
        const Cx<double> d2{1.0 - dt_next * sl.x, -dt_next * sl.y};
        const Cx<double> a = cdiv(Cx<double>{1.0, 0.0}, d1);
        const Cx<double> c = cdiv(Cx<double>{-wl.x, -wl.y}, d2);
        coef[0] = Cx<T>{(T)a.x, (T)a.y};
        coef[1] = Cx<T>{(T)c.x, (T)c.y};
    }
    __syncthreads();
    const Cx<T> a = coef[0], c = coef[1];
    const T dt = (T)dt_prev;
    const long long base = (long long)l * M;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        Cx<T> x = ldcx(X + base + i);
        if (theta) {
            const Cx<T> th = ldcx(theta + i);
            x.x += dt * th.x;
            x.y += dt * th.y;
        }
        const Cx<T> xn = cmul(x, a);
        X[base + i] = xn;
        W[base + i] = cmul(xn, c);
    }
}

g3_status run_gcq_history(g3_ctx* ctx, const g3_freqs* f, int M, void* X, const void* theta, double dt_prev,
                          double dt_next, void* W, int dtype) {
    const int K = f->K;
    dim3 grid((unsigned)std::min((M + 255) / 256, 64), (unsigned)K);
    if (dtype == G3_C128)
        k_gcq_history<double><<<grid, 256, 0, ctx->stream>>>(M, f->d_s_all.as<double2>(), f->d_w_all.as<double2>(),
                                                            dt_prev, dt_next, (Cx<double>*)X,
                                                            (const Cx<double>*)theta, (Cx<double>*)W);
    else
        k_gcq_history<float><<<grid, 256, 0, ctx->stream>>>(M, f->d_s_all.as<double2>(), f->d_w_all.as<double2>(),
                                                           dt_prev, dt_next, (Cx<float>*)X, (const Cx<float>*)theta,
                                                           (Cx<float>*)W);
    ctx->count("k_gcq_history");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

}  // namespace g3

extern "C" g3_status g3_gcq_history(g3_ctx* ctx, const g3_freqs* f, int M, void* X, const void* theta,
                                    double dt_prev, double dt_next, void* W, g3_dtype dtype) {
    using namespace g3;
    if (!ctx || !f || !X || !W) return fail(G3_EINVAL, "g3_gcq_history: NULL argument");
    if (M < 1) return fail(G3_EINVAL, "g3_gcq_history: M = %d", M);
    if (dtype != G3_C64 && dtype != G3_C128) return fail(G3_EINVAL, "g3_gcq_history: bad dtype");
    if (!(dt_prev > 0) || !(dt_next > 0) || !std::isfinite(dt_prev) || !std::isfinite(dt_next))
        return fail(G3_EINVAL, "g3_gcq_history: time steps %g, %g must be positive", dt_prev, dt_next);
    bool has_w = false;
    for (double v : f->omega) has_w |= v != 0.0;
    if (!has_w) return fail(G3_EINVAL, "g3_gcq_history: the frequency set carries no contour weights (gCQ sets do)");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return run_gcq_history(ctx, f, M, X, theta, dt_prev, dt_next, W, dtype);
}
