// Frequencies, device geometry, diagnostic entries and near-field assembly.
#include <algorithm>
#include <cmath>
#include <vector>

#include "g3_device.cuh"

namespace g3 {

// ============================================================================
// Frequencies (float64)
// ============================================================================

// Multistep CQ with the BDF2 generating function: s_k = delta(zeta_k) / dt,
// delta(z) = (1 - z) + (1 - z)^2 / 2, zeta_k = lam exp(2 pi i k / K),
// computed for the unique half k = 0..Ku-1.
__global__ void k_freqs_bdf2(int K, int Ku, double lam, double dt, double2* sd, float2* sf) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ku) return;
    double sn, cs;
    sincospi(2.0 * (double)k / (double)K, &sn, &cs);
    double omr = 1.0 - lam * cs, omi = -lam * sn;             // 1 - zeta
    double sqr = omr * omr - omi * omi, sqi = 2.0 * omr * omi;  // (1 - zeta)^2
    double dr = omr + 0.5 * sqr, di = omi + 0.5 * sqi;
    sd[k] = make_double2(dr / dt, di / dt);
    sf[k] = make_float2((float)(dr / dt), (float)(di / dt));
}

// Complete elliptic integral of the first kind, parameter m: K = pi / (2 AGM(1, sqrt(1 - m))).
__device__ double ellipk_agm(double m) {
    double a = 1.0, b = sqrt(1.0 - m);
    for (int it = 0; it < 40 && fabs(a - b) > 1e-16 * a; ++it) {
        double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
    }
    return 3.141592653589793 / (2.0 * a);
}

// Jacobi sn, cn, dn of a real argument by the arithmetic-geometric mean and
// descending Landen recursion (Abramowitz & Stegun 16.4).
__device__ void jacobi_real(double u, double m, double* sn, double* cn, double* dn) {
    double a[24], c[24];
    a[0] = 1.0;
    double b = sqrt(1.0 - m);
    c[0] = sqrt(m);
    int N = 0;
    while (N < 22 && fabs(c[N]) > 1e-16) {
        double an = 0.5 * (a[N] + b);
        double cn1 = 0.5 * (a[N] - b);
        b = sqrt(a[N] * b);
        ++N;
        a[N] = an;
        c[N] = cn1;
    }
    double phi = ldexp(1.0, N) * a[N] * u;
    double phi_next = phi;
    for (int n = N; n >= 1; --n) {
        phi_next = phi;
        phi = 0.5 * (phi + asin(c[n] * sin(phi) / a[n]));
    }
    *sn = sin(phi);
    *cn = cos(phi);
    *dn = (N == 0) ? 1.0 : cos(phi) / cos(phi_next - phi);
}

// gCQ contour (Appendix A) with q = dt_max / dt_min:
//   s_l = gamma(sigma_l), omega_l = -4 K gamma'(sigma_l) / (2 pi i NQ),
// sn/cn/dn at complex sigma from the addition formula with Jacobi's
// imaginary transformation (A&S 16.21.1-3).
__global__ void k_freqs_gcq(int NQ, double dt_min, double dt_max, double2* s_out, double2* w_out) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= NQ) return;
    double q = dt_max / dt_min;
    double r = sqrt(2.0 * q - 1.0);
    double k = (q - r) / (q + r);
    double m = k * k;
    double Kk = ellipk_agm(m), Kp = ellipk_agm(1.0 - m);
    double x = -Kk + ((double)(l + 1) - 0.5) * 4.0 * Kk / (double)NQ;
    double y = 0.5 * Kp;
    double s, c, d, s1, c1, d1;
    jacobi_real(x, m, &s, &c, &d);
    jacobi_real(y, 1.0 - m, &s1, &c1, &d1);
    double den = c1 * c1 + m * s * s * s1 * s1;
    Cx<double> sn{s * d1 / den, c * d * s1 * c1 / den};
    Cx<double> cn{c * c1 / den, -s * d * s1 * d1 / den};
    Cx<double> dn{d * c1 * d1 / den, -m * s * c * s1 / den};
    double pref = 1.0 / (dt_min * (q - 1.0));
    double ik = 1.0 / k;
    Cx<double> num{ik + sn.x, sn.y}, dnm{ik - sn.x, -sn.y};
    Cx<double> ratio = cdiv(num, dnm);
    double2 sl = make_double2(pref * (r * ratio.x - 1.0), pref * r * ratio.y);
    Cx<double> cd = cmul(cn, dn);
    Cx<double> d2 = cmul(dnm, dnm);
    Cx<double> gp = cdiv(cd, d2);
    double fac = pref * r * 2.0 / k;
    gp.x *= fac;
    gp.y *= fac;
    // omega = -4K gp / (2 pi i NQ) = (4K / (2 pi NQ)) * i * gp
    double wfac = 4.0 * Kk / (2.0 * 3.141592653589793 * (double)NQ);
    s_out[l] = sl;
    w_out[l] = make_double2(-wfac * gp.y, wfac * gp.x);
}

g3_status launch_freqs_bdf2(g3_ctx* ctx, int K, int Ku, double lam, double dt, double* d_sd, float* d_sf) {
    k_freqs_bdf2<<<(Ku + 127) / 128, 128, 0, ctx->stream>>>(K, Ku, lam, dt, (double2*)d_sd, (float2*)d_sf);
    ctx->count("k_freqs_bdf2");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

g3_status launch_freqs_gcq(g3_ctx* ctx, int NQ, double dt_min, double dt_max, double* d_s, double* d_w) {
    k_freqs_gcq<<<(NQ + 127) / 128, 128, 0, ctx->stream>>>(NQ, dt_min, dt_max, (double2*)d_s, (double2*)d_w);
    ctx->count("k_freqs_gcq");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

// ============================================================================
// Geometry in cluster order
// ============================================================================

// One thread per cluster position p (element e = perm[p]): centroid
// ((v0 + v1) + v2) / 3, unit normal and area from the cross product, the
// 7-point degree-5 rule (Radon; constants from their closed forms) and the
// 4-point degree-3 conical-product rule (2-point Gauss-Jacobi in u with
// weight (1 - u), 2-point Gauss-Legendre in v), as offsets from the centroid.
__global__ void k_geometry(int ne, const double* __restrict__ verts, const int* __restrict__ tris,
                           const int* __restrict__ perm, GeomF gf, GeomD gd, float* chw, float* clw, float* qw,
                           float* ww, float* nw, float* q4w, float* w4w, double* cdw, double* qdw, double* wdw,
                           double* ndw, double* vdw, double* q4dw, double* w4dw) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ne) return;
    const int E = ne;
    int e = perm[p];
    double v[3][3];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) v[a][k] = verts[3 * (size_t)tris[3 * e + a] + k];
    double c[3];
    for (int k = 0; k < 3; ++k) c[k] = ((v[0][k] + v[1][k]) + v[2][k]) / 3.0;
    double u[3], w[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = v[1][k] - v[0][k];
        w[k] = v[2][k] - v[0][k];
    }
    double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    double n2 = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double area = 0.5 * n2;
    for (int k = 0; k < 3; ++k) {
        float hi = (float)c[k];
        chw[k * E + p] = hi;
        clw[k * E + p] = (float)(c[k] - (double)hi);
        cdw[k * E + p] = c[k];
        double nk = cr[k] / n2;
        nw[k * E + p] = (float)nk;
        ndw[k * E + p] = nk;
        for (int a = 0; a < 3; ++a) vdw[(a * 3 + k) * E + p] = v[a][k];
    }
    // 7-point rule
    const double r15 = sqrt(15.0);
    const double a1 = (6.0 - r15) / 21.0, b1 = (9.0 + 2.0 * r15) / 21.0;
    const double a2 = (6.0 + r15) / 21.0, b2 = (9.0 - 2.0 * r15) / 21.0;
    const double w1 = (155.0 - r15) / 1200.0, w2 = (155.0 + r15) / 1200.0;
    const double t3 = 1.0 / 3.0;
    const double L[7][3] = {{t3, t3, t3}, {a1, a1, b1}, {a1, b1, a1}, {b1, a1, a1},
                            {a2, a2, b2}, {a2, b2, a2}, {b2, a2, a2}};
    const double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    for (int q = 0; q < 7; ++q) {
        for (int k = 0; k < 3; ++k) {
            double y = L[q][0] * v[0][k] + L[q][1] * v[1][k] + L[q][2] * v[2][k];
            double off = y - c[k];
            qw[(q * 3 + k) * E + p] = (float)off;
            qdw[(q * 3 + k) * E + p] = off;
        }
        ww[q * E + p] = (float)(W[q] * area);
        wdw[q * E + p] = W[q] * area;
    }
    // 4-point conical product rule
    const double r6 = sqrt(6.0);
    const double uu[2] = {(4.0 - r6) / 10.0, (4.0 + r6) / 10.0};
    const double wu[2] = {(9.0 + r6) / 36.0, (9.0 - r6) / 36.0};
    const double vv[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    for (int ia = 0; ia < 2; ++ia)
        for (int ib = 0; ib < 2; ++ib) {
            int q = ia * 2 + ib;
            double l1 = uu[ia], l2 = vv[ib] * (1.0 - uu[ia]), l0 = 1.0 - l1 - l2;
            for (int k = 0; k < 3; ++k) {
                double y = l0 * v[0][k] + l1 * v[1][k] + l2 * v[2][k];
                q4w[(q * 3 + k) * E + p] = (float)(y - c[k]);
                q4dw[(q * 3 + k) * E + p] = y - c[k];
            }
            double wq = 2.0 * wu[ia] * 0.5 * area;
            w4w[q * E + p] = (float)wq;
            w4dw[q * E + p] = wq;
        }
}

g3_status launch_geometry(g3_ctx* ctx, g3_tree* t) {
    const int E = t->ne;
    // float arrays: ch 3, cl 3, q 21, w 7, n 3, q4 12, w4 4 = 53 per element
    const size_t nf = 53;
    // double arrays: c 3, q 21, w 7, n 3, v 9, q4 12, w4 4 = 59 per element
    const size_t nd = 59;
    G3_CUDA(t->d_geom_f.alloc(nf * E * sizeof(float)));
    G3_CUDA(t->d_geom_d.alloc(nd * E * sizeof(double) + 48 * sizeof(double)));
    float* F = t->d_geom_f.as<float>();
    double* D = t->d_geom_d.as<double>();
    GeomF gf{};
    gf.E = E;
    gf.ch = F;
    gf.cl = F + 3 * (size_t)E;
    gf.q = F + 6 * (size_t)E;
    gf.w = F + 27 * (size_t)E;
    gf.n = F + 34 * (size_t)E;
    gf.q4 = F + 37 * (size_t)E;
    gf.w4 = F + 49 * (size_t)E;
    GeomD gd{};
    gd.E = E;
    gd.c = D;
    gd.q = D + 3 * (size_t)E;
    gd.w = D + 24 * (size_t)E;
    gd.n = D + 31 * (size_t)E;
    gd.v = D + 34 * (size_t)E;
    gd.q4 = D + 43 * (size_t)E;
    gd.w4 = D + 55 * (size_t)E;
    gd.gl = D + 59 * (size_t)E;
    G3_CUDA(cudaMemcpyAsync((void*)gd.gl, ctx->gl.p, 48 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    DevBuf dv, dt;
    G3_CUDA(dv.alloc(t->verts.size() * sizeof(double)));
    G3_CUDA(dt.alloc(t->tris.size() * sizeof(int)));
    G3_CUDA(cudaMemcpyAsync(dv.p, t->verts.data(), t->verts.size() * sizeof(double), cudaMemcpyHostToDevice,
                            ctx->stream));
    G3_CUDA(cudaMemcpyAsync(dt.p, t->tris.data(), t->tris.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    k_geometry<<<(E + 127) / 128, 128, 0, ctx->stream>>>(
        E, dv.as<double>(), dt.as<int>(), t->d_perm.as<int>(), gf, gd, (float*)gf.ch, (float*)gf.cl, (float*)gf.q,
        (float*)gf.w, (float*)gf.n, (float*)gf.q4, (float*)gf.w4, (double*)gd.c, (double*)gd.q, (double*)gd.w,
        (double*)gd.n, (double*)gd.v, (double*)gd.q4, (double*)gd.w4);
    ctx->count("k_geometry");
    G3_CUDA(cudaGetLastError());
    G3_CUDA(cudaStreamSynchronize(ctx->stream));  // dv, dt are released on return
    t->gf = gf;
    t->gd = gd;
    return G3_OK;
}

// n-point Gauss-Legendre nodes and weights on [0, 1] (Newton iteration on the
// Legendre recurrence)
static void gauss_legendre01(int n, double* x01, double* w01) {
    for (int i = 0; i < n; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        x01[i] = 0.5 * (x + 1.0);
        w01[i] = 1.0 / ((1.0 - x * x) * dp * dp);  // (2 / ((1 - x^2) P'^2)) / 2
    }
}

// 24-point Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on
// the Legendre recurrence), uploaded once per context.
g3_status gl_table(g3_ctx* ctx) {
    const int n = 24;
    std::vector<double> tab(2 * n);
    for (int i = 0; i < n; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) {
                tab[i] = x;
                tab[n + i] = 2.0 / ((1.0 - x * x) * dp * dp);
                break;
            }
        }
        // recompute the weight at the converged node
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (x * p1 - p0) / (x * x - 1.0);
        tab[i] = x;
        tab[n + i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    G3_CUDA(ctx->gl.alloc(2 * n * sizeof(double)));
    G3_CUDA(cudaMemcpy(ctx->gl.p, tab.data(), 2 * n * sizeof(double), cudaMemcpyHostToDevice));
    return G3_OK;
}

// ============================================================================
// Diagnostic entries
// ============================================================================

// Gauss-Legendre rule of the Sauter-Schwab quadrature (n = SS_N per coordinate)
constexpr int SS_N = 6;
struct SsRule {
    double x[SS_N], w[SS_N];
};

template <int KER, class T>
__global__ void k_entries(GeomF gf, GeomD gd, const int* __restrict__ tv, SsRule gr, const double2* __restrict__ sd,
                          const int* __restrict__ rows, const int* __restrict__ cols, int n,
                          const int* __restrict__ ku, const int* __restrict__ conj, int nk, double2* out) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * nk) return;
    int pr = (int)(idx / nk), m = (int)(idx % nk);
    int i = rows[pr], j = cols[pr];
    double2 s = sd[ku[m]];
    Cx<T> v;
    if constexpr (KER == G3_GAL_P1D || KER == G3_GAL_P1KP) {
        v = p1_entry<KER, T>(gf, gd, i, j, (T)s.x, (T)s.y);  // regular pairs (checked on the host)
    } else if constexpr (KER == G3_GAL_SLP) {
        int8_t px[3], py[3];
        const int cas = ss_classify(tv + 3 * (size_t)i, tv + 3 * (size_t)j, i == j, px, py);
        if (cas == 0) {
            v = gal_regular<T>(gf, gd, i, j, (T)s.x, (T)s.y);
        } else {  // Sauter-Schwab, one thread (diagnostic path)
            SsPanels P;
            ss_panels(gd, i, j, px, py, P);
            Cx<T> acc{0, 0};
            const int nr = ss_regions(cas);
            for (int q = 0; q < SS_N * SS_N * SS_N * SS_N * nr; ++q) {
                const int mreg = q / (SS_N * SS_N * SS_N * SS_N);
                int rem = q % (SS_N * SS_N * SS_N * SS_N);
                double g4[4], gw = 1.0;
                for (int a = 3; a >= 0; --a) {
                    g4[a] = gr.x[rem % SS_N];
                    gw *= gr.w[rem % SS_N];
                    rem /= SS_N;
                }
                double r, w;
                ss_point(P, cas, mreg, g4, gw, r, w);
                const T mm = (T)w * kexp(-(T)s.x * (T)r);
                T sn, cs;
                ksincos((T)s.y * (T)r, &sn, &cs);
                acc.x += mm * cs;
                acc.y -= mm * sn;
            }
            v = acc;
        }
    } else if (i == j && KER == G3_SLP) {  // self entries: float64 with the float64 frequency
        Cx<double> d = slp_self_f64(gd, i, s.x, s.y);
        v = Cx<T>{(T)d.x, (T)d.y};
    } else {
        v = colloc_entry<KER, T>(gf, gd, i, j, (T)s.x, (T)s.y);
    }
    double im = conj[m] ? -(double)v.y : (double)v.y;
    out[idx] = make_double2((double)v.x, im);
}

g3_status launch_entries(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, int kernel, int scheme, int prec,
                         const int* d_rows, const int* d_cols, int n, const int* d_ku, const int* d_conj, int nk,
                         double* d_out) {
    if (!t->p1 && scheme == G3_GALERKIN4x4 && kernel != G3_SLP)
        return fail(G3_EUNSUPPORTED, "g3_entries: the Galerkin scheme is implemented for G3_SLP");
    long long tot = (long long)n * nk;
    int blocks = (int)((tot + 127) / 128);
    if (tot == 0) return G3_OK;
    const double2* sd = f->d_sd.as<double2>();
    double2* out = (double2*)d_out;
    SsRule gr;
    gauss_legendre01(SS_N, gr.x, gr.w);
    const int* tv = t->d_tv.as<int>();
#define G3_ENT(K, T) \
    k_entries<K, T><<<blocks, 128, 0, ctx->stream>>>(t->gf, t->gd, tv, gr, sd, d_rows, d_cols, n, d_ku, d_conj, nk, out)
    if (t->p1 && kernel == G3_GAL_P1D && prec == G3_MIXED) G3_ENT(G3_GAL_P1D, float);
    else if (t->p1 && kernel == G3_GAL_P1D) G3_ENT(G3_GAL_P1D, double);
    else if (t->p1 && prec == G3_MIXED) G3_ENT(G3_GAL_P1KP, float);
    else if (t->p1) G3_ENT(G3_GAL_P1KP, double);
    else if (scheme == G3_GALERKIN4x4 && prec == G3_MIXED) G3_ENT(G3_GAL_SLP, float);
    else if (scheme == G3_GALERKIN4x4) G3_ENT(G3_GAL_SLP, double);
    else if (kernel == G3_SLP && prec == G3_MIXED) G3_ENT(G3_SLP, float);
    else if (kernel == G3_SLP) G3_ENT(G3_SLP, double);
    else if (kernel == G3_DLP && prec == G3_MIXED) G3_ENT(G3_DLP, float);
    else if (kernel == G3_DLP) G3_ENT(G3_DLP, double);
    else return fail(G3_EINVAL, "g3_entries: kernel %d not supported", kernel);
#undef G3_ENT
    ctx->count("k_entries");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

// ============================================================================
// Near-field assembly
// ============================================================================

// One CTA per (near block, chunk of KCH unique frequencies).  Threads run
// over the M_b * N_b entries of the block; each thread sets up the pair
// geometry once and evaluates it at the KCH frequencies.  Layout of a block:
// [k][j][i] (frequency-major, column-major per frequency: the apply reads a
// column of rows with one coalesced load), complex, starting at offs[b].
// Self entries (i == j) are left to k_near_self.
template <int KER, class T, int KCH>
__global__ void __launch_bounds__(256) k_near(GeomF gf, GeomD gd, const double2* __restrict__ sd,
                                              const BlockRange* __restrict__ ranges,
                                              const long long* __restrict__ offs, int Ku, Cx<T>* __restrict__ out) {
    const int b = blockIdx.x;
    const int k0 = blockIdx.y * KCH;
    const BlockRange br = ranges[b];
    const int M = br.re - br.rb, N = br.ce - br.cb;
    const int MN = M * N;
    const long long base = offs[b];
    const int kn = min(KCH, Ku - k0);
    for (int e = threadIdx.x; e < MN; e += blockDim.x) {
        int i = br.rb + e % M, j = br.cb + e / M;
        if (i == j) continue;
        if constexpr (KER == G3_GAL_SLP) {
            // regular rule for every off-diagonal pair; pairs with a common
            // vertex are overwritten by k_near_ss
            Pair16<T> p;
            if constexpr (sizeof(T) == 4)
                gal_setup(gf, i, j, p);
            else
                gal_setup(gd, i, j, p);
            for (int kk = 0; kk < kn; ++kk) {
                double2 s = sd[k0 + kk];
                out[base + (long long)(k0 + kk) * MN + e] = gal_eval<T>(p, (T)s.x, (T)s.y);
            }
        } else {
            Pair7<T> p;
            if constexpr (sizeof(T) == 4)
                pair_setup<KER>(gf, i, j, p);
            else
                pair_setup<KER>(gd, i, j, p);
            for (int kk = 0; kk < kn; ++kk) {
                double2 s = sd[k0 + kk];
                out[base + (long long)(k0 + kk) * MN + e] = pair_eval<KER, T>(p, (T)s.x, (T)s.y);
            }
        }
    }
}

// Galerkin near-field entries of pairs with a common vertex, a common edge or
// identical panels (Sauter-Schwab, SS_N^4 Gauss points per region): one CTA
// per pair.  The points' distances and weights are formed once in float64
// and kept in shared memory (as T); each frequency is then a sum over them
// (exp and sincos in T) reduced across the CTA.
template <class T, int NT>
__global__ void __launch_bounds__(NT) k_near_ss(GeomD gd, SsRule gr, const SsPair* __restrict__ pairs,
                                                 const double2* __restrict__ sd, int Ku, Cx<T>* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* rs = reinterpret_cast<T*>(smem_raw);
    const SsPair pr = pairs[blockIdx.x];
    const int nq = SS_N * SS_N * SS_N * SS_N;
    const int npts = nq * ss_regions(pr.cas);
    T* ws = rs + npts;
    __shared__ SsPanels P;
    if (threadIdx.x == 0) ss_panels(gd, pr.i, pr.j, pr.px, pr.py, P);
    __syncthreads();
    for (int q = threadIdx.x; q < npts; q += NT) {
        const int mreg = q / nq;
        int rem = q % nq;
        double g4[4], gw = 1.0;
        for (int a = 3; a >= 0; --a) {
            g4[a] = gr.x[rem % SS_N];
            gw *= gr.w[rem % SS_N];
            rem /= SS_N;
        }
        double r, w;
        ss_point(P, pr.cas, mreg, g4, gw, r, w);
        rs[q] = (T)r;
        ws[q] = (T)w;
    }
    __syncthreads();
    // each warp owns every (NT / 32)-th frequency: its lanes sum over all the
    // points and the warp reduces, with no block-wide barrier per frequency
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = wid; k < Ku; k += NT / 32) {
        const double2 s = sd[k];
        const T sre = (T)s.x, sim = (T)s.y;
        T ax = 0, ay = 0;
        for (int q = lane; q < npts; q += 32) {
            const T r = rs[q];
            const T m = ws[q] * kexp(-sre * r);
            T sn, cs;
            ksincos(sim * r, &sn, &cs);
            ax += m * cs;
            ay -= m * sn;
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        if (lane == 0) out[pr.off + (long long)k * pr.stride] = Cx<T>{ax, ay};
    }
}

// Linear continuous elements (element-local degrees of freedom): near-field
// entries of element pairs without a common vertex by the 4-point rule on both
// panels, one thread per element pair: the 16 point distances and weights are
// formed once and every frequency gives the pair's nine local entries; the
// pairs with a common vertex are written by k_near_ss_p1.  One CTA per (near
// block, chunk of KCH unique frequencies), layout [k][j][i] as k_near.
template <int OP, class T, int KCH>
__global__ void __launch_bounds__(256) k_near_p1(GeomF gf, GeomD gd, const int* __restrict__ tv,
                                                 const double2* __restrict__ sd, const BlockRange* __restrict__ ranges,
                                                 const long long* __restrict__ offs, int Ku, Cx<T>* __restrict__ out) {
    const int b = blockIdx.x;
    const int k0 = blockIdx.y * KCH;
    const BlockRange br = ranges[b];
    const int M = br.re - br.rb, N = br.ce - br.cb;
    const int Me = M / 3, Ne = N / 3;
    const long long base = offs[b];
    const int kn = min(KCH, Ku - k0);
    for (int e = threadIdx.x; e < Me * Ne; e += blockDim.x) {
        const int pe = br.rb / 3 + e % Me, qe = br.cb / 3 + e / Me;
        bool shared = false;
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) shared |= tv[3 * pe + x] == tv[3 * qe + y];
        if (shared) continue;
        T r[16], m[16], gz[16];
        T cab[9], nn = 0;
        if constexpr (sizeof(T) == 4)
            p1_pair_setup<OP>(gf, pe, qe, r, m, gz, cab, nn);
        else
            p1_pair_setup<OP>(gd, pe, qe, r, m, gz, cab, nn);
        const long long e0 = base + (long long)(3 * (qe - br.cb / 3)) * M + 3 * (pe - br.rb / 3);
        for (int kk = 0; kk < kn; ++kk) {
            const double2 s = sd[k0 + kk];
            Cx<T> v[9];
            p1_pair_eval<OP, T>(r, m, gz, cab, nn, (T)s.x, (T)s.y, v);
            Cx<T>* o = out + (long long)(k0 + kk) * M * N + e0;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) o[a + (long long)c * M] = v[a * 3 + c];
        }
    }
}

// Linear elements, element pairs with a common vertex, a common edge or
// identical panels: the Sauter-Schwab maps (as k_near_ss) with the products
// lambda_a(x) lambda_b(y) of the local functions in the integrand; one CTA per
// element pair writes its 3 x 3 local entries at every frequency.  The points
// of one region (SS_N^4) are set up in float64 and kept in shared memory (their
// reference coordinates, distance and weight, and for the adjoint double layer
// -((x - y) . n_x) / r^2); each frequency's ten sums (the plain integral and
// the nine weighted ones) are reduced over the CTA and added into acc.
template <int OP, class T, int NT>
__global__ void __launch_bounds__(NT) k_near_ss_p1(GeomD gd, SsRule gr, const SsPair* __restrict__ pairs,
                                                   const double2* __restrict__ sd, int Ku, Cx<T>* __restrict__ out) {
    constexpr int NQ = SS_N * SS_N * SS_N * SS_N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* pt = reinterpret_cast<T*>(smem_raw);                    // [7][NQ]: x1, x2, y1, y2, r, w, g
    Cx<T>* acc = reinterpret_cast<Cx<T>*>(pt + 7 * NQ);         // [Ku][10]
    __shared__ SsPanels P;
    const SsPair pr = pairs[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) ss_panels(gd, pr.i, pr.j, pr.px, pr.py, P);
    for (int e = threadIdx.x; e < Ku * 10; e += NT) acc[e] = Cx<T>{0, 0};
    double n[3];
    for (int k = 0; k < 3; ++k) n[k] = gd.n[k * gd.E + pr.i];
    __syncthreads();
    const int nreg = ss_regions(pr.cas);
    for (int mreg = 0; mreg < nreg; ++mreg) {
        for (int q = threadIdx.x; q < NQ; q += NT) {
            int rem = q;
            double g4[4], gw = 1.0;
            for (int a = 3; a >= 0; --a) {
                g4[a] = gr.x[rem % SS_N];
                gw *= gr.w[rem % SS_N];
                rem /= SS_N;
            }
            double xh[2], yh[2];
            const double f = ss_map(pr.cas, mreg, g4[0], g4[1], g4[2], g4[3], xh, yh);
            double z[3], d2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double x = P.P[0][k] + xh[0] * (P.P[1][k] - P.P[0][k]) + xh[1] * (P.P[2][k] - P.P[1][k]);
                const double y = P.Q[0][k] + yh[0] * (P.Q[1][k] - P.Q[0][k]) + yh[1] * (P.Q[2][k] - P.Q[1][k]);
                z[k] = x - y;
                d2 += z[k] * z[k];
            }
            const double r = sqrt(d2);
            pt[0 * NQ + q] = (T)xh[0];
            pt[1 * NQ + q] = (T)xh[1];
            pt[2 * NQ + q] = (T)yh[0];
            pt[3 * NQ + q] = (T)yh[1];
            pt[4 * NQ + q] = (T)r;
            pt[5 * NQ + q] = r > 0.0 ? (T)(gw * f * P.jac / r) : (T)0;
            pt[6 * NQ + q] = r > 0.0 ? (T)(-(z[0] * n[0] + z[1] * n[1] + z[2] * n[2]) / d2) : (T)0;
        }
        __syncthreads();
        // each warp owns every (NT / 32)-th frequency (no block-wide barrier per frequency)
        for (int k = wid; k < Ku; k += NT / 32) {
            const double2 s = sd[k];
            const T sre = (T)s.x, sim = (T)s.y;
            Cx<T> v[10];
#pragma unroll
            for (int u = 0; u < 10; ++u) v[u] = Cx<T>{0, 0};
            for (int q = lane; q < NQ; q += 32) {
                const T r = pt[4 * NQ + q];
                const T m = pt[5 * NQ + q] * kexp(-sre * r);
                T sn, cs;
                ksincos(sim * r, &sn, &cs);
                Cx<T> E{m * cs, -m * sn};
                if (OP == G3_GAL_P1KP) {
                    const T g = pt[6 * NQ + q], fr = (T)1 + sre * r, fi = sim * r;
                    E = Cx<T>{g * m * (fr * cs + fi * sn), g * m * (fi * cs - fr * sn)};
                }
                const T x1 = pt[q], x2 = pt[NQ + q], y1 = pt[2 * NQ + q], y2 = pt[3 * NQ + q];
                const T lx[3] = {(T)1 - x1, x1 - x2, x2}, ly[3] = {(T)1 - y1, y1 - y2, y2};
                v[9].x += E.x;
                v[9].y += E.y;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        v[a * 3 + b].x += lx[a] * ly[b] * E.x;
                        v[a * 3 + b].y += lx[a] * ly[b] * E.y;
                    }
            }
#pragma unroll
            for (int u = 0; u < 10; ++u) {
                v[u].x = warp_sum(v[u].x);
                v[u].y = warp_sum(v[u].y);
            }
            if (lane < 10) {  // frequency k belongs to this warp alone
                Cx<T> t{0, 0};
#pragma unroll
                for (int u = 0; u < 10; ++u)
                    if (u == lane) t = v[u];
                acc[k * 10 + lane].x += t.x;
                acc[k * 10 + lane].y += t.y;
            }
        }
        __syncthreads();  // the region's points are consumed before the next region overwrites them
    }
    // local entries (Sauter-Schwab vertex order c, d = local vertices px[c], py[d])
    for (int e = threadIdx.x; e < Ku * 9; e += NT) {
        const int k = e / 9, c = (e % 9) / 3, dd = e % 3;
        const int a = pr.px[c], b = pr.py[dd];
        Cx<T> val = acc[k * 10 + c * 3 + dd];
        if (OP == G3_GAL_P1D) {
            const double2 s = sd[k];
            const T s2r = (T)(s.x * s.x - s.y * s.y), s2i = (T)(2.0 * s.x * s.y);
            T cab = 0, nn = 0;
            for (int kk = 0; kk < 3; ++kk) {
                cab += (T)(gd.curl[(a * 3 + kk) * gd.E + pr.i] * gd.curl[(b * 3 + kk) * gd.E + pr.j]);
                nn += (T)(gd.n[kk * gd.E + pr.i] * gd.n[kk * gd.E + pr.j]);
            }
            const Cx<T> i0 = acc[k * 10 + 9];
            val = Cx<T>{cab * i0.x + nn * (s2r * val.x - s2i * val.y), cab * i0.y + nn * (s2r * val.y + s2i * val.x)};
        }
        out[pr.off + (long long)k * pr.stride + a + (long long)b * pr.ldm] = val;
    }
}

template <int OP, class T>
static g3_status launch_near_p1_t(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_near* nf) {
    const int nb = (int)nf->order.size();
    constexpr int KCH = 16;
    dim3 grid(nb, (f->Ku + KCH - 1) / KCH);
    Cx<T>* o = reinterpret_cast<Cx<T>*>(nf->data.p);
    k_near_p1<OP, T, KCH><<<grid, 256, 0, ctx->stream>>>(t->gf, t->gd, t->d_tv.as<int>(), f->d_sd.as<double2>(),
                                                          nf->d_ranges.as<BlockRange>(), nf->d_offs.as<long long>(),
                                                          f->Ku, o);
    ctx->count("k_near_p1");
    G3_CUDA(cudaGetLastError());
    if (nf->n_ss > 0) {
        SsRule gr;
        gauss_legendre01(SS_N, gr.x, gr.w);
        constexpr int NT = 256;
        const size_t smem = 7 * (size_t)SS_N * SS_N * SS_N * SS_N * sizeof(T) + 10 * (size_t)f->Ku * sizeof(Cx<T>);
        if (smem > ctx->smem_optin)
            return fail(G3_EUNSUPPORTED, "assemble_near: %zu bytes of shared memory for the singular pairs", smem);
        G3_CUDA(cudaFuncSetAttribute(k_near_ss_p1<OP, T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_near_ss_p1<OP, T, NT><<<nf->n_ss, NT, smem, ctx->stream>>>(t->gd, gr, nf->d_ss.as<SsPair>(),
                                                                      f->d_sd.as<double2>(), f->Ku, o);
        ctx->count("k_near_ss_p1");
        G3_CUDA(cudaGetLastError());
    }
    return G3_OK;
}

// Self entries of the near field, float64: one thread per (element p, unique
// frequency k); the entry (p, p) of the diagonal leaf block sits at
// diag_base[p] + k * diag_mn[p] (diag_base[p] < 0: not in this tree's blocks).
template <int KER, class T>
__global__ void k_near_self(GeomD gd, const double2* __restrict__ sd, int E, int Ku,
                            const long long* __restrict__ diag_base, const int* __restrict__ diag_mn,
                            Cx<T>* __restrict__ out) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)E * Ku) return;
    const int p = (int)(idx % E), k = (int)(idx / E);
    if (diag_base[p] < 0) return;  // the diagonal block belongs to another rank's subset
    Cx<T> v{0, 0};
    if (KER == G3_SLP) {
        double2 s = sd[k];
        Cx<double> d = slp_self_f64(gd, p, s.x, s.y);
        v = Cx<T>{(T)d.x, (T)d.y};
    }
    out[diag_base[p] + (long long)k * diag_mn[p]] = v;
}

// Galerkin: near-field pairs with a common vertex (the list of SsPair records
// built on the host) by k_near_ss, after the regular rule for all pairs
template <class T>
static g3_status launch_near_galerkin(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_near* nf) {
    const int nb = (int)nf->order.size();
    constexpr int KCH = 16;
    dim3 grid(nb, (f->Ku + KCH - 1) / KCH);
    Cx<T>* o = reinterpret_cast<Cx<T>*>(nf->data.p);
    k_near<G3_GAL_SLP, T, KCH><<<grid, 256, 0, ctx->stream>>>(t->gf, t->gd, f->d_sd.as<double2>(),
                                                               nf->d_ranges.as<BlockRange>(),
                                                               nf->d_offs.as<long long>(), f->Ku, o);
    ctx->count("k_near");
    G3_CUDA(cudaGetLastError());
    if (nf->n_ss > 0) {
        SsRule gr;
        gauss_legendre01(SS_N, gr.x, gr.w);
        constexpr int NT = 256;
        const size_t smem = 2 * (size_t)SS_N * SS_N * SS_N * SS_N * 6 * sizeof(T);
        G3_CUDA(cudaFuncSetAttribute(k_near_ss<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_near_ss<T, NT><<<nf->n_ss, NT, smem, ctx->stream>>>(t->gd, gr, nf->d_ss.as<SsPair>(),
                                                              f->d_sd.as<double2>(), f->Ku, o);
        ctx->count("k_near_ss");
        G3_CUDA(cudaGetLastError());
    }
    return G3_OK;
}

g3_status launch_near(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_near* nf, int kernel, int scheme) {
    const int nb = (int)nf->order.size();
    if (nb == 0) return G3_OK;
    if (t->p1) {
        if (kernel == G3_GAL_P1D)
            return nf->prec == G3_MIXED ? launch_near_p1_t<G3_GAL_P1D, float>(ctx, t, f, nf)
                                        : launch_near_p1_t<G3_GAL_P1D, double>(ctx, t, f, nf);
        return nf->prec == G3_MIXED ? launch_near_p1_t<G3_GAL_P1KP, float>(ctx, t, f, nf)
                                    : launch_near_p1_t<G3_GAL_P1KP, double>(ctx, t, f, nf);
    }
    if (scheme == G3_GALERKIN4x4) {
        if (kernel != G3_SLP) return fail(G3_EUNSUPPORTED, "assemble_near: the Galerkin scheme is implemented for G3_SLP");
        return nf->prec == G3_MIXED ? launch_near_galerkin<float>(ctx, t, f, nf)
                                    : launch_near_galerkin<double>(ctx, t, f, nf);
    }
    constexpr int KCH = 16;
    dim3 grid(nb, (f->Ku + KCH - 1) / KCH);
    const double2* sd = f->d_sd.as<double2>();
    const BlockRange* rg = nf->d_ranges.as<BlockRange>();
    const long long* of = nf->d_offs.as<long long>();
    const long long* db = nf->d_diag_base.as<long long>();
    const int* dm = nf->d_diag_mn.as<int>();
    const int sgrid = (int)(((long long)t->ne * f->Ku + 255) / 256);
    if (nf->prec == G3_MIXED) {
        Cx<float>* o = nf->data.as<Cx<float>>();
        if (kernel == G3_SLP) {
            k_near<G3_SLP, float, KCH><<<grid, 256, 0, ctx->stream>>>(t->gf, t->gd, sd, rg, of, f->Ku, o);
            k_near_self<G3_SLP, float><<<sgrid, 256, 0, ctx->stream>>>(t->gd, sd, t->ne, f->Ku, db, dm, o);
        } else {
            k_near<G3_DLP, float, KCH><<<grid, 256, 0, ctx->stream>>>(t->gf, t->gd, sd, rg, of, f->Ku, o);
            k_near_self<G3_DLP, float><<<sgrid, 256, 0, ctx->stream>>>(t->gd, sd, t->ne, f->Ku, db, dm, o);
        }
    } else {
        Cx<double>* o = nf->data.as<Cx<double>>();
        if (kernel == G3_SLP) {
            k_near<G3_SLP, double, KCH><<<grid, 256, 0, ctx->stream>>>(t->gf, t->gd, sd, rg, of, f->Ku, o);
            k_near_self<G3_SLP, double><<<sgrid, 256, 0, ctx->stream>>>(t->gd, sd, t->ne, f->Ku, db, dm, o);
        } else {
            k_near<G3_DLP, double, KCH><<<grid, 256, 0, ctx->stream>>>(t->gf, t->gd, sd, rg, of, f->Ku, o);
            k_near_self<G3_DLP, double><<<sgrid, 256, 0, ctx->stream>>>(t->gd, sd, t->ne, f->Ku, db, dm, o);
        }
    }
    ctx->count("k_near");
    ctx->count("k_near_self");
    G3_CUDA(cudaGetLastError());
    return G3_OK;
}

}  // namespace g3
