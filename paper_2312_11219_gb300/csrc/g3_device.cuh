// Device-side math of the three-way ACA path: complex helpers, the
// Laplace-domain kernel exp(-s r)/(4 pi r) and its normal derivative, the
// collocation entry (7-point rule) and the float64 singular self term.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "g3_internal.h"

namespace g3 {

#define G3_INV4PI 0.07957747154594767

template <class T>
struct Cx {
    T x, y;
};

// One load of a complex element of global memory as a single 64-bit (float)
// or 128-bit (double) access.  Cx<T> has the alignment of T, so a plain
// dereference becomes two accesses; every device buffer of complex values
// here (factor pool, workspace, apply scratch, near field) starts at a
// cudaMalloc'd base and is indexed in whole elements, so its elements are
// aligned to their size.
template <class T>
__device__ __forceinline__ Cx<T> ldcx(const Cx<T>* p) {
    if constexpr (sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        return {v.x, v.y};
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        return {v.x, v.y};
    }
}

template <class T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T>
__device__ __forceinline__ Cx<T> cmulc(Cx<T> a, Cx<T> b) {  // a * conj(b)
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <class T>
__device__ __forceinline__ Cx<T> cconj(Cx<T> a) {
    return {a.x, -a.y};
}
template <class T>
__device__ __forceinline__ T cabs2(Cx<T> a) {
    return a.x * a.x + a.y * a.y;
}
// |a|^2 evaluated in float64 (no underflow for tiny float32 values)
template <class T>
__device__ __forceinline__ double cabs2d(Cx<T> a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}
template <class T>
__device__ __forceinline__ void cfma(Cx<T>& acc, Cx<T> a, Cx<T> b) {  // acc += a * b
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
template <class T>
__device__ __forceinline__ void cfmac(Cx<T>& acc, Cx<T> a, Cx<T> b) {  // acc += a * conj(b)
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.y, b.x, acc.y);
    acc.y = fma(-a.x, b.y, acc.y);
}
__device__ __forceinline__ Cx<double> cdiv(Cx<double> a, Cx<double> b) {
    double d = b.x * b.x + b.y * b.y;
    return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
template <class T, class S>
__device__ __forceinline__ Cx<T> ccast(Cx<S> a) {
    return {(T)a.x, (T)a.y};
}

// exp and sincos in the working precision.  float32: the hardware ex2 / sin /
// cos approximations after an own Cody-Waite reduction of the phase modulo
// 2 pi (two-part constant: 6.28125 is exact in 8 bits, the remainder carries
// the rest), so the approximation sees |t| <= pi.  float64: CUDA's exp and
// sincos.
__device__ __forceinline__ float kexp(float x) { return __expf(x); }
__device__ __forceinline__ double kexp(double x) { return exp(x); }
__device__ __forceinline__ void ksincos(float t, float* s, float* c) {
    float n = rintf(t * 0.15915494309189535f);
    float r = fmaf(-n, 6.28125f, t);
    r = fmaf(-n, 1.9353071795864769e-3f, r);
    __sincosf(r, s, c);
}
__device__ __forceinline__ void ksincos(double t, double* s, double* c) { sincos(t, s, c); }
__device__ __forceinline__ float krsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double krsqrt(double x) { return rsqrt(x); }

// ---- geometry access in the working precision ---------------------------------
// (x_i - c_j) for collocation: centroid difference, float32 via float-float.
__device__ __forceinline__ void cdiff(const GeomF& g, int i, int j, float d[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float hi = g.ch[k * g.E + i] - g.ch[k * g.E + j];
        float lo = g.cl[k * g.E + i] - g.cl[k * g.E + j];
        d[k] = hi + lo;
    }
}
__device__ __forceinline__ void cdiff(const GeomD& g, int i, int j, double d[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = g.c[k * g.E + i] - g.c[k * g.E + j];
}
template <class G>
__device__ __forceinline__ auto qoff(const G& g, int q, int k, int j) {
    return g.q[(q * 3 + k) * g.E + j];
}
template <class G>
__device__ __forceinline__ auto qwt(const G& g, int q, int j) {
    return g.w[q * g.E + j];
}
template <class G>
__device__ __forceinline__ auto nrm(const G& g, int k, int j) {
    return g.n[k * g.E + j];
}

// ---- collocation pair: geometry part of ENTRY(i, j, .) ---------------------------
// For i != j the 7 quadrature points give distances r_q and amplitudes
//   SLP: a_q = w_q / (4 pi r_q)
//   DLP: a_q = w_q d / (4 pi r_q^3), d = (x_i - c_j) . n_j (plane distance)
// and ENTRY(s) = sum_q a_q exp(-s r_q)            (SLP)
//              = sum_q a_q exp(-s r_q) (1 + s r_q) (DLP).
template <class T>
struct Pair7 {
    T r[7];
    T a[7];
};

template <int KER, class G, class T>
__device__ __forceinline__ void pair_setup(const G& g, int i, int j, Pair7<T>& p) {
    T d[3];
    cdiff(g, i, j, d);
    T pd = 0;
    if (KER == G3_DLP) pd = d[0] * nrm(g, 0, j) + d[1] * nrm(g, 1, j) + d[2] * nrm(g, 2, j);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        T rx = d[0] - qoff(g, q, 0, j);
        T ry = d[1] - qoff(g, q, 1, j);
        T rz = d[2] - qoff(g, q, 2, j);
        T r2 = rx * rx + ry * ry + rz * rz;
        T ri = krsqrt(r2);
        p.r[q] = r2 * ri;
        T w = qwt(g, q, j) * (T)G3_INV4PI;
        if (KER == G3_DLP)
            p.a[q] = w * pd * ri * ri * ri;
        else
            p.a[q] = w * ri;
    }
}

template <int KER, class T>
__device__ __forceinline__ Cx<T> pair_eval(const Pair7<T>& p, T sre, T sim) {
    Cx<T> acc{0, 0};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        T m = p.a[q] * kexp(-sre * p.r[q]);
        T sn, cs;
        ksincos(sim * p.r[q], &sn, &cs);
        // exp(-s r) = m' (cos(sim r) - i sin(sim r))
        if (KER == G3_DLP) {
            T fr = (T)1 + sre * p.r[q];
            T fi = sim * p.r[q];
            // (fr + i fi)(cs - i sn)
            acc.x += m * (fr * cs + fi * sn);
            acc.y += m * (fi * cs - fr * sn);
        } else {
            acc.x += m * cs;
            acc.y -= m * sn;
        }
    }
    return acc;
}

// ---- float64 singular self entry V[i, i](s) (collocation at the centroid) ------
// Polar coordinates about x_i over the three sub-triangles (x_i, a, b): with
// d the distance of x_i to the edge line and phi the angle from the foot of
// the perpendicular, r runs to rho(phi) = d / cos(phi), and the radial
// integral is analytic:
//   int_0^rho exp(-s r)/(4 pi r) r dr = rho g(s rho) / (4 pi),
//   g(z) = (1 - exp(-z)) / z  (series for |z| < 0.1).
// The angular integral uses 24-point Gauss-Legendre per edge.
__device__ __forceinline__ Cx<double> g_expm1_over(Cx<double> z) {
    double az = sqrt(z.x * z.x + z.y * z.y);
    if (az < 0.1) {
        // 1 - z/2 + z^2/6 - z^3/24 + ... = sum_{n>=0} (-z)^n / (n+1)!
        Cx<double> term{1.0, 0.0}, sum{1.0, 0.0};
        for (int n = 1; n <= 14; ++n) {
            term = cmul(term, Cx<double>{-z.x, -z.y});
            term.x /= (double)(n + 1);
            term.y /= (double)(n + 1);
            sum.x += term.x;
            sum.y += term.y;
        }
        return sum;
    }
    double e = exp(-z.x), sn, cs;
    sincos(z.y, &sn, &cs);
    Cx<double> one_minus{1.0 - e * cs, e * sn};  // 1 - exp(-z)
    return cdiv(one_minus, z);
}

__device__ inline Cx<double> slp_self_f64(const GeomD& g, int e, double sre, double sim) {
    double x[3], v[3][3];
    for (int k = 0; k < 3; ++k) x[k] = g.c[k * g.E + e];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) v[a][k] = g.v[(a * 3 + k) * g.E + e];
    Cx<double> tot{0.0, 0.0};
    for (int ed = 0; ed < 3; ++ed) {
        const double* A = v[ed];
        const double* B = v[(ed + 1) % 3];
        double t[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double L = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        for (int k = 0; k < 3; ++k) t[k] /= L;
        double t1 = (A[0] - x[0]) * t[0] + (A[1] - x[1]) * t[1] + (A[2] - x[2]) * t[2];
        double t2 = (B[0] - x[0]) * t[0] + (B[1] - x[1]) * t[1] + (B[2] - x[2]) * t[2];
        double f[3] = {A[0] - x[0] - t1 * t[0], A[1] - x[1] - t1 * t[1], A[2] - x[2] - t1 * t[2]};
        double dd = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        double p1 = atan2(t1, dd), p2 = atan2(t2, dd);
        double hm = 0.5 * (p2 - p1), hp = 0.5 * (p2 + p1);
        for (int q = 0; q < 24; ++q) {
            double ph = hm * g.gl[q] + hp;
            double w = hm * g.gl[24 + q];
            double rho = dd / cos(ph);
            Cx<double> gz = g_expm1_over(Cx<double>{sre * rho, sim * rho});
            tot.x += w * rho * gz.x;
            tot.y += w * rho * gz.y;
        }
    }
    tot.x *= G3_INV4PI;
    tot.y *= G3_INV4PI;
    return tot;
}

// ---- full collocation entry (any i, j) in working precision ----------------------
// Self entries (i == j): float64 routine (SLP), 0 (DLP: x_i lies in the plane).
template <int KER, class T>
__device__ __forceinline__ Cx<T> colloc_entry(const GeomF& gf, const GeomD& gd, int i, int j, T sre, T sim) {
    if (i == j) {
        if (KER == G3_DLP) return {0, 0};
        Cx<double> v = slp_self_f64(gd, i, (double)sre, (double)sim);
        return {(T)v.x, (T)v.y};
    }
    Pair7<T> p;
    if constexpr (sizeof(T) == 4)
        pair_setup<KER>(gf, i, j, p);
    else
        pair_setup<KER>(gd, i, j, p);
    return pair_eval<KER>(p, sre, sim);
}

// ---- Galerkin single layer, piecewise-constant elements ---------------------------
// V[i, j](s) = int_{tau_i} int_{tau_j} exp(-s |x - y|) / (4 pi |x - y|) dy dx.
// Pairs without a common vertex: the 4-point conical-product rule on both
// triangles (16 kernel evaluations), points as offsets from the centroids
// (centroid difference in float-float for float32).
template <class G>
__device__ __forceinline__ auto q4off(const G& g, int q, int k, int e) {
    return g.q4[(q * 3 + k) * g.E + e];
}
template <class G>
__device__ __forceinline__ auto q4wt(const G& g, int q, int e) {
    return g.w4[q * g.E + e];
}

template <class T>
struct Pair16 {
    T r[16];
    T a[16];
};

template <class G, class T>
__device__ __forceinline__ void gal_setup(const G& g, int i, int j, Pair16<T>& p) {
    T d[3];
    cdiff(g, i, j, d);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const T xa0 = d[0] + q4off(g, a, 0, i), xa1 = d[1] + q4off(g, a, 1, i), xa2 = d[2] + q4off(g, a, 2, i);
        const T wa = q4wt(g, a, i) * (T)G3_INV4PI;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const T rx = xa0 - q4off(g, b, 0, j), ry = xa1 - q4off(g, b, 1, j), rz = xa2 - q4off(g, b, 2, j);
            const T r2 = rx * rx + ry * ry + rz * rz;
            const T ri = krsqrt(r2);
            p.r[a * 4 + b] = r2 * ri;
            p.a[a * 4 + b] = wa * q4wt(g, b, j) * ri;
        }
    }
}

template <class T>
__device__ __forceinline__ Cx<T> gal_eval(const Pair16<T>& p, T sre, T sim) {
    Cx<T> acc{0, 0};
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const T m = p.a[q] * kexp(-sre * p.r[q]);
        T sn, cs;
        ksincos(sim * p.r[q], &sn, &cs);
        acc.x += m * cs;
        acc.y -= m * sn;
    }
    return acc;
}

// one of the 16 terms (t = 4 a + b)
template <class G, class T>
__device__ __forceinline__ Cx<T> gal_q(const G& g, int i, int j, int t, T sre, T sim) {
    T d[3];
    cdiff(g, i, j, d);
    const int a = t >> 2, b = t & 3;
    const T rx = d[0] + q4off(g, a, 0, i) - q4off(g, b, 0, j);
    const T ry = d[1] + q4off(g, a, 1, i) - q4off(g, b, 1, j);
    const T rz = d[2] + q4off(g, a, 2, i) - q4off(g, b, 2, j);
    const T r2 = rx * rx + ry * ry + rz * rz;
    const T ri = krsqrt(r2);
    const T r = r2 * ri;
    const T m = q4wt(g, a, i) * q4wt(g, b, j) * (T)G3_INV4PI * ri * kexp(-sre * r);
    T sn, cs;
    ksincos(sim * r, &sn, &cs);
    return {m * cs, -m * sn};
}

template <class T>
__device__ __forceinline__ Cx<T> gal_regular(const GeomF& gf, const GeomD& gd, int i, int j, T sre, T sim) {
    Pair16<T> p;
    if constexpr (sizeof(T) == 4)
        gal_setup(gf, i, j, p);
    else
        gal_setup(gd, i, j, p);
    return gal_eval(p, sre, sim);
}

// ---- Galerkin, linear continuous elements (element-local degrees of freedom) ------
// Local function a of element p is the barycentric coordinate lambda_a of its
// vertex a (the element's vertex order).  OP = G3_GAL_P1D: the hypersingular
// operator in the Maue form
//   (curl lambda_a . curl lambda_b) int int U + s^2 (n_p . n_q) int int U lambda_a lambda_b;
// OP = G3_GAL_P1KP: the adjoint double layer int int lambda_a lambda_b dU/dn_x with
//   dU/dn_x = -exp(-s r) (1 + s r) ((x - y) . n_x) / (4 pi r^3).
// Pairs without a common vertex: the 4-point rule on both triangles, whose
// points have the barycentric coordinates below (the rule of the geometry setup).
__device__ __forceinline__ double p1_bary4(int q, int a) {
    const double r6 = sqrt(6.0), r3 = sqrt(3.0);
    const int ia = q >> 1, ib = q & 1;
    const double u = ia == 0 ? (4.0 - r6) / 10.0 : (4.0 + r6) / 10.0;
    const double v = ib == 0 ? 0.5 - 0.5 / r3 : 0.5 + 0.5 / r3;
    const double l1 = u, l2 = v * (1.0 - u);
    return a == 0 ? 1.0 - l1 - l2 : (a == 1 ? l1 : l2);
}

template <int OP, class G, class T>
__device__ __noinline__ Cx<T> p1_regular(const G& g, int p, int a, int q, int b, T sre, T sim) {
    T d[3];
    cdiff(g, p, q, d);
    Cx<T> i0{0, 0}, iab{0, 0};
    const T np0 = (T)nrm(g, 0, p), np1 = (T)nrm(g, 1, p), np2 = (T)nrm(g, 2, p);
#pragma unroll
    for (int qa = 0; qa < 4; ++qa) {
        const T la = (T)p1_bary4(qa, a);
        const T xa0 = d[0] + q4off(g, qa, 0, p), xa1 = d[1] + q4off(g, qa, 1, p), xa2 = d[2] + q4off(g, qa, 2, p);
        const T wa = q4wt(g, qa, p) * (T)G3_INV4PI;
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) {
            const T lb = (T)p1_bary4(qb, b);
            const T rx = xa0 - q4off(g, qb, 0, q), ry = xa1 - q4off(g, qb, 1, q), rz = xa2 - q4off(g, qb, 2, q);
            const T r2 = rx * rx + ry * ry + rz * rz;
            const T ri = krsqrt(r2);
            const T r = r2 * ri;
            const T m = wa * q4wt(g, qb, q) * ri * kexp(-sre * r);   // w w' exp(-Re s r) / (4 pi r)
            T sn, cs;
            ksincos(sim * r, &sn, &cs);
            if (OP == G3_GAL_P1D) {
                const Cx<T> u{m * cs, -m * sn};
                i0.x += u.x;
                i0.y += u.y;
                iab.x += la * lb * u.x;
                iab.y += la * lb * u.y;
            } else {
                // -(1 + s r) exp(-s r) ((x - y) . n_x) / r^2 times the weight above
                const T f = -m * (rx * np0 + ry * np1 + rz * np2) * ri * ri * la * lb;
                const T fr = (T)1 + sre * r, fi = sim * r;
                iab.x += f * (fr * cs + fi * sn);
                iab.y += f * (fi * cs - fr * sn);
            }
        }
    }
    if (OP == G3_GAL_P1KP) return iab;
    T cab = 0, nn = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cab += (T)g.curl[(a * 3 + k) * g.E + p] * (T)g.curl[(b * 3 + k) * g.E + q];
        nn += (T)nrm(g, k, p) * (T)nrm(g, k, q);
    }
    const T s2r = sre * sre - sim * sim, s2i = 2 * sre * sim;
    return {cab * i0.x + nn * (s2r * iab.x - s2i * iab.y), cab * i0.y + nn * (s2r * iab.y + s2i * iab.x)};
}

// all nine local entries of a regular pair: the pair's 16 distances r, weights
// m = w w' / (4 pi r), for the adjoint double layer g = -((x - y) . n_x) / r^2,
// and (hypersingular operator) the curl products and n_p . n_q, formed once ...
template <int OP, class G, class T>
__device__ __forceinline__ void p1_pair_setup(const G& g, int p, int q, T r[16], T m[16], T gz[16], T cab[9], T& nn) {
    T d[3];
    cdiff(g, p, q, d);
    const T np0 = (T)nrm(g, 0, p), np1 = (T)nrm(g, 1, p), np2 = (T)nrm(g, 2, p);
#pragma unroll
    for (int qa = 0; qa < 4; ++qa) {
        const T xa0 = d[0] + q4off(g, qa, 0, p), xa1 = d[1] + q4off(g, qa, 1, p), xa2 = d[2] + q4off(g, qa, 2, p);
        const T wa = q4wt(g, qa, p) * (T)G3_INV4PI;
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) {
            const T rx = xa0 - q4off(g, qb, 0, q), ry = xa1 - q4off(g, qb, 1, q), rz = xa2 - q4off(g, qb, 2, q);
            const T r2 = rx * rx + ry * ry + rz * rz;
            const T ri = krsqrt(r2);
            r[qa * 4 + qb] = r2 * ri;
            m[qa * 4 + qb] = wa * q4wt(g, qb, q) * ri;
            gz[qa * 4 + qb] = OP == G3_GAL_P1KP ? -(rx * np0 + ry * np1 + rz * np2) * ri * ri : (T)0;
        }
    }
    nn = 0;
    if (OP == G3_GAL_P1D) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                T c = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) c += (T)g.curl[(a * 3 + k) * g.E + p] * (T)g.curl[(b * 3 + k) * g.E + q];
                cab[a * 3 + b] = c;
            }
#pragma unroll
        for (int k = 0; k < 3; ++k) nn += (T)nrm(g, k, p) * (T)nrm(g, k, q);
    }
}
// ... and evaluated at one frequency: v[a * 3 + b] (local vertex a of p, b of q)
template <int OP, class T>
__device__ __forceinline__ void p1_pair_eval(const T r[16], const T m[16], const T gz[16], const T cab[9], T nn,
                                             T sre, T sim, Cx<T> v[9]) {
    Cx<T> i0{0, 0};
#pragma unroll
    for (int u = 0; u < 9; ++u) v[u] = Cx<T>{0, 0};
#pragma unroll
    for (int qa = 0; qa < 4; ++qa) {
#pragma unroll
        for (int qb = 0; qb < 4; ++qb) {
            const int q = qa * 4 + qb;
            const T e = m[q] * kexp(-sre * r[q]);
            T sn, cs;
            ksincos(sim * r[q], &sn, &cs);
            Cx<T> u{e * cs, -e * sn};
            if (OP == G3_GAL_P1KP) {
                const T fr = (T)1 + sre * r[q], fi = sim * r[q];
                u = Cx<T>{gz[q] * e * (fr * cs + fi * sn), gz[q] * e * (fi * cs - fr * sn)};
            }
            i0.x += u.x;
            i0.y += u.y;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const T l = (T)(p1_bary4(qa, a) * p1_bary4(qb, b));
                    v[a * 3 + b].x += l * u.x;
                    v[a * 3 + b].y += l * u.y;
                }
        }
    }
    if (OP == G3_GAL_P1D) {
        const T s2r = sre * sre - sim * sim, s2i = 2 * sre * sim;
#pragma unroll
        for (int u = 0; u < 9; ++u) {
            const Cx<T> w = v[u];
            v[u] = Cx<T>{cab[u] * i0.x + nn * (s2r * w.x - s2i * w.y), cab[u] * i0.y + nn * (s2r * w.y + s2i * w.x)};
        }
    }
}

// both geometries: the working precision's copy
template <int OP, class T>
__device__ __forceinline__ Cx<T> p1_entry(const GeomF& gf, const GeomD& gd, int gi, int gj, T sre, T sim) {
    if constexpr (sizeof(T) == 4)
        return p1_regular<OP>(gf, gi / 3, gi % 3, gj / 3, gj % 3, sre, sim);
    else
        return p1_regular<OP>(gd, gi / 3, gi % 3, gj / 3, gj % 3, sre, sim);
}

// Pairs with a common vertex, a common edge or identical panels: the
// Sauter-Schwab transformations (Sauter and Schwab, Boundary Element Methods,
// Section 5.2).  Reference triangle {0 <= x2 <= x1 <= 1}; panel map
// chi(x1, x2) = P0 + x1 (P1 - P0) + x2 (P2 - P1), Jacobian 2 |tau|.  The
// vertices of both panels are ordered with the shared ones first (same order;
// a common edge is x2 = 0 of both maps).  The integrand at (xi, e1, e2, e3) in
// [0, 1]^4 carries the factor returned below; its 1/r singularity is cancelled.
// Regions: identical 6, common edge 5, common vertex 2.
__host__ __device__ inline int ss_regions(int cas) { return cas == SS_IDENTICAL ? 6 : (cas == SS_EDGE ? 5 : 2); }

__device__ inline double ss_map(int cas, int m, double xi, double e1, double e2, double e3, double xh[2],
                                double yh[2]) {
    if (cas == SS_IDENTICAL) {
        const double f = xi * xi * xi * e1 * e1 * e2;
        switch (m) {
            case 0: xh[0] = xi; xh[1] = xi * (1 - e1 + e1 * e2); yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * (1 - e1); break;
            case 1: yh[0] = xi; yh[1] = xi * (1 - e1 + e1 * e2); xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * (1 - e1); break;
            case 2: xh[0] = xi; xh[1] = xi * e1 * (1 - e2 + e2 * e3); yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2); break;
            case 3: yh[0] = xi; yh[1] = xi * e1 * (1 - e2 + e2 * e3); xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2); break;
            case 4: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3); yh[0] = xi; yh[1] = xi * e1 * (1 - e2); break;
            default: yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * (1 - e2 * e3); xh[0] = xi; xh[1] = xi * e1 * (1 - e2); break;
        }
        return f;
    }
    if (cas == SS_EDGE) {
        const double f1 = xi * xi * xi * e1 * e1;
        switch (m) {
            case 0: xh[0] = xi; xh[1] = xi * e1 * e3; yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2); return f1;
            case 1: xh[0] = xi; xh[1] = xi * e1; yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * e2 * (1 - e3); break;
            case 2: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2); yh[0] = xi; yh[1] = xi * e1 * e2 * e3; break;
            case 3: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * e2 * (1 - e3); yh[0] = xi; yh[1] = xi * e1; break;
            default: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3); yh[0] = xi; yh[1] = xi * e1 * e2; break;
        }
        return f1 * e2;
    }
    // common vertex
    if (m == 0) {
        xh[0] = xi; xh[1] = xi * e1; yh[0] = xi * e2; yh[1] = xi * e2 * e3;
    } else {
        yh[0] = xi; yh[1] = xi * e1; xh[0] = xi * e2; xh[1] = xi * e2 * e3;
    }
    return xi * xi * xi * e2;
}

// geometry of one Sauter-Schwab point: r = |chi_x(xh) - chi_y(yh)| and the
// weight w = (Gauss weight) (region factor) (2|tau_x|)(2|tau_y|) / (4 pi r),
// all float64 (the two points can be very close)
struct SsPanels {
    double P[3][3], Q[3][3];   // vertices of tau_x and tau_y in the Sauter-Schwab order
    double jac;                // (2 |tau_x|)(2 |tau_y|) / (4 pi)
};

__device__ inline void ss_panels(const GeomD& g, int i, int j, const int8_t* px, const int8_t* py, SsPanels& S) {
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            S.P[a][k] = g.v[(px[a] * 3 + k) * g.E + i];
            S.Q[a][k] = g.v[(py[a] * 3 + k) * g.E + j];
        }
    auto area2 = [](const double V[3][3]) {
        double u[3] = {V[1][0] - V[0][0], V[1][1] - V[0][1], V[1][2] - V[0][2]};
        double w[3] = {V[2][0] - V[0][0], V[2][1] - V[0][1], V[2][2] - V[0][2]};
        double c0 = u[1] * w[2] - u[2] * w[1], c1 = u[2] * w[0] - u[0] * w[2], c2 = u[0] * w[1] - u[1] * w[0];
        return sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    };
    S.jac = area2(S.P) * area2(S.Q) * G3_INV4PI;
}

__device__ inline void ss_point(const SsPanels& S, int cas, int m, const double g4[4], double gw, double& r,
                                double& w) {
    double xh[2], yh[2];
    const double f = ss_map(cas, m, g4[0], g4[1], g4[2], g4[3], xh, yh);
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double x = S.P[0][k] + xh[0] * (S.P[1][k] - S.P[0][k]) + xh[1] * (S.P[2][k] - S.P[1][k]);
        const double y = S.Q[0][k] + yh[0] * (S.Q[1][k] - S.Q[0][k]) + yh[1] * (S.Q[2][k] - S.Q[1][k]);
        d2 += (x - y) * (x - y);
    }
    r = sqrt(d2);
    w = r > 0.0 ? gw * f * S.jac / r : 0.0;
}

// ---- tensor cores: TF32 products at float32 accuracy ------------------------------
// A real product on the tensor cores as mma.sync m16n8k8 with TF32 inputs and float32
// accumulation, in the three-term split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi =
// a rounded to TF32, a_lo = the rounded remainder), which keeps float32 accuracy (about
// 2^-21 relative per product instead of TF32's 2^-11).
__device__ __forceinline__ unsigned tf32_rna(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
struct Tf32Pair {
    unsigned hi, lo;
};
__device__ __forceinline__ Tf32Pair tf32_split(float x) {
    const unsigned h = tf32_rna(x);
    return Tf32Pair{h, tf32_rna(x - __uint_as_float(h))};
}
// d += a b for one 16 x 8 x 8 tile (fragment layouts of the PTX m16n8k8 .tf32 shape)
__device__ __forceinline__ void mma_tf32(float* d, const unsigned* a, const unsigned* b) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// d += a b in the three-term split (the small terms first)
__device__ __forceinline__ void mma_tf32x3(float* d, const unsigned* ah, const unsigned* al, const unsigned* bh,
                                           const unsigned* bl) {
    mma_tf32(d, ah, bl);
    mma_tf32(d, al, bh);
    mma_tf32(d, ah, bh);
}
// sign flip of TF32 bit patterns (exact)
__device__ __forceinline__ void tf32_neg4(const unsigned* a, unsigned* o) {
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = a[q] ^ 0x80000000u;
}
// ---- asynchronous copies global -> shared (8 bytes; zero-filled when !in) ---------
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool in) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(in ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// ---- block reductions ------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// argmax with ties to the smallest index; v < 0 means "no candidate".  The
// value type is the working precision (float32 compares stay off the float64
// pipe, which runs at a small fraction of the float32 rate on this part).
template <class V>
struct ArgMaxT {
    V v;
    int i;
};
template <class V>
__device__ __forceinline__ ArgMaxT<V> amax_better(ArgMaxT<V> a, ArgMaxT<V> b) {
    if (b.v > a.v) return b;
    if (b.v == a.v && b.i < a.i && b.v >= 0) return b;
    return a;
}
template <class V>
__device__ __forceinline__ ArgMaxT<V> warp_argmax(ArgMaxT<V> a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ArgMaxT<V> b;
        b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
        b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
        a = amax_better(a, b);
    }
    return a;
}
template <class V>
__device__ __forceinline__ ArgMaxT<V> amax_none() {
    return ArgMaxT<V>{(V)-1, 0x7fffffff};
}

}  // namespace g3
