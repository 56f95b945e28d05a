// C ABI entry points (include/g3aca.h): handle management, argument checks,
// host<->device staging.  All compute runs in the kernels of g3_prep.cu,
// g3_aca.cu and g3_apply.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "g3_internal.h"

namespace g3 {

static thread_local char t_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
}

g3_status fail(g3_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return st;
}

g3_status cuda_fail(cudaError_t e, const char* what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? G3_ENOMEM : G3_ECUDA;
}

}  // namespace g3

using namespace g3;

#define G3_CHECK(cond, ...)                                   \
    do {                                                      \
        if (!(cond)) return ::g3::fail(G3_EINVAL, __VA_ARGS__); \
    } while (0)

#define G3_TRY(expr)                       \
    do {                                   \
        g3_status st_ = (expr);            \
        if (st_ != G3_OK) return st_;      \
    } while (0)

static g3_status use_device(const g3_ctx* ctx) {
    G3_CUDA(cudaSetDevice(ctx->device));
    return G3_OK;
}

extern "C" {

const char* g3_last_error(void) { return g3::t_err; }
int g3_version(void) { return G3ACA_VERSION; }

g3_status g3_create(int device, void* cuda_stream, g3_ctx** out) {
    G3_CHECK(out != nullptr, "g3_create: out is NULL");
    *out = nullptr;
    int n = 0;
    G3_CUDA(cudaGetDeviceCount(&n));
    G3_CHECK(device >= 0 && device < n, "g3_create: device %d outside [0, %d)", device, n);
    G3_CUDA(cudaSetDevice(device));
    g3_ctx* c = new (std::nothrow) g3_ctx();
    if (!c) return fail(G3_ENOMEM, "g3_create: out of host memory");
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaGetDeviceProperties");
    }
    c->n_sm = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    for (auto& ev : c->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
            g3_destroy(c);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    for (auto& ev : c->ev_side) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
            g3_destroy(c);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
    // the apply's near-field kernel runs on this stream at the highest priority,
    // next to the far-field kernels on the context's stream: pending near-field
    // CTAs are dispatched first, far-field CTAs fill the rest of each SM
    int prio_least = 0, prio_greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_greatest);
    if (e != cudaSuccess) {
        g3_destroy(c);
        return cuda_fail(e, "side stream / events");
    }
    e = c->status.alloc(64);
    if (e != cudaSuccess) {
        g3_destroy(c);
        return cuda_fail(e, "status buffer");
    }
    g3_status st = gl_table(c);
    if (st != G3_OK) {
        g3_destroy(c);
        return st;
    }
    *out = c;
    return G3_OK;
}

g3_status g3_set_stream(g3_ctx* ctx, void* cuda_stream) {
    G3_CHECK(ctx != nullptr, "g3_set_stream: ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    return G3_OK;
}

g3_status g3_set_apply_tensor_cores(g3_ctx* ctx, int on) {
    G3_CHECK(ctx != nullptr, "g3_set_apply_tensor_cores: ctx is NULL");
    ctx->apply_tensor_cores = on ? 1 : 0;
    return G3_OK;
}

g3_status g3_destroy(g3_ctx* ctx) {
    if (!ctx) return G3_OK;
    cudaSetDevice(ctx->device);
    for (auto& ev : ctx->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& ev : ctx->ev_side)
        if (ev) cudaEventDestroy(ev);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    delete ctx;
    return G3_OK;
}

int64_t g3_launch_count(const g3_ctx* ctx) { return ctx ? ctx->n_launch : 0; }

const char* g3_kernel_name(const g3_ctx* ctx, int i, int64_t* launches) {
    if (!ctx || i < 0 || i >= (int)ctx->launches.size()) return nullptr;
    auto it = ctx->launches.begin();
    std::advance(it, i);
    if (launches) *launches = it->second;
    return it->first.c_str();
}

// ---------------------------------------------------------------------------
// frequencies
// ---------------------------------------------------------------------------

static g3_status finish_freqs(g3_ctx* ctx, g3_freqs* f, const std::vector<double>& su_host) {
    // su_host: unique set as interleaved pairs [2 Ku]; f->s, f->omega: the full set
    G3_CUDA(f->d_s_all.alloc((size_t)f->K * 2 * sizeof(double)));
    G3_CUDA(f->d_w_all.alloc((size_t)f->K * 2 * sizeof(double)));
    G3_CUDA(cudaMemcpy(f->d_s_all.p, f->s.data(), (size_t)f->K * 2 * sizeof(double), cudaMemcpyHostToDevice));
    G3_CUDA(cudaMemcpy(f->d_w_all.p, f->omega.data(), (size_t)f->K * 2 * sizeof(double), cudaMemcpyHostToDevice));
    G3_CUDA(f->d_sd.alloc((size_t)f->Ku * 2 * sizeof(double)));
    G3_CUDA(f->d_sf.alloc((size_t)f->Ku * 2 * sizeof(float)));
    std::vector<float> sf(2 * (size_t)f->Ku);
    for (size_t i = 0; i < sf.size(); ++i) sf[i] = (float)su_host[i];
    G3_CUDA(cudaMemcpy(f->d_sd.p, su_host.data(), su_host.size() * sizeof(double), cudaMemcpyHostToDevice));
    G3_CUDA(cudaMemcpy(f->d_sf.p, sf.data(), sf.size() * sizeof(float), cudaMemcpyHostToDevice));
    G3_CUDA(f->d_uniq.alloc(f->uniq.size() * sizeof(int)));
    G3_CUDA(f->d_partner.alloc(f->partner.size() * sizeof(int)));
    G3_CUDA(cudaMemcpy(f->d_uniq.p, f->uniq.data(), f->uniq.size() * sizeof(int), cudaMemcpyHostToDevice));
    G3_CUDA(cudaMemcpy(f->d_partner.p, f->partner.data(), f->partner.size() * sizeof(int), cudaMemcpyHostToDevice));
    double best = -1;
    for (int u = 0; u < f->Ku; ++u) {
        double a = std::hypot(su_host[2 * u], su_host[2 * u + 1]);
        if (a > best) {
            best = a;
            f->k_maxabs = u;
        }
    }
    (void)ctx;
    return G3_OK;
}

g3_status g3_freqs_bdf2(g3_ctx* ctx, int K, double lambda, double dt, g3_freqs** out) {
    G3_CHECK(ctx && out, "g3_freqs_bdf2: NULL argument");
    *out = nullptr;
    G3_CHECK(K >= 2 && K % 2 == 0 && K <= 2 * 255, "g3_freqs_bdf2: K = %d must be even in [2, 510]", K);
    G3_CHECK(lambda > 0 && lambda < 1, "g3_freqs_bdf2: lambda = %g outside (0, 1)", lambda);
    G3_CHECK(dt > 0 && std::isfinite(dt), "g3_freqs_bdf2: dt = %g must be positive", dt);
    G3_TRY(use_device(ctx));
    g3_freqs* f = new (std::nothrow) g3_freqs();
    if (!f) return fail(G3_ENOMEM, "g3_freqs_bdf2: out of host memory");
    f->ctx = ctx;
    f->device = ctx->device;
    f->kind = 0;
    f->K = K;
    f->Ku = K / 2 + 1;
    DevBuf sd, sf;
    g3_status st = G3_OK;
    if (sd.alloc((size_t)f->Ku * 2 * sizeof(double)) != cudaSuccess || sf.alloc((size_t)f->Ku * 2 * sizeof(float)) != cudaSuccess)
        st = fail(G3_ENOMEM, "g3_freqs_bdf2: device allocation");
    if (st == G3_OK) st = launch_freqs_bdf2(ctx, K, f->Ku, lambda, dt, sd.as<double>(), sf.as<float>());
    std::vector<double> su(2 * (size_t)f->Ku);
    if (st == G3_OK) {
        cudaError_t e = cudaMemcpyAsync(su.data(), sd.p, su.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "g3_freqs_bdf2 copy");
    }
    if (st == G3_OK) {
        f->s.assign(2 * (size_t)K, 0.0);
        f->omega.assign(2 * (size_t)K, 0.0);
        f->uniq.resize(f->Ku);
        f->partner.resize(K);
        for (int k = 0; k < K; ++k) f->partner[k] = (K - k) % K;
        for (int u = 0; u < f->Ku; ++u) {
            f->uniq[u] = u;
            f->s[2 * u] = su[2 * u];
            f->s[2 * u + 1] = su[2 * u + 1];
        }
        for (int k = f->Ku; k < K; ++k) {
            f->s[2 * k] = su[2 * (K - k)];
            f->s[2 * k + 1] = -su[2 * (K - k) + 1];
        }
        st = finish_freqs(ctx, f, su);
    }
    if (st != G3_OK) {
        delete f;
        return st;
    }
    *out = f;
    return G3_OK;
}

g3_status g3_freqs_gcq(g3_ctx* ctx, int NQ, double dt_min, double dt_max, g3_freqs** out) {
    G3_CHECK(ctx && out, "g3_freqs_gcq: NULL argument");
    *out = nullptr;
    G3_CHECK(NQ >= 2 && NQ % 2 == 0 && NQ <= 512, "g3_freqs_gcq: NQ = %d must be even in [2, 512]", NQ);
    G3_CHECK(dt_min > 0 && std::isfinite(dt_max), "g3_freqs_gcq: dt_min must be positive");
    G3_CHECK(dt_max > dt_min,
             "g3_freqs_gcq: dt_max (%g) must exceed dt_min (%g); constant steps give q = 1, k = 0 where the contour "
             "degenerates",
             dt_max, dt_min);
    G3_TRY(use_device(ctx));
    g3_freqs* f = new (std::nothrow) g3_freqs();
    if (!f) return fail(G3_ENOMEM, "g3_freqs_gcq: out of host memory");
    f->ctx = ctx;
    f->device = ctx->device;
    f->kind = 1;
    f->K = NQ;
    f->Ku = NQ / 2;
    DevBuf ds, dw;
    g3_status st = G3_OK;
    if (ds.alloc((size_t)NQ * 2 * sizeof(double)) != cudaSuccess || dw.alloc((size_t)NQ * 2 * sizeof(double)) != cudaSuccess)
        st = fail(G3_ENOMEM, "g3_freqs_gcq: device allocation");
    if (st == G3_OK) st = launch_freqs_gcq(ctx, NQ, dt_min, dt_max, ds.as<double>(), dw.as<double>());
    f->s.assign(2 * (size_t)NQ, 0.0);
    f->omega.assign(2 * (size_t)NQ, 0.0);
    if (st == G3_OK) {
        cudaError_t e = cudaMemcpyAsync(f->s.data(), ds.p, f->s.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(f->omega.data(), dw.p, f->omega.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "g3_freqs_gcq copy");
    }
    if (st == G3_OK) {
        f->uniq.resize(f->Ku);
        f->partner.resize(NQ);
        for (int l = 0; l < NQ; ++l) f->partner[l] = NQ - 1 - l;
        std::vector<double> su(2 * (size_t)f->Ku);
        for (int u = 0; u < f->Ku; ++u) {
            f->uniq[u] = u;
            su[2 * u] = f->s[2 * u];
            su[2 * u + 1] = f->s[2 * u + 1];
        }
        for (double v : f->s)
            if (!std::isfinite(v)) st = fail(G3_ECUDA, "g3_freqs_gcq: non-finite contour point");
        if (st == G3_OK) st = finish_freqs(ctx, f, su);
    }
    if (st != G3_OK) {
        delete f;
        return st;
    }
    *out = f;
    return G3_OK;
}

// Frequencies given by the caller.  Conjugate pairing: l' pairs with l < l'
// when |s_l' - conj(s_l)| <= 1e-12 |s_l| (the first unpaired such l' in index
// order); a frequency with |Im s| <= 1e-12 |s| is its own partner (A(s) is
// real there), as is a complex frequency without a conjugate in the set.
// The unique set is the lower index of each pair plus the self-partnered
// frequencies, in increasing index order.
g3_status g3_freqs_from_array(g3_ctx* ctx, const double* s_re_im, int K, g3_freqs** out) {
    G3_CHECK(ctx && s_re_im && out, "g3_freqs_from_array: NULL argument");
    *out = nullptr;
    G3_CHECK(K >= 1 && K <= 512, "g3_freqs_from_array: K = %d outside [1, 512]", K);
    for (int l = 0; l < 2 * K; ++l)
        G3_CHECK(std::isfinite(s_re_im[l]), "g3_freqs_from_array: s[%d] is not finite", l / 2);
    for (int l = 0; l < K; ++l)
        G3_CHECK(s_re_im[2 * l] > 0.0, "g3_freqs_from_array: Re s[%d] = %g must be positive (the kernel "
                 "exp(-s r) / (4 pi r) of a damped problem)", l, s_re_im[2 * l]);
    std::vector<int32_t> partner(K, -1), uniq;
    const double tol = 1e-12;
    for (int l = 0; l < K; ++l) {
        if (partner[l] >= 0) continue;
        const double re = s_re_im[2 * l], im = s_re_im[2 * l + 1];
        const double mag = std::hypot(re, im);
        uniq.push_back(l);
        partner[l] = l;
        if (std::fabs(im) <= tol * mag) continue;
        for (int m = l + 1; m < K; ++m) {
            if (partner[m] >= 0) continue;
            if (std::hypot(s_re_im[2 * m] - re, s_re_im[2 * m + 1] + im) <= tol * mag) {
                partner[l] = m;
                partner[m] = l;
                break;
            }
        }
    }
    G3_CHECK((int)uniq.size() <= 256, "g3_freqs_from_array: %d unique frequencies, at most 256 are supported",
             (int)uniq.size());
    G3_TRY(use_device(ctx));
    g3_freqs* f = new (std::nothrow) g3_freqs();
    if (!f) return fail(G3_ENOMEM, "g3_freqs_from_array: out of host memory");
    f->ctx = ctx;
    f->device = ctx->device;
    f->kind = 2;
    f->K = K;
    f->Ku = (int)uniq.size();
    f->s.assign(s_re_im, s_re_im + 2 * (size_t)K);
    f->omega.assign(2 * (size_t)K, 0.0);
    f->uniq = uniq;
    f->partner = partner;
    std::vector<double> su(2 * (size_t)f->Ku);
    for (int u = 0; u < f->Ku; ++u) {
        su[2 * u] = s_re_im[2 * uniq[u]];
        su[2 * u + 1] = s_re_im[2 * uniq[u] + 1];
    }
    g3_status st = finish_freqs(ctx, f, su);
    if (st != G3_OK) {
        delete f;
        return st;
    }
    *out = f;
    return G3_OK;
}

g3_status g3_freqs_info(const g3_freqs* f, int* K, int* Ku) {
    G3_CHECK(f != nullptr, "g3_freqs_info: NULL handle");
    if (K) *K = f->K;
    if (Ku) *Ku = f->Ku;
    return G3_OK;
}

g3_status g3_freqs_get(const g3_freqs* f, double* s, double* omega, int32_t* uniq, int32_t* partner) {
    G3_CHECK(f != nullptr, "g3_freqs_get: NULL handle");
    if (s) std::memcpy(s, f->s.data(), f->s.size() * sizeof(double));
    if (omega) std::memcpy(omega, f->omega.data(), f->omega.size() * sizeof(double));
    if (uniq) std::memcpy(uniq, f->uniq.data(), f->uniq.size() * sizeof(int32_t));
    if (partner) std::memcpy(partner, f->partner.data(), f->partner.size() * sizeof(int32_t));
    return G3_OK;
}

g3_status g3_freqs_free(g3_freqs* f) {
    if (f) {
        cudaSetDevice(f->device);
        delete f;
    }
    return G3_OK;
}

// ---------------------------------------------------------------------------
// cluster tree
// ---------------------------------------------------------------------------

g3_status build_cluster_tree(g3_ctx* ctx, const double* verts, int nv, const int32_t* tris, int ne, int leaf,
                             double eta, g3_tree** out) {
    return build_cluster_tree_capped(ctx, verts, nv, tris, ne, leaf, eta, 0, out);
}

g3_status build_cluster_tree_capped(g3_ctx* ctx, const double* verts, int nv, const int32_t* tris, int ne, int leaf,
                                    double eta, int max_block, g3_tree** out) {
    G3_CHECK(ctx && verts && tris && out, "build_cluster_tree: NULL argument");
    *out = nullptr;
    G3_CHECK(nv >= 3 && ne >= 1, "build_cluster_tree: nv = %d, ne = %d", nv, ne);
    G3_CHECK(leaf >= 1, "build_cluster_tree: leaf = %d must be >= 1", leaf);
    G3_CHECK(max_block >= 0, "build_cluster_tree: max_block = %d must be >= 0", max_block);
    G3_CHECK(eta > 0 && std::isfinite(eta), "build_cluster_tree: eta = %g must be positive", eta);
    for (long long i = 0; i < 3LL * nv; ++i)
        G3_CHECK(std::isfinite(verts[i]), "build_cluster_tree: non-finite vertex coordinate at %lld", i);
    G3_TRY(use_device(ctx));
    g3_tree* t = new (std::nothrow) g3_tree();
    if (!t) return fail(G3_ENOMEM, "build_cluster_tree: out of host memory");
    t->ctx = ctx;
    t->device = ctx->device;
    t->ne = ne;
    t->nv = nv;
    t->leaf = leaf;
    t->max_block = max_block;
    t->eta = eta;
    t->verts.assign(verts, verts + 3 * (size_t)nv);
    t->tris.assign(tris, tris + 3 * (size_t)ne);
    g3_status st = build_tree_host(t);
    if (st == G3_OK) {
        if (t->d_perm.alloc(ne * sizeof(int)) != cudaSuccess) st = fail(G3_ENOMEM, "build_cluster_tree: perm");
    }
    if (st == G3_OK) {
        cudaError_t e = cudaMemcpyAsync(t->d_perm.p, t->perm.data(), ne * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "build_cluster_tree: perm copy");
    }
    if (st == G3_OK) {  // vertex ids in cluster order (Galerkin adjacency)
        std::vector<int> tv(3 * (size_t)ne);
        for (int p = 0; p < ne; ++p)
            for (int k = 0; k < 3; ++k) tv[3 * (size_t)p + k] = t->tris[3 * (size_t)t->perm[p] + k];
        cudaError_t e = t->d_tv.alloc(tv.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(t->d_tv.p, tv.data(), tv.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(e, "build_cluster_tree: vertex ids");
    }
    if (st == G3_OK) st = launch_geometry(ctx, t);
    if (st != G3_OK) {
        delete t;
        return st;
    }
    *out = t;
    return G3_OK;
}

g3_status g3_tree_subset(g3_ctx* ctx, const g3_tree* t, const int32_t* owner, int rank, g3_tree** out) {
    G3_CHECK(ctx && t && owner && out, "g3_tree_subset: NULL argument");
    G3_CHECK(!t->p1, "g3_tree_subset: the input must be an element tree");
    *out = nullptr;
    G3_TRY(use_device(ctx));
    g3_tree* s = new (std::nothrow) g3_tree();
    if (!s) return fail(G3_ENOMEM, "g3_tree_subset: out of host memory");
    s->ctx = ctx;
    s->device = ctx->device;
    s->ne = t->ne;
    s->nv = t->nv;
    s->leaf = t->leaf;
    s->max_block = t->max_block;
    s->eta = t->eta;
    s->subset = true;
    s->verts = t->verts;
    s->tris = t->tris;
    s->perm = t->perm;
    s->nodes = t->nodes;
    s->boxes = t->boxes;
    const size_t nb = t->blocks.size() / 5;
    for (size_t b = 0; b < nb; ++b)
        if (owner[b] == rank) s->blocks.insert(s->blocks.end(), &t->blocks[5 * b], &t->blocks[5 * b] + 5);
    tree_index_blocks(s);
    // device copies: the same uploads as build_cluster_tree (deterministic)
    g3_status st = G3_OK;
    cudaError_t e = s->d_perm.alloc(s->ne * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(s->d_perm.p, s->perm.data(), s->ne * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<int> tv(3 * (size_t)s->ne);
        for (int p = 0; p < s->ne; ++p)
            for (int k = 0; k < 3; ++k) tv[3 * (size_t)p + k] = s->tris[3 * (size_t)s->perm[p] + k];
        e = s->d_tv.alloc(tv.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(s->d_tv.p, tv.data(), tv.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) st = cuda_fail(e, "g3_tree_subset: device copies");
    if (st == G3_OK) st = launch_geometry(ctx, s);
    if (st != G3_OK) {
        delete s;
        return st;
    }
    *out = s;
    return G3_OK;
}

// tree of element-local linear shape functions (linear continuous elements):
// position 3 p + a is local vertex a of the element at cluster position p;
// nodes and blocks are the element tree's with tripled ranges; the geometry
// stays per element, with the surface curls of the shape functions added
g3_status build_p1_tree(g3_ctx* ctx, const g3_tree* t, g3_tree** out) {
    G3_CHECK(ctx && t && out, "build_p1_tree: NULL argument");
    *out = nullptr;
    G3_CHECK(!t->p1 && !t->subset, "build_p1_tree: the input must be an element tree of build_cluster_tree");
    G3_TRY(use_device(ctx));
    g3_tree* s = new (std::nothrow) g3_tree();
    if (!s) return fail(G3_ENOMEM, "build_p1_tree: out of host memory");
    const int E = t->ne;
    s->ctx = ctx;
    s->device = ctx->device;
    s->ne = E;  // element count while the geometry is set up (below: 3 E)
    s->nv = t->nv;
    s->leaf = t->leaf;
    s->max_block = t->max_block;
    s->eta = t->eta;
    s->verts = t->verts;
    s->tris = t->tris;
    s->p1 = true;
    s->ne_elem = E;
    s->perm_elem = t->perm;
    s->boxes = t->boxes;
    s->nodes = t->nodes;
    for (size_t n = 0; n < s->nodes.size() / 4; ++n) {
        s->nodes[4 * n] *= 3;
        s->nodes[4 * n + 1] *= 3;
    }
    s->blocks = t->blocks;
    for (size_t b = 0; b < s->blocks.size() / 5; ++b)
        for (int k = 0; k < 4; ++k) s->blocks[5 * b + k] *= 3;
    tree_index_blocks(s);
    g3_status st = G3_OK;
    auto chk = [&](cudaError_t e, const char* w) {
        if (st == G3_OK && e != cudaSuccess) st = cuda_fail(e, w);
    };
    // element geometry (cluster order of the elements)
    chk(s->d_perm.alloc(E * sizeof(int)), "build_p1_tree: perm");
    if (st == G3_OK) chk(cudaMemcpy(s->d_perm.p, t->perm.data(), E * sizeof(int), cudaMemcpyHostToDevice), "copy");
    std::vector<int> tv(3 * (size_t)E);
    for (int p = 0; p < E; ++p)
        for (int k = 0; k < 3; ++k) tv[3 * (size_t)p + k] = t->tris[3 * (size_t)t->perm[p] + k];
    chk(s->d_tv.alloc(tv.size() * sizeof(int)), "build_p1_tree: vertex ids");
    if (st == G3_OK) chk(cudaMemcpy(s->d_tv.p, tv.data(), tv.size() * sizeof(int), cudaMemcpyHostToDevice), "copy");
    if (st == G3_OK) st = launch_geometry(ctx, s);
    // surface curls of the barycentric coordinates, float64 on the host:
    // curl lambda_a = n x grad lambda_a, grad lambda_a = n x (v_{a+2} - v_{a+1}) / (2 area)
    std::vector<double> cd(9 * (size_t)E);
    std::vector<float> cf(9 * (size_t)E);
    for (int p = 0; p < E && st == G3_OK; ++p) {
        double v[3][3];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) v[a][k] = t->verts[3 * (size_t)tv[3 * (size_t)p + a] + k];
        double u[3], w[3];
        for (int k = 0; k < 3; ++k) {
            u[k] = v[1][k] - v[0][k];
            w[k] = v[2][k] - v[0][k];
        }
        double c[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double a2 = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        const double n[3] = {c[0] / a2, c[1] / a2, c[2] / a2};
        for (int a = 0; a < 3; ++a) {
            const double* p2 = v[(a + 2) % 3];
            const double* p1 = v[(a + 1) % 3];
            const double e[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
            const double g[3] = {(n[1] * e[2] - n[2] * e[1]) / a2, (n[2] * e[0] - n[0] * e[2]) / a2,
                                 (n[0] * e[1] - n[1] * e[0]) / a2};
            const double cu[3] = {n[1] * g[2] - n[2] * g[1], n[2] * g[0] - n[0] * g[2], n[0] * g[1] - n[1] * g[0]};
            for (int k = 0; k < 3; ++k) {
                cd[(a * 3 + k) * (size_t)E + p] = cu[k];
                cf[(a * 3 + k) * (size_t)E + p] = (float)cu[k];
            }
        }
    }
    chk(s->d_curl_d.alloc(cd.size() * sizeof(double)), "build_p1_tree: curls");
    chk(s->d_curl_f.alloc(cf.size() * sizeof(float)), "build_p1_tree: curls");
    if (st == G3_OK) chk(cudaMemcpy(s->d_curl_d.p, cd.data(), cd.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
    if (st == G3_OK) chk(cudaMemcpy(s->d_curl_f.p, cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice), "copy");
    // positions of the degrees of freedom: original index 3 e + a and vertex
    std::vector<int32_t> perm3(3 * (size_t)E), src(3 * (size_t)E);
    for (int p = 0; p < E; ++p)
        for (int a = 0; a < 3; ++a) {
            perm3[3 * (size_t)p + a] = 3 * t->perm[p] + a;
            src[3 * (size_t)p + a] = tv[3 * (size_t)p + a];
        }
    if (st == G3_OK) {
        s->gf.curl = s->d_curl_f.as<float>();
        s->gd.curl = s->d_curl_d.as<double>();
        s->perm = perm3;
        s->ne = 3 * E;
        chk(s->d_perm.alloc(perm3.size() * sizeof(int)), "build_p1_tree: perm");
        if (st == G3_OK)
            chk(cudaMemcpy(s->d_perm.p, perm3.data(), perm3.size() * sizeof(int), cudaMemcpyHostToDevice), "copy");
        chk(s->d_src.alloc(src.size() * sizeof(int)), "build_p1_tree: vertices");
        if (st == G3_OK) chk(cudaMemcpy(s->d_src.p, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice), "copy");
    }
    if (st != G3_OK) {
        delete s;
        return st;
    }
    *out = s;
    return G3_OK;
}

g3_status g3_tree_info(const g3_tree* t, int* ne, int* n_nodes, int* n_blocks, int* n_far, int* n_near) {
    G3_CHECK(t != nullptr, "g3_tree_info: NULL handle");
    if (ne) *ne = t->ne;
    if (n_nodes) *n_nodes = (int)(t->nodes.size() / 4);
    if (n_blocks) *n_blocks = (int)(t->blocks.size() / 5);
    if (n_far) *n_far = (int)t->far_index.size();
    if (n_near) *n_near = (int)t->near_index.size();
    return G3_OK;
}

g3_status g3_tree_get(const g3_tree* t, int32_t* perm, int32_t* nodes, double* boxes, int32_t* blocks,
                      int32_t* far_index) {
    G3_CHECK(t != nullptr, "g3_tree_get: NULL handle");
    if (perm) std::memcpy(perm, t->perm.data(), t->perm.size() * sizeof(int32_t));
    if (nodes) std::memcpy(nodes, t->nodes.data(), t->nodes.size() * sizeof(int32_t));
    if (boxes) std::memcpy(boxes, t->boxes.data(), t->boxes.size() * sizeof(double));
    if (blocks) std::memcpy(blocks, t->blocks.data(), t->blocks.size() * sizeof(int32_t));
    if (far_index) std::memcpy(far_index, t->far_index.data(), t->far_index.size() * sizeof(int32_t));
    return G3_OK;
}

g3_status g3_tree_free(g3_tree* t) {
    if (t) {
        cudaSetDevice(t->device);
        delete t;
    }
    return G3_OK;
}

// ---------------------------------------------------------------------------
// entries
// ---------------------------------------------------------------------------

static bool valid_kernel(int k) { return k == G3_SLP || k == G3_DLP; }
// kernel for a tree and scheme: the operators of linear elements need a tree
// of build_p1_tree and the Galerkin scheme, the others an element tree
static bool kernel_fits_tree(int k, int scheme, const g3_tree* t) {
    if (t->p1) return (k == G3_HYPERSINGULAR || k == G3_ADJOINT_DLP) && scheme == G3_GALERKIN4x4;
    return valid_kernel(k);
}
static bool valid_prec(int p) { return p == G3_FP64 || p == G3_MIXED; }

g3_status g3_entries(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, g3_scheme scheme,
                     g3_precision prec, const int32_t* rows, const int32_t* cols, int n, const int32_t* kidx, int nk,
                     double* out) {
    G3_CHECK(ctx && t && f && out, "g3_entries: NULL argument");
    G3_CHECK(n >= 0 && nk >= 0, "g3_entries: negative size");
    G3_CHECK(n == 0 || (rows && cols), "g3_entries: rows/cols NULL");
    G3_CHECK(nk == 0 || kidx, "g3_entries: kidx NULL");
    G3_CHECK(valid_prec(prec), "g3_entries: bad precision");
    G3_CHECK(kernel_fits_tree(kernel, scheme, t), "g3_entries: kernel %d with scheme %d does not fit this tree",
             (int)kernel, (int)scheme);
    if (t->p1)  // linear elements: the regular rule only (pairs of elements without a common vertex)
        for (int i = 0; i < n; ++i) {
            G3_CHECK(rows[i] >= 0 && rows[i] < t->ne && cols[i] >= 0 && cols[i] < t->ne,
                     "g3_entries: pair %d = (%d, %d) outside [0, %d)", i, rows[i], cols[i], t->ne);
            const int* a = &t->tris[3 * (size_t)(rows[i] / 3)];
            const int* b = &t->tris[3 * (size_t)(cols[i] / 3)];
            bool shared = false;
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) shared |= a[x] == b[y];
            if (shared)
                return fail(G3_EUNSUPPORTED, "g3_entries: pair %d of linear elements shares a vertex (near field only)", i);
        }
    if (n == 0 || nk == 0) return G3_OK;
    G3_TRY(use_device(ctx));
    std::vector<int> inv(t->ne);
    for (int p = 0; p < t->ne; ++p) inv[t->perm[p]] = p;
    std::vector<int> r(n), c(n), ku(nk), cj(nk);
    for (int i = 0; i < n; ++i) {
        G3_CHECK(rows[i] >= 0 && rows[i] < t->ne && cols[i] >= 0 && cols[i] < t->ne,
                 "g3_entries: pair %d = (%d, %d) outside [0, %d)", i, rows[i], cols[i], t->ne);
        r[i] = inv[rows[i]];
        c[i] = inv[cols[i]];
    }
    std::vector<int> upos(f->K, -1);
    for (int u = 0; u < f->Ku; ++u) upos[f->uniq[u]] = u;
    for (int m = 0; m < nk; ++m) {
        G3_CHECK(kidx[m] >= 0 && kidx[m] < f->K, "g3_entries: kidx[%d] = %d outside [0, %d)", m, kidx[m], f->K);
        if (upos[kidx[m]] >= 0) {
            ku[m] = upos[kidx[m]];
            cj[m] = 0;
        } else {
            ku[m] = upos[f->partner[kidx[m]]];
            cj[m] = 1;
        }
    }
    DevBuf dr, dc, dk, dj, dout;
    G3_CUDA(dr.alloc(n * sizeof(int)));
    G3_CUDA(dc.alloc(n * sizeof(int)));
    G3_CUDA(dk.alloc(nk * sizeof(int)));
    G3_CUDA(dj.alloc(nk * sizeof(int)));
    G3_CUDA(dout.alloc((size_t)n * nk * 2 * sizeof(double)));
    G3_CUDA(cudaMemcpyAsync(dr.p, r.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    G3_CUDA(cudaMemcpyAsync(dc.p, c.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    G3_CUDA(cudaMemcpyAsync(dk.p, ku.data(), nk * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    G3_CUDA(cudaMemcpyAsync(dj.p, cj.data(), nk * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    G3_TRY(launch_entries(ctx, t, f, kernel, scheme, prec, dr.as<int>(), dc.as<int>(), n, dk.as<int>(), dj.as<int>(), nk,
                          dout.as<double>()));
    G3_CUDA(cudaMemcpyAsync(out, dout.p, (size_t)n * nk * 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    G3_CUDA(cudaStreamSynchronize(ctx->stream));
    return G3_OK;
}

// ---------------------------------------------------------------------------
// near field
// ---------------------------------------------------------------------------

g3_status assemble_near(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, g3_scheme scheme,
                        g3_precision prec, g3_near** out) {
    G3_CHECK(ctx && t && f && out, "assemble_near: NULL argument");
    *out = nullptr;
    G3_CHECK(valid_prec(prec), "assemble_near: bad precision");
    G3_CHECK(scheme == G3_COLLOC7 || scheme == G3_GALERKIN4x4, "assemble_near: bad scheme");
    G3_CHECK(kernel_fits_tree(kernel, scheme, t),
             "assemble_near: kernel %d with scheme %d does not fit this tree (linear-element operators need a "
             "tree of build_p1_tree and G3_GALERKIN4x4)", (int)kernel, (int)scheme);
    if (!t->p1 && scheme == G3_GALERKIN4x4 && kernel != G3_SLP)
        return fail(G3_EUNSUPPORTED, "assemble_near: the Galerkin scheme with piecewise-constant elements is implemented for G3_SLP");
    G3_TRY(use_device(ctx));
    g3_near* nf = new (std::nothrow) g3_near();
    if (!nf) return fail(G3_ENOMEM, "assemble_near: out of host memory");
    nf->ctx = ctx;
    nf->device = ctx->device;
    nf->tree = t;
    nf->freqs = f;
    nf->prec = prec;
    nf->kernel = kernel;
    nf->Ku = f->Ku;
    nf->K = f->K;
    nf->scheme = scheme;
    nf->order = t->near_index;
    std::stable_sort(nf->order.begin(), nf->order.end(), [t](int a, int b) {
        const int32_t* x = &t->blocks[5 * (size_t)a];
        const int32_t* y = &t->blocks[5 * (size_t)b];
        if (x[0] != y[0]) return x[0] < y[0];
        return x[2] < y[2];
    });
    std::vector<BlockRange> rg;
    long long off = 0;
    for (size_t i = 0; i < nf->order.size(); ++i) {
        const int32_t* x = &t->blocks[5 * (size_t)nf->order[i]];
        rg.push_back(BlockRange{x[0], x[1], x[2], x[3]});
        nf->offs.push_back(off);
        off += (long long)(x[1] - x[0]) * (x[3] - x[2]) * f->Ku;
        if (i == 0 || x[0] != rg[i - 1].rb) nf->row_start.push_back((int)i);
    }
    nf->row_start.push_back((int)nf->order.size());
    nf->n_entries = off;
    // position of every self entry (p, p): the diagonal leaf block (tau, tau)
    // is non-admissible (dist = 0), so each element has exactly one
    std::vector<long long> diag_base(t->ne, -1);
    std::vector<int> diag_mn(t->ne, 0);
    for (size_t i = 0; i < rg.size(); ++i) {
        const BlockRange& r = rg[i];
        for (int p = std::max(r.rb, r.cb); p < std::min(r.re, r.ce); ++p) {
            const int N = r.ce - r.cb;
            diag_base[p] = nf->offs[i] + (long long)(p - r.cb) * (r.re - r.rb) + (p - r.rb);  // [k][j][i]
            diag_mn[p] = (r.re - r.rb) * N;
        }
    }
    for (int p = 0; p < t->ne; ++p)
        if (diag_base[p] < 0 && !t->subset) {  // (a rank's subset holds only its rows' diagonal blocks)
            delete nf;
            return fail(G3_EINVAL, "assemble_near: element %d has no diagonal near block", p);
        }
    // Galerkin: the pairs with a common vertex (Sauter-Schwab); they all lie
    // in near blocks (a far block's clusters have disjoint boxes)
    std::vector<SsPair> ss;
    if (t->p1) {
        // element pairs with a common vertex inside each near block; the local
        // entries (a, b) of the pair sit at off + a + b M (frequency stride M N)
        const int E = t->ne_elem;
        std::vector<int> tv(3 * (size_t)E);
        for (int p = 0; p < E; ++p)
            for (int k = 0; k < 3; ++k) tv[3 * (size_t)p + k] = t->tris[3 * (size_t)t->perm_elem[p] + k];
        for (size_t b = 0; b < rg.size(); ++b) {
            const BlockRange& r = rg[b];
            const int M = r.re - r.rb, N = r.ce - r.cb;
            for (int je = r.cb / 3; je < r.ce / 3; ++je)
                for (int ie = r.rb / 3; ie < r.re / 3; ++ie) {
                    SsPair q{};
                    q.cas = ss_classify(&tv[3 * (size_t)ie], &tv[3 * (size_t)je], ie == je, q.px, q.py);
                    if (q.cas == SS_REGULAR) continue;
                    q.i = ie;
                    q.j = je;
                    q.stride = M * N;
                    q.ldm = M;
                    q.off = nf->offs[b] + (long long)(3 * je - r.cb) * M + (3 * ie - r.rb);
                    ss.push_back(q);
                }
        }
        nf->n_ss = (int)ss.size();
    } else if (scheme == G3_GALERKIN4x4) {
        std::vector<int> tv(3 * (size_t)t->ne);
        for (int p = 0; p < t->ne; ++p)
            for (int k = 0; k < 3; ++k) tv[3 * (size_t)p + k] = t->tris[3 * (size_t)t->perm[p] + k];
        for (size_t b = 0; b < rg.size(); ++b) {
            const BlockRange& r = rg[b];
            const int M = r.re - r.rb, N = r.ce - r.cb;
            for (int j = r.cb; j < r.ce; ++j)
                for (int i = r.rb; i < r.re; ++i) {
                    SsPair q{};
                    q.cas = ss_classify(&tv[3 * (size_t)i], &tv[3 * (size_t)j], i == j, q.px, q.py);
                    if (q.cas == SS_REGULAR) continue;
                    q.i = i;
                    q.j = j;
                    q.stride = M * N;
                    q.off = nf->offs[b] + (long long)(j - r.cb) * M + (i - r.rb);  // [k][j][i]
                    ss.push_back(q);
                }
        }
        nf->n_ss = (int)ss.size();
    }
    const size_t esz = prec == G3_MIXED ? 8 : 16;
    g3_status st = G3_OK;
    auto chk = [&](cudaError_t e, const char* w) {
        if (st == G3_OK && e != cudaSuccess) st = cuda_fail(e, w);
    };
    if (!ss.empty()) {
        chk(nf->d_ss.alloc(ss.size() * sizeof(SsPair)), "assemble_near: singular pairs");
        if (st == G3_OK)
            chk(cudaMemcpy(nf->d_ss.p, ss.data(), ss.size() * sizeof(SsPair), cudaMemcpyHostToDevice), "copy");
    }
    chk(nf->data.alloc((size_t)off * esz), "assemble_near: near-field storage");
    chk(nf->d_ranges.alloc(rg.size() * sizeof(BlockRange)), "assemble_near: ranges");
    chk(nf->d_offs.alloc(nf->offs.size() * sizeof(long long)), "assemble_near: offsets");
    chk(nf->d_row_start.alloc(nf->row_start.size() * sizeof(int)), "assemble_near: rows");
    chk(nf->d_diag_base.alloc(t->ne * sizeof(long long)), "assemble_near: diagonal offsets");
    chk(nf->d_diag_mn.alloc(t->ne * sizeof(int)), "assemble_near: diagonal sizes");
    if (st == G3_OK) {
        chk(cudaMemcpyAsync(nf->d_diag_base.p, diag_base.data(), t->ne * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream), "copy");
        chk(cudaMemcpyAsync(nf->d_diag_mn.p, diag_mn.data(), t->ne * sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "copy");
    }
    if (st == G3_OK && !rg.empty()) {
        chk(cudaMemcpyAsync(nf->d_ranges.p, rg.data(), rg.size() * sizeof(BlockRange), cudaMemcpyHostToDevice, ctx->stream), "copy");
        chk(cudaMemcpyAsync(nf->d_offs.p, nf->offs.data(), nf->offs.size() * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream), "copy");
        chk(cudaMemcpyAsync(nf->d_row_start.p, nf->row_start.data(), nf->row_start.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "copy");
    }
    if (st == G3_OK) chk(cudaEventRecord(ctx->ev[0], ctx->stream), "event");
    if (st == G3_OK) st = launch_near(ctx, t, f, nf, kernel, scheme);
    if (st == G3_OK) chk(cudaEventRecord(ctx->ev[1], ctx->stream), "event");
    if (st == G3_OK) chk(cudaEventSynchronize(ctx->ev[1]), "assemble_near: kernel");
    if (st == G3_OK) {
        float ms = 0;
        chk(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]), "event time");
        nf->ms = ms;
    }
    if (st != G3_OK) {
        delete nf;
        return st;
    }
    *out = nf;
    return G3_OK;
}

g3_status g3_near_info(const g3_near* nf, int64_t* n_entries, int64_t* bytes, double* ms) {
    G3_CHECK(nf != nullptr, "g3_near_info: NULL handle");
    if (n_entries) *n_entries = nf->n_entries;
    if (bytes) *bytes = nf->n_entries * (nf->prec == G3_MIXED ? 8 : 16);
    if (ms) *ms = nf->ms;
    return G3_OK;
}

g3_status g3_near_get_block(const g3_near* nf, int block, double* out) {
    G3_CHECK(nf && out, "g3_near_get_block: NULL argument");
    const g3_tree* t = nf->tree;
    G3_CHECK(block >= 0 && block < (int)(t->blocks.size() / 5), "g3_near_get_block: block %d out of range", block);
    auto it = std::find(nf->order.begin(), nf->order.end(), block);
    G3_CHECK(it != nf->order.end(), "g3_near_get_block: block %d is admissible", block);
    const size_t pos = it - nf->order.begin();
    const int32_t* x = &t->blocks[5 * (size_t)block];
    const size_t M = x[1] - x[0], N = x[3] - x[2];
    const size_t n = M * N * nf->Ku;
    G3_TRY(use_device(nf->ctx));
    std::vector<double> tmp(2 * n);
    if (nf->prec == G3_MIXED) {
        std::vector<float> tf(2 * n);
        G3_CUDA(cudaMemcpy(tf.data(), nf->data.as<float>() + 2 * nf->offs[pos], tf.size() * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < tf.size(); ++i) tmp[i] = tf[i];
    } else {
        G3_CUDA(cudaMemcpy(tmp.data(), nf->data.as<double>() + 2 * nf->offs[pos], 2 * n * sizeof(double), cudaMemcpyDeviceToHost));
    }
    // device layout [k][j][i] -> exported [k][i][j]
    for (size_t k = 0; k < (size_t)nf->Ku; ++k)
        for (size_t i = 0; i < M; ++i)
            for (size_t j = 0; j < N; ++j) {
                const size_t src = k * M * N + j * M + i, dst = k * M * N + i * N + j;
                out[2 * dst] = tmp[2 * src];
                out[2 * dst + 1] = tmp[2 * src + 1];
            }
    return G3_OK;
}

g3_status g3_near_free(g3_near* nf) {
    if (nf) {
        cudaSetDevice(nf->device);
        delete nf;
    }
    return G3_OK;
}

// ---------------------------------------------------------------------------
// compression
// ---------------------------------------------------------------------------

static g3_opts defaults(const g3_opts* o) {
    g3_opts d{};
    if (o) d = *o;
    return d;
}

g3_status aca3_compress(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, g3_scheme scheme,
                        g3_precision prec, double eps3, const g3_opts* opts, g3_factors** out) {
    G3_CHECK(ctx && t && f && out, "aca3_compress: NULL argument");
    *out = nullptr;
    G3_CHECK(valid_prec(prec), "aca3_compress: bad precision");
    G3_CHECK(scheme == G3_COLLOC7 || scheme == G3_GALERKIN4x4, "aca3_compress: bad scheme");
    G3_CHECK(kernel_fits_tree(kernel, scheme, t),
             "aca3_compress: kernel %d with scheme %d does not fit this tree (linear-element operators need a "
             "tree of build_p1_tree and G3_GALERKIN4x4)", (int)kernel, (int)scheme);
    G3_CHECK(eps3 > 0 && eps3 < 1, "aca3_compress: eps3 = %g outside (0, 1)", eps3);
    g3_opts o = defaults(opts);
    if (t->p1) {
        G3_CHECK(o.threads == 0 || o.threads == 256, "aca3_compress: linear-element operators run with 256 threads");
        G3_CHECK(o.mlp == nullptr && !o.whole_matrix && !o.unbatched,
                 "aca3_compress: linear-element operators take no predictor, whole-matrix or unbatched run");
    }
    G3_CHECK(o.face_rank_max >= 0 && o.face_rank_max <= 64, "aca3_compress: face_rank_max = %d outside [0, 64]", o.face_rank_max);
    G3_CHECK(o.threads == 0 || o.threads == 128 || o.threads == 256 || o.threads == 384 || o.threads == 512,
             "aca3_compress: threads must be 0, 128, 256, 384 or 512");
    G3_CHECK(o.mlp_use >= 0 && o.mlp_use <= 7, "aca3_compress: mlp_use = %d outside [0, 7]", o.mlp_use);
    G3_TRY(use_device(ctx));
    g3_factors* fa = new (std::nothrow) g3_factors();
    if (!fa) return fail(G3_ENOMEM, "aca3_compress: out of host memory");
    fa->ctx = ctx;
    fa->device = ctx->device;
    fa->tree = t;
    fa->freqs = f;
    fa->prec = prec;
    fa->kernel = kernel;
    fa->Ku = f->Ku;
    fa->K = f->K;
    g3_status st = run_aca(ctx, t, f, fa, kernel, scheme, eps3, o, nullptr, nullptr, nullptr, 0);
    if (st != G3_OK) {
        delete fa;
        return st;
    }
    *out = fa;
    return G3_OK;
}

static int log2_ceil(int x) {
    int b = 0;
    while ((1 << b) < x) ++b;
    return b;
}

g3_status g3_autotune(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, g3_scheme scheme,
                      g3_precision prec, double eps3, g3_opts* opts, double* best_ms) {
    G3_CHECK(ctx && t && f && opts, "g3_autotune: NULL argument");
    G3_CHECK(kernel == G3_SLP || kernel == G3_DLP, "g3_autotune: kernel must be G3_SLP or G3_DLP");
    G3_CHECK(valid_prec(prec), "g3_autotune: bad precision");
    G3_CHECK(eps3 > 0 && eps3 < 1, "g3_autotune: eps3 = %g outside (0, 1)", eps3);
    const int side = std::max(t->max_far_m, t->max_far_n);
    const long long key = (((long long)log2_ceil(f->Ku) * 32 + log2_ceil(std::max(side, 1))) * 8 + kernel) * 8 +
                          scheme * 2 + prec;
    if (best_ms) *best_ms = 0.0;
    auto hit = ctx->tune_cache.find(key);
    if (hit != ctx->tune_cache.end()) {
        opts->threads = hit->second[0];
        opts->dense_face_max = hit->second[1];
        opts->residual_face_max = hit->second[2];
        return G3_OK;
    }
    G3_TRY(use_device(ctx));
    const int threads[4] = {256, 384, 128, 512};
    const int dmax[3] = {24 * 24, 48 * 48, 64 * 64};
    double best = -1.0;
    int bt = 256, bd = 48 * 48;
    for (int a = 0; a < (prec == G3_MIXED ? 4 : 1); ++a)
        for (int b = 0; b < 3; ++b) {
            g3_opts o = *opts;
            o.threads = threads[a];
            o.dense_face_max = dmax[b];
            g3_factors* fa = nullptr;
            G3_TRY(aca3_compress(ctx, t, f, kernel, scheme, prec, eps3, &o, &fa));
            const double ms = fa->stats.ms;
            g3_factors_free(fa);
            if (best < 0 || ms < best) {
                best = ms;
                bt = threads[a];
                bd = dmax[b];
            }
        }
    // the dense residual working faces (on by default in float32) against
    // rows and columns evaluated on demand, at the fastest shape: which wins
    // depends on how many ACA steps a face takes against its M_b N_b entries
    int br = opts->residual_face_max;
    if (prec == G3_MIXED && br >= 0) {
        g3_opts o = *opts;
        o.threads = bt;
        o.dense_face_max = bd;
        o.residual_face_max = -1;
        g3_factors* fa = nullptr;
        G3_TRY(aca3_compress(ctx, t, f, kernel, scheme, prec, eps3, &o, &fa));
        const double ms = fa->stats.ms;
        g3_factors_free(fa);
        if (ms < best) {
            best = ms;
            br = -1;
        }
    }
    ctx->tune_cache[key] = {bt, bd, br};
    opts->threads = bt;
    opts->dense_face_max = bd;
    opts->residual_face_max = br;
    if (best_ms) *best_ms = best;
    return G3_OK;
}

g3_status aca3_compress_batch(g3_ctx* ctx, const g3_tree* const* trees, const g3_freqs* const* freqs, int n_geom,
                              g3_kernel kernel, g3_scheme scheme, g3_precision prec, double eps3, const g3_opts* opts,
                              g3_factors** out) {
    G3_CHECK(ctx && trees && freqs && out, "aca3_compress_batch: NULL argument");
    G3_CHECK(n_geom >= 1, "aca3_compress_batch: n_geom = %d", n_geom);
    for (int j = 0; j < n_geom; ++j) {
        out[j] = nullptr;
        G3_CHECK(trees[j] && freqs[j], "aca3_compress_batch: NULL tree or frequencies for mesh %d", j);
    }
    G3_CHECK(kernel == G3_SLP || kernel == G3_DLP, "aca3_compress_batch: kernel must be G3_SLP or G3_DLP");
    G3_CHECK(valid_prec(prec), "aca3_compress_batch: bad precision");
    G3_CHECK(scheme == G3_COLLOC7 || scheme == G3_GALERKIN4x4, "aca3_compress_batch: bad scheme");
    G3_CHECK(eps3 > 0 && eps3 < 1, "aca3_compress_batch: eps3 = %g outside (0, 1)", eps3);
    g3_opts o = defaults(opts);
    G3_CHECK(o.k1 == nullptr && o.cost == nullptr, "aca3_compress_batch: opts->k1 and opts->cost are per mesh; not accepted");
    G3_CHECK(o.face_rank_max >= 0 && o.face_rank_max <= 64, "aca3_compress_batch: face_rank_max = %d outside [0, 64]",
             o.face_rank_max);
    G3_CHECK(o.threads == 0 || o.threads == 128 || o.threads == 256 || o.threads == 384 || o.threads == 512,
             "aca3_compress_batch: threads must be 0, 128, 256, 384 or 512");
    G3_CHECK(o.mlp_use >= 0 && o.mlp_use <= 7, "aca3_compress_batch: mlp_use = %d outside [0, 7]", o.mlp_use);
    G3_CHECK(!o.unbatched, "aca3_compress_batch: unbatched is not accepted");
    G3_TRY(use_device(ctx));
    std::vector<g3_factors*> fas(n_geom, nullptr);
    for (int j = 0; j < n_geom; ++j) {
        g3_factors* fa = new (std::nothrow) g3_factors();
        if (!fa) {
            for (auto* x : fas) delete x;
            return fail(G3_ENOMEM, "aca3_compress_batch: out of host memory");
        }
        fa->ctx = ctx;
        fa->device = ctx->device;
        fa->tree = trees[j];
        fa->freqs = freqs[j];
        fa->prec = prec;
        fa->kernel = kernel;
        fa->Ku = freqs[j]->Ku;
        fa->K = freqs[j]->K;
        fas[j] = fa;
    }
    g3_status st = run_aca_batch(ctx, trees, freqs, n_geom, fas.data(), kernel, scheme, eps3, o);
    if (st != G3_OK) {
        for (auto* x : fas) delete x;
        return st;
    }
    for (int j = 0; j < n_geom; ++j) out[j] = fas[j];
    return G3_OK;
}

g3_status aca3_compress_separable(g3_ctx* ctx, const double* a, const double* b, const double* c, int R, int M, int N,
                                  int Ku, g3_precision prec, double eps3, const g3_opts* opts, g3_factors** out) {
    G3_CHECK(ctx && a && b && c && out, "aca3_compress_separable: NULL argument");
    *out = nullptr;
    G3_CHECK(R >= 1 && M >= 1 && N >= 1 && Ku >= 1 && Ku <= 256, "aca3_compress_separable: bad sizes");
    G3_CHECK(valid_prec(prec), "aca3_compress_separable: bad precision");
    G3_CHECK(eps3 > 0 && eps3 < 1, "aca3_compress_separable: eps3 = %g outside (0, 1)", eps3);
    g3_opts o = defaults(opts);
    G3_TRY(use_device(ctx));
    g3_factors* fa = new (std::nothrow) g3_factors();
    if (!fa) return fail(G3_ENOMEM, "aca3_compress_separable: out of host memory");
    fa->ctx = ctx;
    fa->device = ctx->device;
    fa->prec = prec;
    fa->kernel = G3_SEPARABLE;
    fa->Ku = Ku;
    fa->K = Ku;
    fa->M_sep = M;
    fa->N_sep = N;
    g3_status st = run_aca(ctx, nullptr, nullptr, fa, G3_SEPARABLE, G3_COLLOC7, eps3, o, a, b, c, R);
    if (st != G3_OK) {
        delete fa;
        return st;
    }
    *out = fa;
    return G3_OK;
}

g3_status g3_factors_stats(const g3_factors* fa, g3_stats* out) {
    G3_CHECK(fa && out, "g3_factors_stats: NULL argument");
    *out = fa->stats;
    return G3_OK;
}

g3_status g3_factors_ranks(const g3_factors* fa, int32_t* r3) {
    G3_CHECK(fa && r3, "g3_factors_ranks: NULL argument");
    std::memcpy(r3, fa->r3.data(), fa->r3.size() * sizeof(int32_t));
    return G3_OK;
}

g3_status g3_factors_block_cycles(const g3_factors* fa, int64_t* cycles) {
    G3_CHECK(fa && cycles, "g3_factors_block_cycles: NULL argument");
    for (size_t i = 0; i < fa->cycles.size(); ++i) cycles[i] = (int64_t)fa->cycles[i];
    return G3_OK;
}

g3_status g3_factors_block_phases(const g3_factors* fa, int64_t* out) {
    G3_CHECK(fa && out, "g3_factors_block_phases: NULL argument");
    for (size_t i = 0; i < fa->phases.size(); ++i) out[i] = (int64_t)fa->phases[i];
    return G3_OK;
}

g3_status g3_factors_get_block(const g3_factors* fa, int i, int32_t* r3, int32_t* face_ranks, double* U, double* V,
                               double* fib, int32_t* piv) {
    G3_CHECK(fa != nullptr, "g3_factors_get_block: NULL handle");
    G3_CHECK(i >= 0 && i < fa->n_far, "g3_factors_get_block: block %d outside [0, %d)", i, fa->n_far);
    const int nc = fa->r3[i];
    if (r3) *r3 = nc;
    const BlockRange br = fa->ranges[i];
    const int M = br.re - br.rb, N = br.ce - br.cb, Ku = fa->Ku;
    G3_TRY(use_device(fa->ctx));
    size_t ou = 0, ov = 0;
    for (int p = 0; p < nc; ++p) {
        const CrossRec& c = fa->crec(i, p);
        const bool dense = c.r < 0;
        const int rr = dense ? N : c.r;
        if (face_ranks) face_ranks[p] = rr;
        if (piv) {
            piv[3 * p] = c.ip;
            piv[3 * p + 1] = c.jp;
            piv[3 * p + 2] = c.kp;
        }
        const size_t nu = (size_t)rr * M, nv = (size_t)rr * N;
        // stored: low-rank U, V, f  |  dense H (M x N column-major), f
        const size_t tot = dense ? (size_t)M * N + Ku : nu + nv + Ku;
        std::vector<double> tmp(2 * tot);
        if (fa->prec == G3_MIXED) {
            std::vector<float> tf(2 * tot);
            G3_CUDA(cudaMemcpy(tf.data(), fa->pool->as<float>() + 2 * c.off, tf.size() * sizeof(float), cudaMemcpyDeviceToHost));
            for (size_t k = 0; k < tf.size(); ++k) tmp[k] = tf[k];
        } else {
            G3_CUDA(cudaMemcpy(tmp.data(), fa->pool->as<double>() + 2 * c.off, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
        }
        if (dense) {
            if (U) std::memcpy(U + 2 * ou, tmp.data(), 2 * nu * sizeof(double));
            if (V) {
                std::memset(V + 2 * ov, 0, 2 * nv * sizeof(double));
                for (int j = 0; j < N; ++j) V[2 * (ov + (size_t)j * N + j)] = 1.0;
            }
            if (fib) std::memcpy(fib + 2 * (size_t)p * Ku, tmp.data() + 2 * (size_t)M * N, 2 * (size_t)Ku * sizeof(double));
        } else {
            if (U) std::memcpy(U + 2 * ou, tmp.data(), 2 * nu * sizeof(double));
            if (V) std::memcpy(V + 2 * ov, tmp.data() + 2 * nu, 2 * nv * sizeof(double));
            if (fib) std::memcpy(fib + 2 * (size_t)p * Ku, tmp.data() + 2 * (nu + nv), 2 * (size_t)Ku * sizeof(double));
        }
        ou += nu;
        ov += nv;
    }
    return G3_OK;
}

g3_status g3_factors_free(g3_factors* fa) {
    if (fa) {
        cudaSetDevice(fa->device);
        delete fa;
    }
    return G3_OK;
}

// ---------------------------------------------------------------------------
// apply
// ---------------------------------------------------------------------------

g3_status apply_gcq(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa, const void* W, void* Y,
                    g3_dtype dtype, g3_apply_mode mode, g3_memory mem) {
    G3_CHECK(ctx && t && W && Y, "apply_gcq: NULL argument");
    G3_CHECK(nf || fa, "apply_gcq: near field and factors are both NULL");
    G3_CHECK(dtype == G3_C64 || dtype == G3_C128, "apply_gcq: bad dtype");
    G3_CHECK(mode == G3_APPLY_SUM || mode == G3_APPLY_PERFREQ, "apply_gcq: bad mode");
    G3_CHECK(mem == G3_DEVICE || mem == G3_HOST, "apply_gcq: bad memory kind");
    G3_CHECK(!nf || nf->tree == t, "apply_gcq: near field built on another tree");
    G3_CHECK(!fa || fa->tree == t, "apply_gcq: factors built on another tree");
    G3_CHECK(!t->p1 || mode == G3_APPLY_SUM, "apply_gcq: linear-element trees take G3_APPLY_SUM");
    G3_TRY(use_device(ctx));
    const g3_freqs* f = nf ? nf->freqs : fa->freqs;
    const size_t esz = dtype == G3_C128 ? 16 : 8;
    const size_t rows = t->p1 ? (size_t)t->nv : (size_t)t->ne;  // linear elements: nodal W and Y
    const size_t wbytes = rows * f->K * esz;
    const size_t ybytes = rows * (mode == G3_APPLY_SUM ? 1 : f->K) * esz;
    if (mem == G3_DEVICE) return run_apply(ctx, t, nf, fa, W, Y, dtype, mode);
    // host buffers: staged through context-owned device buffers (kept for reuse)
    G3_CUDA(ctx->stage_w.ensure(wbytes));
    G3_CUDA(ctx->stage_y.ensure(ybytes));
    G3_CUDA(cudaMemcpyAsync(ctx->stage_w.p, W, wbytes, cudaMemcpyHostToDevice, ctx->stream));
    G3_TRY(run_apply(ctx, t, nf, fa, ctx->stage_w.p, ctx->stage_y.p, dtype, mode));
    G3_CUDA(cudaMemcpyAsync(Y, ctx->stage_y.p, ybytes, cudaMemcpyDeviceToHost, ctx->stream));
    G3_CUDA(cudaStreamSynchronize(ctx->stream));
    return G3_OK;
}

g3_status g3_peak(g3_ctx* ctx, int kind, double* ops_per_s, double* ms) {
    G3_CHECK(ctx && ops_per_s, "g3_peak: NULL argument");
    G3_CHECK(kind >= 0 && kind <= 5, "g3_peak: kind %d outside [0, 5]", kind);
    G3_TRY(use_device(ctx));
    return run_peak(ctx, kind, ops_per_s, ms);
}

g3_status g3_apply_last(const g3_ctx* ctx, double* ms, int64_t* bytes, double* near_ms, int64_t* near_bytes) {
    G3_CHECK(ctx != nullptr, "g3_apply_last: NULL handle");
    if (ms) *ms = ctx->last_apply_ms;
    if (bytes) *bytes = ctx->last_apply_bytes;
    if (near_ms) *near_ms = ctx->last_near_ms;
    if (near_bytes) *near_bytes = ctx->last_near_bytes;
    return G3_OK;
}

// ---- block predictor ---------------------------------------------------------

static g3_status mlp_alloc(g3_ctx* ctx, const float* params, const float* mean, const float* inv_std, uint64_t seed,
                           g3_mlp** out) {
    g3_mlp* m = new (std::nothrow) g3_mlp();
    if (!m) return fail(G3_ENOMEM, "g3_mlp: out of host memory");
    std::vector<float> P(G3_MLP_NP), Z(G3_MLP_NP, 0.f);
    if (params) {
        for (int i = 0; i < G3_MLP_NP; ++i)
            if (!std::isfinite(params[i])) {
                delete m;
                return fail(G3_EINVAL, "g3_mlp_create: params[%d] is not finite", i);
            }
        std::memcpy(P.data(), params, sizeof(float) * G3_MLP_NP);
    } else {
        mlp_init_params(seed, P.data());
    }
    for (int i = 0; i < G3_MLP_NF; ++i) {
        m->mean[i] = mean ? mean[i] : 0.f;
        m->inv_std[i] = inv_std ? inv_std[i] : 1.f;
    }
    m->ctx = ctx;
    m->device = ctx->device;
    auto up = [&](g3::DevBuf& d, const void* src, size_t bytes) -> cudaError_t {
        cudaError_t e = d.alloc(bytes);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(d.p, src, bytes, cudaMemcpyHostToDevice);
    };
    const long long t0 = 0;
    cudaError_t e;
    if ((e = up(m->d_params, P.data(), sizeof(float) * G3_MLP_NP)) != cudaSuccess ||
        (e = up(m->d_m, Z.data(), sizeof(float) * G3_MLP_NP)) != cudaSuccess ||
        (e = up(m->d_v, Z.data(), sizeof(float) * G3_MLP_NP)) != cudaSuccess ||
        (e = up(m->d_t, &t0, sizeof(t0))) != cudaSuccess ||
        (e = up(m->d_mean, m->mean, sizeof(float) * G3_MLP_NF)) != cudaSuccess ||
        (e = up(m->d_inv_std, m->inv_std, sizeof(float) * G3_MLP_NF)) != cudaSuccess) {
        delete m;
        return cuda_fail(e, "g3_mlp_create: upload");
    }
    *out = m;
    return G3_OK;
}

g3_status g3_mlp_create(g3_ctx* ctx, const float* params, const float* mean, const float* inv_std, uint64_t seed,
                        g3_mlp** out) {
    G3_CHECK(ctx && out, "g3_mlp_create: NULL argument");
    *out = nullptr;
    G3_TRY(use_device(ctx));
    return mlp_alloc(ctx, params, mean, inv_std, seed, out);
}

struct TrainCfg {
    int epochs, batch, graph;
    double lr, b1, b2, eps;
    uint64_t seed;
};

static g3_status train_cfg(const g3_train_opts* o, TrainCfg& c) {
    g3_train_opts d{};
    if (o) d = *o;
    c.epochs = d.epochs > 0 ? d.epochs : 200;
    c.batch = d.batch > 0 ? d.batch : 256;
    c.lr = d.lr > 0 ? d.lr : 1e-3;
    c.b1 = d.beta1 > 0 ? d.beta1 : 0.9;
    c.b2 = d.beta2 > 0 ? d.beta2 : 0.999;
    c.eps = d.adam_eps > 0 ? d.adam_eps : 1e-8;
    c.seed = d.seed;
    c.graph = d.no_graph ? 0 : 1;
    G3_CHECK(d.epochs >= 0 && d.batch >= 0, "g3_mlp: negative epochs or batch");
    G3_CHECK(c.b1 < 1 && c.b2 < 1, "g3_mlp: Adam decay rates must be below 1");
    return G3_OK;
}

static g3_status upload_samples(const float* feats, const float* labels, int n, g3::DevBuf& dx, g3::DevBuf& dy) {
    G3_CUDA(dx.alloc((size_t)n * G3_MLP_NF * sizeof(float)));
    G3_CUDA(cudaMemcpy(dx.p, feats, (size_t)n * G3_MLP_NF * sizeof(float), cudaMemcpyHostToDevice));
    if (labels) {
        G3_CUDA(dy.alloc((size_t)n * 2 * sizeof(float)));
        G3_CUDA(cudaMemcpy(dy.p, labels, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice));
    }
    return G3_OK;
}

static g3_status fit(g3_ctx* ctx, g3_mlp* m, const float* feats, const float* labels, int n, const TrainCfg& c,
                     float* losses) {
    g3::DevBuf dx, dy, dl;
    G3_TRY(upload_samples(feats, labels, n, dx, dy));
    const long long nb = ((long long)n + c.batch - 1) / c.batch;
    G3_CUDA(dl.alloc((size_t)c.epochs * nb * sizeof(float)));
    G3_TRY(mlp_fit_dev(ctx, m, dx.as<float>(), dy.as<float>(), n, c.epochs, c.batch, c.lr, c.b1, c.b2, c.eps, c.graph,
                       dl.as<float>()));
    if (losses) G3_CUDA(cudaMemcpy(losses, dl.p, (size_t)c.epochs * nb * sizeof(float), cudaMemcpyDeviceToHost));
    return G3_OK;
}

g3_status g3_mlp_train(g3_ctx* ctx, const float* feats, const float* labels, int n, const g3_train_opts* opts,
                       g3_mlp** out) {
    G3_CHECK(ctx && feats && labels && out, "g3_mlp_train: NULL argument");
    *out = nullptr;
    G3_CHECK(n >= 1, "g3_mlp_train: n = %d", n);
    TrainCfg c;
    G3_TRY(train_cfg(opts, c));
    G3_TRY(use_device(ctx));
    // standardisation from the samples (float64 sums on the host)
    float mean[G3_MLP_NF], inv[G3_MLP_NF];
    for (int f = 0; f < G3_MLP_NF; ++f) {
        double s = 0, s2 = 0;
        for (int i = 0; i < n; ++i) s += feats[(size_t)i * G3_MLP_NF + f];
        const double mu = s / n;
        for (int i = 0; i < n; ++i) {
            const double d = feats[(size_t)i * G3_MLP_NF + f] - mu;
            s2 += d * d;
        }
        const double sd = std::sqrt(s2 / n);
        G3_CHECK(std::isfinite(mu) && std::isfinite(sd), "g3_mlp_train: feature %d is not finite", f);
        mean[f] = (float)mu;
        inv[f] = sd > 1e-6 ? (float)(1.0 / sd) : 1.0f;
    }
    g3_mlp* m = nullptr;
    G3_TRY(mlp_alloc(ctx, nullptr, mean, inv, c.seed, &m));
    const g3_status st = fit(ctx, m, feats, labels, n, c, nullptr);
    if (st != G3_OK) {
        delete m;
        return st;
    }
    *out = m;
    return G3_OK;
}

g3_status g3_mlp_fit(g3_ctx* ctx, g3_mlp* m, const float* feats, const float* labels, int n,
                     const g3_train_opts* opts, float* losses) {
    G3_CHECK(ctx && m && feats && labels, "g3_mlp_fit: NULL argument");
    G3_CHECK(n >= 1, "g3_mlp_fit: n = %d", n);
    TrainCfg c;
    G3_TRY(train_cfg(opts, c));
    G3_TRY(use_device(ctx));
    return fit(ctx, m, feats, labels, n, c, losses);
}

g3_status g3_mlp_grad(g3_ctx* ctx, const g3_mlp* m, const float* feats, const float* labels, int n, float* grad,
                      float* loss) {
    G3_CHECK(ctx && m && feats && labels && grad, "g3_mlp_grad: NULL argument");
    G3_CHECK(n >= 1, "g3_mlp_grad: n = %d", n);
    G3_TRY(use_device(ctx));
    g3::DevBuf dx, dy, dg, dl;
    G3_TRY(upload_samples(feats, labels, n, dx, dy));
    G3_CUDA(dg.alloc(G3_MLP_NP * sizeof(float)));
    G3_CUDA(dl.alloc(sizeof(float)));
    G3_TRY(mlp_grad_dev(ctx, m, dx.as<float>(), dy.as<float>(), n, dg.as<float>(), dl.as<float>()));
    G3_CUDA(cudaMemcpy(grad, dg.p, G3_MLP_NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss) G3_CUDA(cudaMemcpy(loss, dl.p, sizeof(float), cudaMemcpyDeviceToHost));
    return G3_OK;
}

g3_status g3_mlp_predict(g3_ctx* ctx, const g3_mlp* m, const float* feats, int n, float* out) {
    G3_CHECK(ctx && m && feats && out, "g3_mlp_predict: NULL argument");
    G3_CHECK(n >= 0, "g3_mlp_predict: n = %d", n);
    if (n == 0) return G3_OK;
    G3_TRY(use_device(ctx));
    g3::DevBuf dx, dy, dout;
    G3_TRY(upload_samples(feats, nullptr, n, dx, dy));
    G3_CUDA(dout.alloc((size_t)n * 2 * sizeof(float)));
    G3_TRY(mlp_forward_dev(ctx, m, dx.as<float>(), n, dout.as<float>()));
    G3_CUDA(cudaMemcpyAsync(out, dout.p, (size_t)n * 2 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    G3_CUDA(cudaStreamSynchronize(ctx->stream));
    return G3_OK;
}

g3_status g3_mlp_get(const g3_mlp* m, float* params, float* adam_m, float* adam_v, int64_t* t, float* mean,
                     float* inv_std) {
    G3_CHECK(m != nullptr, "g3_mlp_get: NULL handle");
    G3_TRY(use_device(m->ctx));
    G3_CUDA(cudaStreamSynchronize(m->ctx->stream));
    if (params) G3_CUDA(cudaMemcpy(params, m->d_params.p, G3_MLP_NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (adam_m) G3_CUDA(cudaMemcpy(adam_m, m->d_m.p, G3_MLP_NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (adam_v) G3_CUDA(cudaMemcpy(adam_v, m->d_v.p, G3_MLP_NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (t) *t = m->t;
    if (mean) std::memcpy(mean, m->mean, sizeof(m->mean));
    if (inv_std) std::memcpy(inv_std, m->inv_std, sizeof(m->inv_std));
    return G3_OK;
}

g3_status g3_mlp_free(g3_mlp* m) {
    if (!m) return G3_OK;
    if (m->ctx) cudaSetDevice(m->device);
    delete m;
    return G3_OK;
}

g3_status g3_block_features(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, double eps3,
                            float* out) {
    G3_CHECK(ctx && t && f && out, "g3_block_features: NULL argument");
    G3_CHECK(kernel == G3_SLP || kernel == G3_DLP, "g3_block_features: kernel must be G3_SLP or G3_DLP");
    G3_CHECK(!t->p1, "g3_block_features: the tree must be an element tree (features are per element block)");
    G3_CHECK(eps3 > 0 && eps3 < 1, "g3_block_features: eps3 = %g outside (0, 1)", eps3);
    const int n_far = (int)t->far_index.size();
    if (n_far == 0) return G3_OK;
    G3_TRY(use_device(ctx));
    g3::DevBuf d;
    G3_CUDA(d.alloc((size_t)n_far * G3_MLP_NF * sizeof(float)));
    G3_TRY(mlp_features_dev(ctx, t, f, kernel, eps3, d.as<float>()));
    G3_CUDA(cudaMemcpyAsync(out, d.p, (size_t)n_far * G3_MLP_NF * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    G3_CUDA(cudaStreamSynchronize(ctx->stream));
    return G3_OK;
}

g3_status g3_factors_labels(g3_ctx* ctx, const g3_factors* fa, float* out) {
    G3_CHECK(ctx && fa && out, "g3_factors_labels: NULL argument");
    if (fa->n_far == 0) return G3_OK;
    G3_TRY(use_device(ctx));
    g3::DevBuf dr, d;
    G3_CUDA(dr.alloc(fa->ranges.size() * sizeof(BlockRange)));
    G3_CUDA(cudaMemcpy(dr.p, fa->ranges.data(), fa->ranges.size() * sizeof(BlockRange), cudaMemcpyHostToDevice));
    G3_CUDA(d.alloc((size_t)fa->n_far * 2 * sizeof(float)));
    G3_TRY(mlp_labels_dev(ctx, fa, dr.as<BlockRange>(), d.as<float>()));
    G3_CUDA(cudaMemcpyAsync(out, d.p, (size_t)fa->n_far * 2 * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    G3_CUDA(cudaStreamSynchronize(ctx->stream));
    return G3_OK;
}

}  // extern "C"
