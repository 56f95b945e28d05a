// Host driver of the three-way ACA (kernel and device routines: g3_aca_dev.cuh;
// kernel instantiations: g3_aca_slp.cu, g3_aca_dlp.cu, g3_aca_sep.cu).
#include <chrono>
#include <cmath>

#include "g3_aca_dev.cuh"

namespace g3 {

#define G3_ACA_EXTERN(KER, T, NT, DENSE)                                                                 \
    extern template g3_status launch_aca_t<KER, T, NT, DENSE>(g3_ctx*, AcaArgs<T>&, int, size_t);      \
    extern template int occupancy<KER, T, NT, DENSE>(size_t);
#define G3_ACA_EXTERN_KIND(KER)              \
    G3_ACA_EXTERN(KER, float, 256, false)    \
    G3_ACA_EXTERN(KER, float, 256, true)     \
    G3_ACA_EXTERN(KER, float, 128, false)    \
    G3_ACA_EXTERN(KER, float, 512, false)    \
    G3_ACA_EXTERN(KER, float, 384, false)    \
    G3_ACA_EXTERN(KER, double, 256, false)   \
    G3_ACA_EXTERN(KER, double, 256, true)
G3_ACA_EXTERN_KIND(G3_SLP)
G3_ACA_EXTERN_KIND(G3_DLP)
G3_ACA_EXTERN_KIND(G3_SEPARABLE)
G3_ACA_EXTERN_KIND(G3_GAL_SLP)
// linear-element operators: the 256-thread launches only
G3_ACA_EXTERN(G3_GAL_P1D, float, 256, false)
G3_ACA_EXTERN(G3_GAL_P1D, float, 256, true)
G3_ACA_EXTERN(G3_GAL_P1D, double, 256, false)
G3_ACA_EXTERN(G3_GAL_P1D, double, 256, true)
G3_ACA_EXTERN(G3_GAL_P1KP, float, 256, false)
G3_ACA_EXTERN(G3_GAL_P1KP, float, 256, true)
G3_ACA_EXTERN(G3_GAL_P1KP, double, 256, false)
G3_ACA_EXTERN(G3_GAL_P1KP, double, 256, true)

#define G3_WHOLE_EXTERN(KER, T)                                                                              \
    extern template g3_status launch_whole_t<KER, T>(g3_ctx*, AcaArgs<T>&, int, size_t, int, int, const double*, \
                                                     WholeCand*, Cx<double>*, double*);                         \
    extern template g3_status launch_whole_fiber_t<KER, T>(g3_ctx*, AcaArgs<T>&, int, int, int, int, Cx<double>*, \
                                                           Cx<double>*, double*, int, const Cx<double>*,          \
                                                           const double*, double*, double*);
G3_WHOLE_EXTERN(G3_SLP, float)
G3_WHOLE_EXTERN(G3_SLP, double)
G3_WHOLE_EXTERN(G3_DLP, float)
G3_WHOLE_EXTERN(G3_DLP, double)
G3_WHOLE_EXTERN(G3_GAL_SLP, float)
G3_WHOLE_EXTERN(G3_GAL_SLP, double)

template <class T, int NT, bool DENSE>
static g3_status launch_kind(g3_ctx* ctx, int kernel, AcaArgs<T>& A, int grid, size_t smem) {
    if (kernel == G3_SLP) return launch_aca_t<G3_SLP, T, NT, DENSE>(ctx, A, grid, smem);
    if (kernel == G3_DLP) return launch_aca_t<G3_DLP, T, NT, DENSE>(ctx, A, grid, smem);
    if (kernel == G3_GAL_SLP) return launch_aca_t<G3_GAL_SLP, T, NT, DENSE>(ctx, A, grid, smem);
    if (kernel == G3_GAL_P1D || kernel == G3_GAL_P1KP) {
        if constexpr (NT == 256)
            return kernel == G3_GAL_P1D ? launch_aca_t<G3_GAL_P1D, T, NT, DENSE>(ctx, A, grid, smem)
                                        : launch_aca_t<G3_GAL_P1KP, T, NT, DENSE>(ctx, A, grid, smem);
        return fail(G3_EUNSUPPORTED, "aca3_compress: linear-element operators run with 256 threads per CTA");
    }
    return launch_aca_t<G3_SEPARABLE, T, NT, DENSE>(ctx, A, grid, smem);
}

template <class T, int NT, bool DENSE>
static int occupancy_kind(int kernel, size_t smem) {
    if (kernel == G3_SLP) return occupancy<G3_SLP, T, NT, DENSE>(smem);
    if (kernel == G3_DLP) return occupancy<G3_DLP, T, NT, DENSE>(smem);
    if (kernel == G3_GAL_SLP) return occupancy<G3_GAL_SLP, T, NT, DENSE>(smem);
    if (kernel == G3_GAL_P1D || kernel == G3_GAL_P1KP) {
        if constexpr (NT == 256)
            return kernel == G3_GAL_P1D ? occupancy<G3_GAL_P1D, T, NT, DENSE>(smem)
                                        : occupancy<G3_GAL_P1KP, T, NT, DENSE>(smem);
        return 1;
    }
    return occupancy<G3_SEPARABLE, T, NT, DENSE>(smem);
}

// one mesh of a (possibly batched) compression: its tree, frequencies and
// output; its blocks are [first, first + n) of the concatenated block list
struct AcaJob {
    const g3_tree* t;
    const g3_freqs* f;
    g3_factors* fa;
    int first = 0, n = 0, Ku = 0;
};

// the kept records of every block, packed: block b's r3[b] records go to
// out[off[b]], ...  (the device keeps the [n_far][Cmax] layout; the host
// copy is compact)
__global__ void __launch_bounds__(256) k_rec_pack(const CrossRec* __restrict__ rec, const int* __restrict__ r3,
                                                  const long long* __restrict__ off, int Cmax, long long n,
                                                  CrossRec* __restrict__ out) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(idx / Cmax), p = (int)(idx % Cmax);
        if (p < r3[b]) out[off[b] + p] = rec[idx];
    }
}

// pinned host staging of the context (grown, never shrunk)
static g3_status stage_ensure(g3_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->h_stage_bytes) return G3_OK;
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    const size_t want = std::max(bytes, (size_t)1 << 20);
    const cudaError_t e = cudaMallocHost(&ctx->h_stage, want);
    if (e != cudaSuccess) {
        ctx->h_stage = nullptr;
        return cuda_fail(e, "pinned staging buffer");
    }
    ctx->h_stage_bytes = want;
    return G3_OK;
}

// host copies of the records in compact form from a [n][Cmax] host array
static void compact_records(g3_factors* fa, const std::vector<CrossRec>& full, int Cmax) {
    const int n = (int)fa->r3.size();
    fa->rec_off.assign((size_t)n + 1, 0);
    for (int b = 0; b < n; ++b) fa->rec_off[b + 1] = fa->rec_off[b] + std::max(0, fa->r3[b]);
    fa->rec.resize((size_t)fa->rec_off[n]);
    for (int b = 0; b < n; ++b) {
        const auto src = full.begin() + (size_t)b * Cmax;
        std::copy(src, src + (fa->rec_off[b + 1] - fa->rec_off[b]), fa->rec.begin() + fa->rec_off[b]);
    }
}

// move a device buffer's ownership
static void take(DevBuf& dst, DevBuf& src) {
    dst.release();
    dst.p = src.p;
    dst.bytes = src.bytes;
    src.p = nullptr;
    src.bytes = 0;
}

template <class T>
static g3_status run_aca_t(g3_ctx* ctx, std::vector<AcaJob>& jobs, int kernel, double eps3, const g3_opts& o,
                           const void* sep_a, const void* sep_b, const void* sep_c, int sep_R) {
    const auto th0 = std::chrono::steady_clock::now();
    auto ms_since = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
    };
    const bool sep = kernel == G3_SEPARABLE;
    const int n_jobs = (int)jobs.size();
    const bool batched = n_jobs > 1;
    // face rank cap: 48, and RF_MAX for the linear-element operators, whose
    // hypersingular faces at high frequencies need ranks of 70 and more on
    // blocks of 40 elements a side (capped at 48 they stay unresolved)
    const bool p1_kind = kernel == G3_GAL_P1D || kernel == G3_GAL_P1KP;
    const int RF = o.face_rank_max > 0 ? std::min(o.face_rank_max, RF_MAX) : (p1_kind ? RF_MAX : 48);
    // face tolerance: eps3 / 100 (eps = 100 eps_ACA); in float32 arithmetic not
    // below 1e-5, the relative noise level of float32 entries
    const double eps_face = o.eps_face > 0 ? o.eps_face : (sizeof(T) == 4 ? std::max(eps3 / 100.0, 1e-5) : eps3 / 100.0);
    // concatenated block list (far order of each mesh, meshes in order)
    std::vector<BlockRange> ranges;
    std::vector<int> bgeo;
    int Ku = 0;  // largest unique-frequency count (sizes, cross-record stride)
    for (int j = 0; j < n_jobs; ++j) {
        AcaJob& J = jobs[j];
        J.first = (int)ranges.size();
        J.Ku = J.fa->Ku;
        Ku = std::max(Ku, J.Ku);
        if (sep) {
            ranges.push_back(BlockRange{0, J.fa->M_sep, 0, J.fa->N_sep});
        } else {
            for (int b : J.t->far_index) {
                const int32_t* r = &J.t->blocks[5 * (size_t)b];
                ranges.push_back(BlockRange{r[0], r[1], r[2], r[3]});
            }
        }
        J.n = (int)ranges.size() - J.first;
        bgeo.insert(bgeo.end(), J.n, j);
        J.fa->n_far = J.n;
        J.fa->ranges.assign(ranges.begin() + J.first, ranges.end());
        J.fa->r3.assign(J.n, 0);
    }
    const int Cmax = Ku;
    for (auto& J : jobs) J.fa->Cmax = Cmax;
    const int n_far = (int)ranges.size();
    if (n_far == 0) {  // no admissible block: empty work lists, the apply runs the near field alone
        for (auto& J : jobs) {
            const g3_status pst = far_plan_build(J.fa);
            if (pst != G3_OK) return pst;
        }
        return G3_OK;
    }
    int Mmax = 0, Nmax = 0;
    for (auto& r : ranges) {
        Mmax = std::max(Mmax, r.re - r.rb);
        Nmax = std::max(Nmax, r.ce - r.cb);
    }
    const int dense_max = o.dense_face_max > 0 ? o.dense_face_max : (o.dense_face_max < 0 ? -1 : 48 * 48);
    auto is_dense = [&](const BlockRange& r) { return (long long)(r.re - r.rb) * (r.ce - r.cb) <= dense_max; };
    auto ku_of = [&](int b) { return jobs[bgeo[b]].Ku; };
    // block predictor: rank and first frequency of every block before the
    // compression starts (features and forward pass on the device)
    int mlp_use = 0;
    std::vector<double> rhat;
    std::vector<int> k1_mlp;
    double ms_mlp = 0;
    if (o.mlp && !sep) {
        mlp_use = o.mlp_use ? o.mlp_use : 7;
        DevBuf d_feat, d_pred;
        G3_CUDA(d_feat.alloc((size_t)n_far * G3_MLP_NF * sizeof(float)));
        G3_CUDA(d_pred.alloc((size_t)n_far * 2 * sizeof(float)));
        G3_CUDA(cudaEventRecord(ctx->ev[3], ctx->stream));
        for (auto& J : jobs) {
            const g3_status st = mlp_features_dev(ctx, J.t, J.f, kernel, eps3,
                                                  d_feat.as<float>() + (size_t)J.first * G3_MLP_NF);
            if (st != G3_OK) return st;
        }
        g3_status st = mlp_forward_dev(ctx, o.mlp, d_feat.as<float>(), n_far, d_pred.as<float>());
        if (st != G3_OK) return st;
        G3_CUDA(cudaEventRecord(ctx->ev[4], ctx->stream));
        std::vector<float> pred((size_t)n_far * 2);
        G3_CUDA(cudaMemcpyAsync(pred.data(), d_pred.p, pred.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
        float mm = 0;
        G3_CUDA(cudaEventElapsedTime(&mm, ctx->ev[3], ctx->ev[4]));
        ms_mlp = mm;
        rhat.resize(n_far);
        k1_mlp.resize(n_far);
        for (int i = 0; i < n_far; ++i) {
            const int ku = ku_of(i);
            const double y0 = std::isfinite(pred[2 * i]) ? pred[2 * i] : 0.0;
            const double y1 = std::isfinite(pred[2 * i + 1]) ? pred[2 * i + 1] : 0.0;
            rhat[i] = std::min((double)ku, std::max(0.0, std::exp2(std::min(y0, 16.0)) - 1.0));
            k1_mlp[i] = (int)std::min<long long>(ku - 1, std::max<long long>(0, std::llround(y1 * ku)));
        }
        if (o.cost) mlp_use &= ~1;
        if (o.k1) mlp_use &= ~4;
    }
    std::vector<int> queue(n_far);
    std::iota(queue.begin(), queue.end(), 0);
    // optional bounded run: only the first max_blocks blocks of the far order
    const int n_run = o.max_blocks > 0 ? std::min(n_far, o.max_blocks) : n_far;
    const int order = o.order_by_cost;  // 0 given -> default on
    if (order >= 0) {
        std::vector<double> cost(n_far);
        for (int i = 0; i < n_far; ++i) {
            double mm = ranges[i].re - ranges[i].rb, nn = ranges[i].ce - ranges[i].cb;
            if (o.cost)
                cost[i] = (double)o.cost[i];
            else if (mlp_use & 1)  // predicted work: crosses x entries per cross
                cost[i] = (rhat[i] + 1.0) * (is_dense(ranges[i]) ? mm * nn : mm + nn);
            else
                cost[i] = mm * nn;
        }
        std::stable_sort(queue.begin(), queue.begin() + n_run, [&](int a, int b) { return cost[a] > cost[b]; });
    }
    // two block classes, each in cost order: low-rank faces, then dense faces
    std::vector<int> qcat;
    qcat.reserve(n_run);
    for (int pass = 0; pass < 2; ++pass)
        for (int q = 0; q < n_run; ++q)
            if (is_dense(ranges[queue[q]]) == (pass == 1)) qcat.push_back(queue[q]);
    int n_low = 0;
    for (int q = 0; q < n_run; ++q) n_low += !is_dense(ranges[queue[q]]);
    const int n_dense = n_run - n_low;
    DevBuf d_ranges, d_queue, d_head, d_k1, d_counters, d_ctr, d_spill, d_spill_n, d_geos, d_bgeo;
    G3_CUDA(d_ranges.alloc(n_far * sizeof(BlockRange)));
    G3_CUDA(d_queue.alloc(std::max(n_run, 1) * sizeof(int)));
    G3_CUDA(d_head.alloc(2 * sizeof(int)));
    G3_CUDA(d_counters.alloc(32 * sizeof(unsigned long long)));
    G3_CUDA(d_ctr.alloc(sizeof(unsigned long long)));
    G3_CUDA(d_spill.alloc(std::max(n_far, 1) * sizeof(int)));
    G3_CUDA(d_spill_n.alloc(sizeof(int)));
    G3_CUDA(cudaMemcpyAsync(d_ranges.p, ranges.data(), n_far * sizeof(BlockRange), cudaMemcpyHostToDevice, ctx->stream));
    if (n_run > 0)
        G3_CUDA(cudaMemcpyAsync(d_queue.p, qcat.data(), n_run * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    const int* k1_host = o.k1 ? o.k1 : ((mlp_use & 4) ? k1_mlp.data() : nullptr);
    if (k1_host) {
        for (int i = 0; i < n_far; ++i)
            if (k1_host[i] < 0 || k1_host[i] >= ku_of(i))
                return fail(G3_EINVAL, "opts->k1[%d] = %d outside [0, %d)", i, k1_host[i], ku_of(i));
        G3_CUDA(d_k1.alloc(n_far * sizeof(int)));
        G3_CUDA(cudaMemcpy(d_k1.p, k1_host, n_far * sizeof(int), cudaMemcpyHostToDevice));
    }
    if (batched) {
        std::vector<GeoDesc> geos(n_jobs);
        for (int j = 0; j < n_jobs; ++j)
            geos[j] = GeoDesc{jobs[j].t->gf, jobs[j].t->gd, jobs[j].f->d_sd.as<double2>(),
                              jobs[j].f->d_sf.as<float2>(), jobs[j].Ku, jobs[j].f->k_maxabs};
        G3_CUDA(d_geos.alloc(n_jobs * sizeof(GeoDesc)));
        G3_CUDA(d_bgeo.alloc(n_far * sizeof(int)));
        G3_CUDA(cudaMemcpy(d_geos.p, geos.data(), n_jobs * sizeof(GeoDesc), cudaMemcpyHostToDevice));
        G3_CUDA(cudaMemcpy(d_bgeo.p, bgeo.data(), n_far * sizeof(int), cudaMemcpyHostToDevice));
    }
    // separable inputs (converted to T)
    DevBuf d_sa, d_sb, d_sc;
    SepView<T> sv{};
    if (sep) {
        g3_factors* fa = jobs[0].fa;
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
    // dynamic shared memory arena, reused phase by phase: the four RS x RS
    // matrices of the recompression (+ Gram staging; float32: + the working-
    // precision copies of the two Cholesky factors), the pivot-search
    // tiles (2 RF TM complex T, TM = 64 float / 32 double) and the eq. (norm)
    // staging ((NORM_RC + 1) (32 + RF) + 32 RF complex T, then 64 column pointers)
    const size_t recomp_bytes = 2 * (size_t)RS * RS * sizeof(Cx<double>) +
                                std::max(2 * (size_t)RS * RS * sizeof(Cx<T>), 33 * (size_t)RF * sizeof(Cx<T>)) +
                                (sizeof(T) == 4 ? 2 * (size_t)RS * RS * sizeof(Cx<T>) : 0);
    const size_t tile_bytes = 2 * (size_t)RF * (sizeof(T) == 4 ? 64 : 32) * sizeof(Cx<T>);
    const size_t gram_bytes = ((NORM_RC<T> + 1) * (size_t)(32 + RF) + 32 * (size_t)RF) * sizeof(Cx<T>) + 64 * sizeof(void*);
    const size_t tab_bytes = 2 * TABMAX * sizeof(long long) + TABMAX * sizeof(short) +
                             (TABMAX + RF_MAX) * sizeof(Cx<T>) + ROWMAX * sizeof(Cx<T>) + 64;
    // dense residual working faces (float32 low-rank faces of blocks with M N <= drf):
    // a per-CTA buffer of the largest such face and shared-memory staging after
    // the face tables (sized for the widest launch shape)
    long long drf_elems = 0;
    int drf = -1;
    if (sizeof(T) == 4 && kernel != G3_SEPARABLE) {
        drf = o.residual_face_max > 0 ? o.residual_face_max : (o.residual_face_max == 0 ? 192 * 192 : -1);
        for (int q = 0; q < n_run && drf > 0; ++q) {
            const BlockRange& r = ranges[queue[q]];
            const long long mn = (long long)(r.re - r.rb) * (r.ce - r.cb);
            if (!is_dense(r) && mn <= drf) drf_elems = std::max(drf_elems, mn);
        }
        if (drf_elems == 0) drf = -1;
    }
    const size_t drf_smem =
        drf > 0 ? drf_stage_offset<T>() + std::max(drf_stage_bytes<T, 256>(), drf_stage_bytes<T, 512>()) : 0;
    const size_t smem =
        std::max(std::max(std::max(std::max(recomp_bytes, tile_bytes), gram_bytes), tab_bytes), drf_smem);
    // low-rank class: 128, 256, 384 or 512 threads per CTA (float32 path); more
    // threads shorten each block, which matters for the largest blocks at the
    // end, fewer keep more blocks in flight per SM
    const int nt_low = (sizeof(T) == 4 && (o.threads == 128 || o.threads == 384 || o.threads == 512)) ? o.threads
                                                                                                         : NT;
    int per_low = o.ctas_per_sm;
    if (per_low <= 0) {
        if constexpr (sizeof(T) == 4)
            per_low = nt_low == 512   ? occupancy_kind<T, 512, false>(kernel, smem)
                      : nt_low == 384 ? occupancy_kind<T, 384, false>(kernel, smem)
                      : nt_low == 128 ? occupancy_kind<T, 128, false>(kernel, smem)
                                      : occupancy_kind<T, NT, false>(kernel, smem);
        else
            per_low = occupancy_kind<T, NT, false>(kernel, smem);
    }
    const int per_dense = o.ctas_per_sm > 0 ? o.ctas_per_sm : occupancy_kind<T, NT, true>(kernel, smem);
    const int grid_low = o.unbatched ? 1 : std::max(1, std::min(n_low, ctx->n_sm * per_low));
    const int grid_dense = o.unbatched ? 1 : std::max(1, std::min(n_dense, ctx->n_sm * per_dense));
    const int grid = std::max(grid_low, grid_dense);
    const size_t drf_off = al256(ws_bytes<T>(RF, Mmax, Nmax, Cmax, Ku));
    const size_t stride = drf_off + al256((size_t)drf_elems * sizeof(Cx<T>));
    // per-CTA workspace, kept by the context between compressions
    G3_CUDA(ctx->aca_ws.ensure(stride * grid));
    DevBuf& d_ws = ctx->aca_ws;
    // outputs of all meshes (sliced per mesh at the end)
    DevBuf g_rec, g_r3, g_cyc;
    G3_CUDA(g_rec.alloc((size_t)n_far * Cmax * sizeof(CrossRec)));
    G3_CUDA(g_r3.alloc((size_t)n_far * sizeof(int)));
    G3_CUDA(g_cyc.alloc((size_t)n_far * NPH * sizeof(long long)));
    // factor pool (shared by the meshes of a batch): initial estimate; blocks
    // that find it full go to a spill queue and are rerun in a further launch
    // with an enlarged pool
    double pf = o.pool_factor > 0 ? o.pool_factor : 1.0;
    // estimate per block (complex elements).  Plain: low-rank blocks ~256 (M + N),
    // dense blocks ~12 M N, fibers 24 Ku.  Predicted: ceil(1.25 r3) + 2 crosses of
    // 16 (M + N) + Ku (low-rank, a typical kept face rank of 16) or M N + Ku.
    // Each is scaled by what earlier compressions on this context needed
    // relative to the same estimate.
    const bool pool_mlp = (mlp_use & 2) != 0;
    auto block_est = [&](int b) {
        const BlockRange& r = ranges[b];
        const double m = r.re - r.rb, n = r.ce - r.cb, ku = ku_of(b);
        if (pool_mlp) {
            const double slots = std::ceil(1.25 * rhat[b]) + 2.0;
            return slots * ((is_dense(r) ? m * n : 16.0 * (m + n)) + ku);
        }
        return (is_dense(r) ? 12.0 * m * n : 256.0 * (m + n)) + 24.0 * ku;
    };
    // learned per kernel kind and precision: operators alternating on one
    // context (single and double layer) need different pool sizes per estimate
    double& scale = ctx->pool_scale[pool_mlp ? 1 : 0][(kernel >= 0 && kernel < 6) ? kernel : 2][sizeof(T) == 4 ? 1 : 0];
    double est = 0.0;
    for (int q = 0; q < n_run; ++q) est += block_est(queue[q]);
    long long cap = (long long)(pf * scale * est);
    cap = std::max(cap, (long long)1 << 16);
    // never ask for more than 85 % of the free device memory: an estimate
    // above it is served by spill rounds instead
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b > 0)
        cap = std::min(cap, std::max((long long)1 << 16, (long long)(0.85 * (double)free_b / sizeof(Cx<T>))));
    auto pool = std::make_shared<DevBuf>();
    G3_CUDA(pool->alloc((size_t)cap * sizeof(Cx<T>)));
    G3_CUDA(cudaMemsetAsync(d_head.p, 0, 2 * sizeof(int), ctx->stream));
    G3_CUDA(cudaMemsetAsync(d_counters.p, 0, 32 * sizeof(unsigned long long), ctx->stream));
    G3_CUDA(cudaMemsetAsync(g_r3.p, 0, (size_t)n_far * sizeof(int), ctx->stream));
    G3_CUDA(cudaMemsetAsync(g_cyc.p, 0, (size_t)n_far * NPH * sizeof(long long), ctx->stream));
    std::vector<int> qpos(n_far, 0);
    for (int q = 0; q < n_run; ++q) qpos[qcat[q]] = q;
    unsigned long long base = 0;  // pool elements in use before this launch round
    int n_lo = n_low, n_de = n_dense;
    int regrows = 0, spilled_total = 0;
    unsigned status_all = 0;
    cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1];
    double ms_total = 0, ms_low_total = 0, ms_dense_total = 0;
    unsigned long long ctr = 0;
    const g3_tree* t0 = jobs[0].t;
    const g3_freqs* f0 = jobs[0].f;
    const double ms_setup = ms_since(th0);
    const auto th1 = std::chrono::steady_clock::now();
    for (int round = 0;; ++round) {
        // the first round can run as one captured CUDA graph (opts->graph):
        // the queue resets and both persistent launches become one graph launch
        const bool graph = o.graph && round == 0 && !o.unbatched;
        cudaGraph_t cg = nullptr;
        cudaStream_t main_stream = ctx->stream;
        if (graph) {
            // captured on the context's side stream (the context's stream may be
            // the legacy default stream, which cannot be captured), ordered
            // after the work already on the context's stream
            G3_CUDA(cudaEventRecord(ctx->fork, main_stream));
            G3_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork, 0));
            ctx->stream = ctx->side;
            const cudaError_t ce = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
            if (ce != cudaSuccess) {
                ctx->stream = main_stream;
                return cuda_fail(ce, "aca3_compress: cudaStreamBeginCapture");
            }
        }
        G3_CUDA(cudaMemsetAsync(d_head.p, 0, 2 * sizeof(int), ctx->stream));
        G3_CUDA(cudaMemsetAsync(d_spill_n.p, 0, sizeof(int), ctx->stream));
        G3_CUDA(cudaMemsetAsync(ctx->status.p, 0, sizeof(unsigned), ctx->stream));
        if (graph)  // base = 0 in the first round
            G3_CUDA(cudaMemsetAsync(d_ctr.p, 0, sizeof(base), ctx->stream));
        else
            G3_CUDA(cudaMemcpyAsync(d_ctr.p, &base, sizeof(base), cudaMemcpyHostToDevice, ctx->stream));
        AcaArgs<T> A{};
        A.geos = batched ? d_geos.as<GeoDesc>() : nullptr;
        A.bgeo = batched ? d_bgeo.as<int>() : nullptr;
        A.gf = t0 ? t0->gf : GeomF{};
        A.gd = t0 ? t0->gd : GeomD{};
        A.sep = sv;
        A.sd = f0 ? f0->d_sd.as<double2>() : nullptr;
        A.sf = f0 ? f0->d_sf.as<float2>() : nullptr;
        A.Ku = Ku;
        A.k_maxabs = f0 ? f0->k_maxabs : Ku - 1;
        A.ranges = d_ranges.as<BlockRange>();
        A.n_far = n_far;
        A.queue = d_queue.as<int>();
        A.queue_head = d_head.as<int>();
        A.single = -1;
        A.k1 = k1_host ? d_k1.as<int>() : nullptr;
        A.Cmax = Cmax;
        A.RF = RF;
        A.dense_max = dense_max;
        A.sample_check = o.literal_stop ? 0 : 1;
        A.pivot_index = o.pivot_index;
        A.eps3 = eps3;
        A.eps_face = eps_face;
        A.face_floor = sizeof(T) == 4 ? eps_face * (o.face_floor_scale > 0 ? o.face_floor_scale : 1.0) : 0.0;
        A.trunc_floor = sizeof(T) == 4 ? eps_face * (o.trunc_floor_scale > 0 ? o.trunc_floor_scale : 1.0) : 0.0;
        A.no_recompress = o.no_recompress;
        A.pool = pool->as<Cx<T>>();
        A.pool_cap = cap;
        A.pool_ctr = d_ctr.as<unsigned long long>();
        A.spill = d_spill.as<int>();
        A.spill_n = d_spill_n.as<int>();
        A.spill_cap = n_far;
        A.rec = g_rec.as<CrossRec>();
        A.r3 = g_r3.as<int>();
        A.blk_cycles = g_cyc.as<long long>();
        A.counters = d_counters.as<unsigned long long>();
        A.status = ctx->status.as<unsigned>();
        A.ws = d_ws.as<char>();
        A.ws_stride = stride;
        A.Mmax = Mmax;
        A.Nmax = Nmax;
        A.drf_max = drf > 0 ? drf : 0;
        A.drf_off = drf > 0 ? drf_off : 0;
        if (!graph) G3_CUDA(cudaEventRecord(e0, ctx->stream));
        g3_status st = G3_OK;
        for (int cls = 0; cls < 2 && st == G3_OK; ++cls) {
            if (cls == 1 && !graph) G3_CUDA(cudaEventRecord(ctx->ev[2], ctx->stream));
            const int cnt = cls == 0 ? n_lo : n_de;
            if (cnt == 0) continue;
            AcaArgs<T> B = A;
            B.queue = d_queue.as<int>() + (cls == 0 ? 0 : n_lo);
            B.queue_head = d_head.as<int>() + cls;
            B.n_far = cnt;
            const int launches = o.unbatched ? cnt : 1;
            const int g = std::min(cls == 0 ? grid_low : grid_dense, o.unbatched ? 1 : cnt);
            for (int l = 0; l < launches && st == G3_OK; ++l) {
                if (o.unbatched) B.single = l;
                if (cls == 1)
                    st = launch_kind<T, NT, true>(ctx, kernel, B, g, smem);
                else if constexpr (sizeof(T) == 4)
                    st = nt_low == 512   ? launch_kind<T, 512, false>(ctx, kernel, B, g, smem)
                         : nt_low == 384 ? launch_kind<T, 384, false>(ctx, kernel, B, g, smem)
                         : nt_low == 128 ? launch_kind<T, 128, false>(ctx, kernel, B, g, smem)
                                         : launch_kind<T, NT, false>(ctx, kernel, B, g, smem);
                else
                    st = launch_kind<T, NT, false>(ctx, kernel, B, g, smem);
            }
        }
        if (graph) {
            cudaError_t ce = cudaStreamEndCapture(ctx->stream, &cg);
            if (st != G3_OK || ce != cudaSuccess) {
                ctx->stream = main_stream;
                if (cg) cudaGraphDestroy(cg);
                if (st != G3_OK) return st;
                return cuda_fail(ce, "aca3_compress: stream capture of the compression");
            }
            cudaGraphExec_t ge = nullptr;
            ce = cudaGraphInstantiate(&ge, cg, 0);
            if (ce == cudaSuccess) ce = cudaEventRecord(e0, ctx->stream);
            if (ce == cudaSuccess) ce = cudaGraphLaunch(ge, ctx->stream);
            if (ce == cudaSuccess) ce = cudaEventRecord(ctx->ev[2], ctx->stream);  // no split inside the graph
            if (ce == cudaSuccess) ce = cudaEventRecord(ctx->join, ctx->stream);
            ctx->stream = main_stream;
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ctx->stream, ctx->join, 0);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
            if (ge) cudaGraphExecDestroy(ge);
            cudaGraphDestroy(cg);
            if (ce != cudaSuccess) return cuda_fail(ce, "aca3_compress: graph launch of the compression");
            ctx->count("graph_launch");
        }
        if (st != G3_OK) return st;
        G3_CUDA(cudaEventRecord(e1, ctx->stream));
        unsigned status = 0;
        int n_spill = 0;
        G3_CUDA(cudaMemcpyAsync(&status, ctx->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaMemcpyAsync(&ctr, d_ctr.p, sizeof(ctr), cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaMemcpyAsync(&n_spill, d_spill_n.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
        float ms = 0, ms_low = 0;
        G3_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        G3_CUDA(cudaEventElapsedTime(&ms_low, e0, ctx->ev[2]));
        ms_total += ms;
        ms_low_total += ms_low;
        ms_dense_total += ms - ms_low;
        status_all |= status & ~ST_POOL_OVERFLOW;
        if (!(status & ST_POOL_OVERFLOW)) break;
        if (++regrows > 8 || n_spill <= 0 || n_spill > n_far)
            return fail(G3_EOVERFLOW, "aca3_compress: factor pool overflow after %d spill rounds", regrows);
        spilled_total += n_spill;
        // spilled blocks, in their original queue order, split by class
        std::vector<int> sp(n_spill);
        G3_CUDA(cudaMemcpy(sp.data(), d_spill.p, n_spill * sizeof(int), cudaMemcpyDeviceToHost));
        std::sort(sp.begin(), sp.end(), [&](int a, int b) { return qpos[a] < qpos[b]; });
        std::vector<int> nq;
        nq.reserve(n_spill);
        double est2 = 0.0;
        for (int pass = 0; pass < 2; ++pass)
            for (int b : sp)
                if (is_dense(ranges[b]) == (pass == 1)) {
                    nq.push_back(b);
                    est2 += block_est(b);
                }
        n_lo = 0;
        for (int b : sp) n_lo += !is_dense(ranges[b]);
        n_de = n_spill - n_lo;
        // enlarged pool: the used part [0, cap) is kept at the same offsets
        // at least 1.5 times the spilled blocks' plain estimate (which
        // over-reserves): one round, even after the learned scale has shrunk
        long long add = (long long)(1.5 * std::max(scale, 1.0) * est2);
        add = std::max(add, (long long)(ctr - std::min<unsigned long long>(ctr, (unsigned long long)cap)));
        add = std::max(add, (long long)1 << 16);
        // the enlarged pool and the copy of the old one must fit together
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const long long room = (long long)(0.9 * (double)free_b / sizeof(Cx<T>)) - cap;
            if (room < (long long)1 << 16)
                return fail(G3_ENOMEM, "aca3_compress: the factors need more than the free device memory");
            add = std::min(add, room);
        }
        DevBuf grown;
        G3_CUDA(grown.alloc((size_t)(cap + add) * sizeof(Cx<T>)));
        G3_CUDA(cudaMemcpyAsync(grown.p, pool->p, (size_t)cap * sizeof(Cx<T>), cudaMemcpyDeviceToDevice, ctx->stream));
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
        take(*pool, grown);
        base = (unsigned long long)cap;
        cap += add;
        G3_CUDA(cudaMemcpy(d_queue.p, nq.data(), n_spill * sizeof(int), cudaMemcpyHostToDevice));
    }
    const double ms_rounds = ms_since(th1);
    const auto th2 = std::chrono::steady_clock::now();
    // the pool's scale against the estimate, learned from what this run
    // needed (+15 %): it grows at once and shrinks by at most half per run,
    // so that an over-reserving estimate stops costing the trim copy below on
    // every compression while a problem that needs more than the last one
    // rarely spills
    if (est > 0) {
        const double need = 1.15 * (double)ctr / est;
        scale = need >= scale ? need : std::max(need, 0.5 * scale);
    }
    // give back what the estimate over-reserved: a pool much larger than its
    // use is moved into an exact-size buffer (its offsets stay valid)
    if (ctr > 0 && (double)cap > 1.25 * (double)ctr && ((long long)cap - (long long)ctr) * (long long)sizeof(Cx<T>) > (256LL << 20)) {
        DevBuf exact;
        if (exact.alloc((size_t)ctr * sizeof(Cx<T>)) == cudaSuccess) {
            G3_CUDA(cudaMemcpyAsync(exact.p, pool->p, (size_t)ctr * sizeof(Cx<T>), cudaMemcpyDeviceToDevice,
                                    ctx->stream));
            G3_CUDA(cudaStreamSynchronize(ctx->stream));
            take(*pool, exact);
            cap = (long long)ctr;
        } else {
            cudaGetLastError();  // keep the large pool
        }
    }
    // read-back: counters and ranks, then the kept records packed on the
    // device and the per-block cycles, through the pinned staging buffer
    unsigned long long cnt[32];
    G3_CUDA(cudaMemcpy(cnt, d_counters.p, sizeof(cnt), cudaMemcpyDeviceToHost));
    std::vector<int32_t> r3(n_far);
    G3_CUDA(cudaMemcpy(r3.data(), g_r3.p, n_far * sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<long long> roff((size_t)n_far + 1, 0);
    for (int b = 0; b < n_far; ++b) {
        if (r3[b] < 0 || r3[b] > Cmax) return fail(G3_ECUDA, "aca3_compress: block %d has %d crosses", b, r3[b]);
        roff[b + 1] = roff[b] + r3[b];
    }
    const size_t rec_bytes = (size_t)roff[n_far] * sizeof(CrossRec);
    const size_t ph_bytes = (size_t)n_far * NPH * sizeof(long long);
    {
        const g3_status sst = stage_ensure(ctx, al256(rec_bytes) + ph_bytes);
        if (sst != G3_OK) return sst;
    }
    CrossRec* h_rec = static_cast<CrossRec*>(ctx->h_stage);
    long long* h_ph = reinterpret_cast<long long*>(static_cast<char*>(ctx->h_stage) + al256(rec_bytes));
    {
        DevBuf d_off, d_pack;
        G3_CUDA(d_off.alloc(roff.size() * sizeof(long long)));
        G3_CUDA(d_pack.alloc(std::max(rec_bytes, (size_t)16)));
        G3_CUDA(cudaMemcpyAsync(d_off.p, roff.data(), roff.size() * sizeof(long long), cudaMemcpyHostToDevice,
                                ctx->stream));
        const long long n_all = (long long)n_far * Cmax;
        const int g_pack = (int)std::min<long long>((n_all + 255) / 256, (long long)ctx->n_sm * 8);
        k_rec_pack<<<std::max(g_pack, 1), 256, 0, ctx->stream>>>(g_rec.as<CrossRec>(), g_r3.as<int>(),
                                                                 d_off.as<long long>(), Cmax, n_all,
                                                                 d_pack.as<CrossRec>());
        G3_CUDA(cudaGetLastError());
        ctx->count("k_rec_pack");
        if (rec_bytes > 0)
            G3_CUDA(cudaMemcpyAsync(h_rec, d_pack.p, rec_bytes, cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaMemcpyAsync(h_ph, g_cyc.p, ph_bytes, cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    // per mesh: device slices (the whole buffers for a single mesh), host
    // copies and statistics; the pool is shared
    for (int j = 0; j < n_jobs; ++j) {
        AcaJob& J = jobs[j];
        g3_factors* fa = J.fa;
        fa->pool = pool;
        fa->pool_cap = cap;
        if (!batched) {
            take(fa->d_rec, g_rec);
            take(fa->d_r3, g_r3);
            take(fa->d_cycles, g_cyc);
        } else {
            G3_CUDA(fa->d_rec.alloc((size_t)std::max(J.n, 1) * Cmax * sizeof(CrossRec)));
            G3_CUDA(fa->d_r3.alloc((size_t)std::max(J.n, 1) * sizeof(int)));
            G3_CUDA(fa->d_cycles.alloc((size_t)std::max(J.n, 1) * NPH * sizeof(long long)));
            if (J.n > 0) {
                G3_CUDA(cudaMemcpy(fa->d_rec.p, g_rec.as<CrossRec>() + (size_t)J.first * Cmax,
                                   (size_t)J.n * Cmax * sizeof(CrossRec), cudaMemcpyDeviceToDevice));
                G3_CUDA(cudaMemcpy(fa->d_r3.p, g_r3.as<int>() + J.first, (size_t)J.n * sizeof(int),
                                   cudaMemcpyDeviceToDevice));
                G3_CUDA(cudaMemcpy(fa->d_cycles.p, g_cyc.as<long long>() + (size_t)J.first * NPH,
                                   (size_t)J.n * NPH * sizeof(long long), cudaMemcpyDeviceToDevice));
            }
        }
        fa->r3.assign(r3.begin() + J.first, r3.begin() + J.first + J.n);
        fa->phases.assign(h_ph + (size_t)J.first * NPH, h_ph + (size_t)(J.first + J.n) * NPH);
        fa->cycles.assign(J.n, 0);
        for (int b = 0; b < J.n; ++b)
            for (int i = 0; i < 7; ++i) fa->cycles[b] += fa->phases[(size_t)b * NPH + i];
        fa->rec.assign(h_rec + roff[J.first], h_rec + roff[J.first + J.n]);
        fa->rec_off.resize((size_t)J.n + 1);
        for (int b = 0; b <= J.n; ++b) fa->rec_off[b] = roff[J.first + b] - roff[J.first];
        // batch-wide counters and times (a batched compression is one launch)
        g3_stats& S = fa->stats;
        S = g3_stats{};
        S.n_far = J.n;
        S.blocks_run = std::max(0, std::min(J.n, n_run - J.first));
        S.entries = (int64_t)cnt[0];
        S.crosses_computed = (int64_t)cnt[1];
        S.zero_blocks = (int32_t)cnt[2];
        S.capped_faces = (int32_t)cnt[3];
        S.pool_regrows = regrows;
        S.recompress_fallbacks = (int32_t)cnt[4];
        S.status_bits = (int32_t)status_all;
        S.ms = ms_total;
        S.ms_lowrank = ms_low_total;
        S.ms_dense = ms_dense_total;
        S.spilled_blocks = spilled_total;
        S.entries_face_dense = (int64_t)cnt[7];
        S.face_check_restarts = (int64_t)cnt[5];
        S.stop_check_overrides = (int64_t)cnt[6];
        S.mlp_used = mlp_use;
        S.ms_mlp = ms_mlp;
        for (int i = 0; i < 7; ++i) S.phase_cycles[i] = (int64_t)cnt[8 + i];
        for (int i = 0; i < NSUB; ++i) S.sub_cycles[i] = (int64_t)cnt[16 + i];
        S.ctas = grid;
        for (int b = 0; b < J.n; ++b) {
            const BlockRange& rg = fa->ranges[b];
            const int M = rg.re - rg.rb, N = rg.ce - rg.cb;
            S.crosses += fa->r3[b];
            S.r3_max = std::max(S.r3_max, fa->r3[b]);
            S.dense_bytes += (int64_t)M * N * J.Ku * (int64_t)sizeof(Cx<T>);
            for (int p = 0; p < fa->r3[b]; ++p) {
                const CrossRec& c = fa->crec(b, p);
                if (c.r < 0) {  // dense face
                    S.dense_crosses += 1;
                    S.factor_bytes += ((int64_t)M * N + J.Ku) * (int64_t)sizeof(Cx<T>);
                } else {
                    S.face_rank_sum += c.r;
                    S.face_rank_max = std::max(S.face_rank_max, c.r);
                    S.factor_bytes += ((int64_t)c.r * (M + N) + J.Ku) * (int64_t)sizeof(Cx<T>);
                }
            }
        }
        S.ms_host[0] = ms_setup;
        S.ms_host[1] = ms_rounds;
        S.ms_host[2] = ms_since(th2);
        const auto th3 = std::chrono::steady_clock::now();
        const g3_status pst = far_plan_build(fa);
        if (pst != G3_OK) return pst;
        S.ms_host[3] = ms_since(th3);
    }
    return G3_OK;
}

// ---------------------------------------------------------------------------
// Three-way ACA of the H-matrix as a whole (Section 4, first implementation
// remark; kernels in g3_aca_dev.cuh): the host runs Algorithm 1's loop over
// crosses with one face launch over all admissible blocks per cross, the
// global pivot, one shared fiber and eq. (norm) summed over the blocks; the
// literal stopping test (rank l - 1).  Low-rank faces for every block.
// ---------------------------------------------------------------------------
template <class T>
static g3_status run_aca_whole_t(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_factors* fa, int kernel,
                                 double eps3, const g3_opts& o) {
    const int RF = o.face_rank_max > 0 ? std::min(o.face_rank_max, RF_MAX) : 48;
    const double eps_face = o.eps_face > 0 ? o.eps_face : (sizeof(T) == 4 ? std::max(eps3 / 100.0, 1e-5) : eps3 / 100.0);
    std::vector<BlockRange> ranges;
    for (int b : t->far_index) {
        const int32_t* r = &t->blocks[5 * (size_t)b];
        ranges.push_back(BlockRange{r[0], r[1], r[2], r[3]});
    }
    const int n_far = (int)ranges.size();
    const int Ku = fa->Ku, Cmax = Ku;
    fa->n_far = n_far;
    fa->ranges = ranges;
    fa->r3.assign(n_far, 0);
    fa->Cmax = Cmax;
    if (n_far == 0) return far_plan_build(fa);
    int Mmax = 0, Nmax = 0;
    long long worst = 0;  // pool elements one cross can take
    for (auto& r : ranges) {
        const int M = r.re - r.rb, N = r.ce - r.cb;
        Mmax = std::max(Mmax, M);
        Nmax = std::max(Nmax, N);
        worst += (long long)std::min(RF, std::min(M, N)) * (M + N) + Ku;
    }
    std::vector<int> queue(n_far);
    std::iota(queue.begin(), queue.end(), 0);
    std::stable_sort(queue.begin(), queue.end(), [&](int a, int b) {
        return (long long)(ranges[a].re - ranges[a].rb) * (ranges[a].ce - ranges[a].cb) >
               (long long)(ranges[b].re - ranges[b].rb) * (ranges[b].ce - ranges[b].cb);
    });
    const size_t recomp_bytes = 2 * (size_t)RS * RS * sizeof(Cx<double>) +
                                std::max(2 * (size_t)RS * RS * sizeof(Cx<T>), 33 * (size_t)RF * sizeof(Cx<T>)) +
                                (sizeof(T) == 4 ? 2 * (size_t)RS * RS * sizeof(Cx<T>) : 0);
    const size_t gram_bytes = ((NORM_RC<T> + 1) * (size_t)(32 + RF) + 32 * (size_t)RF) * sizeof(Cx<T>) + 64 * sizeof(void*);
    const size_t tab_bytes = 2 * TABMAX * sizeof(long long) + TABMAX * sizeof(short) +
                             (TABMAX + RF_MAX) * sizeof(Cx<T>) + ROWMAX * sizeof(Cx<T>) + 64;
    const size_t smem = std::max(std::max(recomp_bytes, gram_bytes), tab_bytes);
    const int grid = std::max(1, std::min(n_far, 2 * ctx->n_sm));
    const size_t stride = al256(ws_bytes<T>(RF, Mmax, Nmax, Cmax, Ku));
    DevBuf d_ws, d_ranges, d_queue, d_head, d_counters, d_ctr, d_rec, d_r3, d_normb, d_cand, d_hh, d_hself, d_fib,
        d_ff, d_scal, d_tot;
    G3_CUDA(d_ws.alloc(stride * grid));
    G3_CUDA(d_ranges.alloc(n_far * sizeof(BlockRange)));
    G3_CUDA(d_queue.alloc(n_far * sizeof(int)));
    G3_CUDA(d_head.alloc(sizeof(int)));
    G3_CUDA(d_counters.alloc(32 * sizeof(unsigned long long)));
    G3_CUDA(d_ctr.alloc(sizeof(unsigned long long)));
    G3_CUDA(d_rec.alloc((size_t)n_far * Cmax * sizeof(CrossRec)));
    G3_CUDA(d_r3.alloc(n_far * sizeof(int)));
    G3_CUDA(d_normb.alloc(n_far * sizeof(double)));
    G3_CUDA(d_cand.alloc(n_far * sizeof(WholeCand)));
    G3_CUDA(d_hh.alloc((size_t)n_far * Cmax * sizeof(Cx<double>)));
    G3_CUDA(d_hself.alloc(n_far * sizeof(double)));
    G3_CUDA(d_fib.alloc((size_t)Cmax * Ku * sizeof(Cx<double>)));
    G3_CUDA(d_ff.alloc((size_t)(Cmax + 1) * sizeof(Cx<double>)));
    G3_CUDA(d_scal.alloc(2 * sizeof(double)));
    G3_CUDA(d_tot.alloc(2 * sizeof(double)));
    G3_CUDA(cudaMemcpy(d_ranges.p, ranges.data(), n_far * sizeof(BlockRange), cudaMemcpyHostToDevice));
    G3_CUDA(cudaMemcpy(d_queue.p, queue.data(), n_far * sizeof(int), cudaMemcpyHostToDevice));
    G3_CUDA(cudaMemset(d_counters.p, 0, 32 * sizeof(unsigned long long)));
    G3_CUDA(cudaMemset(d_ctr.p, 0, sizeof(unsigned long long)));
    G3_CUDA(cudaMemset(d_normb.p, 0, n_far * sizeof(double)));
    G3_CUDA(cudaMemset(d_r3.p, 0, n_far * sizeof(int)));
    auto pool = std::make_shared<DevBuf>();
    long long cap = 4 * worst;
    G3_CUDA(pool->alloc((size_t)cap * sizeof(Cx<T>)));
    AcaArgs<T> A{};
    A.gf = t->gf;
    A.gd = t->gd;
    A.sd = f->d_sd.as<double2>();
    A.sf = f->d_sf.as<float2>();
    A.Ku = Ku;
    A.k_maxabs = f->k_maxabs;
    A.ranges = d_ranges.as<BlockRange>();
    A.n_far = n_far;
    A.queue = d_queue.as<int>();
    A.queue_head = d_head.as<int>();
    A.single = -1;
    A.Cmax = Cmax;
    A.RF = RF;
    A.dense_max = -1;
    A.sample_check = 0;
    A.eps3 = eps3;
    A.eps_face = eps_face;
    A.face_floor = sizeof(T) == 4 ? eps_face * (o.face_floor_scale > 0 ? o.face_floor_scale : 1.0) : 0.0;
    A.trunc_floor = sizeof(T) == 4 ? eps_face * (o.trunc_floor_scale > 0 ? o.trunc_floor_scale : 1.0) : 0.0;
    A.no_recompress = o.no_recompress;
    A.pool_ctr = d_ctr.as<unsigned long long>();
    A.rec = d_rec.as<CrossRec>();
    A.r3 = d_r3.as<int>();
    A.counters = d_counters.as<unsigned long long>();
    A.status = ctx->status.as<unsigned>();
    A.ws = d_ws.as<char>();
    A.ws_stride = stride;
    A.Mmax = Mmax;
    A.Nmax = Nmax;
    auto face = [&](int kf, int nc) -> g3_status {
        if (kernel == G3_SLP)
            return launch_whole_t<G3_SLP, T>(ctx, A, grid, smem, kf, nc, d_normb.as<double>(), d_cand.as<WholeCand>(),
                                             d_hh.as<Cx<double>>(), d_hself.as<double>());
        if (kernel == G3_DLP)
            return launch_whole_t<G3_DLP, T>(ctx, A, grid, smem, kf, nc, d_normb.as<double>(), d_cand.as<WholeCand>(),
                                             d_hh.as<Cx<double>>(), d_hself.as<double>());
        return launch_whole_t<G3_GAL_SLP, T>(ctx, A, grid, smem, kf, nc, d_normb.as<double>(), d_cand.as<WholeCand>(),
                                             d_hh.as<Cx<double>>(), d_hself.as<double>());
    };
    auto fiber = [&](int pb, int pi, int pj, int nc) -> g3_status {
        if (kernel == G3_SLP)
            return launch_whole_fiber_t<G3_SLP, T>(ctx, A, pb, pi, pj, nc, d_fib.as<Cx<double>>(), d_ff.as<Cx<double>>(),
                                                   d_scal.as<double>(), n_far, d_hh.as<Cx<double>>(),
                                                   d_hself.as<double>(), d_normb.as<double>(), d_tot.as<double>());
        if (kernel == G3_DLP)
            return launch_whole_fiber_t<G3_DLP, T>(ctx, A, pb, pi, pj, nc, d_fib.as<Cx<double>>(), d_ff.as<Cx<double>>(),
                                                   d_scal.as<double>(), n_far, d_hh.as<Cx<double>>(),
                                                   d_hself.as<double>(), d_normb.as<double>(), d_tot.as<double>());
        return launch_whole_fiber_t<G3_GAL_SLP, T>(ctx, A, pb, pi, pj, nc, d_fib.as<Cx<double>>(),
                                                   d_ff.as<Cx<double>>(), d_scal.as<double>(), n_far,
                                                   d_hh.as<Cx<double>>(), d_hself.as<double>(), d_normb.as<double>(),
                                                   d_tot.as<double>());
    };
    std::vector<char> used(Ku, 0);
    std::vector<WholeCand> cand(n_far);
    std::vector<Cx<double>> fib((size_t)Ku);
    double norm2 = 0.0;
    int k = 0, R = 0, computed = 0;
    unsigned status_all = 0;
    cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1];
    G3_CUDA(cudaEventRecord(e0, ctx->stream));
    for (int ell = 0; ell < Ku; ++ell) {
        // the face at k, else up to three more unused frequencies (zero faces everywhere)
        const int tries[4] = {k, Ku - 1, Ku / 2, f->k_maxabs};
        int pb = -1;
        for (int c = 0; c < 4 && pb < 0; ++c) {
            const int kk = tries[c];
            bool dup = c > 0 && used[kk];
            for (int d = 1; d < c; ++d) dup |= tries[d] == kk;
            if (dup) continue;
            // pool room for one more cross of every block
            unsigned long long ctr = 0;
            G3_CUDA(cudaMemcpy(&ctr, d_ctr.p, sizeof(ctr), cudaMemcpyDeviceToHost));
            if ((long long)ctr + worst > cap) {
                const long long ncap = std::max((long long)ctr + 4 * worst, cap + cap / 2);
                DevBuf grown;
                G3_CUDA(grown.alloc((size_t)ncap * sizeof(Cx<T>)));
                G3_CUDA(cudaMemcpy(grown.p, pool->p, (size_t)ctr * sizeof(Cx<T>), cudaMemcpyDeviceToDevice));
                take(*pool, grown);
                cap = ncap;
            }
            A.pool = pool->as<Cx<T>>();
            A.pool_cap = cap;
            G3_CUDA(cudaMemsetAsync(d_head.p, 0, sizeof(int), ctx->stream));
            G3_CUDA(cudaMemsetAsync(ctx->status.p, 0, sizeof(unsigned), ctx->stream));
            { const g3_status st_ = face(kk, ell); if (st_ != G3_OK) return st_; }
            unsigned status = 0;
            G3_CUDA(cudaMemcpyAsync(cand.data(), d_cand.p, n_far * sizeof(WholeCand), cudaMemcpyDeviceToHost,
                                    ctx->stream));
            G3_CUDA(cudaMemcpyAsync(&status, ctx->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
            G3_CUDA(cudaStreamSynchronize(ctx->stream));
            status_all |= status;
            if (status & ST_POOL_OVERFLOW) return fail(G3_EOVERFLOW, "aca3_compress: whole-matrix factor pool overflow");
            used[kk] = 1;
            ++computed;
            double best = sizeof(T) == 4 ? 1.1754944e-38 : 2.2250738585072014e-308;
            for (int b = 0; b < n_far; ++b)
                if (cand[b].v > best) {
                    best = cand[b].v;
                    pb = b;
                }
            if (pb >= 0) k = kk;
        }
        if (pb < 0) break;  // zero faces at every tested frequency: the rank is ell
        G3_CUDA(cudaMemsetAsync(d_tot.p, 0, 2 * sizeof(double), ctx->stream));
        { const g3_status st_ = fiber(pb, cand[pb].i, cand[pb].j, ell); if (st_ != G3_OK) return st_; }
        double scal[2], tot[2];
        G3_CUDA(cudaMemcpyAsync(scal, d_scal.p, sizeof(scal), cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaMemcpyAsync(tot, d_tot.p, sizeof(tot), cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaMemcpyAsync(fib.data(), d_fib.as<Cx<double>>() + (size_t)ell * Ku, Ku * sizeof(Cx<double>),
                                cudaMemcpyDeviceToHost, ctx->stream));
        G3_CUDA(cudaStreamSynchronize(ctx->stream));
        norm2 += tot[0];
        const double nH2 = tot[1], nf2 = scal[0];
        if (std::sqrt(std::max(nH2 * nf2, 0.0)) <= eps3 * std::sqrt(std::max(norm2, 0.0))) break;  // rank ell
        R = ell + 1;
        bool all = true;
        for (int q = 0; q < Ku; ++q) all &= used[q] != 0;
        if (all) break;
        double bv = -1.0;
        int bk = -1;
        for (int q = 0; q < Ku; ++q)
            if (!used[q]) {
                const double v = fib[q].x * fib[q].x + fib[q].y * fib[q].y;
                if (v > bv) {
                    bv = v;
                    bk = q;
                }
            }
        if (bk < 0) break;
        k = bk;
    }
    G3_CUDA(cudaEventRecord(e1, ctx->stream));
    G3_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    G3_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    // every block keeps the R crosses before the dropped one
    fa->r3.assign(n_far, R);
    G3_CUDA(cudaMemcpy(d_r3.p, fa->r3.data(), n_far * sizeof(int), cudaMemcpyHostToDevice));
    {
        std::vector<CrossRec> full((size_t)n_far * Cmax);
        G3_CUDA(cudaMemcpy(full.data(), d_rec.p, full.size() * sizeof(CrossRec), cudaMemcpyDeviceToHost));
        compact_records(fa, full, Cmax);
    }
    unsigned long long cnt[32];
    G3_CUDA(cudaMemcpy(cnt, d_counters.p, sizeof(cnt), cudaMemcpyDeviceToHost));
    unsigned long long ctr = 0;
    G3_CUDA(cudaMemcpy(&ctr, d_ctr.p, sizeof(ctr), cudaMemcpyDeviceToHost));
    fa->pool = pool;
    fa->pool_cap = cap;
    take(fa->d_rec, d_rec);
    take(fa->d_r3, d_r3);
    fa->phases.assign((size_t)n_far * NPH, 0);
    fa->cycles.assign(n_far, 0);
    g3_stats& S = fa->stats;
    S = g3_stats{};
    S.n_far = n_far;
    S.blocks_run = n_far;
    S.entries = (int64_t)cnt[0];
    S.crosses_computed = (int64_t)computed * n_far;
    S.status_bits = (int32_t)(status_all & ~ST_POOL_OVERFLOW);
    S.ms = ms;
    S.ms_lowrank = ms;
    S.ctas = grid;
    for (int b = 0; b < n_far; ++b) {
        const int M = ranges[b].re - ranges[b].rb, N = ranges[b].ce - ranges[b].cb;
        S.crosses += R;
        S.r3_max = std::max(S.r3_max, R);
        S.dense_bytes += (int64_t)M * N * Ku * (int64_t)sizeof(Cx<T>);
        for (int p = 0; p < R; ++p) {
            const CrossRec& c = fa->crec(b, p);
            S.face_rank_sum += c.r;
            S.face_rank_max = std::max(S.face_rank_max, c.r);
            S.factor_bytes += ((int64_t)c.r * (M + N) + Ku) * (int64_t)sizeof(Cx<T>);
        }
    }
    (void)ctr;
    return far_plan_build(fa);
}

g3_status run_aca(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_factors* fa, int kernel, int scheme,
                  double eps3, const g3_opts& o, const void* sep_a, const void* sep_b, const void* sep_c, int sep_R) {
    if (o.whole_matrix) {
        if (kernel == G3_GAL_P1D || kernel == G3_GAL_P1KP)
            return fail(G3_EUNSUPPORTED, "aca3_compress: whole_matrix is not implemented for linear elements");
        if (kernel == G3_SEPARABLE || o.unbatched)
            return fail(G3_EUNSUPPORTED, "aca3_compress: whole_matrix applies to boundary element operators, not unbatched");
        if (scheme == G3_GALERKIN4x4 && kernel != G3_SLP)
            return fail(G3_EUNSUPPORTED, "aca3_compress: the Galerkin scheme is implemented for G3_SLP");
        if (fa->Ku > KU_MAX) return fail(G3_EINVAL, "aca3_compress: %d unique frequencies exceed %d", fa->Ku, KU_MAX);
        const int kk = scheme == G3_GALERKIN4x4 ? G3_GAL_SLP : kernel;
        if (fa->prec == G3_MIXED) return run_aca_whole_t<float>(ctx, t, f, fa, kk, eps3, o);
        return run_aca_whole_t<double>(ctx, t, f, fa, kk, eps3, o);
    }
    const bool p1 = kernel == G3_GAL_P1D || kernel == G3_GAL_P1KP;
    if (scheme == G3_GALERKIN4x4 && kernel != G3_SLP && !p1)
        return fail(G3_EUNSUPPORTED, "aca3_compress: the Galerkin scheme is implemented for G3_SLP");
    if (scheme == G3_GALERKIN4x4 && !p1) kernel = G3_GAL_SLP;
    if (fa->Ku > KU_MAX) return fail(G3_EINVAL, "aca3_compress: %d unique frequencies exceed %d", fa->Ku, KU_MAX);
    std::vector<AcaJob> jobs(1);
    jobs[0].t = t;
    jobs[0].f = f;
    jobs[0].fa = fa;
    if (fa->prec == G3_MIXED) return run_aca_t<float>(ctx, jobs, kernel, eps3, o, sep_a, sep_b, sep_c, sep_R);
    return run_aca_t<double>(ctx, jobs, kernel, eps3, o, sep_a, sep_b, sep_c, sep_R);
}

g3_status run_aca_batch(g3_ctx* ctx, const g3_tree* const* trees, const g3_freqs* const* freqs, int n,
                        g3_factors* const* fas, int kernel, int scheme, double eps3, const g3_opts& o) {
    if (scheme == G3_GALERKIN4x4 && kernel != G3_SLP)
        return fail(G3_EUNSUPPORTED, "aca3_compress_batch: the Galerkin scheme is implemented for G3_SLP");
    if (scheme == G3_GALERKIN4x4) kernel = G3_GAL_SLP;
    std::vector<AcaJob> jobs(n);
    for (int j = 0; j < n; ++j) {
        if (fas[j]->Ku > KU_MAX)
            return fail(G3_EINVAL, "aca3_compress_batch: mesh %d has %d unique frequencies (max %d)", j, fas[j]->Ku,
                        KU_MAX);
        jobs[j].t = trees[j];
        jobs[j].f = freqs[j];
        jobs[j].fa = fas[j];
    }
    if (fas[0]->prec == G3_MIXED) return run_aca_t<float>(ctx, jobs, kernel, eps3, o, nullptr, nullptr, nullptr, 0);
    return run_aca_t<double>(ctx, jobs, kernel, eps3, o, nullptr, nullptr, nullptr, 0);
}

}  // namespace g3
