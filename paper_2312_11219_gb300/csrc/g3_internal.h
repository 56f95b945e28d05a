// Internal declarations shared by the host C++ and the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/g3aca.h"

namespace g3 {

// ---- error handling -------------------------------------------------------

void set_error(const char* fmt, ...);
g3_status fail(g3_status st, const char* fmt, ...);
g3_status cuda_fail(cudaError_t e, const char* what);

#define G3_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::g3::cuda_fail(e_, #call);            \
    } while (0)

// ---- device status bits (written by kernels with atomicOr) ----------------
enum : unsigned {
    ST_POOL_OVERFLOW = 1u << 0,   // factor pool exhausted
    ST_FACE_CAPPED = 1u << 1,     // a face ACA hit its rank cap
    ST_CHOL_FALLBACK = 1u << 2,   // recompression skipped (Cholesky breakdown)
    ST_BAD_INDEX = 1u << 3,       // an index check failed (access skipped)
    ST_JACOBI_NOCONV = 1u << 4,   // Jacobi SVD hit its sweep limit
};

// ---- owned device buffer ----------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t n) {
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        else p = nullptr;
        return e;
    }
    cudaError_t ensure(size_t n) { return n <= bytes ? cudaSuccess : alloc(n); }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ---- geometry views passed to kernels (cluster order, SoA) ------------------
// float32 view: centroid as an unevaluated float-float sum (hi + lo) so that
// centroid differences keep float32 relative accuracy; quadrature points as
// float offsets from the centroid.
struct GeomF {
    int E;
    const float* ch;   // [3][E]
    const float* cl;   // [3][E]
    const float* q;    // [7][3][E] 7-point rule offsets  y_q - c
    const float* w;    // [7][E] weight * area
    const float* n;    // [3][E] unit normal
    const float* q4;   // [4][3][E] 4-point (Galerkin) rule offsets
    const float* w4;   // [4][E]
    const float* curl; // [3 local][3][E] surface curls of the linear shape functions (linear-element trees)
};
struct GeomD {
    int E;
    const double* c;   // [3][E]
    const double* q;   // [7][3][E]
    const double* w;   // [7][E]
    const double* n;   // [3][E]
    const double* v;   // [3 vertices][3 coords][E] absolute vertex coordinates
    const double* q4;  // [4][3][E]
    const double* w4;  // [4][E]
    const double* gl;  // 24-point Gauss-Legendre nodes [24] then weights [24] on [-1, 1]
    const double* curl; // [3 local][3][E] surface curls of the linear shape functions (linear-element trees)
};

#ifdef __CUDACC__
#define G3_HD __host__ __device__
#else
#define G3_HD
#endif

// internal kernel kind of the Galerkin single layer (the C ABI passes G3_SLP
// with G3_GALERKIN4x4)
constexpr int G3_GAL_SLP = 3;
// kernel kinds of the Galerkin operators with linear continuous elements (the
// same values as their public g3_kernel names): hypersingular operator D and
// adjoint double layer K', on element-local degrees of freedom
constexpr int G3_GAL_P1D = 4;
constexpr int G3_GAL_P1KP = 5;

// Galerkin pairs with a common vertex: classification and vertex order for
// the Sauter-Schwab rules (shared vertices first, in the same order in both
// panels; a common edge keeps the orientation it has in the first panel)
enum : int { SS_REGULAR = 0, SS_VERTEX = 1, SS_EDGE = 2, SS_IDENTICAL = 3 };

G3_HD inline int ss_classify(const int* a, const int* b, bool same, int8_t px[3], int8_t py[3]) {
    if (same) {
        for (int k = 0; k < 3; ++k) px[k] = py[k] = (int8_t)k;
        return SS_IDENTICAL;
    }
    int ia[3], ib[3], nc = 0;
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y)
            if (a[x] == b[y]) {
                ia[nc] = x;
                ib[nc] = y;
                ++nc;
            }
    if (nc == 0) return SS_REGULAR;
    if (nc == 1) {
        px[0] = (int8_t)ia[0];
        py[0] = (int8_t)ib[0];
        for (int k = 0, u = 1, v = 1; k < 3; ++k) {
            if (k != ia[0]) px[u++] = (int8_t)k;
            if (k != ib[0]) py[v++] = (int8_t)k;
        }
        return SS_VERTEX;
    }
    if (nc == 2) {
        int e0 = 0, e1 = 1;
        if ((ia[0] + 1) % 3 != ia[1]) {
            e0 = 1;
            e1 = 0;
        }
        px[0] = (int8_t)ia[e0];
        px[1] = (int8_t)ia[e1];
        px[2] = (int8_t)(3 - ia[0] - ia[1]);
        py[0] = (int8_t)ib[e0];
        py[1] = (int8_t)ib[e1];
        py[2] = (int8_t)(3 - ib[0] - ib[1]);
        return SS_EDGE;
    }
    for (int k = 0; k < 3; ++k) {  // three common vertices: the same triangle
        px[k] = (int8_t)k;
        py[k] = (int8_t)ib[k];
    }
    return SS_IDENTICAL;
}

// one Galerkin near-field pair for the Sauter-Schwab kernel
struct SsPair {
    int i, j;          // cluster positions of tau_x, tau_y
    int cas;           // SS_VERTEX, SS_EDGE or SS_IDENTICAL
    int stride;        // M_b N_b: distance between frequencies in the block
    long long off;     // near-field offset of the entry at the first frequency (linear
                       // elements: of the entry of local functions (0, 0))
    int8_t px[3], py[3];
    int ldm;           // linear elements: rows M_b of the block (column stride of the local entries)
};

// synthetic separable tensor sum_t a[t][i] b[t][j] c[t][k] (complex, interleaved)
template <class T>
struct SepView {
    int R, M, N, Ku;
    const T* a;  // [R][M][2]
    const T* b;  // [R][N][2]
    const T* c;  // [R][Ku][2]
};

struct BlockRange {
    int rb, re, cb, ce;
};

// per-cross record written by the compression kernel
struct CrossRec {
    long long off;   // pool offset (complex elements) of U (M x r), then V (N x r), then f (Ku)
    int r;           // face rank
    int ip, jp, kp;  // pivot (local row, local column, unique-frequency index)
};

}  // namespace g3

// ---- opaque handle definitions ---------------------------------------------

struct g3_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int apply_tensor_cores = 1;  // float32 far-field x formation on the tensor cores
    int n_sm = 0;
    size_t smem_optin = 0;
    std::map<std::string, int64_t> launches;
    int64_t n_launch = 0;
    std::vector<std::string> names_cache;
    g3::DevBuf gl;           // Gauss-Legendre table for self terms
    g3::DevBuf scratch;      // apply scratch (cluster-order densities, partial y)
    g3::DevBuf aca_ws;       // per-CTA workspace of the compression (grown, never shrunk)
    g3::DevBuf status;       // device status word(s)
    g3::DevBuf stage_w, stage_y;  // device staging of host W / Y in apply_gcq
    void* h_stage = nullptr;      // pinned host staging of read-backs (grown, never shrunk)
    size_t h_stage_bytes = 0;
    cudaEvent_t ev[6] = {};
    // a second stream on which the apply runs its near field next to the far
    // field (fork / join through events; ev_side times the near field there)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t ev_side[2] = {};
    double last_apply_ms = 0, last_near_ms = 0;
    // factor-pool size / estimate needed by earlier compressions, per kernel
    // kind (slot 4: anything else) and working precision, [0] plain estimate,
    // [1] the predictor-based one
    // factor-pool scale against the plain estimate, per predictor use, kernel
    // kind (single, double layer, separable, Galerkin single layer,
    // hypersingular, adjoint double layer) and precision
    double pool_scale[2][6][2] = {{{1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}},
                                  {{1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}}};
    std::map<long long, std::array<int, 3>> tune_cache;  // autotuner: key -> (threads, dense_face_max,
                                                         // residual_face_max)
    int64_t last_apply_bytes = 0, last_near_bytes = 0;
    void count(const char* name, int64_t n = 1) {
        launches[name] += n;
        n_launch += n;
    }
};

struct g3_freqs {
    g3_ctx* ctx = nullptr;
    int device = 0;                // the context's device (freeing needs no context)
    int kind = 0;  // 0 = bdf2, 1 = gcq, 2 = given by the caller
    int K = 0, Ku = 0;
    std::vector<double> s;      // [2K]
    std::vector<double> omega;  // [2K]
    std::vector<int32_t> uniq;  // [Ku]
    std::vector<int32_t> partner;  // [K]
    int k_maxabs = 0;           // unique index of the largest |s|
    g3::DevBuf d_s_all, d_w_all; // [K] double2: all frequencies and contour weights
    g3::DevBuf d_sd;            // [Ku] double2 (unique set)
    g3::DevBuf d_sf;            // [Ku] float2
    g3::DevBuf d_uniq, d_partner;
};

struct g3_tree {
    g3_ctx* ctx = nullptr;
    int device = 0;                // the context's device (freeing needs no context)
    int ne = 0, nv = 0, leaf = 0;  // ne: rows (elements; linear-element trees: 3 per element)
    // linear-element tree (build_p1_tree): degree of freedom 3 e + a is the shape
    // function of local vertex a of element e; cluster position 3 p + a; blocks
    // are the element tree's with tripled ranges.  Geometry arrays stay per element.
    bool p1 = false;
    int ne_elem = 0;               // elements (p1)
    std::vector<int32_t> perm_elem;  // element of each element cluster position (p1)
    g3::DevBuf d_src;              // int32 [ne]: vertex (row of nodal W and Y) of each position (p1)
    g3::DevBuf d_curl_f, d_curl_d; // surface curls [3][3][E] (p1)
    int max_block = 0;             // cap of the larger side of a far block (0 = none)
    bool subset = false;           // a rank's share of another tree's blocks (g3_tree_subset)
    double eta = 0;
    std::vector<double> verts;
    std::vector<int32_t> tris;
    std::vector<int32_t> perm;     // cluster position -> element
    std::vector<int32_t> nodes;    // [n][4]
    std::vector<double> boxes;     // [n][6]
    std::vector<int32_t> blocks;   // [nb][5]
    std::vector<int32_t> far_index, near_index;
    int max_far_m = 0, max_far_n = 0;
    // device
    g3::DevBuf d_perm;             // int32 [ne]
    g3::DevBuf d_tv;               // int32 [ne][3]: vertex ids of the element at each cluster position
    g3::DevBuf d_geom_f, d_geom_d; // packed SoA arrays
    g3::GeomF gf{};
    g3::GeomD gd{};
};

struct g3_near {
    g3_ctx* ctx = nullptr;
    int device = 0;                // the context's device (freeing needs no context)
    const g3_tree* tree = nullptr;
    int prec = 0, kernel = 0, Ku = 0, K = 0;
    std::vector<int32_t> order;       // near blocks (tree block ids) sorted by (row, col)
    std::vector<long long> offs;      // entry offset (complex elements) of each sorted block
    std::vector<int32_t> row_start;   // [n_rows+1] into `order`, grouped by row cluster
    long long n_entries = 0;
    double ms = 0;
    g3::DevBuf data;                  // complex64 or complex128
    g3::DevBuf d_ranges;              // BlockRange per sorted near block
    g3::DevBuf d_offs;                // long long per sorted near block
    g3::DevBuf d_row_start;
    g3::DevBuf d_diag_base;           // long long [ne]: offset of entry (p, p) at k = 0
    g3::DevBuf d_diag_mn;             // int [ne]: M_b * N_b of the diagonal block of p
    g3::DevBuf d_ss;                  // SsPair [n_ss] (Galerkin)
    int n_ss = 0;
    int scheme = 0;
    const g3_freqs* freqs = nullptr;
    std::vector<int32_t> partner_u;   // unique index -> full index of partner (or -1)
};

struct g3_factors {
    g3_ctx* ctx = nullptr;
    int device = 0;                // the context's device (freeing needs no context)
    const g3_tree* tree = nullptr;
    int prec = 0, kernel = 0, Ku = 0, K = 0, n_far = 0, Cmax = 0;
    int M_sep = 0, N_sep = 0;          // separable mode: one block
    std::shared_ptr<g3::DevBuf> pool = std::make_shared<g3::DevBuf>();  // complex elements; shared by
                                                                          // the meshes of a batch
    long long pool_cap = 0;            // elements
    g3::DevBuf d_rec;                  // CrossRec [n_far][Cmax]
    g3::DevBuf d_r3;                   // int [n_far]
    g3::DevBuf d_cycles;               // long long [n_far][8]
    std::vector<long long> cycles;     // per-block cycle totals
    std::vector<long long> phases;     // [n_far][8]: cycles per phase, then face ACA steps
    std::vector<int32_t> r3;
    std::vector<g3::CrossRec> rec;     // host copy, compact: block b's r3[b] records from rec_off[b]
    std::vector<long long> rec_off;    // [n_far + 1]
    const g3::CrossRec& crec(int b, int p) const { return rec[(size_t)rec_off[b] + p]; }
    std::vector<g3::BlockRange> ranges;
    g3_stats stats{};
    // far-field apply work lists, built when the compression ends and kept
    // on the device with the factors (the apply does no host work for them)
    bool plan_ready = false;
    std::vector<int> plan;             // host copy
    int plan_nd = 0, plan_n1 = 0, plan_n2 = 0;
    int plan_mmax_dense = 0;           // most rows of a dense-face block
    int plan_nmax_dense = 0;           // most columns of a dense-face block
    long long plan_ab = 0;             // complex values of the a/b buffer
    g3::DevBuf d_plan;                 // int [plan.size()]
    g3::DevBuf d_franges;              // BlockRange [n_far]
    const g3_freqs* freqs = nullptr;
};

struct g3_mlp {
    g3_ctx* ctx = nullptr;
    int device = 0;                // the context's device (freeing needs no context)
    g3::DevBuf d_params, d_m, d_v;     // float [G3_MLP_NP]: master weights, Adam moments
    g3::DevBuf d_t;                    // long long: Adam steps taken
    g3::DevBuf d_mean, d_inv_std;      // float [G3_MLP_NF]
    long long t = 0;                   // host copy of the step count
    float mean[G3_MLP_NF] = {}, inv_std[G3_MLP_NF] = {};
};

namespace g3 {

// ---- launchers implemented in the .cu files ----------------------------------
g3_status launch_freqs_bdf2(g3_ctx* ctx, int K, int Ku, double lam, double dt, double* d_sd, float* d_sf);
g3_status launch_freqs_gcq(g3_ctx* ctx, int NQ, double dt_min, double dt_max, double* d_s, double* d_w);
g3_status launch_geometry(g3_ctx* ctx, g3_tree* t);
g3_status far_plan_build(g3_factors* fa);
g3_status launch_entries(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, int kernel, int scheme, int prec,
                         const int* d_rows, const int* d_cols, int n, const int* d_ku, const int* d_conj, int nk,
                         double* d_out);
g3_status launch_near(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_near* nf, int kernel, int scheme);
g3_status mlp_forward_dev(g3_ctx* ctx, const g3_mlp* net, const float* d_x, long long n, float* d_out);
g3_status mlp_features_dev(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, int kernel, double eps3, float* d_out);
g3_status mlp_labels_dev(g3_ctx* ctx, const g3_factors* fa, const BlockRange* d_ranges, float* d_out);
g3_status mlp_grad_dev(g3_ctx* ctx, const g3_mlp* net, const float* d_x, const float* d_y, long long n,
                       float* d_grad, float* d_loss);
g3_status mlp_fit_dev(g3_ctx* ctx, g3_mlp* net, const float* d_x, const float* d_y, long long n, int epochs,
                      int batch, double lr, double b1, double b2, double eps, int use_graph, float* d_loss);
void mlp_init_params(uint64_t seed, float* P);
g3_status run_aca_batch(g3_ctx* ctx, const g3_tree* const* trees, const g3_freqs* const* freqs, int n,
                        g3_factors* const* fas, int kernel, int scheme, double eps3, const g3_opts& o);
g3_status run_aca(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_factors* fa, int kernel, int scheme,
                  double eps3, const g3_opts& o, const void* sep_a, const void* sep_b, const void* sep_c, int sep_R);
g3_status run_apply(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa, const void* W, void* Y,
                    int dtype, int mode);
g3_status gl_table(g3_ctx* ctx);
g3_status run_peak(g3_ctx* ctx, int kind, double* ops_per_s, double* ms);

// host tree builder (bit-exact specification)
g3_status build_tree_host(g3_tree* t);
void tree_index_blocks(g3_tree* t);

}  // namespace g3
