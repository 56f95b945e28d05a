/*
 * g3aca.h -- C ABI of the GB300 three-way ACA library.
 *
 * The library generates and compresses the three-way array
 *     A[i, j, k] = ENTRY(i, j, s_k)
 * of Laplace-domain boundary element entries (single layer V, double layer
 * K) over complex (g)CQ frequencies s_k, block by block with the generalised
 * (three-way) adaptive cross approximation, and applies the compressed
 * factors plus the dense near field to densities at all frequencies.
 *
 * Paper: "Generalised Adaptive Cross Approximation for Convolution
 * Quadrature based Boundary Element Formulation" (Haider, Rjasanow, Schanz,
 * arXiv 2312.11219).  Each entry point names the section, equation or
 * algorithm that defines its operation.
 *
 * Conventions (all entry points):
 *  - Every function returns g3_status; 0 (G3_OK) is success, negative values
 *    are errors.  g3_last_error() returns a message for the calling thread's
 *    most recent error (static storage, valid until the next call on that
 *    thread).  No function exits, aborts or traps.
 *  - Handles (g3_ctx, g3_freqs, g3_tree, g3_near, g3_factors) are opaque,
 *    owned by the library and released with the matching *_free / destroy.
 *    A handle is used on the device and stream of the context it was created
 *    with.  Handles are not thread-safe; distinct handles may be used from
 *    distinct threads.
 *  - Host arrays passed in are copied (or fully consumed) before return;
 *    the caller keeps ownership.  Device pointers passed in (W, Y of
 *    apply_gcq) belong to the caller; the library reads/writes them in
 *    stream order on the context's stream and never frees them.
 *  - Complex numbers are interleaved (re, im) pairs; "c128" = 2 doubles,
 *    "c64" = 2 floats.  Matrices are column-major unless stated otherwise.
 *  - Element indices at the boundary are ORIGINAL element indices (the row of
 *    `tris`), not cluster order, unless stated otherwise.
 *  - Device errors are reported through a device status word that the host
 *    reads after the launch; they surface as G3_ECUDA, G3_ENOCONV or
 *    G3_EOVERFLOW.  No kernel spins on a flag written by another block.
 */
#ifndef G3ACA_H
#define G3ACA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define G3ACA_VERSION 1

typedef enum {
    G3_OK = 0,
    G3_EINVAL = -1,     /* invalid argument (null handle, bad size, bad enum) */
    G3_ENOMEM = -2,     /* host or device allocation failed */
    G3_ECUDA = -3,      /* a CUDA runtime call or a kernel failed */
    G3_ETIMEOUT = -4,   /* reserved: a bounded device wait ran out */
    G3_ENOCONV = -5,    /* a face ACA reached its rank cap before its tolerance */
    G3_EOVERFLOW = -6,  /* the factor pool was too small even after regrowth */
    G3_EUNSUPPORTED = -7 /* combination not implemented (e.g. DLP + Galerkin) */
} g3_status;

/* Integral kernel (paper Section 2: single layer eq. (slp), double layer
 * eq. (dlp); Laplace-domain fundamental solution exp(-s r)/(4 pi r), c = 1). */
typedef enum {
    G3_SLP = 0,          /* V: exp(-s r)/(4 pi r)                                  */
    G3_DLP = 1,          /* K: exp(-s r)(1 + s r)((x - y).n_y)/(4 pi r^3)          */
    G3_SEPARABLE = 2,    /* synthetic sum_t a_t[i] b_t[j] c_t[k] (test tensors)     */
    /* Galerkin with linear continuous elements (eq. (bie_semi_neum), the Neumann
     * problem), on a tree of build_p1_tree and with G3_GALERKIN4x4: rows and
     * columns are element-local shape functions, the nodal matrix is
     * P^T A P (P: element-local function -> its vertex). */
    G3_HYPERSINGULAR = 4, /* D in the integration-by-parts (Maue) form:
                             (curl phi_i . curl phi_j) int int U + s^2 (n_x . n_y) int int U phi_i phi_j */
    G3_ADJOINT_DLP = 5    /* K': int int phi_i(x) dU/dn_x phi_j(y),
                             dU/dn_x = -exp(-s r)(1 + s r)((x - y).n_x)/(4 pi r^3)          */
} g3_kernel;

/* Spatial scheme (paper Section 3, eq. (bie_semi_diri), eq. (bie_semi_indirect)). */
typedef enum {
    G3_COLLOC7 = 0,      /* collocation at centroids, 7-point degree-5 rule        */
    G3_GALERKIN4x4 = 1   /* Galerkin, 4-point x 4-point rule (single layer only)   */
} g3_scheme;

/* Arithmetic of the path. */
typedef enum {
    G3_FP64 = 0,   /* everything in float64; factors and near field complex128       */
    G3_MIXED = 1   /* float32 entries and face arithmetic, float64 singular entries,
                      fiber residuals, norms, recompression and frequencies;
                      factors and near field complex64                                */
} g3_precision;

typedef enum { G3_C64 = 0, G3_C128 = 1 } g3_dtype;
typedef enum { G3_DEVICE = 0, G3_HOST = 1 } g3_memory;
typedef enum {
    G3_APPLY_SUM = 0,     /* y = sum_{l=1}^{K} A(s_l) w_l              (eq. (product)) */
    G3_APPLY_PERFREQ = 1  /* Y[:, l] = A(s_l) w_l for every l: the terms of eq. (product)
                             before the sum over l (a per-frequency check of the
                             compressed operator; not tuned for speed)                 */
} g3_apply_mode;

typedef struct g3_ctx g3_ctx;
typedef struct g3_freqs g3_freqs;
typedef struct g3_tree g3_tree;
typedef struct g3_near g3_near;
typedef struct g3_factors g3_factors;
typedef struct g3_mlp g3_mlp;

/* Block predictor: features per admissible block and parameters. */
#define G3_MLP_NF 12
#define G3_MLP_NP 5122

/* Options of aca3_compress.  Zero-initialise and set what you need;
 * a NULL pointer means all defaults. */
typedef struct {
    int face_rank_max;    /* cap of a face ACA's rank (0 = 48, 64 for G3_HYPERSINGULAR and
                             G3_ADJOINT_DLP; max 64)                                      */
    int unbatched;        /* 1 = one block per launch sequence, host loop (plain baseline) */
    int ctas_per_sm;      /* persistent CTAs per SM (0 = from the occupancy calculator)    */
    int threads;          /* threads per CTA of the low-rank-face launch: 128, 256, 384 or
                             512 (all but 256: G3_MIXED only); 0 = 256                    */
    int no_recompress;    /* 1 = keep raw ACA faces (no QR+SVD)                            */
    int order_by_cost;    /* 1 (default when 0 is given: 1) = longest-first queue order    */
    const int32_t* k1;    /* optional host array [n_far]: first frequency per block
                             (unique-set index); NULL = 0 for every block                 */
    const float* cost;    /* optional host array [n_far]: predicted cost per block used
                             for the queue order instead of M_b * N_b                      */
    double pool_factor;   /* initial factor-pool size multiplier (0 = 1.0)                 */
    double eps_face;      /* face ACA / recompression tolerance (0 = eps3/100; in G3_MIXED
                             not below 1e-5, the relative noise of float32 entries)        */
    int max_blocks;       /* > 0: compress only the first max_blocks admissible blocks (far
                             order); the others get rank 0 (bounded timing samples)         */
    int dense_face_max;   /* blocks with M_b N_b <= this use exact dense faces (no low-rank
                             face, the paper's "No Lwr" variant); 0 = 48*48, < 0 = never    */
    int literal_stop;     /* 1 = stop on Algorithm 1's newest-cross test alone; 0 (default)
                             = confirm each stop on 32 fixed sample entries over all
                             frequencies (keeps the cross and continues when the sampled
                             relative residual exceeds eps3)                               */
    const g3_mlp* mlp;    /* optional block predictor (no counterpart in the paper): its
                             predictions of every block's rank r3 and first frequency set
                             the factor-pool size, the queue order and k1.  Algorithm 1's
                             stopping test still decides every rank.  Ignored (with the
                             plain defaults) when opts->k1 or opts->cost is given for the
                             respective use.                                               */
    int mlp_use;          /* bit mask of the predictor's uses: 1 = queue order, 2 = pool
                             size, 4 = k1 seeding; 0 = all three                          */
    double face_floor_scale;  /* G3_MIXED: the face ACA tests stop at the absolute level
                                 scale * eps_face * ||C^(l-1)||_F / sqrt(Ku) (0 = 1)     */
    double trunc_floor_scale; /* G3_MIXED: the recompression drops singular values below
                                 scale * eps_face * ||C^(l-1)||_F / sqrt(Ku) (0 = 1)     */
    int pivot_index;      /* 1 = pivot of each low-rank face by the estimate of eq. (index)
                             (Section 4, last implementation remark): the row
                             i = argmax_i sum_b |U'[i,b]| ||V'[:,b]|| of the recompressed
                             factors (the paper's sum_k |u_ik sigma_k|), then the largest
                             entry of row i, j = argmax_j |(U' V'^H)[i,j]|; O((M + N) r)
                             instead of the dense expansion's O(M N r).  Single layer
                             only: G3_DLP keeps the dense expansion, the paper's
                             fallback.  0 (default) = dense expansion                   */
    int graph;            /* 1 = the compression's launch sequence (queue resets and both
                             persistent launches) is captured into a CUDA graph on the
                             context's stream and launched as one graph; blocks that spill
                             rerun as plain launches.  The low-rank / dense split of the
                             device time is not available then (ms_lowrank = ms).  Not
                             with unbatched.  The graph is captured and launched on the
                             context's side stream, ordered after and joined back into the
                             context's stream.  0 (default) = plain launches              */
    int whole_matrix;     /* 1 = the three-way ACA of the H-matrix as a whole (Section 4,
                             first implementation remark): all admissible blocks share the
                             frequency sequence and one fiber per cross; a face is every
                             block's residual face (face ACA + recompression), the pivot the
                             largest entry over all blocks, eq. (norm) summed over the blocks
                             and the stopping test taken once for all (rank l - 1, no
                             sampled confirmation); every block keeps the same number of
                             crosses.  Low-rank faces only, one launch per cross; not with
                             unbatched, the batch or the separable test tensor.
                             0 (default) = block by block                                */
    int residual_face_max; /* G3_MIXED, low-rank faces: blocks with M_b N_b <= this evaluate
                             each face's residual ENTRY(i, j, k_l) - sum_p f_p[k_l]
                             (U_p V_p^H)[i, j] for the whole face in one parallel pass into
                             a per-CTA working buffer before the face ACA, which then reads
                             its rows and columns there (same pivots, same stored factors;
                             only the order of float32 sums differs).  No counterpart in
                             the paper (an evaluation order; the sum over the earlier
                             crosses is a dense product, formed on the tensor cores).
                             0 = 192 * 192 (default), < 0 = never (rows and columns
                             evaluated on demand)                                         */
} g3_opts;

/* Statistics of one compression. */
typedef struct {
    int64_t n_far;            /* admissible blocks compressed                             */
    int64_t entries;          /* ENTRY evaluations done (rows, columns, fibers)           */
    int64_t crosses;          /* kept crosses, sum of r3 over blocks                     */
    int64_t crosses_computed; /* crosses computed (incl. the dropped last one per block)  */
    int64_t face_rank_sum;    /* sum of kept face ranks                                   */
    int64_t factor_bytes;     /* bytes of kept factors (U, V, f)                          */
    int64_t dense_bytes;      /* bytes of the same blocks stored densely (Ku freqs)       */
    int32_t r3_max;           /* largest block rank                                       */
    int32_t face_rank_max;    /* largest kept face rank                                   */
    int32_t zero_blocks;      /* blocks detected as zero                                  */
    int32_t capped_faces;     /* faces whose ACA hit face_rank_max                         */
    int32_t pool_regrows;     /* times the factor pool had to be enlarged                 */
    int32_t status_bits;      /* OR of device status flags                                */
    double ms;                /* device time of the compression (CUDA events)             */
    int64_t phase_cycles[7];  /* SM cycles summed over CTAs: face ACA, recompression,
                                 factor formation, pivot search, fiber, eq. (norm), next k  */
    int32_t ctas;             /* persistent CTAs launched                                 */
    int32_t recompress_fallbacks; /* faces kept unrecompressed (Cholesky breakdown)       */
    int32_t blocks_run;       /* blocks compressed (n_far unless opts->max_blocks)        */
    int64_t dense_crosses;    /* kept crosses with a dense face (face_rank_sum excludes them) */
    double ms_lowrank;        /* device time of the low-rank-face launch (last attempt)   */
    double ms_dense;          /* device time of the dense-face launch (last attempt)      */
    int32_t spilled_blocks;   /* blocks rerun from the spill queue after the factor pool
                                 filled up (their work up to the overflow is repeated)     */
    int32_t mlp_used;         /* the predictor's uses applied (mask as opts->mlp_use)      */
    double ms_mlp;            /* device time of the block features + predictor forward     */
    int64_t face_check_restarts;  /* face ACAs continued after a failed sample check       */
    int64_t stop_check_overrides; /* 3D stops overruled by the sampled residual check      */
    int64_t sub_cycles[12];   /* SM cycles of sub-steps (thread 0 of each CTA, diagnostics):
                                 recompression Gram, Cholesky, core, core factorisation,
                                 rest; face ACA table set-up, residual rows, residual
                                 columns, approximant norm, sample checks; of the residual
                                 rows and columns: the entries; dense residual faces      */
    double ms_host[4];        /* host wall time of the call: set-up before the first launch
                                 (predictor, queue, allocations, uploads), the launch rounds
                                 up to the last synchronize, the read-back of records and
                                 statistics, the apply's work lists                       */
    int64_t entries_face_dense; /* ENTRY evaluations into dense residual working faces
                                 (opts->residual_face_max); not part of `entries`, which
                                 counts the rows, columns, samples and fibers Algorithm 1
                                 takes                                                   */
} g3_stats;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (may be NULL for the legacy default stream); the library enqueues all its
 * work on it. */
g3_status g3_create(int device, void* cuda_stream, g3_ctx** out);
g3_status g3_set_stream(g3_ctx* ctx, void* cuda_stream);
/* Where the float32 (complex64) apply forms the far-field vectors
 * x_p = sum_k f_p[k] w_k of eq. (product): on = 1 (default) on the tensor cores
 * (mma.sync m16n8k8 TF32 in a three-term split, float32 accumulation, about
 * float32 accuracy), on = 0 on the CUDA cores (float32 fused multiply-adds).
 * Applies to apply_gcq (SUM) and apply_gcq_noalloc; float64 applies always
 * use the CUDA cores. */
g3_status g3_set_apply_tensor_cores(g3_ctx* ctx, int on);
g3_status g3_destroy(g3_ctx* ctx);
const char* g3_last_error(void);
int g3_version(void);
/* Number of kernel launches the library has issued on this context. */
int64_t g3_launch_count(const g3_ctx* ctx);
/* Name of the kernel that issued the most launches / the i-th kernel name
 * and its launch count (diagnostics; i >= count returns NULL). */
const char* g3_kernel_name(const g3_ctx* ctx, int i, int64_t* launches);

/* ---- frequencies (Appendix A; multistep CQ) ------------------------------ */

/* Multistep-CQ frequencies with the BDF2 generating function,
 *   s_k = delta(zeta_k)/dt, delta(z) = (1 - z) + (1 - z)^2/2,
 *   zeta_k = lambda exp(2 pi i k / K), k = 0..K-1.
 * Unique set: k = 0..K/2 (K even); partner(k) = (K - k) mod K.
 * Computed on the device in float64.  K >= 2 and even, 0 < lambda < 1, dt > 0. */
g3_status g3_freqs_bdf2(g3_ctx* ctx, int K, double lambda, double dt, g3_freqs** out);

/* gCQ contour points and weights (paper Appendix A) for time steps in
 * [dt_min, dt_max], N_Q = NQ points:
 *   q = dt_max/dt_min (implicit-Euler reading), k = (q - sqrt(2q-1))/(q + sqrt(2q-1)),
 *   sigma_l = -K(k^2) + (l - 1/2) 4K(k^2)/NQ + i K(1-k^2)/2,
 *   s_l = gamma(sigma_l), omega_l = -4K(k^2) gamma'(sigma_l) / (2 pi i NQ).
 * Unique set: l = 0..NQ/2-1 (0-based); partner(l) = NQ - 1 - l.
 * Returns G3_EINVAL for dt_max <= dt_min (q = 1 gives k = 0, the degenerate
 * constant-step case the paper warns about) or odd NQ. */
g3_status g3_freqs_gcq(g3_ctx* ctx, int NQ, double dt_min, double dt_max, g3_freqs** out);

/* A frequency set given by the caller (any rule: another CQ generating
 * function, a Runge-Kutta gCQ, a measured set).  s_re_im [2K] holds
 * interleaved (Re s_l, Im s_l), l = 0..K-1, copied on entry; 1 <= K <= 512,
 * every Re s_l > 0 and finite (G3_EINVAL otherwise).  The set keeps the
 * caller's order.  Conjugate pairing (Appendix A: a real operator gives
 * A(conj s) = conj A(s), so half of a conjugate-closed set suffices): for
 * l in increasing order, an unpaired l is unique and is paired with the
 * first unpaired l' > l with |s_l' - conj(s_l)| <= 1e-12 |s_l|; a frequency
 * with |Im s_l| <= 1e-12 |s_l|, or without such a partner, is its own
 * partner.  At most 256 unique frequencies (G3_EINVAL beyond).  omega is
 * zero (g3_freqs_get). */
g3_status g3_freqs_from_array(g3_ctx* ctx, const double* s_re_im, int K, g3_freqs** out);

/* Sizes of a frequency set: K (all) and Ku (unique). */
g3_status g3_freqs_info(const g3_freqs* f, int* K, int* Ku);
/* Copy to host: s [2K] (c128, all K), omega [2K] or NULL (gCQ only; zeros for
 * multistep CQ), uniq [Ku] (full index of each unique frequency) and partner [K]
 * (full index of the conjugate); any output may be NULL. */
g3_status g3_freqs_get(const g3_freqs* f, double* s, double* omega, int32_t* uniq, int32_t* partner);
g3_status g3_freqs_free(g3_freqs* f);

/* ---- cluster tree and block partition (Section 4, eq. (outerProd)) --------- */

/* Build the balanced binary cluster tree and the geometric block partition
 * of a flat-triangle surface mesh, and upload the element geometry to the
 * device in cluster order.
 *   verts [nv*3] float64 (x, y, z per vertex), tris [ne*3] int32 (outward,
 *   counter-clockwise), leaf >= 1 (clusters with more elements are split),
 *   eta > 0 (admissibility min(diam) <= eta * dist, dist > 0).
 * Splitting: longest side of the cluster's vertex box (lowest axis on
 * ties); stable sort by (centroid[axis], element index); left = first half.
 * Admissibility in float64 without fused multiply-adds.  The result is
 * bit-identical on every machine.  Degenerate triangles -> G3_EINVAL. */
g3_status build_cluster_tree(g3_ctx* ctx, const double* verts, int nv, const int32_t* tris, int ne,
                             int leaf, double eta, g3_tree** out);
/* The same with a cap on far blocks (no counterpart in the paper; it bounds
 * the work of the largest block, the tail of the batched compression): an
 * admissible pair whose larger cluster has more than max_block elements is
 * split like an inadmissible pair unless both are leaves (children of an
 * admissible pair are admissible).  max_block = 0: no cap (build_cluster_tree). */
g3_status build_cluster_tree_capped(g3_ctx* ctx, const double* verts, int nv, const int32_t* tris, int ne,
                                    int leaf, double eta, int max_block, g3_tree** out);
/* Sharding of the block partition over ranks by row cluster (no counterpart
 * in the paper, whose code runs OpenMP threads over H-matrix blocks on one
 * node; Section 5.1).  Blocks are independent units of assembly and
 * compression, and the apply adds each block's product into the rows of its
 * row cluster, so ranks that own whole row clusters split the work with
 * disjoint output rows and no exchange on the data path.
 * Host only (no GPU, no context): nodes [n_nodes*4] and blocks [n_blocks*5]
 * as g3_tree_get returns them; cost [n_blocks] per-block work estimates
 * (NULL = M_b N_b); n_ranks >= 1.  Units are the clusters at the smallest
 * depth that holds a block's row cluster (plus the leaves above it); each
 * block belongs to the unit that contains its row cluster.  Units are
 * assigned longest first (cost = the sum of their blocks' costs; ties: lower
 * first element) to the least loaded rank (ties: lower rank).
 * Outputs: owner [n_blocks] rank of each block; load [n_ranks] (may be NULL)
 * summed cost per rank; n_units (may be NULL).  Deterministic: every rank
 * computes the same partition.  Balance needs n_units >= n_ranks (a far-block
 * cap, build_cluster_tree_capped, lowers the depth of the units). */
g3_status g3_shard_rows(const int32_t* nodes, int n_nodes, const int32_t* blocks, int n_blocks, const double* cost,
                        int n_ranks, int32_t* owner, double* load, int* n_units);
/* A tree whose block list is the blocks of t with owner[b] == rank (owner
 * [n_blocks] as from g3_shard_rows), in t's order; the clusters, permutation
 * and device geometry are t's (uploaded again).  assemble_near, aca3_compress
 * and apply_gcq on it handle only those blocks; the apply's y then holds the
 * rank's rows, zero elsewhere, and the ranks' y add up to t's. */
g3_status g3_tree_subset(g3_ctx* ctx, const g3_tree* t, const int32_t* owner, int rank, g3_tree** out);
/* The host half of build_cluster_tree_capped alone, with no context and no
 * device: the same permutation (perm [ne], may be NULL) and block list
 * (blocks [n_blocks*5] as from g3_tree_get, may be NULL; blocks_cap = its
 * capacity in blocks, G3_EINVAL if smaller than the count) for host-side use
 * and checks; n_blocks (may be NULL) gets the count.  Errors as
 * build_cluster_tree. */
g3_status g3_tree_partition_host(const double* verts, int nv, const int32_t* tris, int ne, int leaf, double eta,
                                 int max_block, int32_t* perm, int32_t* blocks, int64_t blocks_cap,
                                 int64_t* n_blocks);
/* Tree of element-local linear shape functions (linear continuous elements,
 * eq. (bie_semi_neum)) over an element tree `elem` of build_cluster_tree (no
 * counterpart beyond the paper's choice of shape functions): row 3 e + a is the
 * shape function of local vertex a (the element's vertex order) of element e;
 * cluster position 3 p + a; the nodes and blocks are those of `elem` with
 * tripled index ranges, so the block partition is the element partition.  The
 * tree owns copies of everything it needs (`elem` may be freed).  Use with
 * G3_HYPERSINGULAR / G3_ADJOINT_DLP and G3_GALERKIN4x4 in assemble_near,
 * aca3_compress (G3_MIXED or G3_FP64, block by block; not batched, whole-matrix
 * or with a predictor) and apply_gcq (G3_APPLY_SUM; W and Y are NODAL, nv rows:
 * the apply gathers w at each shape function's vertex and adds the rows of
 * y into their vertices).  Errors: G3_EINVAL for a NULL argument or a tree that
 * is not an element tree. */
g3_status build_p1_tree(g3_ctx* ctx, const g3_tree* elem, g3_tree** out);
g3_status g3_tree_info(const g3_tree* t, int* ne, int* n_nodes, int* n_blocks, int* n_far, int* n_near);
/* Copy to host (any output may be NULL):
 *   perm [ne]            cluster position -> original element index
 *   nodes [n_nodes*4]    (begin, end, left, right) per preorder node; -1 = no child
 *   boxes [n_nodes*6]    (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z)
 *   blocks [n_blocks*5]  (row_begin, row_end, col_begin, col_end, admissible),
 *                        cluster-order ranges, depth-first order
 *   far_index [n_far]    block index of the i-th admissible block */
g3_status g3_tree_get(const g3_tree* t, int32_t* perm, int32_t* nodes, double* boxes, int32_t* blocks,
                      int32_t* far_index);
g3_status g3_tree_free(g3_tree* t);

/* ---- entries (Section 3, eq. (bie_semi_diri) / (bie_semi_indirect)) ------- */

/* ENTRY(rows[n], cols[n], s_{kidx[m]}) for n pairs and nk frequency indices
 * (indices into the FULL set 0..K-1; frequencies outside the unique set are
 * evaluated as conj of their partner's entry) -> out [n*nk] c128 row-major
 * (pair-major), host memory.  Evaluated by the same device routines the
 * compression uses, in the given precision.  Diagnostic entry point. */
g3_status g3_entries(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, g3_scheme scheme,
                     g3_precision prec, const int32_t* rows, const int32_t* cols, int n, const int32_t* kidx,
                     int nk, double* out);

/* ---- near field ---------------------------------------------------------- */

/* Assemble the dense near field: every entry of every non-admissible block
 * at every unique frequency (self entries in float64).  Storage: complex64
 * (G3_MIXED) or complex128 (G3_FP64), grouped by row cluster.  The paper
 * keeps non-admissible blocks dense (last implementation remark, Section 4). */
g3_status assemble_near(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, g3_scheme scheme,
                        g3_precision prec, g3_near** out);
g3_status g3_near_info(const g3_near* nf, int64_t* n_entries, int64_t* bytes, double* ms);
/* Copy the near field of block `block` (index into the tree's block list; must
 * be non-admissible) to host: out [M_b*N_b*Ku] c128, layout [k][i][j] with i, j
 * local cluster-order indices. */
g3_status g3_near_get_block(const g3_near* nf, int block, double* out);
g3_status g3_near_free(g3_near* nf);

/* ---- compression (Algorithm 1, eq. (norm), Section 4 remarks) -------------- */

/* Compress every admissible block of `t` with the three-way ACA of
 * Algorithm 1 on the unique frequencies of `f`:
 *   face H_l by partial-pivot ACA of the residual face at k_l (tolerance
 *   eps3/100) with QR+SVD recompression; pivot (i_l, j_l) = argmax |H_l| over
 *   the dense expansion of the low-rank face; fiber f_l from the residual
 *   fiber; ||C^(l)||_F by eq. (norm); stop when ||H_l|| ||f_l|| <= eps3 ||C^(l)||
 *   (rank l - 1) or when all unique frequencies are used (rank l);
 *   k_{l+1} = argmax of |f_l| over unused frequencies.
 * All blocks run in one persistent launch unless opts->unbatched.
 * kernel: G3_SLP or G3_DLP on an element tree, G3_HYPERSINGULAR or
 * G3_ADJOINT_DLP (G3_GALERKIN4x4) on a tree of build_p1_tree.  eps3 in (0, 1). */
g3_status aca3_compress(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, g3_scheme scheme,
                        g3_precision prec, double eps3, const g3_opts* opts, g3_factors** out);

/* Autotuner of the compression's launch shape (no counterpart in the paper).
 * Times aca3_compress on (t, f) for each candidate -- threads per CTA of the
 * low-rank launch 128, 256, 384 or 512 (all but 256: G3_MIXED only) and the dense-face
 * threshold M_b N_b <= 24^2, 48^2 or 64^2 -- and writes the fastest into
 * opts->threads and opts->dense_face_max; in G3_MIXED it then times the
 * fastest shape once more without the dense residual working faces and sets
 * opts->residual_face_max to -1 when that is faster (the other fields of
 * *opts are used as given).  The choice is cached in ctx by (K_u bucket, largest far-block
 * bucket, kernel, scheme, precision) and reused without timing.  best_ms
 * (may be NULL): the fastest time, 0 on a cache hit. */
g3_status g3_autotune(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, g3_scheme scheme,
                      g3_precision prec, double eps3, g3_opts* opts, double* best_ms);

/* Algorithm 1 on every admissible block of n_geom meshes in ONE persistent
 * launch (blocks of all meshes share one longest-first queue and one factor
 * pool).  trees[j], freqs[j]: mesh j and its frequency set (K may differ per
 * mesh).  out [n_geom]: one factors handle per mesh, each usable with
 * apply_gcq on trees[j] and freed separately (the pool is freed with the
 * last).  Times and counters in each handle's stats are those of the whole
 * batch; ranks, bytes and per-block data are the mesh's own.  opts->k1,
 * opts->cost and opts->unbatched are not accepted. */
g3_status aca3_compress_batch(g3_ctx* ctx, const g3_tree* const* trees, const g3_freqs* const* freqs, int n_geom,
                              g3_kernel kernel, g3_scheme scheme, g3_precision prec, double eps3, const g3_opts* opts,
                              g3_factors** out);

/* Same algorithm on ONE synthetic block A[i,j,k] = sum_{t<R} a[t,i] b[t,j] c[t,k]
 * (host arrays a [R*M], b [R*N], c [R*Ku], c128, row t contiguous).  Used to
 * check exact recovery of separable tensors. */
g3_status aca3_compress_separable(g3_ctx* ctx, const double* a, const double* b, const double* c, int R, int M,
                                  int N, int Ku, g3_precision prec, double eps3, const g3_opts* opts,
                                  g3_factors** out);

g3_status g3_factors_stats(const g3_factors* fa, g3_stats* out);
/* Per admissible block i (in the tree's far order): r3[i] kept crosses. */
g3_status g3_factors_ranks(const g3_factors* fa, int32_t* r3);
/* Per admissible block i: SM clock cycles its compression took (one CTA;
 * diagnostics and cost labels for scheduling). */
g3_status g3_factors_block_cycles(const g3_factors* fa, int64_t* cycles);
/* Per admissible block i: out[10 i + q] = SM cycles of phase q (0 face ACA,
 * 1 recompression, 2 factor formation, 3 pivot search, 4 fiber, 5 eq. (norm),
 * 6 next frequency), out[10 i + 7] = face ACA steps (face ranks before
 * recompression, summed over the block's faces), out[10 i + 8] and
 * out[10 i + 9] = start and end of the block's (last) compression on the GPU's
 * global timer (ns).  Diagnostics. */
g3_status g3_factors_block_phases(const g3_factors* fa, int64_t* out);
/* Export block i's crosses to host.  Sizes first: call with U = V = fib = NULL
 * to get r3 and the face ranks in face_ranks [r3] (if non-NULL; a dense face
 * is exported as U = H (M_b x N_b), V = identity (N_b x N_b), rank N_b).  Then:
 *   U [sum_p M_b r_p] c128, column-major per cross, crosses concatenated;
 *   V [sum_p N_b r_p] c128, likewise (face_p = U_p V_p^H);
 *   fib [r3 * Ku] c128; piv [r3*3] int32 (i_l, j_l, k_l) local indices. */
g3_status g3_factors_get_block(const g3_factors* fa, int i, int32_t* r3, int32_t* face_ranks, double* U, double* V,
                               double* fib, int32_t* piv);
g3_status g3_factors_free(g3_factors* fa);

/* ---- block predictor (no counterpart in the paper) -------------------------- */

/* Algorithm 1 starts each block at an arbitrary frequency and learns the
 * block's rank only as it goes.  A small network, trained on earlier
 * compressions, predicts both before a compression starts, so that the factor
 * pool is sized, the queue ordered longest first and k1 chosen up front:
 *
 *   x (G3_MLP_NF = 12 features) -> 64 ReLU -> 64 ReLU -> 2 outputs
 *   y0 = log2(1 + r3),  y1 = k* / Ku  (k* = argmax_k |f_1[k]|, the frequency of
 *                                      the block's largest pivot entry)
 *
 * Parameters (G3_MLP_NP = 5,122 float32, row-major, output index first):
 *   W1 [64][12], b1 [64], W2 [64][64], b2 [64], W3 [2][64], b3 [2].
 * Inputs are standardised as (x - mean) * inv_std in float32 and rounded to
 * bfloat16; weights are used rounded to bfloat16 (float32 master copy);
 * activations, sums, gradients and Adam are float32.
 *
 * Features of an admissible block (tau, sigma), from the vertex bounding boxes
 * (diam = box diagonal, dist = box distance), the area-weighted normal sums
 * nA = sum a_i n_i and area-weighted centroids c, and the unique frequencies:
 *   0 log2 M_b      1 log2 N_b     2 log2(diam_tau / dist)  3 log2(diam_sigma / dist)
 *   4 log2(dist max|s|)            5 log2(dist min Re s)
 *   6 log2(1 + max(diam) max|Im s| / (2 pi))                 7 log2 Ku
 *   8 -log10 eps3   9 kernel (0 SLP, 1 DLP)
 *   10 |nA_tau . nA_sigma| / (A_tau A_sigma)
 *   11 |(c_sigma - c_tau) . nA_tau| / (|nA_tau| |c_sigma - c_tau|)  (0: coplanar) */
typedef struct {
    int epochs;           /* passes over the samples (0 = 200)                           */
    int batch;            /* minibatch size (0 = 256); batches are consecutive slices    */
    double lr;            /* Adam step size (0 = 1e-3)                                   */
    double beta1, beta2;  /* Adam decay rates (0 = 0.9, 0.999)                           */
    double adam_eps;      /* Adam epsilon (0 = 1e-8)                                     */
    uint64_t seed;        /* He-uniform initial weights from splitmix64 (g3_mlp_train)   */
    int no_graph;         /* 1 = launch each step; 0 = replay one CUDA graph per epoch   */
} g3_train_opts;

/* New model.  params [G3_MLP_NP] (NULL = He-uniform from seed), mean and
 * inv_std [G3_MLP_NF] (NULL = 0 and 1).  Host arrays, copied. */
g3_status g3_mlp_create(g3_ctx* ctx, const float* params, const float* mean, const float* inv_std, uint64_t seed,
                        g3_mlp** out);
/* New model trained on n samples: feats [n*12], labels [n*2] (host, row-major).
 * mean / inv_std come from the samples (inv_std = 1 for a constant feature). */
g3_status g3_mlp_train(g3_ctx* ctx, const float* feats, const float* labels, int n, const g3_train_opts* opts,
                       g3_mlp** out);
/* Further Adam epochs on an existing model (its Adam state continues).
 * losses: optional host [epochs * ceil(n / batch)], the loss of every step. */
g3_status g3_mlp_fit(g3_ctx* ctx, g3_mlp* m, const float* feats, const float* labels, int n,
                     const g3_train_opts* opts, float* losses);
/* Loss 0.5/n sum |y - t|^2 and its gradient [G3_MLP_NP] at the model's
 * current weights over n samples (host arrays). */
g3_status g3_mlp_grad(g3_ctx* ctx, const g3_mlp* m, const float* feats, const float* labels, int n, float* grad,
                      float* loss);
/* Outputs out [n*2] for feats [n*12] (host arrays). */
g3_status g3_mlp_predict(g3_ctx* ctx, const g3_mlp* m, const float* feats, int n, float* out);
/* Copy out the state (any pointer may be NULL): params, Adam moments m and v
 * [G3_MLP_NP], Adam step count t, mean and inv_std [G3_MLP_NF]. */
g3_status g3_mlp_get(const g3_mlp* m, float* params, float* adam_m, float* adam_v, int64_t* t, float* mean,
                     float* inv_std);
g3_status g3_mlp_free(g3_mlp* m);
/* Features [n_far*12] of the admissible blocks of t (far order), computed on
 * the device. */
g3_status g3_block_features(g3_ctx* ctx, const g3_tree* t, const g3_freqs* f, g3_kernel kernel, double eps3,
                            float* out);
/* Training labels [n_far*2] (y0, y1 above) of a compression, computed on the
 * device from its ranks and first fibers. */
g3_status g3_factors_labels(g3_ctx* ctx, const g3_factors* fa, float* out);

/* ---- application (eq. (product)) ------------------------------------------ */

/* y = sum_{l=1}^{K} A(s_l) w_l with the compressed far field and the dense
 * near field (near may be NULL: far field only; fa may be NULL: near only).
 *   W [M*K] complex (dtype), column l = w_l, ORIGINAL element order;
 *   Y [M] (SUM) or [M*K] (PERFREQ), complex (dtype), overwritten.
 * mem = G3_DEVICE: W, Y are device pointers (caller-owned).
 * mem = G3_HOST:   W, Y are host pointers; the library copies W in and Y out
 *                  on the context's stream and synchronises before return.
 * Frequencies outside the unique set use A(conj s) = conj A(s).
 * G3_APPLY_SUM: with both parts present the near-field kernel runs on a
 * second, high-priority stream owned by the context (forked from and joined
 * back into the context's stream, next to the far-field kernels on the
 * context's stream), so work the caller orders after this call on the
 * context's stream sees y complete.  G3_APPLY_PERFREQ runs on the context's stream only; its
 * scratch holds 4 Ku M complex values (context-owned, grown on demand), and
 * face ranks above 64 return G3_EUNSUPPORTED.  The call synchronises the
 * context's stream before it returns (the device time is recorded for
 * g3_apply_last). */
g3_status apply_gcq(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa, const void* W, void* Y,
                    g3_dtype dtype, g3_apply_mode mode, g3_memory mem);
/* Allocation-free variant of apply_gcq (no counterpart in the paper).  For
 * callers that cannot allocate device memory while this step runs (a
 * memory-capped or pre-reserved arena, a runtime that forbids cudaMalloc or
 * the device synchronisation it may cause on its hot path).  Computes the same
 * y = sum_l A(s_l) w_l as apply_gcq with mem = G3_DEVICE and G3_APPLY_SUM:
 * W [M*K] and Y [M] are caller-owned device buffers (layout as apply_gcq).
 * Its scratch is a fixed 32 MiB device array inside the library (held by
 * every GPU that loads the library until the process exits); no
 * cudaMalloc/cudaFree or other allocating routine is called.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the process; under lazy module loading (the CUDA
 * default) that lookup also loads the module and so reserves the 32 MiB
 * then.  Make that first call before any stream capture, and do not call
 * after cudaDeviceReset (the kept address would be stale).  Problems needing more
 * scratch than 32 MiB (2 Ku M + M complex values, each part rounded up to
 * 256 bytes) return G3_EINVAL.  All calls
 * share the array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  Element trees
 * only (a tree of build_p1_tree returns G3_EUNSUPPORTED). */
g3_status apply_gcq_noalloc(g3_ctx* ctx, const g3_tree* t, const g3_near* nf, const g3_factors* fa, const void* W,
                            void* Y, g3_dtype dtype);
/* The gCQ time-stepping consumer of the apply (eq. (gCQ_xn) and the weight
 * vectors of eq. (gcq_formula)), implicit-Euler reading (one stage,
 * A = b = 1).  For every frequency l of f (all K) and element i < M:
 *   X[:, l] <- (X[:, l] + dt_prev theta) / (1 - dt_prev s_l)   (x_{n-1} from x_{n-2})
 *   W[:, l]  = -omega_l X[:, l] / (1 - dt_next s_l)             (weights for apply_gcq)
 * where dt_prev = dt_{n-1} (the step of theta = theta_{n-1}) and dt_next =
 * dt_n.  The sign: the contour integral of eq. (conv_discrete) runs so that
 * the pole of (1 - dt_n s)^{-1} gives +V((dt_n A)^{-1}); omega_l
 * (g3_freqs_gcq) is normalised the other way round.  apply_gcq(W) then
 * returns the history sum of eq. (gcq_formula).  X, W [M*K] complex (dtype)
 * column-major device buffers (column l = frequency l, caller's element
 * order), X updated in place (start from zeros: x_0 = 0); theta [M] complex
 * device buffer, or NULL for zero.  f must carry contour weights (a gCQ set;
 * G3_EINVAL otherwise).  Runs on the context's stream, no synchronisation. */
g3_status g3_gcq_history(g3_ctx* ctx, const g3_freqs* f, int M, void* X, const void* theta, double dt_prev,
                         double dt_next, void* W, g3_dtype dtype);
/* Device time (ms) of the last apply on this context and its algorithmic
 * bytes (near field, factors, W read once, Y written once). */
g3_status g3_apply_last(const g3_ctx* ctx, double* ms, int64_t* bytes, double* near_ms, int64_t* near_bytes);

/* ---- diagnostics -------------------------------------------------------------- */

/* Throughput of one arithmetic pipe on the context's GPU (no counterpart in
 * the paper; it measures the denominators of the compression's ALU roofline):
 * kind 0 = float32 FMA, 1 = rsqrt.approx, 2 = ex2.approx, 3 = sin.approx,
 * 4 = cos.approx (special-function unit), 5 = float64 FMA.  Writes
 * operations per second (one FMA = one operation) and the timed ms. */
g3_status g3_peak(g3_ctx* ctx, int kind, double* ops_per_s, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* G3ACA_H */
