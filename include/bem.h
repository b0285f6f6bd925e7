/*
 * bem.h -- C ABI of the GB300 Galerkin boundary-element quadrature library.
 *
 * The library computes entries of Galerkin boundary-element matrices
 * (Section 2.1, Eq. 1)
 *
 *     g_ij = int_Gamma phi_i(x) int_Gamma k(x, y) psi_j(y) dy dx
 *
 * on flat-triangle surface meshes, as sums over triangle pairs of integrals on
 * the reference triangle D = {(s,t): 0 <= t <= s <= 1} (Section 2.2), with
 *   - kernels (Eq. 2, Section 4): Laplace single layer 1/(4 pi |x-y|),
 *     Laplace double layer (x-y).n_y / (4 pi |x-y|^3) (outward n_y),
 *     Helmholtz single layer exp(i kappa |x-y|) / (4 pi |x-y|);
 *   - bases: piecewise constant (index = triangle) or continuous piecewise
 *     linear (index = vertex), the same space for test and trial functions;
 *   - quadrature (Section 2.2): tensor Gauss-Legendre after the Duffy map for
 *     disjoint triangles (or the 7-point Radon rule on each triangle), and
 *     Sauter-Schwab subdomain rules for identical, common-edge and
 *     common-vertex pairs.  "Touching" means sharing a vertex index.
 *
 * Conventions for every call:
 *   - Every call returns an int status: BEM_OK (0) or a negative BEM_ERR_*.
 *     bem_last_error() returns a message for the last failure on a context.
 *   - Bulk data pointers (index lists, outputs) are DEVICE pointers owned by
 *     the caller, except bem_mesh_upload, which takes HOST arrays and keeps
 *     its own device copy until bem_mesh_free / bem_destroy.
 *   - Index arrays are int32 and 0-based.  Output matrices are column-major.
 *     Real kernels write double; the Helmholtz kernel writes interleaved
 *     complex (re, im) double pairs (16 bytes per entry, 16-byte aligned).
 *     The mixed-precision mode still writes double.
 *   - Compute calls are asynchronous on the context's CUDA stream.  Errors
 *     detected on the device (an index out of range, a touching pair inside a
 *     block that must be disjoint) are recorded in a device status word that
 *     bem_sync() returns; the entries concerned are left unwritten.
 *   - A context serves one thread at a time.
 */
#ifndef BEM_GB300_H
#define BEM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define BEM_OK               0
#define BEM_ERR_INVALID_ARG (-1)  /* bad argument or index (host or device check) */
#define BEM_ERR_CUDA        (-2)  /* a CUDA runtime call failed                  */
#define BEM_ERR_OOM         (-3)  /* device allocation failed                    */
#define BEM_ERR_TIMEOUT     (-4)  /* a bounded device wait gave up               */
#define BEM_ERR_DEGENERATE  (-5)  /* zero-area triangle / repeated vertex        */
#define BEM_ERR_UNSUPPORTED (-6)  /* option combination not implemented          */

/* ---- enumerations -------------------------------------------------------- */
enum { BEM_LAPLACE_SLP = 0, BEM_LAPLACE_DLP = 1, BEM_HELMHOLTZ_SLP = 2, BEM_HELMHOLTZ_DLP = 3,
       BEM_HELMHOLTZ_BW = 4 };
enum { BEM_P0 = 0, BEM_P1 = 1 };
enum { BEM_RULE_DUFFY = 0, BEM_RULE_TRI7 = 1 };
enum { BEM_FP64 = 0, BEM_MIXED = 1, BEM_MIXED_FULL = 2 };
enum { BEM_ORDER_FIXED = 0, BEM_ORDER_LEARNED = 1 };

typedef struct bem_ctx bem_ctx;

/* Kernel function (Eq. 2 and Section 4), k(x, y) with r = |x - y|:
 *   BEM_LAPLACE_SLP    1 / (4 pi r)
 *   BEM_LAPLACE_DLP    (x - y).n_y / (4 pi r^3)
 *   BEM_HELMHOLTZ_SLP  exp(i kappa r) / (4 pi r)
 *   BEM_HELMHOLTZ_DLP  d/dn_y exp(i kappa r)/(4 pi r)
 *                      = (x - y).n_y (1 - i kappa r) exp(i kappa r) / (4 pi r^3)
 *   BEM_HELMHOLTZ_BW   the Brakhage-Werner combination of Section 4, the
 *                      double layer minus i eta times the single layer.
 * kappa: wave number (Helmholtz kinds); eta: coupling parameter of
 * BEM_HELMHOLTZ_BW (ignored by the others).  The Helmholtz kinds give complex
 * entries ((re, im) double pairs, 16-byte aligned outputs).
 * BEM_HELMHOLTZ_DLP and BEM_HELMHOLTZ_BW run in FP64 in every precision (the
 * float forms cover the first three kinds), take fixed orders only, and are not
 * kernels of the Green matrices (bem_green_matrices) or of the allocation-free
 * call. */
typedef struct {
    int32_t kind;
    double kappa;
    double eta;
} bem_kernel_desc;

/* Quadrature orders (Section 2.2 and the "higher quadrature orders" study of
 * Section 4): q_* = Gauss-Legendre points per axis of [0,1]^4.  The paper's
 * default is 3 for disjoint pairs and 5 for the singular cases.
 *   regular_rule: BEM_RULE_DUFFY (q_regular^4 points) or BEM_RULE_TRI7
 *                 (7 x 7 = 49 points, q_regular ignored).
 *   precision:    BEM_FP64, or BEM_MIXED: disjoint and common-vertex pairs in
 *                 FP32 arithmetic (double-float set-up of vertex differences,
 *                 double-layer heights and the Helmholtz reference phase
 *                 kappa |c_a - c_b| of the centroids, compensated sums);
 *                 identical and common-edge pairs stay FP64, and so do the
 *                 disjoint Helmholtz pairs of the piecewise-linear basis and
 *                 bem_pivot_entries.
 *                 BEM_MIXED_FULL: as BEM_MIXED, and identical and common-edge
 *                 pairs in FP32 too (x - y from the rule's difference columns
 *                 and float edge vectors, double-layer numerators from
 *                 double-float plane heights, Kahan-compensated sums).
 *   order_mode:   BEM_ORDER_FIXED (the orders above) or BEM_ORDER_LEARNED: for
 *                 bem_near_field and bem_coupling_blocks on piecewise-constant
 *                 meshes, every disjoint pair gets the rule class the context's
 *                 order model (bem_set_order_model) predicts; touching pairs
 *                 keep the fixed singular orders above.  Such a call reads one value
 *                 back from the device to size its scratch (it synchronises). */
typedef struct {
    int32_t q_regular;
    int32_t regular_rule;
    int32_t q_identical;
    int32_t q_edge;
    int32_t q_vertex;
    int32_t precision;
    int32_t order_mode;
} bem_quad_desc;

/* A list of matrix blocks G|_{t x s} of one mesh (Section 2.3: blocks of the
 * block tree; near-field blocks t x s, coupling blocks t~ x s~).
 *   Row clusters: cluster c holds indices row_idx[row_ptr[c] .. row_ptr[c+1]).
 *   Column clusters: likewise with col_ptr / col_idx.
 *   Block b is G restricted to (row cluster blk_row[b]) x (column cluster
 *   blk_col[b]) and is written column-major (leading dimension = number of
 *   rows of the block) at element offset blk_off[b] of `out`.
 * All arrays are device arrays.  Blocks must not overlap in `out`. */
typedef struct {
    int32_t mesh_id;
    bem_kernel_desc kernel;
    bem_quad_desc quad;
    const int32_t *row_ptr;      /* n_row_clusters + 1 */
    const int32_t *row_idx;
    int32_t n_row_clusters;
    const int32_t *col_ptr;      /* n_col_clusters + 1 */
    const int32_t *col_idx;
    int32_t n_col_clusters;
    const int32_t *blk_row;      /* n_blocks */
    const int32_t *blk_col;      /* n_blocks */
    const int64_t *blk_off;      /* n_blocks */
    int64_t n_blocks;
    void *out;                   /* double or (re,im) double pairs */
} bem_block_job;

/* Counters of an uploaded mesh (filled by bem_mesh_info). */
typedef struct {
    int64_t n_vertices;
    int64_t n_triangles;
    int64_t n_identical;    /* ordered touching pairs per case */
    int64_t n_edge;
    int64_t n_vertex;
    int32_t max_vertex_degree;
    int32_t basis;
} bem_mesh_stats;

/* ---- context --------------------------------------------------------------
 * bem_create: context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream is not
 * owned.  bem_destroy frees everything the context allocated (meshes,
 * rules, scratch) after synchronising its stream. */
int bem_create(bem_ctx **ctx, int device, void *cuda_stream);
int bem_destroy(bem_ctx *ctx);
/* Message of the last failure on this context ("" if none).  Owned by ctx. */
const char *bem_last_error(bem_ctx *ctx);
/* Waits for all work on the context's stream; returns the first error
 * recorded by a kernel since the previous bem_sync (and clears it), a CUDA
 * error, or BEM_OK. */
int bem_sync(bem_ctx *ctx);

/* ---- mesh (a1: per-triangle precompute; a2: touching-pair classification) --
 * Copies a flat-triangle mesh to the device and precomputes per triangle the
 * vertices, the edge vectors of the affine map Phi(s,t) = v0 + s (v1 - v0) +
 * t (v2 - v1) (Section 2.2), the Gram factor sqrt(g) = |(v1-v0) x (v2-v1)|
 * and the unit normal (v1-v0) x (v2-v1) / sqrt(g) (outward for outward-
 * oriented meshes: the double layer uses it).  It also classifies every pair
 * of triangles that share a vertex index into identical / common edge /
 * common vertex (Section 2.2) with the vertex orders the Sauter-Schwab maps
 * expect, and builds the vertex-to-triangle adjacency the piecewise-linear
 * basis needs.
 *   verts: HOST double[nv][3];  tris: HOST int32[nt][3].
 *   basis: BEM_P0 or BEM_P1 (index space of every call on this mesh).
 * Errors: BEM_ERR_INVALID_ARG (vertex index out of range, nv or nt < 1),
 * BEM_ERR_DEGENERATE (zero-area triangle, repeated vertex in a triangle),
 * BEM_ERR_OOM. */
int bem_mesh_upload(bem_ctx *ctx, const double *verts, int64_t nv, const int32_t *tris,
                    int64_t nt, int32_t basis, int32_t *mesh_id);
int bem_mesh_free(bem_ctx *ctx, int32_t mesh_id);
int bem_mesh_info(bem_ctx *ctx, int32_t mesh_id, bem_mesh_stats *stats);

/* ---- matrix entries ------------------------------------------------------- */

/* Near-field blocks (Section 2.3: inadmissible leaves of the block tree), the
 * paper's per-case work lists (Section 3) formed on the device: every triangle
 * pair of every block is classified by its shared vertex indices; disjoint
 * pairs use the regular rule, touching pairs the Sauter-Schwab rules.
 * n_jobs jobs (any meshes, kernels and orders) run in one call. */
int bem_near_field(bem_ctx *ctx, const bem_block_job *jobs, int32_t n_jobs);

/* Coupling blocks G|_{t~ x s~} of admissible blocks (Section 2.4): the same
 * block layout as bem_near_field, with the pivot sets t~, s~ as clusters.
 * Admissible blocks contain only disjoint pairs; a touching pair found in a
 * coupling block is a caller error, recorded as BEM_ERR_INVALID_ARG in the
 * device status word, and that block is left unwritten. */
int bem_coupling_blocks(bem_ctx *ctx, const bem_block_job *jobs, int32_t n_jobs);

/* Arbitrary entries (pivot rows / columns, Section 2.3-2.4):
 * out[k] = g_{rows[k], cols[k]} for k < n.  rows, cols, out: device arrays.
 * Here the regular rule may be any Duffy order 1..20 (the block calls take
 * Duffy 2..4 or TRI7). */
int bem_pivot_entries(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                      const bem_quad_desc *quad, const int32_t *rows, const int32_t *cols,
                      int64_t n, void *out);

/* Full dense matrix, n x n column-major (n = triangles for P0, vertices for
 * P1).  lower_only != 0 writes only entries with row >= column (the single
 * layer is symmetric, Section 4); the rest of `out` is not touched. */
int bem_assemble_dense(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                       const bem_quad_desc *quad, int32_t lower_only, void *out);

/* Sum of the magnitudes of the quadrature terms of each requested entry,
 * A_k = sum over pairs sqrt(g_a g_b)/(4 pi) sum_p |w_p phi psi k|, with the
 * same rules as bem_pivot_entries (real double output for every kernel).
 * A_k bounds the rounding error of any floating-point evaluation of the
 * entry's sum (up to a multiple of the unit roundoff); it is the error scale
 * used to label rule classes for the order model. */
int bem_pivot_entries_absolute(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                               const bem_quad_desc *quad, const int32_t *rows, const int32_t *cols,
                               int64_t n, double *out);

/* ---- learned quadrature orders ----------------------------------------------
 * The paper fixes one rule per case (Section 2.2; Section 4 compares fixed
 * orders 3/5 and 4/6).  The order model is a small multilayer perceptron,
 * 8 pair features -> 64 -> 64 -> 6 classes (ReLU), that predicts, for a
 * disjoint pair, the cheapest of six rules meeting an error target, on a
 * ladder of increasing accuracy and cost:
 *   class 0: Duffy q=2 (16 points)  1: Radon 7x7 (49)   2: Duffy q=4 (256)
 *   class 3: Duffy q=5 (625)        4: Duffy q=6 (1296) 5: Duffy q=8 (4096).
 * Features (bem_pair_features, normalised by the model's mean / std):
 * log2 centroid distance / D, log2 closest-vertex distance / D, cos of the
 * normals' angle, log2 area ratio, test centroid height above the trial
 * plane / distance, kernel id / 2, kappa D, log2 aspect ratio; D = larger
 * triangle diameter.  Training runs on the device (FP32 forward, backward
 * and Adam, deterministic); inference uses BF16 weights on the tensor cores.
 * Parameters: W1[64][8] b1[64] W2[64][64] b2[64] W3[6][64] b3[6] (floats);
 * normalisation: mean[8] then 1/std[8]. All X / y / grads / logits pointers
 * are device arrays (X: n x 8 floats row-major, y: n int32 classes). */
typedef struct bem_mlp bem_mlp;
int bem_mlp_create(bem_ctx *ctx, uint64_t seed, bem_mlp **mlp);
int bem_mlp_destroy(bem_ctx *ctx, bem_mlp *mlp);
int bem_mlp_num_params(void);
int bem_mlp_set_params(bem_ctx *ctx, bem_mlp *mlp, const float *host_params, const float *host_norm);
int bem_mlp_get_params(bem_ctx *ctx, bem_mlp *mlp, float *host_params, float *host_norm);
/* gradients of the mean cross-entropy over the n rows (grads: device, num_params floats) */
int bem_mlp_gradients(bem_ctx *ctx, bem_mlp *mlp, const float *X, const int32_t *y, int32_t n,
                      float *grads, float *loss);
/* one Adam step (beta 0.9 / 0.999) on the n rows; loss = mean loss before the step */
int bem_mlp_train_step(bem_ctx *ctx, bem_mlp *mlp, const float *X, const int32_t *y, int32_t n,
                       float lr, float *loss);
/* Normalisation from raw features: the mean and population standard
 * deviation of each of the 8 columns of X (device, n x 8 raw features), in
 * FP64 with a fixed reduction order; stored as the model's mean and 1/std
 * (a standard deviation below 1e-6 counts as 1). */
int bem_mlp_fit_norm(bem_ctx *ctx, bem_mlp *mlp, const float *X, int64_t n);
/* One epoch of training on RAW features: for every minibatch of `batch` rows
 * of the permutation perm (device int64[n], row indices of X and y), the rows
 * are gathered and normalised with the model's mean / std, then one Adam step
 * as bem_mlp_train_step.  mean_loss (may be NULL) = the per-row mean of the
 * minibatch losses, each taken before its step; waits for the stream once. */
int bem_mlp_train_epoch(bem_ctx *ctx, bem_mlp *mlp, const float *X, const int32_t *y, int64_t n,
                        const int64_t *perm, int32_t batch, float lr, float *mean_loss);
/* Training labels from the method itself, for disjoint pairs (a[k], b[k]) of a
 * piecewise-constant mesh (device int32 arrays): the pair is integrated with
 * the six classes' rules and with Duffy q_ref (FP64, bem_pivot_entries), and
 * err_c = |g_c - g_ref| / A_ref (A_ref: the sum of the magnitudes of the
 * reference's terms, the forward-error scale); labels[k] (device int32) = the
 * cheapest class with err_c <= tol, else class 5.  errors (device n x 6
 * floats, may be NULL) receives err_c.  Waits for the stream. */
int bem_order_labels(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                     const int32_t *a, const int32_t *b, int64_t n, float tol, int32_t q_ref,
                     int32_t *labels, float *errors);
/* logits (n x 6, device) of the BF16 tensor-core inference */
int bem_mlp_infer(bem_ctx *ctx, bem_mlp *mlp, const float *X, int64_t n, float *logits);
/* features of pairs (a[k], b[k]) of a piecewise-constant mesh (normalised by the
 * model when mlp != NULL, raw otherwise) */
int bem_pair_features(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel, bem_mlp *mlp,
                      const int32_t *a, const int32_t *b, int64_t n, float *X);
/* model used by BEM_ORDER_LEARNED calls (NULL to clear); every disjoint pair
 * gets the cheapest class whose cumulative predicted probability (classes 0..c)
 * reaches `confidence`, so an uncertain prediction moves up the ladder (the
 * most accurate class is the fallback).  The model must outlive the calls. */
int bem_set_order_model(bem_ctx *ctx, bem_mlp *mlp, float confidence);
/* number of disjoint pairs per class of the last BEM_ORDER_LEARNED job */
int bem_learned_counts(bem_ctx *ctx, int64_t *counts /* [6] */);

/* ---- persistent batched driver ---------------------------------------------
 * A plan replaces the paper's CPU-side list machinery (Section 3, Algorithms
 * 1-4: per-case lists, list-size limit, worker threads, result scatter) for a
 * fixed set of jobs: the near-field jobs (as bem_near_field) and coupling
 * jobs (as bem_coupling_blocks) of any meshes and kernels.  Jobs that share
 * a kernel instantiation (basis, kernel, regular rule and order, precision)
 * form one bucket, and each bucket is drained by ONE persistent launch over
 * the tiles of all its jobs; touching pairs are likewise batched per (case,
 * order).  Each near-field job gets its own touching table inside the plan.
 *   flags: BEM_PLAN_GRAPH     capture the whole launch sequence into a CUDA
 *                             graph at creation; bem_plan_run replays it;
 *          BEM_PLAN_AUTOTUNE  time candidate grid sizes per bucket on the
 *                             plan's data at creation and keep the fastest
 *                             (cached in the context);
 *          BEM_PLAN_PROFILE   record launch-profiling events in the plan
 *                             (read with bem_profile_read while profiling is
 *                             enabled);
 *          BEM_PLAN_STATIC_LISTS  the index lists' contents (cluster lists,
 *                             block lists) stay as they are at creation: the
 *                             passes derived from them alone (tile prefix sums,
 *                             piecewise-linear support records, a learned
 *                             job's prefix sums) run once at creation and the
 *                             runs issue only the quadrature and guard passes.
 *                             Changing the lists afterwards gives wrong entries
 *                             (the kernels still check every index).
 * The plan keeps the jobs' device pointers (index lists, outputs) and uses
 * the meshes' device data: both must stay valid until bem_plan_destroy; the
 * index lists' contents are read at every run (unless BEM_PLAN_STATIC_LISTS).
 * bem_plan_create runs the plan's kernels once (or several times when
 * autotuning), so outputs are written at creation too.  Results are the
 * same, bit for bit, as those of bem_near_field / bem_coupling_blocks.
 * Piecewise-linear near-field jobs read support records (the triangles
 * around each 32-index slice of a cluster), built once per run for every
 * distinct cluster list; their storage is sized from the lists' total length
 * at creation (one device read), and a later run whose lists need more
 * records reports BEM_ERR_INVALID_ARG through the status word.
 * A job with order_mode BEM_ORDER_LEARNED (piecewise-constant basis only,
 * else BEM_ERR_UNSUPPORTED) runs the learned path of bem_near_field inside the
 * plan (tile prefix sums, selection by the order model, compaction by class,
 * one evaluation per class), with the order model and confidence set by
 * bem_set_order_model at plan creation (BEM_ERR_INVALID_ARG if none): the
 * model must stay alive until bem_plan_destroy.  Its scratch is sized from
 * the job's tile count at creation; its results equal bem_near_field's.
 * The cancellation guard below covers fixed-order jobs only.
 * In the float forms a piecewise-linear Laplace single-layer job and a
 * double-layer job of the same kind (both near field or both coupling) with
 * the same mesh, the same block-list pointers and the same regular rule,
 * order and precision run fused: one launch evaluates both layers and shares
 * the points, distances and reciprocal square roots (Eq. 1 for both kernels
 * over the same pairs); the results are unchanged.  The outputs of a plan's
 * jobs must not overlap.
 * Errors as bem_near_field; BEM_ERR_CUDA if graph capture fails. */
typedef struct bem_plan bem_plan;
#define BEM_PLAN_GRAPH    1
#define BEM_PLAN_AUTOTUNE 2
#define BEM_PLAN_PROFILE  4
#define BEM_PLAN_STATIC_LISTS 8
int bem_plan_create(bem_ctx *ctx, const bem_block_job *near_jobs, int32_t n_near,
                    const bem_block_job *coupling_jobs, int32_t n_coupling, int32_t flags,
                    bem_plan **plan);
int bem_plan_run(bem_ctx *ctx, bem_plan *plan);
int bem_plan_destroy(bem_ctx *ctx, bem_plan *plan);
/* Kernel launches of one plan run: touching buckets, block buckets, and the
 * auxiliary launches (per block bucket its tile prefix sums, per distinct
 * piecewise-linear cluster list its support records, per guard set its three
 * or four passes, per learned job its prefix sums (one launch, two above 8192
 * blocks), selection, three scan passes, offsets, compaction and six class
 * evaluations; BEM_PLAN_STATIC_LISTS leaves out the list-derived passes); the
 * chosen CTAs per SM of up to `cap` block buckets.  Any pointer may be NULL. */
int bem_plan_info(bem_ctx *ctx, bem_plan *plan, int32_t *n_touch_launches,
                  int32_t *n_block_launches, int32_t *n_aux_launches, int32_t *grid_mult,
                  int32_t cap);

/* Cancellation guard of the float forms (piecewise-constant double layer).
 * A double-layer entry whose test triangle straddles the trial triangle's
 * plane sums terms of both signs (Eq. 1 with the kernel of Section 4's K);
 * its float value then carries an error of a few float ulps of the sum of
 * the magnitudes of its terms, A, which can exceed 1e-6 of the entry or of a
 * thousandth of the largest entry of its row.  Plans (and bem_near_field /
 * bem_coupling_blocks) running a BEM_LAPLACE_DLP job in BEM_MIXED or
 * BEM_MIXED_FULL on a BEM_P0 mesh therefore check every entry after the float
 * pass: if 8e-7 A > 1e-6 max(|g|, 1e-3 max over the job's row of |g|), the
 * entry is recomputed with the FP64 form's rules in double-float arithmetic
 * (float hi + lo pairs, about 44 bits).  This call waits for
 * the context's stream and returns the number of guarded entries of the plan
 * and how many of them the last run recomputed.  The per-call entry points
 * read the job's cluster and block arrays to size the guard's scratch, so a
 * guarded job makes them wait for the stream. */
int bem_plan_guard_stats(bem_ctx *ctx, bem_plan *plan, int64_t *guarded_entries,
                         int64_t *recomputed);

/* Rule-class counts of the plan's learned-order jobs in its last run (HOST
 * int64[6], classes in the order of bem_learned_counts); waits for the
 * context's stream. */
int bem_plan_learned_counts(bem_ctx *ctx, bem_plan *plan, int64_t *counts);

/* ---- sharding (multi-GPU) ----------------------------------------------------
 * Every matrix entry is independent (Section 3: the work lists need no
 * exchange), so block lists shard across GPUs without communication.  Splits
 * blocks 0..n_blocks-1 (HOST array cost[b] >= 0, e.g. quadrature points of
 * the block) into n_shards contiguous ranges of nearly equal total cost:
 * shard k owns blocks bounds[k] .. bounds[k+1]-1 (bounds: HOST, n_shards+1).
 * Whole blocks, so every output block has one owner.  Needs no device. */
int bem_shard_blocks(const int64_t *cost, int64_t n_blocks, int32_t n_shards, int64_t *bounds);

/* ---- touching pairs (host) ---------------------------------------------------
 * The case test of bem_mesh_upload (Section 2.2: pairs of triangles that share
 * one, two or three vertex indices are common-vertex, common-edge and
 * identical pairs; Section 3 / Algorithm 3 sorts pairs by this test), run on
 * the host without a device.  tris: HOST, nt x 3 vertex indices in [0, nv),
 * distinct within each triangle.  Lists every ordered pair (a, b) of triangles
 * sharing at least one vertex index, a == b included, ascending in (a, b):
 * src[k] = a, dst[k] = b, cas[k] = number of shared indices (1 vertex, 2 edge,
 * 3 identical) and ord[6k .. 6k+5] = the vertex orders the Sauter-Schwab maps
 * use, a's local indices at positions 0, 1, 2 followed by b's: the shared
 * vertex first; a shared edge as positions 0 -> 1 in the direction it has in
 * a, with b's same two vertices in the same order; identical pairs with b in
 * a's order; the remaining vertices in cyclic order.  *n_pairs receives the
 * number of pairs and min(cap, *n_pairs) are written (cap = 0 sizes the
 * arrays; they may then be NULL).  All arrays are HOST memory owned by the
 * caller.  Errors: BEM_ERR_INVALID_ARG (NULL pointers, an index out of
 * range), BEM_ERR_DEGENERATE (a triangle with a repeated index, two triangles
 * with the same three indices), BEM_ERR_UNSUPPORTED (beyond 32-bit indices).
 * Needs no context and no device. */
int bem_touching_pairs(const int32_t *tris, int64_t nt, int64_t nv, int32_t *src, int32_t *dst,
                       int32_t *cas, int32_t *ord, int64_t cap, int64_t *n_pairs);

/* ---- GCA pivots (host) -------------------------------------------------------
 * Pivot rows t~ of every cluster for the H^2 coupling matrices G|t~ x s~
 * (Sections 2.3-2.4).  For a cluster t: B_t = bounding box of the supports
 * of its basis functions, delta_t = diam(B_t), omega_t = B_t grown by
 * delta_t / 2 on every side; a gauss_per_face x gauss_per_face Gauss rule on
 * each of the six faces of omega_t (m = 6 gauss_per_face^2 points z_nu,
 * weights w_nu) gives the matrix A_t = (A_t+, A_t-) of Green's representation
 * formula, a_{t+,i nu} = sqrt(w_nu) int phi_i g(., z_nu) and
 * a_{t-,i nu} = sqrt(w_nu) delta_t int phi_i dg/dn(z_nu)(., z_nu) (g the
 * Laplace Green function for kappa = 0, exp(i kappa r)/(4 pi r) otherwise).
 * Cross approximation with complete pivoting on A_t chooses at most max_rank
 * rows, stopping once the largest remaining entry is <= eps times the first
 * pivot.  A cluster with sons restricts A_t to the rows t^ = t~_1 u t~_2 of
 * its sons' pivots (nested bases), so its pivots are a subset of theirs.
 *   verts   HOST double[nv][3]; tris HOST int32[nt][3] (as bem_mesh_upload)
 *   basis   BEM_P0 (indices are triangles) or BEM_P1 (vertices)
 *   cl_ptr, cl_idx  HOST cluster CSR: cluster c holds the indices
 *                   cl_idx[cl_ptr[c] .. cl_ptr[c+1]-1] (cl_ptr[0] = 0)
 *   cl_son  HOST int32[n_clusters][2]: the sons of c, -1 where absent; every
 *           cluster has at most one parent, and the sons' index sets make up
 *           the father's
 *   n_threads  host threads (0 = all hardware threads); the result does not
 *              depend on it
 *   piv_ptr, piv_idx  HOST outputs: pivots of c (sorted ascending) are
 *           piv_idx[piv_ptr[c] .. piv_ptr[c+1]-1]; piv_ptr holds n_clusters+1
 *           entries, piv_idx `cap` (n_clusters * max_rank always suffices).
 * Returns BEM_OK, or BEM_ERR_INVALID_ARG for bad arguments, an index out of
 * range, a cluster with two parents or a cycle, or cap too small.  Needs no
 * device and no context; all arrays stay the caller's. */
int bem_gca_pivots(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, int32_t basis,
                   double kappa, const int32_t *cl_ptr, const int32_t *cl_idx,
                   const int32_t *cl_son, int32_t n_clusters, int32_t gauss_per_face, double eps,
                   int32_t max_rank, int32_t n_threads, int32_t *piv_ptr, int32_t *piv_idx,
                   int64_t cap);

/* GCA pivots and interpolation matrices (Section 2.3: V_t = (A_t)|rows x tau
 * ((A_t)|t~ x tau)^-1 with the pivot rows t~ and pivot columns tau that the
 * cross approximation chose; Section 2.4: nested bases).  Same arguments and
 * pivots as bem_gca_pivots, plus the matrices: cluster c's matrix has one row
 * per row of its Green problem -- every index of a leaf in cl_idx order, or
 * for a cluster with sons the sons' pivots (first son first, each ascending),
 * the rows t^ of its transfer matrix V^_t -- and one column per pivot of c
 * (ascending), row-major, at element offset v_off[c] of V (v_off HOST
 * int64[n_clusters + 1], v_off[c + 1] - v_off[c] = rows x K_c).  V is a HOST
 * array of v_cap elements: doubles for kappa = 0, (re, im) double pairs
 * otherwise; (n_indices + 2 max_rank n_clusters) max_rank elements always
 * suffice.  The rows at the pivots form the identity (the interpolation
 * property R_t V_t = I), up to rounding.  Errors as bem_gca_pivots, and
 * BEM_ERR_INVALID_ARG for NULL v_off or V or v_cap too small. */
int bem_gca_bases(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, int32_t basis,
                  double kappa, const int32_t *cl_ptr, const int32_t *cl_idx,
                  const int32_t *cl_son, int32_t n_clusters, int32_t gauss_per_face, double eps,
                  int32_t max_rank, int32_t n_threads, int32_t *piv_ptr, int32_t *piv_idx,
                  int64_t cap, int64_t *v_off, double *V, int64_t v_cap);

/* ---- Green quadrature matrices (device) --------------------------------------
 * The matrices A_t = (A_t+, A_t-) of Green's representation formula that the
 * cross approximation above works on (Section 2.3), for a list of clusters in
 * one launch.  Cluster c has rows r_k = row_idx[row_ptr[c] + k], k < n_c
 * (n_c = row_ptr[c+1] - row_ptr[c]; P0: triangles, P1: vertices of the mesh)
 * and points z_nu with unit normals n_nu, nu = pt_ptr[c] + l, l < m_c
 * (m_c = pt_ptr[c+1] - pt_ptr[c]).  Its block, column-major with leading
 * dimension n_c, n_c x 2 m_c, at element offset out_off[c] of `out`, holds
 *   column l        A_t+[k, l] = sp_nu int phi_{r_k}(x) g(x, z_nu) dx
 *   column m_c + l  A_t-[k, l] = sm_nu int phi_{r_k}(x) d/dn(z_nu) g(x, z_nu) dx
 * with g(x, z) = exp(i kappa r)/(4 pi r), r = |x - z| (kappa = 0 for
 * BEM_LAPLACE_SLP and BEM_LAPLACE_DLP, which share Green's function) and
 * n . grad_z g = (x - z).n (1 - i kappa r) exp(i kappa r)/(4 pi r^3).  The GCA
 * takes sp = sqrt(w_nu), sm = sqrt(w_nu) delta_t (quadrature weights w_nu on
 * the boundary of omega_t, delta_t = diam of the cluster's box).  Every
 * support triangle is integrated in FP64 by a rule on the reference triangle
 * (Section 2.2): BEM_RULE_TRI7 (Radon's 7 points) or BEM_RULE_DUFFY with q in
 * [1, 5] Gauss points per axis of the Duffy square.  The integrands are smooth
 * only for points away from the supports (the GCA keeps them delta_t / 2 away);
 * this is not checked, and a point on a support gives non-finite entries.
 *   All pointers are DEVICE arrays owned by the caller:
 *     row_ptr, pt_ptr  int32[n_clusters + 1], non-decreasing
 *     row_idx          int32[n_row_idx]
 *     z, nz            double[n_points][3]
 *     sp, sm           double[n_points], or NULL for a factor of 1
 *     out_off          int64[n_clusters]
 *     out              double[out_len] (Laplace) or 16-byte aligned (re, im)
 *                      double pairs [out_len] (Helmholtz); blocks must not
 *                      overlap.
 * Asynchronous on the context's stream.  Host errors: BEM_ERR_INVALID_ARG
 * (unknown mesh, bad kernel, rule or counts, NULL pointers, misaligned
 * complex output).  Found on the device and reported by bem_sync as
 * BEM_ERR_INVALID_ARG: pointer ranges beyond n_row_idx / n_points or
 * decreasing, a cluster with 2^30 or more rows or points, a block beyond
 * out_len (that cluster is skipped), a row index out of range (that row is
 * skipped). */
typedef struct {
    int32_t mesh_id;
    bem_kernel_desc kernel;
    int32_t rule;                /* BEM_RULE_TRI7 or BEM_RULE_DUFFY */
    int32_t q;                   /* Gauss points per axis (BEM_RULE_DUFFY) */
    int32_t n_clusters;
    const int32_t *row_ptr;
    const int32_t *row_idx;
    int64_t n_row_idx;
    const int32_t *pt_ptr;
    const double *z;
    const double *nz;
    const double *sp;
    const double *sm;
    int64_t n_points;
    const int64_t *out_off;
    void *out;
    int64_t out_len;
} bem_green_job;

int bem_green_matrices(bem_ctx *ctx, const bem_green_job *job);

/* GCA pivots with the Green matrices on the device: the pivots of
 * bem_gca_pivots (same arguments, same host arrays and outputs), with every
 * A_t assembled by the kernel of bem_green_matrices (FP64, Radon's 7 points
 * per support triangle) instead of on the host.  The tree is processed level by
 * level from the deepest: a level's A_t in one launch, copied back, and their
 * cross approximation on host threads, as in bem_gca_pivots.  The pivots equal
 * those of bem_gca_pivots except where rounding of A_t's entries decides between
 * two candidates of equal magnitude.
 *   ctx, mesh_id  the context and the id of the same mesh uploaded with
 *                 bem_mesh_upload (vertex and triangle counts and basis must
 *                 match; the host arrays give the clusters' boxes)
 * Synchronises the context's stream once per level.  Allocates one device
 * buffer for the largest level and frees it before returning.  Errors: those
 * of bem_gca_pivots; BEM_ERR_INVALID_ARG for an unknown or different mesh;
 * BEM_ERR_CUDA / BEM_ERR_OOM from the device. */
int bem_gca_pivots_device(bem_ctx *ctx, int32_t mesh_id, const double *verts, int64_t nv,
                          const int32_t *tris, int64_t nt, int32_t basis, double kappa,
                          const int32_t *cl_ptr, const int32_t *cl_idx, const int32_t *cl_son,
                          int32_t n_clusters, int32_t gauss_per_face, double eps,
                          int32_t max_rank, int32_t n_threads, int32_t *piv_ptr, int32_t *piv_idx,
                          int64_t cap);

/* ---- quadrature rules ------------------------------------------------------
 * Copies the library's 4D rule on D x D for a case (Section 2.2; case 0 =
 * disjoint pairs with regular_rule BEM_RULE_DUFFY / BEM_RULE_TRI7, 1 = common
 * vertex, 2 = common edge, 3 = identical; q = Gauss points per axis) into the
 * HOST array `out` as 7 columns of n values: x1, x2, y1, y2, w, x1-y1,
 * x2-y2 (x in the test triangle's reference domain, y in the trial's, w the
 * weight including the Jacobian; the differences are formed from each
 * subdomain map's own factors).  Returns n, or a negative BEM_ERR_* for an
 * unknown case or order.  If out is NULL or cap < 7 n, only n is returned.
 * Needs no device and no context. */
int64_t bem_rule_points(int32_t cas, int32_t regular_rule, int32_t q, double *out, int64_t cap);

/* The touching rule of case cas (1 = common vertex, 2 = common edge,
 * 3 = identical) and order q with xi integrated out, in the layout of
 * bem_rule_points: the q^3 points per subdomain at xi = 1, weight J(eta)
 * times the Gauss weights of (eta1, eta2, eta3).  Under the Sauter-Schwab
 * maps of Section 2.2 every coordinate and difference is xi times a function
 * of eta and the weight xi^3 times one, so for the Laplace kernels the
 * integrand of a moment is xi^n times a function of eta (single layer n = 2,
 * double layer n = 1, one more per piecewise-linear coordinate factor); where
 * the q-point Gauss rule in xi is exact for degree n, the q^4-point sum equals
 * 1/(n+1) times the sum over these points.  The library evaluates Laplace
 * touching pairs this way wherever that holds (2q - 1 >= n); the Helmholtz
 * kernels keep the q^4 rule.  Returns n, or a negative BEM_ERR_* for another
 * case or order.  Needs no device and no context. */
int64_t bem_rule_points_xi(int32_t cas, int32_t q, double *out, int64_t cap);

/* ---- allocation-free near field --------------------------------------------
 * The paper has no counterpart of this call; it exists for callers that must
 * not allocate device memory (a service whose device memory belongs to its own
 * pool allocator, a loop that cannot afford the implicit device-wide
 * synchronisation cudaMalloc/cudaFree may cause, a host program that has
 * handed out all device memory before assembling).
 *
 * Computes the same near-field blocks as bem_near_field for ONE job, with the
 * same kernels, but calls no cudaMalloc, cudaFree or other allocating routine.
 * Its scratch (the singular-case rule tables of every order 1..6 and the
 * per-block tile sums) is a static device array of 2,053,088 bytes inside the
 * library, present on every GPU that loads the library until the process
 * exits.  The mesh, the context's status word and the outputs are the ones
 * set up by earlier calls (bem_create, bem_mesh_upload) and by the caller.
 *
 * Supported: the FP64 form (precision BEM_FP64) with fixed orders
 * (BEM_ORDER_FIXED), regular rule BEM_RULE_TRI7 or BEM_RULE_DUFFY with
 * q_regular in [2, 4], singular orders q_vertex, q_edge, q_identical in
 * [1, 6], at most 65536 blocks.  Rejections (nothing is launched):
 *   BEM_ERR_INVALID_ARG  null context or job, unknown mesh id, bad kernel
 *                        descriptor, a singular order outside [1, 6] or more
 *                        than 65536 blocks (the message names the static
 *                        scratch's limit), negative block count, null pointer
 *                        or empty cluster list, complex output not 16-byte
 *                        aligned;
 *   BEM_ERR_UNSUPPORTED  the mixed or float-full forms, learned orders, any
 *                        other regular rule or order, piecewise-linear meshes
 *                        with a vertex of degree above 16;
 *   BEM_ERR_CUDA         a failed CUDA call (message from the runtime).
 *   - The first call on a device sets the array up with that device current:
 *     it looks up the array's device address (cudaGetSymbolAddress) and
 *     copies the rule tables into it (synchronous host-to-device copies).
 *     Make that first call before any stream capture.  Later calls copy
 *     nothing from the host and only launch kernels on the context's stream.
 *   - Every call shares the one array and the mesh's touching table, and
 *     leaves its contents behind: calls on the same stream are ordered, but
 *     calls that overlap on the GPU (other streams or contexts on the same
 *     device) race and may produce wrong entries. */
int bem_near_field_noalloc(bem_ctx *ctx, const bem_block_job *job);

/* ---- H2 matrix-vector product and conjugate gradients -----------------------
 * The H2 matrix of Section 2.4 built from the blocks this library assembles,
 * and the solve of Section 4 (the interior Dirichlet problem V a = (1/2 M + K) b
 * by conjugate gradients, V symmetric positive definite):
 *     G ~ sum over near blocks (t, s) of N_ts  +  sum over admissible blocks of
 *         V_t S_ts V_s^T,   S_ts = G|t~ x s~ (coupling entries at the pivots),
 * with the nested cluster bases of bem_gca_bases (V_t = diag(V_t1, V_t2) V^_t
 * for a cluster with sons).  Real (FP64) matrices: the Laplace kernels.
 *   n             number of indices (basis functions)
 *   cl_ptr, cl_idx, cl_son, n_clusters  HOST cluster tree as for bem_gca_pivots
 *   piv_ptr, piv_idx, v_off, V          HOST output of bem_gca_bases (kappa = 0;
 *                                        at most 32 pivots per cluster)
 *   near_row, near_col, near_off  HOST near blocks (row cluster, column cluster,
 *                 element offset): leaves only, column-major |t| x |s| over the
 *                 clusters' index sets at near_vals + near_off (DEVICE, the
 *                 output of bem_near_field for the same blocks)
 *   far_row, far_col, far_off     HOST admissible blocks, column-major
 *                 |t~| x |s~| over the pivots at far_vals + far_off (DEVICE, the
 *                 output of bem_coupling_blocks over the pivot sets)
 *   diag          HOST double[n] added to the diagonal (Section 4's 1/2 M for
 *                 the operator 1/2 M + K of the right-hand side), or NULL
 * The library copies the tree, the bases, the block lists and diag to the
 * device; near_vals and far_vals stay the caller's and must outlive the
 * handle.
 * bem_h2_matvec: y = G x for DEVICE vectors of n doubles (x != y),
 * asynchronous on the context's stream; bitwise reproducible (no atomics).
 * bem_h2_cg: conjugate gradients (Hestenes-Stiefel) from x = 0 until
 * |r| <= tol |b| or maxit iterations; b, x DEVICE vectors of n doubles; waits
 * for the stream once per iteration (the residual check); returns the
 * iterations and |r|/|b|.  Errors: BEM_ERR_INVALID_ARG (bad tree, bases of the
 * wrong shape, a block out of range or a near block on a non-leaf row
 * cluster), BEM_ERR_UNSUPPORTED (more than 32 pivots in a cluster),
 * BEM_ERR_DEGENERATE (a non-finite residual: the matrix is not positive
 * definite), BEM_ERR_CUDA. */
typedef struct bem_h2 bem_h2;
int bem_h2_create(bem_ctx *ctx, int64_t n, int32_t n_clusters, const int32_t *cl_ptr,
                  const int32_t *cl_idx, const int32_t *cl_son, const int32_t *piv_ptr,
                  const int32_t *piv_idx, const int64_t *v_off, const double *V, int64_t n_near,
                  const int32_t *near_row, const int32_t *near_col, const int64_t *near_off,
                  const double *near_vals, int64_t n_far, const int32_t *far_row,
                  const int32_t *far_col, const int64_t *far_off, const double *far_vals,
                  const double *diag, bem_h2 **out);
int bem_h2_matvec(bem_ctx *ctx, bem_h2 *h2, const double *x, double *y);
int bem_h2_cg(bem_ctx *ctx, bem_h2 *h2, const double *b, double *x, double tol, int32_t maxit,
              int32_t *iters, double *rel_res);
int bem_h2_destroy(bem_ctx *ctx, bem_h2 *h2);

/* ---- potentials and the exterior Helmholtz problem -----------------------
 * Section 4's exterior Dirichlet problem in the Brakhage-Werner form: the
 * density w on the surface solves (1/2 M + K - i eta V) w = F, F_i = int phi_i f,
 * and the field outside is u(z) = sum_j w_j int_{T_j} (dg/dn_y - i eta g)(z, y) dy.
 * bem_potentials: u(z_k) = sum_j w_j int_{T_j} k(z_k, y) dy for n_points points
 *   z (DEVICE double[n_points][3], off the surface: the integrands must be
 *   smooth) and a piecewise-constant complex density (DEVICE (re, im) double
 *   pairs, one per triangle), with the kernel of `kernel` (any kind) and a
 *   Duffy q x q rule per triangle (q in [1, 5]), FP64; out: DEVICE complex
 *   [n_points].  Asynchronous.  Errors: BEM_ERR_INVALID_ARG (unknown mesh, bad
 *   kernel, order or pointers, complex arrays not 16-byte aligned),
 *   BEM_ERR_UNSUPPORTED (a piecewise-linear mesh).
 * bem_dense_gmres: restarted GMRES for (A + diag(d)) x = b with A a DEVICE
 *   column-major complex n x n matrix (e.g. from bem_assemble_dense), d a
 *   DEVICE complex vector or NULL, b and x DEVICE complex vectors (x is
 *   overwritten, starting from 0); classical Gram-Schmidt applied twice,
 *   `restart` Krylov vectors per cycle (<= 500), at most maxit iterations,
 *   until |b - (A + D) x| <= tol |b|.  Allocates (restart + 1) n complex
 *   values of scratch per call and waits for the stream at every Arnoldi
 *   step.  Returns the iterations and the relative residual. */
int bem_potentials(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel, int32_t q,
                   const double *points, int64_t n_points, const double *density, double *out);
int bem_dense_gmres(bem_ctx *ctx, int64_t n, const double *A, const double *diag,
                    const double *b, double *x, double tol, int32_t restart, int32_t maxit,
                    int32_t *iters, double *rel_res);

/* ---- arithmetic-pipe probes -------------------------------------------------
 * Not part of the paper's method: measurement kernels that give the
 * quadrature kernels' rooflines a measured denominator on the GPU at hand.
 * Launches one probe on the context's stream (asynchronously) and stores in
 * *ops the number of operations that launch performs; the caller times the
 * launch with CUDA events on that stream.  kind: 0 = FP32 FMA (2 operations
 * each), 1 = FP64 FMA (2 each), 2 = reciprocal square root of the special
 * function unit (rsqrt.approx.ftz.f32, 1 each), 3 = its sine and cosine
 * (2 per argument), 4 = packed FP32 pair FMA (fma.rn.f32x2, 4 each).  Every
 * thread of 8 CTAs of 256 threads per SM runs 8 independent chains of 16
 * instructions per trip, `trips` times.  Errors: BEM_ERR_INVALID_ARG for a
 * kind outside [0, 4] or trips outside [1, 2^30]. */
int bem_peak_probe(bem_ctx *ctx, int32_t kind, int64_t trips, double *ops);

/* ---- launch profiling (tracing) ------------------------------------------
 * When enabled, every kernel launch of the context is bracketed by CUDA
 * events recorded on the context's stream.  bem_profile_read waits for the
 * stream, adds the elapsed times of all finished launches to per-kernel
 * totals and copies up to `cap` totals to `out` (*n_out = number of kernel
 * classes).  bem_profile_enable(ctx, 0) stops recording; bem_profile_reset
 * clears the totals.  No effect on results. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} bem_kernel_time;

int bem_profile_enable(bem_ctx *ctx, int32_t on);
int bem_profile_reset(bem_ctx *ctx);
int bem_profile_read(bem_ctx *ctx, bem_kernel_time *out, int32_t cap, int32_t *n_out);

#ifdef __cplusplus
}
#endif
#endif /* BEM_GB300_H */
