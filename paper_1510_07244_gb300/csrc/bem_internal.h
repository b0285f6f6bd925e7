// Internal declarations shared by the host planner (bem_api.cpp), the rule
// generator (bem_rules.cpp) and the device code (bem_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "bem.h"

namespace bem {

constexpr int kGeomStride = 16;      // doubles per triangle record (128 bytes)
// record layout: v0[3] v1[3] v2[3] n[3] sqrt_g pad[3]
constexpr int kGeomFStride = 32;     // floats per triangle record of the mixed form (128 bytes)
// layout: vertex hi[9] | vertex lo[9] (x = hi + lo exactly to ~2^-48) | e1[3] e2[3]
//         (FP64 differences rounded once) | n hi[3] | n lo[3] | sqrt_g | pad
constexpr int kMaxDegP1 = 16;        // vertex degree bound of the P1 block engine
constexpr int kTile = 32;            // rows / columns of one block tile
constexpr int kP0Tile = 256;         // entries of one piecewise-constant tile (one per thread)
constexpr int kMaxNp = 25;           // points of a 2D regular rule (Duffy q <= 5)

enum Case { kRegular = 0, kVertex = 1, kEdge = 2, kIdentical = 3 };

// The six permutations of (0,1,2); a code c in [0,6) names kPerm[c].
// Canonical orders are stored as (code_a * 6 + code_b).
extern const int kPerm[6][3];

// 2D rule on the reference triangle D, passed by value to the kernels.
struct Rule2D {
    int np;
    double s[kMaxNp], t[kMaxNp], w[kMaxNp];
    float sf[kMaxNp], tf[kMaxNp], wf[kMaxNp];   // the same rule rounded to float
    // w_k lambda_q(s_k, t_k) in float: the weights times the three linear
    // basis functions of the reference triangle, lambda = (1 - s, s - t, t)
    float wl[3][kMaxNp];
};

// 4D rule on D x D, device SoA with kRuleCols columns of n values:
// x1 | x2 | y1 | y2 | w | x1-y1 | x2-y2 (the differences are formed from each
// subdomain map's own factors, so they keep full precision near the singular set).
constexpr int kRuleCols = 7;
struct Rule4D {
    int n = 0;
    int q = 0;             // Gauss points per axis (touching rules)
    double *d = nullptr;   // device, kRuleCols n doubles
    float *f = nullptr;    // device, kRuleCols n floats (mixed form), may be null
    float *fl = nullptr;   // device, kRuleCols n floats: d - f (double-float form), may be null
    int xi = 0;            // 1: a touching rule with xi integrated out (at xi = 1)
};
// Rule id of the touching rules with xi integrated out (the rule cache's key).
constexpr int kRuleXiOut = 1;

// The q-point Gauss rule in xi on [0, 1] for the Helmholtz sums at fixed eta:
// sum_k w_k xi_k^(2+m) exp(i th xi_k) = exp(i th / 2) (cmid[m] + sum_j
// (cp[j][m] cos(th t_j) + i cm[j][m] sin(th t_j))) over the node pairs
// xi = 1/2 -+ t_j (the nodes and weights are symmetric about 1/2), cmid the
// middle node's term for odd q; m = 0, 1, 2.
constexpr int kMaxXiPairs = 10;
struct XiRule {
    int npair = 0;
    float t[kMaxXiPairs];
    float cp[kMaxXiPairs][3], cm[kMaxXiPairs][3];
    float cmid[3] = {0.0f, 0.0f, 0.0f};
};
bool make_xi_rule(int q, XiRule &out);

// Device view of an uploaded mesh.
struct MeshView {
    int64_t nv, nt;
    int basis;
    int maxdeg;
    const double *geom;        // nt * kGeomStride
    const float *geomf;        // nt * kGeomFStride (mixed form)
    const int4 *tvid;          // nt (v0, v1, v2, 0)
    const int *vt_ptr;         // nv + 1
    const int *vt_tri;         // 3 nt, ascending triangle ids per vertex
    const int *nb_ptr;         // nt + 1: touching neighbours of each triangle
    const int *nb_tri;         // ntouch, ascending per triangle
    const int *nb_src;         // ntouch: the triangle a of entry k (b = nb_tri[k])
    const unsigned char *nb_case;   // ntouch
    const unsigned char *nb_perm;   // ntouch: code_a * 6 + code_b
    double2 *table;            // ntouch * (1 or 9): touching-pair integrals
    int64_t ntouch;
};

// Scratch of one learned-order job: class per tile slot, records grouped by
// class, counters (int [8] + fill [8]) and class offsets (int64 [7]).
struct LearnedScratch {
    unsigned char *cls = nullptr;   // class per entry slot (cap slots)
    void *rec = nullptr;            // records by class (cap int4)
    int64_t *small = nullptr;       // class counts and offsets
    int *tcount = nullptr;          // per class and tile warp: count, then scanned offset
    int64_t cap = 0;                // entry slots: a multiple of the flat tile
};

struct Mesh {
    MeshView v{};
    bem_mesh_stats stats{};
    std::vector<void *> allocs;
    int *list[4] = {nullptr, nullptr, nullptr, nullptr};   // touching indices per case
    int64_t nlist[4] = {0, 0, 0, 0};
    std::vector<int> hlist[4];                              // host copies of the lists
    int *iota = nullptr;       // 0 .. n-1 (dense calls)
    int *dense_csr = nullptr;  // {0, n} and the block {0, 0, off 0}
    uint64_t host_hash = 0;    // mesh_hash of the uploaded vertex and triangle arrays
};

// FNV-1a over the bytes of the vertex and triangle arrays: calls that take the
// host mesh again (bem_gca_pivots_device) check it is the uploaded one.
inline uint64_t mesh_hash(const double *verts, int64_t nv, const int32_t *tris, int64_t nt)
{
    uint64_t h = 1469598103934665603ull;
    auto add = [&h](const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t k = 0; k < n; ++k) {
            h ^= c[k];
            h *= 1099511628211ull;
        }
    };
    add(verts, (size_t)nv * 3 * sizeof(double));
    add(tris, (size_t)nt * 3 * sizeof(int32_t));
    return h;
}

}  // namespace bem

struct bem_prof_rec {
    std::string name;
    cudaEvent_t a, b;
    bool skipped = false;   // a launch group the runs do not issue (static plans)
};

struct bem_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int *status = nullptr;                 // device status word
    int64_t *tile_prefix = nullptr;        // scratch: per-block tile prefix sums
    int64_t tile_prefix_cap = 0;
    void *guard_buf = nullptr;             // scratch: cancellation guard of one call
    size_t guard_cap = 0;
    int num_sms = 0;
    std::map<int, bem::Mesh *> meshes;
    int next_mesh = 1;
    std::map<std::tuple<int, int, int>, bem::Rule4D> rules4;   // (case, rule, q)
    bool profile = false;
    std::vector<bem_prof_rec> prof_pending;
    std::vector<cudaEvent_t> prof_free;
    std::map<std::string, std::pair<int64_t, double>> prof_total;
    std::vector<struct bem_plan *> prof_plans;   // plans whose last run's events are unread
    std::map<std::string, int> tuned;            // autotuner cache: bucket key -> CTAs per SM
    // learned order selection
    struct bem_mlp *order_model = nullptr;
    float order_conf = 0.0f;
    bem::LearnedScratch learned;                 // scratch of the per-call learned path
    int64_t learned_counts[6] = {0, 0, 0, 0, 0, 0};
};

namespace bem {
// Brackets one launch with profiling events when the context profiles.
struct ProfScope {
    bem_ctx *ctx;
    bem_prof_rec rec;
    bool on;
    ProfScope(bem_ctx *c, const char *name);
    ~ProfScope();
};
}  // namespace bem

namespace bem {

// bem_api.cpp helpers shared with the plan driver
int api_fail(bem_ctx *ctx, int code, const char *msg);
int api_ensure_prefix(bem_ctx *ctx, int64_t n);   // grows the tile-prefix scratch
int api_cuda_fail(bem_ctx *ctx, cudaError_t e, const char *where);
int api_check_job(bem_ctx *ctx, const bem_block_job &J, Rule2D &r2, Mesh **mesh);
int api_get_rule4(bem_ctx *ctx, int cas, int rule, int q, Rule4D &out);
// The touching rule of case cas and order q for a kernel, basis and
// precision of the touching kernel (f32): xi integrated out where
// touch_xi_out allows it, else the q^4 rule.
int api_touch_rule(bem_ctx *ctx, int cas, int q, int kind, int basis, bool f32, Rule4D &out);
void prof_accumulate(bem_ctx *ctx, const bem_prof_rec &r);
// bem_plan.cpp: adds the unread launch times of plans run since the last read
void plan_drain_profile(bem_ctx *ctx);
void plan_forget(bem_ctx *ctx);   // context teardown

// bem_gca.cpp: the GCA of a cluster tree level by level (deepest first), the
// Green matrices A_t of each level from a producer.  A level is given in the
// cluster-CSR layout of bem_green_matrices: cluster k's rows
// rows[row_ptr[k] .. row_ptr[k+1]) (all indices of a leaf, the sons' pivots
// otherwise), its box points z / normals nz (3 doubles each) with factors sp =
// sqrt(w), sm = sqrt(w) delta_t, and its block at element off[k].
struct GreenLevel {
    std::vector<int32_t> row_ptr, rows, pt_ptr;
    std::vector<double> z, nz, sp, sm;
    std::vector<int64_t> off;
    int64_t total = 0;
};
// Fills out (total doubles, or total (re, im) pairs when cplx_out) with the
// level's blocks as bem_green_matrices writes them; returns BEM_OK or an error.
using GreenLevelProducer =
    std::function<int(const GreenLevel &L, bool cplx_out, std::vector<double> &out)>;
int gca_pivots_levels(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                      int32_t basis, double kappa, const int32_t *cl_ptr, const int32_t *cl_idx,
                      const int32_t *cl_son, int32_t n_clusters, int32_t gauss_per_face,
                      double eps, int32_t max_rank, int32_t n_threads,
                      const GreenLevelProducer &produce, int32_t *piv_ptr, int32_t *piv_idx,
                      int64_t cap);

// bem_rules.cpp
bool gauss_legendre_unit(int q, std::vector<double> &x, std::vector<double> &w);
bool make_rule2d(int regular_rule, int q, Rule2D &out);
bool make_rule4d_host(int cas, int regular_rule, int q, std::vector<double> &soa,
                      bool xi_out = false);

// bem_kernels.cu: launchers (return a cudaError_t of the launch)
struct BlockLaunch {
    const int32_t *row_ptr, *row_idx, *col_ptr, *col_idx;
    int32_t n_row_clusters, n_col_clusters;
    const int32_t *blk_row, *blk_col;
    const int64_t *blk_off;
    int64_t n_blocks;
    void *out;
    int kind;
    double kappa;
    double eta = 0.0;   // Brakhage-Werner coupling (BEM_HELMHOLTZ_BW)
    int lower_only;
    int allow_touching;
    int mixed;        // 1: regular pairs in FP32 (BEM_MIXED, BEM_MIXED_FULL)
    // piecewise-linear tile engine: support records of the 32-index slices of
    // the row / column clusters, built once per run (null: built per tile);
    // slice_*[c] = first record of cluster c, cap_* = records allocated
    const int32_t *sup_r = nullptr, *sup_c = nullptr;
    const int32_t *slice_r = nullptr, *slice_c = nullptr;
    int64_t cap_r = 0, cap_c = 0;
    // fused jobs (single and double layer of the same blocks): the double-layer
    // output (the single-layer one is `out`) and, for the near field, the
    // double layer's touching table (the single layer's is the mesh view's)
    void *out2 = nullptr;
    const double2 *table2 = nullptr;
    // cancellation guard (piecewise-constant double layer, float forms): the
    // engine writes each entry as the float pair (value, sum of |terms|) for
    // the guard pass (bem_guard.cu), which widens or recomputes it
    int guard = 0;
};

// Internal kernel id of the fused single + double layer (never a public kind).
constexpr int kFusedLaplace = 16;

// One support record (int32 words, 16-byte multiple): list lengths [kTile],
// per-vertex lists [kMaxDegP1][kTile], triangles [kTile * kMaxDegP1], count.
constexpr int kSupListN = 0;
constexpr int kSupLists = kTile;
constexpr int kSupTris = kSupLists + kMaxDegP1 * kTile;
constexpr int kSupCount = kSupTris + kTile * kMaxDegP1;
constexpr int kSupInts = (kSupCount + 1 + 3) & ~3;

// Precision forms: float arithmetic for disjoint pairs, and for the touching
// pairs of case `cas`.
inline bool is_mixed(int precision) { return precision == BEM_MIXED || precision == BEM_MIXED_FULL; }
// kernels with complex values, and kernels that run in FP64 in every precision
__host__ __device__ constexpr bool kind_complex(int kind)
{
    return kind == BEM_HELMHOLTZ_SLP || kind == BEM_HELMHOLTZ_DLP || kind == BEM_HELMHOLTZ_BW;
}
__host__ __device__ constexpr bool kind_fp64_only(int kind)
{
    return kind == BEM_HELMHOLTZ_DLP || kind == BEM_HELMHOLTZ_BW;
}
// kernels whose numerator is the height (x - y).n_y of x above the trial plane
__host__ __device__ constexpr bool kind_has_height(int kind)
{
    return kind == BEM_LAPLACE_DLP || kind == BEM_HELMHOLTZ_DLP || kind == BEM_HELMHOLTZ_BW;
}
// Touching pairs with xi integrated out.  Under the Sauter-Schwab maps the
// Laplace integrands are xi^n times a function of (eta1, eta2, eta3): the
// single layer xi^2 (Jacobian xi^3 over r = xi |u|), the double layer xi
// (height xi h over r^3 = xi^3 |u|^3), and each piecewise-linear moment
// (1, x1, x2) x (1, y1, y2) one more power per factor x or y.  The q-point
// Gauss rule in xi integrates degree 2q - 1 exactly, so where n stays within
// it the sum over xi is 1 / (n + 1), and the rule at xi = 1 with that factor
// gives the q^4-point result (up to rounding) with q^3 points per subdomain.
__host__ __device__ constexpr int xi_base(int kind) { return kind == BEM_LAPLACE_SLP ? 2 : 1; }
inline bool touch_xi_out(int kind, int basis, int q, bool f32)
{
    // the float Helmholtz single layer sums over xi at each point (XiRule)
    if (kind == BEM_HELMHOLTZ_SLP) return f32 && q <= 2 * kMaxXiPairs;
    if (kind != BEM_LAPLACE_SLP && kind != BEM_LAPLACE_DLP) return false;
    const int deg = xi_base(kind) + (basis == BEM_P1 ? 2 : 0);
    return 2 * q - 1 >= deg;
}
// factor of the moment with i (test) and j (trial) coordinate factors
__host__ __device__ constexpr double xi_moment(int kind, int i, int j)
{
    return 1.0 / (double)(xi_base(kind) + (i > 0 ? 1 : 0) + (j > 0 ? 1 : 0) + 1);
}
inline int touch_in_float(int precision, int cas, int kind)
{
    if (kind_fp64_only(kind)) return 0;
    return precision == BEM_MIXED_FULL || (precision == BEM_MIXED && cas == kVertex);
}

// One block list of a batched launch (device table entry).
struct BatchJob {
    MeshView m;
    BlockLaunch L;
    const int64_t *prefix;     // per-block tile prefix sums of this list
};

// One guarded job (bem_guard.cu): its mesh and blocks, and a per-row maximum
// (float bits of |value|, zeroed before every pass) over n_rows row indices.
struct GuardJob {
    MeshView m;
    BlockLaunch L;
    unsigned *rowmax;
    int64_t n_rows;
};

// An entry of a guarded job recomputed in FP64: row and column triangles and
// the output offset.
struct GuardItem {
    int32_t job, row, col, pad;
    int64_t off;
};

// Forward-error bound of the float forms' double-layer entries, relative to the
// sum of the magnitudes of the quadrature terms; entries whose bound can exceed
// the relative-error bar are recomputed in FP64.
constexpr float kGuardRel = 8e-7f;

// Guarded jobs with the same orders, and their device buffers.  Built on the
// host (guard_add reads each job's cluster and block arrays once to count its
// entries), laid out in one device allocation by guard_layout, run by
// guard_run: zero the row maxima and the list counter, row maxima, selection,
// FP64 recomputation (rules: the FP64 rules of the jobs' orders).
struct GuardSet {
    std::vector<GuardJob> host;
    std::vector<int64_t> blk_end;        // inclusive prefix of the block counts
    int64_t rows = 0, entries = 0, cap = 0, cap_t = 0;
    Rule4D rules[4];                     // FP64 rules: regular, vertex, edge, identical
    Rule2D r2;                           // the regular rule's 2D points (one per set)
    GuardJob *d_jobs = nullptr;
    int64_t *d_blk_end = nullptr;
    unsigned *d_rowmax = nullptr;
    unsigned long long *d_count = nullptr;   // [0]: disjoint entries listed, [1]: touching
    GuardItem *d_list = nullptr;             // disjoint pairs (capacity cap)
    GuardItem *d_list_t = nullptr;           // touching pairs (capacity cap_t)
};
cudaError_t guard_add(GuardSet &g, const MeshView &m, const BlockLaunch &L, cudaStream_t st);
size_t guard_bytes(const GuardSet &g);
// buf: guard_bytes(g) bytes, 256-byte aligned; uploads the job table on st
cudaError_t guard_layout(GuardSet &g, void *buf, cudaStream_t st);
cudaError_t guard_run(const GuardSet &g, int num_sms, int *status, cudaStream_t st);

// One mesh / kernel of a batched touching launch.
struct TouchJob {
    MeshView m;                // m.table = this job's touching table
    double kappa;
    double eta = 0.0;
};

// Launch shape of a block-engine bucket (autotuned).
struct Shape {
    int grid_mult;             // CTAs per SM
};

cudaError_t launch_tile_prefix(const BlockLaunch &L, int tr, int tc, int64_t *prefix,
                               int *status, cudaStream_t st);
// Blocks per CTA of the many-CTA prefix pass, and its chunk count (the
// chunk_total scratch holds one int64 per chunk).
constexpr int64_t kPrefixChunk = 8192;
inline int64_t prefix_chunks(int64_t n_blocks) { return (n_blocks + kPrefixChunk - 1) / kPrefixChunk; }
// The same prefix sums as launch_tile_prefix; lists longer than one chunk take
// two launches over many CTAs.
cudaError_t launch_tile_prefix_wide(const BlockLaunch &L, int tr, int tc, int64_t *prefix,
                                    int64_t *chunk_total, int *status, cudaStream_t st);
cudaError_t launch_touching(const MeshView &m, int cas, const int *list, int64_t n,
                            const Rule4D &rule, int kind, double kappa, int f32,
                            cudaStream_t st, double eta = 0.0);
cudaError_t launch_block_engine(const MeshView &m, const BlockLaunch &L, const Rule2D &rule,
                                const int64_t *prefix, int *status, int grid, cudaStream_t st);
size_t p1_smem_bytes(bool cplx, bool mixed, bool fused = false);
// bem_block_p1_{fp64,mixed}.cu: piecewise-linear block engine per precision
cudaError_t launch_p1_single_fp64(int kind, int np, const MeshView &m, const BlockLaunch &L,
                                  const Rule2D &R, const int64_t *prefix, int *status, int grid,
                                  cudaStream_t st);
cudaError_t launch_p1_single_mixed(int kind, int np, const MeshView &m, const BlockLaunch &L,
                                   const Rule2D &R, const int64_t *prefix, int *status, int grid,
                                   cudaStream_t st);
cudaError_t launch_p1_batch_fp64(int kind, int np, const BatchJob *jobs, int n_jobs,
                                 const int64_t *job_end, const Rule2D &R, int *status, int grid,
                                 cudaStream_t st);
cudaError_t launch_p1_batch_mixed(int kind, int np, const BatchJob *jobs, int n_jobs,
                                  const int64_t *job_end, const Rule2D &R, int *status, int grid,
                                  cudaStream_t st);
// Per-job block prefix sums of tiles tr x tc (tr = tc = 1: entries) and the
// inclusive scan of the job totals in units of `unit` per tile.
cudaError_t launch_tile_prefix_batch(BatchJob *jobs, int n_jobs, int tr, int tc, int unit,
                                     int64_t *job_total, int64_t *job_end, int *status,
                                     cudaStream_t st);
// bem_coupling.cu: coupling blocks of the piecewise-linear basis, mixed form
// (Laplace kernels), one entry per lane in warp tiles of 16 rows x 2 columns.
constexpr int kCouplingRows = 16, kCouplingCols = 2;
// Tile shape of the block engines: rows x columns per tile for the prefix
// sums, and prefix units per tile (the piecewise-constant engine counts
// entries and takes kP0Tile consecutive ones per tile).
struct TileShape {
    int tr, tc, unit;
};
inline TileShape block_tile_shape(int basis, bool coupling)
{
    if (coupling) return {kCouplingRows, kCouplingCols, 1};
    if (basis == BEM_P0) return {1, 1, kP0Tile};
    return {kTile, kTile, 1};
}
bool use_coupling_engine(int basis, int kind, int mixed, int allow_touching);
cudaError_t launch_coupling_p1(const MeshView &m, const BlockLaunch &L, const Rule2D &R,
                               const int64_t *prefix, int *status, int grid, cudaStream_t st);
cudaError_t launch_coupling_p1_batch(const BatchJob *jobs, int n_jobs, const int64_t *job_end,
                                     int kind, const Rule2D &R, int *status, int grid,
                                     cudaStream_t st);
// Single and double layer of the same coupling blocks in one pass (the
// distance and its reciprocal square root are shared): jobs carry both outputs.
cudaError_t launch_coupling_p1_fused_batch(const BatchJob *jobs, int n_jobs,
                                           const int64_t *job_end, const Rule2D &R, int *status,
                                           int grid, cudaStream_t st);
// bem_block.cu: support records of all 32-index slices of a cluster list
// (ptr, idx, n_clusters) into sup (cap records); slice gets n_clusters + 1
// entries (exclusive prefix of the slice counts).
cudaError_t launch_build_supports(const MeshView &m, const int32_t *ptr, const int32_t *idx,
                                  int32_t n_clusters, int32_t *slice, int32_t *sup, int64_t cap,
                                  int *status, int grid, cudaStream_t st);
cudaError_t launch_touching_batch(const TouchJob *jobs, int basis, int kind, int cas, int mixed,
                                  const int2 *items, int64_t n, const Rule4D &rule, cudaStream_t st);
// Block buckets of many jobs: job_end[j] = tiles of jobs 0..j (inclusive
// prefix); job_end holds n_jobs + 1 entries, the last one the tile counter of
// the piecewise-linear tile engine (reset by the launch).
cudaError_t launch_block_batch(const BatchJob *jobs, int n_jobs, const int64_t *job_end, int basis,
                               int kind, int mixed, const Rule2D &R, int *status, int grid,
                               cudaStream_t st);
cudaError_t launch_pivot_entries(const MeshView &m, const int32_t *rows, const int32_t *cols,
                                 int64_t n, void *out, const Rule4D *rules /*[4]*/, int kind,
                                 double kappa, int *status, cudaStream_t st, bool absolute,
                                 double eta = 0.0);

// bem_order.cu: learned-order near field of one piecewise-constant job
cudaError_t learned_alloc(LearnedScratch &S, int64_t tiles);
void learned_free(LearnedScratch &S);
int learned_rules(bem_ctx *ctx, Rule4D *rules);   // the 6 classes' FP64 4D rules
cudaError_t learned_launches(const MeshView &mv, const BlockLaunch &L, const int64_t *prefix,
                             const ::bem_mlp *model, float conf, const LearnedScratch &S,
                             const Rule4D *rules, int precision, int num_sms, int *status,
                             cudaStream_t st, bem_ctx *prof_ctx);
int run_learned_p0(bem_ctx *ctx, const MeshView &mv, const BlockLaunch &L, const int64_t *prefix,
                   int precision);

}  // namespace bem
