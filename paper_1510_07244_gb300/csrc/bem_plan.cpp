// Persistent batched driver: a plan gathers many block lists (near-field and
// coupling jobs of any meshes and kernels), groups them into buckets that
// share one kernel instantiation (basis, kernel, regular rule, precision; for
// touching pairs also the case and its order), and issues one launch per
// bucket: every bucket's kernel drains the tiles of all its jobs.  The launch
// sequence can be captured once into a CUDA graph and replayed per step, and
// each bucket's grid can be picked by an autotuner that times candidates on
// the plan's own data.  This replaces the paper's CPU list building, list
// size tuning and worker threads (Section 3, Algorithms 1-4) by device-side
// lists and one graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "bem_internal.h"

using namespace bem;

namespace {

struct TouchBucket {
    int basis, kind, cas, mixed;
    Rule4D rule;
    int2 *items = nullptr;
    int64_t n = 0;
    std::string name;
};

struct BlockBucket {
    int basis, kind, mixed;
    bool coupling = false;   // coupling engine (16 x 2 entry tiles) instead of the tile engine
    bool fused = false;      // coupling engine, single and double layer of the same blocks
    Rule2D r2;
    std::vector<BatchJob> host_jobs;
    BatchJob *jobs = nullptr;
    int64_t *job_total = nullptr, *job_end = nullptr;
    int grid_mult = 0;
    std::string key, name;
};

// Support records of one cluster list of one mesh, shared by every P1 tile
// engine job that uses the list (rows or columns).
struct SupTable {
    MeshView m;
    const int32_t *ptr, *idx;
    int32_t n;
    int32_t *slice = nullptr, *sup = nullptr;
    int64_t cap = 0;
};

}  // namespace

struct bem_plan {
    int flags = 0;
    cudaStream_t cap = nullptr;
    std::vector<void *> allocs;
    TouchJob *touch_jobs = nullptr;
    std::vector<TouchBucket> tb;
    std::vector<BlockBucket> bb;
    std::vector<SupTable> sup;
    std::vector<GuardSet> guards;     // cancellation guard per set of orders
    // learned-order jobs (piecewise constant): each with its tile prefix sums
    // and scratch; the order model and confidence captured at creation
    struct Learned {
        MeshView m;
        BlockLaunch L;
        int64_t *prefix = nullptr;
        LearnedScratch S;
        int precision = 0;
    };
    std::vector<Learned> learned;
    const ::bem_mlp *model = nullptr;
    float conf = 0.0f;
    Rule4D lrules[6];
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<bem_prof_rec> prof;   // event pairs recorded around each launch
    bool prof_outstanding = false;
};

namespace {

template <class T>
cudaError_t plan_alloc(bem_plan *p, T **ptr, size_t count)
{
    cudaError_t e = cudaMalloc((void **)ptr, std::max<size_t>(1, count) * sizeof(T));
    if (e == cudaSuccess) p->allocs.push_back(*ptr);
    return e;
}

template <class T>
cudaError_t plan_upload(bem_plan *p, T **ptr, const std::vector<T> &h)
{
    cudaError_t e = plan_alloc(p, ptr, h.size());
    if (e == cudaSuccess && !h.empty())
        e = cudaMemcpy(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

void plan_free(bem_plan *p)
{
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto &r : p->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (void *a : p->allocs) cudaFree(a);
    for (auto &l : p->learned) learned_free(l.S);
    if (p->cap) cudaStreamDestroy(p->cap);
    delete p;
}

int default_mult(const BlockBucket &b)
{
    if (b.coupling) return 4;
    return b.basis == BEM_P0 ? 8 : (b.mixed ? 4 : 2);
}

std::vector<int> candidates(const BlockBucket &b)
{
    if (b.coupling) return {3, 4, 6};
    if (b.basis == BEM_P0) return {4, 8, 16};
    return b.mixed ? std::vector<int>{4, 8, 12} : std::vector<int>{1, 2, 3};
}

// The support table of (mesh, cluster list), created on first use.  Its size
// comes from the list's current total length (one read from the device):
// sum ceil(|c| / 32) <= total / 32 + n records.
cudaError_t plan_support(bem_plan *p, const MeshView &m, const int32_t *ptr, const int32_t *idx,
                         int32_t n, int *out)
{
    for (size_t k = 0; k < p->sup.size(); ++k) {
        const SupTable &s = p->sup[k];
        if (s.m.geom == m.geom && s.ptr == ptr && s.idx == idx && s.n == n) {
            *out = (int)k;
            return cudaSuccess;
        }
    }
    int32_t total = 0;
    cudaError_t e = cudaMemcpy(&total, ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    SupTable s;
    s.m = m;
    s.ptr = ptr;
    s.idx = idx;
    s.n = n;
    s.cap = (int64_t)std::max(total, 0) / kTile + n + 1;
    if ((e = plan_alloc(p, &s.slice, (size_t)n + 1)) != cudaSuccess) return e;
    if ((e = plan_alloc(p, &s.sup, (size_t)s.cap * kSupInts)) != cudaSuccess) return e;
    *out = (int)p->sup.size();
    p->sup.push_back(s);
    return cudaSuccess;
}

cudaError_t bucket_prefix(bem_ctx *ctx, const BlockBucket &b, cudaStream_t st)
{
    const TileShape ts = block_tile_shape(b.basis, b.coupling);
    return launch_tile_prefix_batch(b.jobs, (int)b.host_jobs.size(), ts.tr, ts.tc, ts.unit,
                                    b.job_total, b.job_end, ctx->status, st);
}

cudaError_t launch_bucket(bem_ctx *ctx, const BlockBucket &b, int mult, cudaStream_t st)
{
    if (b.fused && b.coupling)
        return launch_coupling_p1_fused_batch(b.jobs, (int)b.host_jobs.size(), b.job_end, b.r2,
                                              ctx->status, ctx->num_sms * mult, st);
    if (b.fused)
        return launch_block_batch(b.jobs, (int)b.host_jobs.size(), b.job_end, b.basis, kFusedLaplace,
                                  b.mixed, b.r2, ctx->status, ctx->num_sms * mult, st);
    if (b.coupling)
        return launch_coupling_p1_batch(b.jobs, (int)b.host_jobs.size(), b.job_end, b.kind, b.r2,
                                        ctx->status, ctx->num_sms * mult, st);
    return launch_block_batch(b.jobs, (int)b.host_jobs.size(), b.job_end, b.basis, b.kind, b.mixed,
                              b.r2, ctx->status, ctx->num_sms * mult, st);
}

// Issues the plan's launches on stream st (profiling events when prof != null).
// Events recorded while the stream is being captured must be external record
// nodes, or the graph only uses them for ordering and never records them.
// structure: also issue the passes that only depend on the index lists (the
// support records and the tile prefix sums); static plans skip them after
// creation.
cudaError_t issue(bem_ctx *ctx, bem_plan *p, cudaStream_t st, bool record_prof,
                  bool capturing = false, bool structure = true)
{
    cudaError_t e = cudaSuccess;
    size_t pi = 0;
    auto rec = [&](cudaEvent_t ev) {
        if (capturing) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
        else cudaEventRecord(ev, st);
    };
    auto ev_begin = [&](void) {
        if (record_prof) rec(p->prof[pi].a);
    };
    auto ev_end = [&](void) {
        if (record_prof) rec(p->prof[pi].b);
        ++pi;
    };
    for (auto &t : p->tb) {
        ev_begin();
        e = launch_touching_batch(p->touch_jobs, t.basis, t.kind, t.cas, t.mixed, t.items, t.n, t.rule, st);
        ev_end();
        if (e != cudaSuccess) return e;
    }
    for (auto &s : p->sup) {
        if (!structure) {
            ++pi;
            continue;
        }
        ev_begin();
        e = launch_build_supports(s.m, s.ptr, s.idx, s.n, s.slice, s.sup, s.cap, ctx->status,
                                  ctx->num_sms * 4, st);
        ev_end();
        if (e != cudaSuccess) return e;
    }
    for (auto &b : p->bb) {
        if (!structure) {
            ++pi;
            continue;
        }
        ev_begin();
        e = bucket_prefix(ctx, b, st);
        ev_end();
        if (e != cudaSuccess) return e;
    }
    for (auto &b : p->bb) {
        ev_begin();
        e = launch_bucket(ctx, b, b.grid_mult, st);
        ev_end();
        if (e != cudaSuccess) return e;
    }
    for (auto &l : p->learned) {
        ev_begin();
        if (structure)
            e = launch_tile_prefix_wide(l.L, 1, 1, l.prefix, l.prefix + l.L.n_blocks, ctx->status,
                                        st);
        if (e == cudaSuccess)
            e = learned_launches(l.m, l.L, l.prefix, p->model, p->conf, l.S, p->lrules, l.precision,
                                 ctx->num_sms, ctx->status, st, nullptr);
        ev_end();
        if (e != cudaSuccess) return e;
    }
    for (auto &g : p->guards) {
        ev_begin();
        e = guard_run(g, ctx->num_sms, ctx->status, st);
        ev_end();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int autotune(bem_ctx *ctx, bem_plan *p)
{
    cudaStream_t st = p->cap;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // prerequisites once: touching tables and tile prefix sums
    for (auto &t : p->tb)
        launch_touching_batch(p->touch_jobs, t.basis, t.kind, t.cas, t.mixed, t.items, t.n, t.rule, st);
    for (auto &s : p->sup)
        launch_build_supports(s.m, s.ptr, s.idx, s.n, s.slice, s.sup, s.cap, ctx->status,
                              ctx->num_sms * 4, st);
    for (auto &bk : p->bb)
        bucket_prefix(ctx, bk, st);
    cudaError_t e = cudaStreamSynchronize(st);
    for (auto &bk : p->bb) {
        if (e != cudaSuccess) break;
        auto it = ctx->tuned.find(bk.key);
        if (it != ctx->tuned.end()) {
            bk.grid_mult = it->second;
            continue;
        }
        float best = 1e30f;
        int best_m = bk.grid_mult;
        for (int mult : candidates(bk)) {
            float t_min = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(a, st);
                e = launch_bucket(ctx, bk, mult, st);
                cudaEventRecord(b, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                if (e != cudaSuccess) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, a, b);
                t_min = std::min(t_min, ms);
            }
            if (e != cudaSuccess) break;
            if (t_min < best) {
                best = t_min;
                best_m = mult;
            }
        }
        bk.grid_mult = best_m;
        ctx->tuned[bk.key] = best_m;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "autotune");
    return BEM_OK;
}

}  // namespace

namespace bem {

void plan_drain_profile(bem_ctx *ctx)
{
    for (bem_plan *p : ctx->prof_plans) {
        if (!p->prof_outstanding || p->prof.empty()) continue;
        cudaEventSynchronize(p->prof.back().b);
        for (auto &r : p->prof) prof_accumulate(ctx, r);
        p->prof_outstanding = false;
    }
    ctx->prof_plans.clear();
}

void plan_forget(bem_ctx *ctx) { ctx->prof_plans.clear(); }

}  // namespace bem

extern "C" {

int bem_plan_create(bem_ctx *ctx, const bem_block_job *near_jobs, int32_t n_near,
                    const bem_block_job *coupling_jobs, int32_t n_coupling, int32_t flags,
                    bem_plan **out)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!out || n_near < 0 || n_coupling < 0 || (n_near > 0 && !near_jobs) ||
        (n_coupling > 0 && !coupling_jobs))
        return api_fail(ctx, BEM_ERR_INVALID_ARG, "bad plan arguments");
    *out = nullptr;
    cudaSetDevice(ctx->device);
    bem_plan *p = new bem_plan();
    p->flags = flags;
    cudaError_t e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        plan_free(p);
        return api_cuda_fail(ctx, e, "cudaStreamCreate");
    }

    struct JobInfo {
        const bem_block_job *J;
        Mesh *m;
        Rule2D r2;
        bool near;
        int touch_job;   // index into touch_jobs (near jobs), -1 otherwise
    };
    std::vector<JobInfo> jobs;
    for (int k = 0; k < n_near + n_coupling; ++k) {
        const bem_block_job &J = k < n_near ? near_jobs[k] : coupling_jobs[k - n_near];
        JobInfo ji;
        ji.J = &J;
        ji.near = k < n_near;
        ji.touch_job = -1;
        int rc = api_check_job(ctx, J, ji.r2, &ji.m);
        if (rc == BEM_OK && J.quad.order_mode == BEM_ORDER_LEARNED) {
            if (ji.m->v.basis != BEM_P0)
                rc = api_fail(ctx, BEM_ERR_UNSUPPORTED, "learned orders need the piecewise-constant basis");
            else if (kind_fp64_only(J.kernel.kind))
                rc = api_fail(ctx, BEM_ERR_UNSUPPORTED,
                              "learned orders cover the Laplace kernels and the Helmholtz single layer");
            else if (!ctx->order_model)
                rc = api_fail(ctx, BEM_ERR_INVALID_ARG, "order_mode LEARNED needs bem_set_order_model");
        }
        if (rc) {
            plan_free(p);
            return rc;
        }
        jobs.push_back(ji);
    }

    // touching work of the near jobs: one table per job, items bucketed
    std::vector<TouchJob> tj;
    std::map<std::tuple<int, int, int, int, int>, std::vector<int2>> titems;   // basis,kind,case,mixed,q
    for (auto &ji : jobs) {
        if (!ji.near || ji.J->n_blocks == 0) continue;
        const MeshView &mv = ji.m->v;
        const size_t per = mv.basis == BEM_P0 ? 1 : 9;
        double2 *table = nullptr;
        if ((e = plan_alloc(p, &table, (size_t)mv.ntouch * per)) != cudaSuccess) {
            plan_free(p);
            return api_cuda_fail(ctx, e, "cudaMalloc(plan touching table)");
        }
        TouchJob t;
        t.m = mv;
        t.m.table = table;
        t.kappa = ji.J->kernel.kappa;
        t.eta = ji.J->kernel.eta;
        ji.touch_job = (int)tj.size();
        tj.push_back(t);
        const int qs[4] = {0, ji.J->quad.q_vertex, ji.J->quad.q_edge, ji.J->quad.q_identical};
        for (int c = kVertex; c <= kIdentical; ++c) {
            auto &v = titems[std::make_tuple(mv.basis, ji.J->kernel.kind, c,
                                             touch_in_float(ji.J->quad.precision, c,
                                                            ji.J->kernel.kind), qs[c])];
            for (int idx : ji.m->hlist[c]) v.push_back(make_int2(ji.touch_job, idx));
        }
    }
    if ((e = plan_upload(p, &p->touch_jobs, tj)) != cudaSuccess) {
        plan_free(p);
        return api_cuda_fail(ctx, e, "plan upload");
    }
    static const char *cname[4] = {"", "vertex", "edge", "identical"};
    for (auto &kv : titems) {
        if (kv.second.empty()) continue;
        TouchBucket t;
        std::tie(t.basis, t.kind, t.cas, t.mixed, std::ignore) = kv.first;
        const int q = std::get<4>(kv.first);
        int rc = api_touch_rule(ctx, t.cas, q, t.kind, t.basis, t.mixed != 0, t.rule);
        if (rc) {
            plan_free(p);
            return rc;
        }
        t.n = (int64_t)kv.second.size();
        if ((e = plan_upload(p, &t.items, kv.second)) != cudaSuccess) {
            plan_free(p);
            return api_cuda_fail(ctx, e, "plan upload");
        }
        t.name = std::string("touching_") + cname[t.cas];
        p->tb.push_back(t);
    }

    // jobs of the single and the double layer over the same blocks of the same
    // mesh (same device arrays, same regular rule, both near field or both
    // coupling) run fused in the float forms of the piecewise-linear basis: the
    // double-layer job's output (and touching table) ride on the single-layer
    // job, which then computes both
    std::vector<void *> out2(jobs.size(), nullptr);
    std::vector<const double2 *> table2(jobs.size(), nullptr);
    std::vector<char> absorbed(jobs.size(), 0);
    auto same_blocks = [](const bem_block_job &x, const bem_block_job &y) {
        return x.mesh_id == y.mesh_id && x.row_ptr == y.row_ptr && x.row_idx == y.row_idx &&
               x.col_ptr == y.col_ptr && x.col_idx == y.col_idx && x.blk_row == y.blk_row &&
               x.blk_col == y.blk_col && x.blk_off == y.blk_off && x.n_blocks == y.n_blocks &&
               x.n_row_clusters == y.n_row_clusters && x.n_col_clusters == y.n_col_clusters &&
               x.quad.precision == y.quad.precision && x.quad.regular_rule == y.quad.regular_rule &&
               x.quad.q_regular == y.quad.q_regular;
    };
    for (size_t x = 0; x < jobs.size(); ++x) {
        const bem_block_job &Jx = *jobs[x].J;
        if (Jx.n_blocks == 0 || Jx.kernel.kind != BEM_LAPLACE_SLP || out2[x] ||
            jobs[x].m->v.basis != BEM_P1 || !is_mixed(Jx.quad.precision))
            continue;
        for (size_t y = 0; y < jobs.size(); ++y) {
            const bem_block_job &Jy = *jobs[y].J;
            if (y == x || jobs[y].near != jobs[x].near || absorbed[y] ||
                Jy.kernel.kind != BEM_LAPLACE_DLP || !same_blocks(Jx, Jy) || Jy.out == Jx.out)
                continue;
            out2[x] = Jy.out;
            if (jobs[x].near) table2[x] = tj[jobs[y].touch_job].m.table;
            absorbed[y] = 1;
            break;
        }
    }

    // block buckets
    std::map<std::string, int> bindex;
    std::map<std::string, int> gindex;   // guard sets by orders
    for (size_t jx = 0; jx < jobs.size(); ++jx) {
        auto &ji = jobs[jx];
        const bem_block_job &J = *ji.J;
        if (J.n_blocks == 0 || absorbed[jx]) continue;
        if (J.quad.order_mode == BEM_ORDER_LEARNED) {
            bem_plan::Learned l;
            l.m = ji.m->v;
            l.m.table = ji.touch_job >= 0 ? tj[ji.touch_job].m.table : nullptr;
            BlockLaunch &L = l.L;
            L.row_ptr = J.row_ptr;
            L.row_idx = J.row_idx;
            L.col_ptr = J.col_ptr;
            L.col_idx = J.col_idx;
            L.n_row_clusters = J.n_row_clusters;
            L.n_col_clusters = J.n_col_clusters;
            L.blk_row = J.blk_row;
            L.blk_col = J.blk_col;
            L.blk_off = J.blk_off;
            L.n_blocks = J.n_blocks;
            L.out = J.out;
            L.kind = J.kernel.kind;
            L.kappa = J.kernel.kappa;
            L.lower_only = 0;
            L.allow_touching = ji.near ? 1 : 0;
            L.mixed = is_mixed(J.quad.precision) ? 1 : 0;
            l.precision = J.quad.precision;
            // the entry count sizes the job's scratch: one prefix pass now
            int64_t entries = 0;
            // prefix sums, then the many-CTA pass's chunk totals
            if ((e = plan_alloc(p, &l.prefix, (size_t)(J.n_blocks + prefix_chunks(J.n_blocks)))) !=
                    cudaSuccess ||
                (e = launch_tile_prefix_wide(L, 1, 1, l.prefix, l.prefix + J.n_blocks, ctx->status,
                                             p->cap)) != cudaSuccess ||
                (e = cudaMemcpyAsync(&entries, l.prefix + (J.n_blocks - 1), sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, p->cap)) != cudaSuccess ||
                (e = cudaStreamSynchronize(p->cap)) != cudaSuccess ||
                (e = learned_alloc(l.S, (entries + kP0Tile - 1) / kP0Tile)) != cudaSuccess) {
                learned_free(l.S);
                plan_free(p);
                return api_cuda_fail(ctx, e, "learned plan job");
            }
            p->learned.push_back(l);
            continue;
        }
        const int mixed = is_mixed(J.quad.precision) && !kind_fp64_only(J.kernel.kind) &&
                          !(J.kernel.kind == BEM_HELMHOLTZ_SLP && ji.m->v.basis == BEM_P1);
        const bool coupling = use_coupling_engine(ji.m->v.basis, J.kernel.kind, mixed, ji.near ? 1 : 0);
        const bool fused = out2[jx] != nullptr;
        char key[96];
        std::snprintf(key, sizeof key, "b%d k%d np%d m%d r%d q%d c%d f%d", ji.m->v.basis,
                      J.kernel.kind, ji.r2.np, mixed, J.quad.regular_rule, J.quad.q_regular,
                      coupling ? 1 : 0, fused ? 1 : 0);
        auto it = bindex.find(key);
        if (it == bindex.end()) {
            BlockBucket b;
            b.basis = ji.m->v.basis;
            b.kind = J.kernel.kind;
            b.mixed = mixed;
            b.coupling = coupling;
            b.fused = fused;
            b.r2 = ji.r2;
            b.key = key;
            b.name = coupling ? "coupling_p1" : (b.basis == BEM_P0 ? "block_p0" : "block_p1");
            b.grid_mult = default_mult(b);
            bindex[key] = (int)p->bb.size();
            p->bb.push_back(b);
            it = bindex.find(key);
        }
        BlockBucket &b = p->bb[it->second];
        BatchJob bj;
        bj.m = ji.m->v;
        bj.m.table = ji.touch_job >= 0 ? tj[ji.touch_job].m.table : nullptr;
        BlockLaunch &L = bj.L;
        L.row_ptr = J.row_ptr;
        L.row_idx = J.row_idx;
        L.col_ptr = J.col_ptr;
        L.col_idx = J.col_idx;
        L.n_row_clusters = J.n_row_clusters;
        L.n_col_clusters = J.n_col_clusters;
        L.blk_row = J.blk_row;
        L.blk_col = J.blk_col;
        L.blk_off = J.blk_off;
        L.n_blocks = J.n_blocks;
        L.out = J.out;
        L.out2 = out2[jx];
        L.table2 = table2[jx];
        L.kind = J.kernel.kind;
        L.kappa = J.kernel.kappa;
        L.lower_only = 0;
        L.allow_touching = ji.near ? 1 : 0;
        L.mixed = mixed;
        L.eta = J.kernel.eta;
        if (b.basis == BEM_P0 && b.kind == BEM_LAPLACE_DLP && mixed) {
            // cancellation guard: packed (value, sum of |terms|) outputs, then
            // the guard pass of this job's orders
            L.guard = 1;
            char gk[64];
            std::snprintf(gk, sizeof gk, "%d %d %d %d %d", J.quad.regular_rule, J.quad.q_regular,
                          J.quad.q_vertex, J.quad.q_edge, J.quad.q_identical);
            auto gi = gindex.find(gk);
            if (gi == gindex.end()) {
                GuardSet g;
                g.r2 = ji.r2;
                const int qq[4] = {J.quad.q_regular, J.quad.q_vertex, J.quad.q_edge, J.quad.q_identical};
                for (int c = 0; c < 4; ++c) {
                    int rc = c == kRegular
                                 ? api_get_rule4(ctx, c, J.quad.regular_rule, qq[c], g.rules[c])
                                 : api_touch_rule(ctx, c, qq[c], L.kind, b.basis, true, g.rules[c]);
                    if (rc) {
                        plan_free(p);
                        return rc;
                    }
                }
                gindex[gk] = (int)p->guards.size();
                p->guards.push_back(g);
                gi = gindex.find(gk);
            }
            cudaError_t eg = guard_add(p->guards[gi->second], bj.m, L, p->cap);
            if (eg != cudaSuccess) {
                plan_free(p);
                return api_cuda_fail(ctx, eg, "guard set-up");
            }
        }
        if (b.basis == BEM_P1 && !b.coupling) {
            // the tile engine reads per-slice support records built once per run
            int rows = -1, cols = -1;
            cudaError_t es = plan_support(p, ji.m->v, J.row_ptr, J.row_idx, J.n_row_clusters, &rows);
            if (es == cudaSuccess)
                es = plan_support(p, ji.m->v, J.col_ptr, J.col_idx, J.n_col_clusters, &cols);
            if (es != cudaSuccess) {
                plan_free(p);
                return api_cuda_fail(ctx, es, "plan support tables");
            }
            L.sup_r = p->sup[rows].sup;
            L.slice_r = p->sup[rows].slice;
            L.cap_r = p->sup[rows].cap;
            L.sup_c = p->sup[cols].sup;
            L.slice_c = p->sup[cols].slice;
            L.cap_c = p->sup[cols].cap;
        }
        int64_t *prefix = nullptr;
        if ((e = plan_alloc(p, &prefix, (size_t)J.n_blocks)) != cudaSuccess) {
            plan_free(p);
            return api_cuda_fail(ctx, e, "cudaMalloc(plan prefix)");
        }
        bj.prefix = prefix;
        b.host_jobs.push_back(bj);
    }
    for (auto &b : p->bb) {
        const size_t nj = b.host_jobs.size();
        if ((e = plan_upload(p, &b.jobs, b.host_jobs)) != cudaSuccess ||
            (e = plan_alloc(p, &b.job_total, nj)) != cudaSuccess ||
            (e = plan_alloc(p, &b.job_end, nj + 1)) != cudaSuccess) {   // + tile counter
            plan_free(p);
            return api_cuda_fail(ctx, e, "plan upload");
        }
    }
    if (!p->learned.empty()) {
        p->model = ctx->order_model;
        p->conf = ctx->order_conf;
        int rc = learned_rules(ctx, p->lrules);
        if (rc) {
            plan_free(p);
            return rc;
        }
    }
    for (auto &g : p->guards) {
        char *buf = nullptr;
        if ((e = plan_alloc(p, &buf, guard_bytes(g))) != cudaSuccess ||
            (e = guard_layout(g, buf, p->cap)) != cudaSuccess ||
            (e = cudaStreamSynchronize(p->cap)) != cudaSuccess) {
            plan_free(p);
            return api_cuda_fail(ctx, e, "guard buffers");
        }
    }
    // profiling events: one pair per launch group of issue()
    const size_t nt = p->tb.size(), ns = p->sup.size(), nb = p->bb.size(), ng = p->guards.size();
    const size_t nl = p->learned.size();
    for (size_t k = 0; k < nt + ns + 2 * nb + nl + ng; ++k) {
        bem_prof_rec r;
        cudaEventCreate(&r.a);
        cudaEventCreate(&r.b);
        if (k < nt) r.name = p->tb[k].name;
        else if (k < nt + ns) r.name = "supports";
        else if (k < nt + ns + nb) r.name = "tile_prefix";
        else if (k < nt + ns + 2 * nb) r.name = p->bb[k - nt - ns - nb].name;
        else if (k < nt + ns + 2 * nb + nl) r.name = "learned";
        else r.name = "guard";
        // static plans build the support records and tile prefix sums once
        r.skipped = (flags & BEM_PLAN_STATIC_LISTS) && k >= nt && k < nt + ns + nb;
        p->prof.push_back(r);
    }

    if (flags & BEM_PLAN_AUTOTUNE) {
        int rc = autotune(ctx, p);
        if (rc) {
            plan_free(p);
            return rc;
        }
    } else {
        // one direct issue sets the kernels' shared-memory attributes before any capture
        e = issue(ctx, p, p->cap, false);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->cap);
        if (e != cudaSuccess) {
            plan_free(p);
            return api_cuda_fail(ctx, e, "plan warm-up");
        }
    }
    if (flags & BEM_PLAN_GRAPH) {
        e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = issue(ctx, p, p->cap, (flags & BEM_PLAN_PROFILE) != 0, true,
                                   !(flags & BEM_PLAN_STATIC_LISTS));
            e = cudaStreamEndCapture(p->cap, &p->graph);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (e != cudaSuccess) {
            plan_free(p);
            return api_cuda_fail(ctx, e, "graph capture");
        }
    }
    *out = p;
    return BEM_OK;
}

int bem_plan_run(bem_ctx *ctx, bem_plan *p)
{
    if (!ctx || !p) return BEM_ERR_INVALID_ARG;
    const bool prof = (p->flags & BEM_PLAN_PROFILE) && ctx->profile && !p->prof.empty();
    if (p->prof_outstanding && !p->prof.empty()) {
        // the previous run's launch times are added before the events are reused
        cudaEventSynchronize(p->prof.back().b);
        for (auto &r : p->prof) prof_accumulate(ctx, r);
        p->prof_outstanding = false;
    }
    cudaError_t e;
    if (p->exec) e = cudaGraphLaunch(p->exec, ctx->stream);
    else e = issue(ctx, p, ctx->stream, prof, false, !(p->flags & BEM_PLAN_STATIC_LISTS));
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "plan run");
    if (prof) {
        p->prof_outstanding = true;
        if (std::find(ctx->prof_plans.begin(), ctx->prof_plans.end(), p) == ctx->prof_plans.end())
            ctx->prof_plans.push_back(p);
    }
    return BEM_OK;
}

int bem_plan_destroy(bem_ctx *ctx, bem_plan *p)
{
    if (!ctx || !p) return BEM_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    cudaStreamSynchronize(p->cap);
    ctx->prof_plans.erase(std::remove(ctx->prof_plans.begin(), ctx->prof_plans.end(), p),
                          ctx->prof_plans.end());
    plan_free(p);
    return BEM_OK;
}

int bem_plan_info(bem_ctx *ctx, bem_plan *p, int32_t *n_touch_launches, int32_t *n_block_launches,
                  int32_t *n_aux_launches, int32_t *grid_mult, int32_t cap)
{
    if (!ctx || !p) return BEM_ERR_INVALID_ARG;
    if (n_touch_launches) *n_touch_launches = (int32_t)p->tb.size();
    if (n_block_launches) *n_block_launches = (int32_t)p->bb.size();
    // per block bucket: tile prefix sums and job scan; per support table:
    // slice prefix and record build
    // (static plans: without the list-derived passes); a guard set launches
    // row maxima, selection and the disjoint recomputation, plus the touching
    // one when it has near-field jobs; a learned job selection, scan (three
    // launches), offsets, compaction and six class evaluations after its prefix
    // sums
    const bool stat = (p->flags & BEM_PLAN_STATIC_LISTS) != 0;
    int64_t guard_launches = 0;
    for (const auto &g : p->guards) guard_launches += g.cap_t > 0 ? 4 : 3;
    int64_t n_learned = 12 * (int64_t)p->learned.size();
    if (!stat)   // prefix sums: one CTA, or two launches over many CTAs for long lists
        for (const auto &l : p->learned) n_learned += l.L.n_blocks > kPrefixChunk ? 2 : 1;
    if (n_aux_launches)
        *n_aux_launches = (int32_t)((stat ? 0 : 2 * p->bb.size() + 2 * p->sup.size()) +
                                    guard_launches + n_learned);
    for (int k = 0; grid_mult && k < cap && k < (int)p->bb.size(); ++k) grid_mult[k] = p->bb[k].grid_mult;
    return BEM_OK;
}

int bem_plan_learned_counts(bem_ctx *ctx, bem_plan *p, int64_t *counts)
{
    if (!ctx || !p || !counts) return BEM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    for (int c = 0; c < 6; ++c) counts[c] = 0;
    for (auto &l : p->learned) {
        int k[8] = {0};
        if (e == cudaSuccess) e = cudaMemcpy(k, l.S.small, sizeof(k), cudaMemcpyDeviceToHost);
        for (int c = 0; c < 6; ++c) counts[c] += k[c];
    }
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "learned counts");
    return BEM_OK;
}

int bem_plan_guard_stats(bem_ctx *ctx, bem_plan *p, int64_t *guarded_entries, int64_t *recomputed)
{
    if (!ctx || !p || !guarded_entries || !recomputed) return BEM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    int64_t n = 0, r = 0;
    for (auto &g : p->guards) {
        unsigned long long c[2] = {0, 0};   // disjoint and touching entries listed
        if (e == cudaSuccess)
            e = cudaMemcpy(c, g.d_count, sizeof(c), cudaMemcpyDeviceToHost);
        n += g.entries;
        r += std::min<int64_t>((int64_t)c[0], g.cap) + std::min<int64_t>((int64_t)c[1], g.cap_t);
    }
    if (e != cudaSuccess) return api_cuda_fail(ctx, e, "guard statistics");
    *guarded_entries = n;
    *recomputed = r;
    return BEM_OK;
}

}  // extern "C"
