// Host side of the C ABI: context, mesh upload with the touching-pair
// classification (host planner), argument validation and kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "bem_internal.h"
#include "bem_mesh_plan.h"

using namespace bem;

namespace bem {

static cudaEvent_t prof_event(bem_ctx *c)
{
    if (!c->prof_free.empty()) {
        cudaEvent_t e = c->prof_free.back();
        c->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(bem_ctx *c, const char *name) : ctx(c), on(c && c->profile)
{
    if (!on) return;
    rec.name = name;
    rec.a = prof_event(c);
    rec.b = prof_event(c);
    cudaEventRecord(rec.a, c->stream);
}

ProfScope::~ProfScope()
{
    if (!on) return;
    cudaEventRecord(rec.b, ctx->stream);
    ctx->prof_pending.push_back(rec);
}

}  // namespace bem

namespace {

int fail(bem_ctx *ctx, int code, const char *msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(bem_ctx *ctx, cudaError_t e, const char *where)
{
    if (ctx) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
        ctx->err = buf;
    }
    return e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA;
}

template <class T>
int upload(bem_ctx *ctx, Mesh *m, const std::vector<T> &h, T **d)
{
    const size_t bytes = std::max<size_t>(1, h.size()) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)d, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    m->allocs.push_back(*d);
    if (!h.empty()) {
        e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy");
    }
    return BEM_OK;
}

void free_mesh(Mesh *m)
{
    for (void *p : m->allocs) cudaFree(p);
    delete m;
}

Mesh *get_mesh(bem_ctx *ctx, int id)
{
    auto it = ctx->meshes.find(id);
    return it == ctx->meshes.end() ? nullptr : it->second;
}

int check_quad(bem_ctx *ctx, const bem_quad_desc *q, Rule2D &r2, bool block_rule = true)
{
    if (!q) return fail(ctx, BEM_ERR_INVALID_ARG, "null quadrature descriptor");
    if (q->precision != BEM_FP64 && !is_mixed(q->precision))
        return fail(ctx, BEM_ERR_INVALID_ARG,
                    "precision must be BEM_FP64, BEM_MIXED or BEM_MIXED_FULL");
    if (q->order_mode != BEM_ORDER_FIXED && q->order_mode != BEM_ORDER_LEARNED)
        return fail(ctx, BEM_ERR_INVALID_ARG, "order_mode must be BEM_ORDER_FIXED or BEM_ORDER_LEARNED");
    for (int v : {q->q_identical, q->q_edge, q->q_vertex})
        if (v < 1 || v > 20) return fail(ctx, BEM_ERR_INVALID_ARG, "singular order must be in [1, 20]");
    if (!block_rule) {
        // entries evaluated with 4D tables: any Duffy order up to 20, or TRI7
        if (q->regular_rule != BEM_RULE_TRI7 &&
            (q->regular_rule != BEM_RULE_DUFFY || q->q_regular < 1 || q->q_regular > 20))
            return fail(ctx, BEM_ERR_INVALID_ARG, "regular rule must be TRI7 or DUFFY with q in [1, 20]");
        return BEM_OK;
    }
    if (!make_rule2d(q->regular_rule, q->q_regular, r2))
        return fail(ctx, BEM_ERR_UNSUPPORTED, "regular rule must be TRI7 or DUFFY with q in [2, 4]");
    if (r2.np != 4 && r2.np != 7 && r2.np != 9 && r2.np != 16)
        return fail(ctx, BEM_ERR_UNSUPPORTED, "regular rule must be TRI7 or DUFFY with q in [2, 4]");
    return BEM_OK;
}

int check_kernel(bem_ctx *ctx, const bem_kernel_desc *k)
{
    if (!k) return fail(ctx, BEM_ERR_INVALID_ARG, "null kernel descriptor");
    if (k->kind < BEM_LAPLACE_SLP || k->kind > BEM_HELMHOLTZ_BW)
        return fail(ctx, BEM_ERR_INVALID_ARG, "unknown kernel kind");
    if (!std::isfinite(k->kappa)) return fail(ctx, BEM_ERR_INVALID_ARG, "kappa is not finite");
    if (!std::isfinite(k->eta)) return fail(ctx, BEM_ERR_INVALID_ARG, "eta is not finite");
    return BEM_OK;
}

// Rules of the context, built on first use: regular rules by (rule, q),
// touching rules by q with rule 0 (q^4 points) or kRuleXiOut (xi integrated out).
int get_rule4(bem_ctx *ctx, int cas, int rule, int q, Rule4D &out)
{
    const bool xi = cas != kRegular && rule == kRuleXiOut;
    auto key = std::make_tuple(cas, cas == kRegular || xi ? rule : 0, q);
    auto it = ctx->rules4.find(key);
    if (it != ctx->rules4.end()) {
        out = it->second;
        return BEM_OK;
    }
    std::vector<double> soa;
    if (!make_rule4d_host(cas, rule, q, soa, xi)) return fail(ctx, BEM_ERR_INVALID_ARG, "bad rule");
    Rule4D r;
    r.xi = xi ? 1 : 0;
    r.q = q;
    r.n = (int)(soa.size() / kRuleCols);
    cudaError_t e = cudaMalloc((void **)&r.d, soa.size() * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(rule)");
    e = cudaMemcpy(r.d, soa.data(), soa.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(rule)");
    std::vector<float> sf(soa.begin(), soa.end());
    e = cudaMalloc((void **)&r.f, sf.size() * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(rule)");
    e = cudaMemcpy(r.f, sf.data(), sf.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(rule)");
    // the rounding remainders: (f, fl) is the rule as double-float pairs
    std::vector<float> sl(soa.size());
    for (size_t k = 0; k < soa.size(); ++k) sl[k] = (float)(soa[k] - (double)sf[k]);
    e = cudaMalloc((void **)&r.fl, sl.size() * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(rule)");
    e = cudaMemcpy(r.fl, sl.data(), sl.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(rule)");
    ctx->rules4[key] = r;
    out = r;
    return BEM_OK;
}

int touch_rule(bem_ctx *ctx, int cas, int q, int kind, int basis, bool f32, Rule4D &out)
{
    return get_rule4(ctx, cas, touch_xi_out(kind, basis, q, f32) ? kRuleXiOut : 0, q, out);
}

// Evaluates every touching pair of the mesh into its touching table.
int run_touching(bem_ctx *ctx, Mesh *m, const bem_kernel_desc *k, const bem_quad_desc *q)
{
    const int qs[4] = {0, q->q_vertex, q->q_edge, q->q_identical};
    for (int cas = kVertex; cas <= kIdentical; ++cas) {
        if (m->nlist[cas] == 0) continue;
        Rule4D r;
        const int f32 = touch_in_float(q->precision, cas, k->kind);
        int rc = touch_rule(ctx, cas, qs[cas], k->kind, m->v.basis, f32 != 0, r);
        if (rc) return rc;
        static const char *names[4] = {"", "touching_vertex", "touching_edge",
                                       "touching_identical"};
        ProfScope ps(ctx, names[cas]);
        cudaError_t e = launch_touching(m->v, cas, m->list[cas], m->nlist[cas], r, k->kind,
                                        k->kappa, f32, ctx->stream, k->eta);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "touching kernel");
    }
    return BEM_OK;
}

int ensure_prefix(bem_ctx *ctx, int64_t n)
{
    if (n <= ctx->tile_prefix_cap) return BEM_OK;
    if (ctx->tile_prefix) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->tile_prefix);
        ctx->tile_prefix = nullptr;
    }
    const int64_t cap = std::max<int64_t>(n, 1024);
    cudaError_t e = cudaMalloc((void **)&ctx->tile_prefix, cap * sizeof(int64_t));
    if (e != cudaSuccess) {
        ctx->tile_prefix_cap = 0;
        return cuda_fail(ctx, e, "cudaMalloc(tile prefix)");
    }
    ctx->tile_prefix_cap = cap;
    return BEM_OK;
}

// Guard pass of one guarded job (bem_guard.cu) in the context's scratch.
int run_guard(bem_ctx *ctx, Mesh *m, const BlockLaunch &L, const bem_quad_desc &q,
              const Rule2D &r2)
{
    GuardSet g;
    g.r2 = r2;
    const int qq[4] = {q.q_regular, q.q_vertex, q.q_edge, q.q_identical};
    for (int c = 0; c < 4; ++c) {
        int rc = c == kRegular ? get_rule4(ctx, c, q.regular_rule, qq[c], g.rules[c])
                               : touch_rule(ctx, c, qq[c], L.kind, m->v.basis, true, g.rules[c]);
        if (rc) return rc;
    }
    cudaError_t e = guard_add(g, m->v, L, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "guard set-up");
    const size_t bytes = guard_bytes(g);
    if (bytes > ctx->guard_cap) {
        if (ctx->guard_buf) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->guard_buf);
            ctx->guard_buf = nullptr;
            ctx->guard_cap = 0;
        }
        e = cudaMalloc(&ctx->guard_buf, bytes);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(guard)");
        ctx->guard_cap = bytes;
    }
    e = guard_layout(g, ctx->guard_buf, ctx->stream);
    if (e == cudaSuccess) {
        ProfScope ps(ctx, "guard");
        e = guard_run(g, ctx->num_sms, ctx->status, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "guard pass");
    return BEM_OK;
}

int run_blocks(bem_ctx *ctx, const bem_block_job *jobs, int32_t n_jobs, bool allow_touching,
               int lower_only)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(ctx, BEM_ERR_INVALID_ARG, "bad job list");
    for (int j = 0; j < n_jobs; ++j) {
        const bem_block_job &J = jobs[j];
        Mesh *m = get_mesh(ctx, J.mesh_id);
        if (!m) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
        int rc = check_kernel(ctx, &J.kernel);
        if (rc) return rc;
        Rule2D r2;
        rc = check_quad(ctx, &J.quad, r2);
        if (rc) return rc;
        if (J.n_blocks < 0) return fail(ctx, BEM_ERR_INVALID_ARG, "negative block count");
        if (J.n_blocks == 0) continue;
        if (!J.row_ptr || !J.row_idx || !J.col_ptr || !J.col_idx || !J.blk_row || !J.blk_col ||
            !J.blk_off || !J.out || J.n_row_clusters < 1 || J.n_col_clusters < 1)
            return fail(ctx, BEM_ERR_INVALID_ARG, "null pointer or empty cluster list");
        if (kind_complex(J.kernel.kind) && (reinterpret_cast<uintptr_t>(J.out) & 15))
            return fail(ctx, BEM_ERR_INVALID_ARG, "complex output must be 16-byte aligned");
        if (m->v.basis == BEM_P1 && m->v.maxdeg > kMaxDegP1)
            return fail(ctx, BEM_ERR_UNSUPPORTED, "vertex degree above 16 (piecewise linear)");
        if (allow_touching) {
            rc = run_touching(ctx, m, &J.kernel, &J.quad);
            if (rc) return rc;
        }
        rc = ensure_prefix(ctx, J.n_blocks + prefix_chunks(J.n_blocks));   // + chunk totals
        if (rc) return rc;
        BlockLaunch L;
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
        L.lower_only = lower_only;
        L.allow_touching = allow_touching ? 1 : 0;
        L.mixed = is_mixed(J.quad.precision) && !kind_fp64_only(L.kind) ? 1 : 0;
        L.eta = J.kernel.eta;
        const bool coupling = J.quad.order_mode == BEM_ORDER_FIXED &&
                              use_coupling_engine(m->v.basis, L.kind, L.mixed, L.allow_touching);
        // learned orders run on the piecewise-constant engine's flat tiles
        const bool learned = J.quad.order_mode == BEM_ORDER_LEARNED;
        const TileShape ts = block_tile_shape(learned ? BEM_P0 : m->v.basis, coupling);
        const int tr = ts.tr, tc = ts.tc;
        cudaError_t e;
        {
            ProfScope ps(ctx, "tile_prefix");
            e = launch_tile_prefix_wide(L, tr, tc, ctx->tile_prefix, ctx->tile_prefix + J.n_blocks,
                                        ctx->status, ctx->stream);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tile prefix kernel");
        if (J.quad.order_mode == BEM_ORDER_LEARNED) {
            if (kind_fp64_only(J.kernel.kind))
                return fail(ctx, BEM_ERR_UNSUPPORTED,
                            "learned orders cover the Laplace kernels and the Helmholtz single layer");
            if (m->v.basis != BEM_P0)
                return fail(ctx, BEM_ERR_UNSUPPORTED, "learned orders need the piecewise-constant basis");
            if (lower_only)
                return fail(ctx, BEM_ERR_UNSUPPORTED,
                            "learned orders are available for bem_near_field and bem_coupling_blocks");
            ProfScope ps(ctx, "learned_p0");
            rc = run_learned_p0(ctx, m->v, L, ctx->tile_prefix, J.quad.precision);
            if (rc) return rc;
            continue;
        }
        if (coupling) {
            ProfScope ps(ctx, "coupling_p1");
            e = launch_coupling_p1(m->v, L, r2, ctx->tile_prefix, ctx->status, ctx->num_sms * 4,
                                   ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "coupling kernel");
            continue;
        }
        const int grid = ctx->num_sms * (m->v.basis == BEM_P0 ? 8 : 2);
        // cancellation guard of the float double layer (not for the lower
        // triangle alone: the guard pass reads every entry of the blocks)
        L.guard = m->v.basis == BEM_P0 && L.kind == BEM_LAPLACE_DLP && L.mixed && !lower_only;
        {
            ProfScope ps(ctx, m->v.basis == BEM_P0 ? "block_p0" : "block_p1");
            e = launch_block_engine(m->v, L, r2, ctx->tile_prefix, ctx->status, grid, ctx->stream);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "block kernel");
        if (L.guard) {
            rc = run_guard(ctx, m, L, J.quad, r2);
            if (rc) return rc;
        }
    }
    return BEM_OK;
}

}  // namespace

namespace bem {

int api_fail(bem_ctx *ctx, int code, const char *msg) { return fail(ctx, code, msg); }
int api_ensure_prefix(bem_ctx *ctx, int64_t n) { return ensure_prefix(ctx, n); }
int api_cuda_fail(bem_ctx *ctx, cudaError_t e, const char *where) { return cuda_fail(ctx, e, where); }
int api_touch_rule(bem_ctx *ctx, int cas, int q, int kind, int basis, bool f32, Rule4D &out)
{
    return touch_rule(ctx, cas, q, kind, basis, f32, out);
}

int api_get_rule4(bem_ctx *ctx, int cas, int rule, int q, Rule4D &out)
{
    return get_rule4(ctx, cas, rule, q, out);
}

int api_check_job(bem_ctx *ctx, const bem_block_job &J, Rule2D &r2, Mesh **mesh)
{
    Mesh *m = get_mesh(ctx, J.mesh_id);
    if (!m) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    int rc = check_kernel(ctx, &J.kernel);
    if (rc) return rc;
    rc = check_quad(ctx, &J.quad, r2);
    if (rc) return rc;
    if (J.n_blocks < 0) return fail(ctx, BEM_ERR_INVALID_ARG, "negative block count");
    if (J.n_blocks > 0 &&
        (!J.row_ptr || !J.row_idx || !J.col_ptr || !J.col_idx || !J.blk_row || !J.blk_col ||
         !J.blk_off || !J.out || J.n_row_clusters < 1 || J.n_col_clusters < 1))
        return fail(ctx, BEM_ERR_INVALID_ARG, "null pointer or empty cluster list");
    if (kind_complex(J.kernel.kind) && (reinterpret_cast<uintptr_t>(J.out) & 15))
        return fail(ctx, BEM_ERR_INVALID_ARG, "complex output must be 16-byte aligned");
    if (m->v.basis == BEM_P1 && m->v.maxdeg > kMaxDegP1)
        return fail(ctx, BEM_ERR_UNSUPPORTED, "vertex degree above 16 (piecewise linear)");
    *mesh = m;
    return BEM_OK;
}

void prof_accumulate(bem_ctx *ctx, const bem_prof_rec &r)
{
    if (r.skipped) return;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto &t = ctx->prof_total[r.name];
    t.first += 1;
    t.second += ms;
}

}  // namespace bem

extern "C" {

int bem_create(bem_ctx **out, int device, void *cuda_stream)
{
    if (!out) return BEM_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return BEM_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return BEM_ERR_CUDA;
    bem_ctx *ctx = new bem_ctx();
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    e = cudaMalloc((void **)&ctx->status, sizeof(int));
    if (e != cudaSuccess) {
        delete ctx;
        return BEM_ERR_OOM;
    }
    cudaMemset(ctx->status, 0, sizeof(int));
    *out = ctx;
    return BEM_OK;
}

int bem_destroy(bem_ctx *ctx)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    plan_forget(ctx);
    for (auto &kv : ctx->meshes) free_mesh(kv.second);
    for (auto &kv : ctx->rules4) {
        cudaFree(kv.second.d);
        cudaFree(kv.second.f);
        cudaFree(kv.second.fl);
    }
    for (auto &r : ctx->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->prof_free) cudaEventDestroy(e);
    cudaFree(ctx->status);
    cudaFree(ctx->tile_prefix);
    cudaFree(ctx->guard_buf);
    learned_free(ctx->learned);
    delete ctx;
    return BEM_OK;
}

const char *bem_last_error(bem_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int bem_sync(bem_ctx *ctx)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    int st = 0;
    e = cudaMemcpy(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    if (st != 0) {
        cudaMemset(ctx->status, 0, sizeof(int));
        return fail(ctx, st, "a kernel reported invalid input (index out of range, or a "
                             "touching pair in a coupling block)");
    }
    return BEM_OK;
}

int bem_mesh_upload(bem_ctx *ctx, const double *verts, int64_t nv, const int32_t *tris,
                    int64_t nt, int32_t basis, int32_t *mesh_id)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!verts || !tris || !mesh_id || nv < 1 || nt < 1 || (basis != BEM_P0 && basis != BEM_P1))
        return fail(ctx, BEM_ERR_INVALID_ARG, "bad mesh arguments");
    if (nt > (int64_t)1 << 28 || nv > (int64_t)1 << 30)
        return fail(ctx, BEM_ERR_UNSUPPORTED, "mesh too large for 32-bit indices");
    for (int64_t k = 0; k < 3 * nt; ++k)
        if (tris[k] < 0 || tris[k] >= nv) return fail(ctx, BEM_ERR_INVALID_ARG, "vertex index out of range");
    for (int64_t k = 0; k < 3 * nv; ++k)
        if (!std::isfinite(verts[k])) return fail(ctx, BEM_ERR_INVALID_ARG, "non-finite vertex");

    // a1: per-triangle records
    std::vector<double> geom((size_t)nt * kGeomStride, 0.0);
    std::vector<int4> tvid((size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *T = tris + 3 * t;
        if (T[0] == T[1] || T[1] == T[2] || T[0] == T[2])
            return fail(ctx, BEM_ERR_DEGENERATE, "triangle with a repeated vertex");
        double v[3][3];
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) v[k][c] = verts[3 * (int64_t)T[k] + c];
        double e1[3], e2[3];
        for (int c = 0; c < 3; ++c) {
            e1[c] = v[1][c] - v[0][c];
            e2[c] = v[2][c] - v[1][c];
        }
        const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double sg = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        const double l2 = std::sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
        if (!(sg > 1e-14 * l1 * l2)) return fail(ctx, BEM_ERR_DEGENERATE, "zero-area triangle");
        double *g = &geom[(size_t)t * kGeomStride];
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) g[3 * k + c] = v[k][c];
        for (int c = 0; c < 3; ++c) g[9 + c] = n[c] / sg;
        g[12] = sg;
        tvid[t] = make_int4(T[0], T[1], T[2], 0);
    }

    // mixed-form records: vertices as float hi + lo, FP64 edge vectors and
    // normal rounded to float (normal also as hi + lo), Gram factor
    std::vector<float> geomf((size_t)nt * kGeomFStride, 0.0f);
    for (int64_t t = 0; t < nt; ++t) {
        const double *g = &geom[(size_t)t * kGeomStride];
        float *f = &geomf[(size_t)t * kGeomFStride];
        for (int k = 0; k < 9; ++k) {
            const float hi = (float)g[k];
            f[k] = hi;
            f[9 + k] = (float)(g[k] - (double)hi);
        }
        for (int c = 0; c < 3; ++c) {
            f[18 + c] = (float)(g[3 + c] - g[c]);
            f[21 + c] = (float)(g[6 + c] - g[3 + c]);
            const float nh = (float)g[9 + c];
            f[24 + c] = nh;
            f[27 + c] = (float)(g[9 + c] - (double)nh);
        }
        f[30] = (float)g[12];
    }

    // vertex -> triangle adjacency and the touching pairs of every triangle
    // with case and vertex orders (a2, mesh part; bem_mesh_plan.cpp)
    TouchPlan P;
    {
        const char *err = nullptr;
        const int rc = plan_touching(tris, nt, nv, P, &err);
        if (rc != BEM_OK) return fail(ctx, rc, err ? err : "touching pairs");
    }
    const std::vector<int> &vt_ptr = P.vt_ptr, &vt_tri = P.vt_tri;
    const std::vector<int> &nb_ptr = P.nb_ptr, &nb_tri = P.nb_tri, &nb_src = P.nb_src;
    const std::vector<unsigned char> &nb_case = P.nb_case, &nb_perm = P.nb_perm;
    const int maxdeg = P.maxdeg;
    std::vector<int> *lists = P.lists;
    // reject coordinates shared by two different vertex indices (such pairs
    // would be treated as disjoint although their triangles touch)
    if (find_duplicate_vertex(verts, nv) >= 0)
        return fail(ctx, BEM_ERR_DEGENERATE, "two vertex indices with equal coordinates");

    cudaSetDevice(ctx->device);
    Mesh *m = new Mesh();
    m->host_hash = mesh_hash(verts, nv, tris, nt);
    MeshView &V = m->v;
    V.nv = nv;
    V.nt = nt;
    V.basis = basis;
    V.maxdeg = maxdeg;
    V.ntouch = (int64_t)nb_tri.size();
    int rc = BEM_OK;
    double *d_geom;
    float *d_geomf;
    int4 *d_tvid;
    int *d_vtp, *d_vtt, *d_nbp, *d_nbt, *d_nbs;
    unsigned char *d_nbc, *d_nbperm;
    if ((rc = upload(ctx, m, geom, &d_geom)) || (rc = upload(ctx, m, geomf, &d_geomf)) ||
        (rc = upload(ctx, m, tvid, &d_tvid)) ||
        (rc = upload(ctx, m, vt_ptr, &d_vtp)) || (rc = upload(ctx, m, vt_tri, &d_vtt)) ||
        (rc = upload(ctx, m, nb_ptr, &d_nbp)) || (rc = upload(ctx, m, nb_tri, &d_nbt)) ||
        (rc = upload(ctx, m, nb_src, &d_nbs)) || (rc = upload(ctx, m, nb_case, &d_nbc)) ||
        (rc = upload(ctx, m, nb_perm, &d_nbperm))) {
        free_mesh(m);
        return rc;
    }
    V.geom = d_geom;
    V.geomf = d_geomf;
    V.tvid = d_tvid;
    V.vt_ptr = d_vtp;
    V.vt_tri = d_vtt;
    V.nb_ptr = d_nbp;
    V.nb_tri = d_nbt;
    V.nb_src = d_nbs;
    V.nb_case = d_nbc;
    V.nb_perm = d_nbperm;
    for (int c = kVertex; c <= kIdentical; ++c) {
        m->nlist[c] = (int64_t)lists[c].size();
        m->hlist[c] = lists[c];
        if ((rc = upload(ctx, m, lists[c], &m->list[c]))) {
            free_mesh(m);
            return rc;
        }
    }
    {
        const size_t per = basis == BEM_P0 ? 1 : 9;
        const size_t bytes = std::max<size_t>(1, (size_t)V.ntouch * per) * sizeof(double2);
        cudaError_t e = cudaMalloc((void **)&V.table, bytes);
        if (e != cudaSuccess) {
            free_mesh(m);
            return cuda_fail(ctx, e, "cudaMalloc(touching table)");
        }
        m->allocs.push_back(V.table);
    }
    {
        const int64_t n = basis == BEM_P0 ? nt : nv;
        std::vector<int> iota((size_t)n);
        for (int64_t k = 0; k < n; ++k) iota[k] = (int)k;
        std::vector<int> csr = {0, (int)n, 0, 0};   // ptr {0, n}, blk_row 0, blk_col 0
        if ((rc = upload(ctx, m, iota, &m->iota)) || (rc = upload(ctx, m, csr, &m->dense_csr))) {
            free_mesh(m);
            return rc;
        }
    }
    m->stats.n_vertices = nv;
    m->stats.n_triangles = nt;
    m->stats.n_identical = m->nlist[kIdentical];
    m->stats.n_edge = m->nlist[kEdge];
    m->stats.n_vertex = m->nlist[kVertex];
    m->stats.max_vertex_degree = maxdeg;
    m->stats.basis = basis;
    const int id = ctx->next_mesh++;
    ctx->meshes[id] = m;
    *mesh_id = id;
    return BEM_OK;
}

int bem_mesh_free(bem_ctx *ctx, int32_t mesh_id)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    cudaStreamSynchronize(ctx->stream);
    free_mesh(m);
    ctx->meshes.erase(mesh_id);
    return BEM_OK;
}

int bem_mesh_info(bem_ctx *ctx, int32_t mesh_id, bem_mesh_stats *stats)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m || !stats) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id or null stats");
    *stats = m->stats;
    return BEM_OK;
}

int bem_near_field(bem_ctx *ctx, const bem_block_job *jobs, int32_t n_jobs)
{
    return run_blocks(ctx, jobs, n_jobs, true, 0);
}

int bem_coupling_blocks(bem_ctx *ctx, const bem_block_job *jobs, int32_t n_jobs)
{
    return run_blocks(ctx, jobs, n_jobs, false, 0);
}

static int pivot_impl(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                      const bem_quad_desc *quad, const int32_t *rows, const int32_t *cols,
                      int64_t n, void *out, bool absolute)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    int rc = check_kernel(ctx, kernel);
    if (rc) return rc;
    Rule2D r2;
    rc = check_quad(ctx, quad, r2, false);
    if (rc) return rc;
    if (n < 0) return fail(ctx, BEM_ERR_INVALID_ARG, "negative entry count");
    if (n == 0) return BEM_OK;
    if (!rows || !cols || !out) return fail(ctx, BEM_ERR_INVALID_ARG, "null pointer");
    if (!absolute && kind_complex(kernel->kind) && (reinterpret_cast<uintptr_t>(out) & 15))
        return fail(ctx, BEM_ERR_INVALID_ARG, "complex output must be 16-byte aligned");
    Rule4D rules[4];
    if ((rc = get_rule4(ctx, kRegular, quad->regular_rule, quad->q_regular, rules[kRegular])) ||
        (rc = get_rule4(ctx, kVertex, 0, quad->q_vertex, rules[kVertex])) ||
        (rc = get_rule4(ctx, kEdge, 0, quad->q_edge, rules[kEdge])) ||
        (rc = get_rule4(ctx, kIdentical, 0, quad->q_identical, rules[kIdentical])))
        return rc;
    cudaError_t e;
    {
        ProfScope ps(ctx, "pivot");
        e = launch_pivot_entries(m->v, rows, cols, n, out, rules, kernel->kind, kernel->kappa,
                                 ctx->status, ctx->stream, absolute, kernel->eta);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pivot kernel");
    return BEM_OK;
}

int bem_pivot_entries(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                      const bem_quad_desc *quad, const int32_t *rows, const int32_t *cols,
                      int64_t n, void *out)
{
    return pivot_impl(ctx, mesh_id, kernel, quad, rows, cols, n, out, false);
}

int bem_pivot_entries_absolute(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                               const bem_quad_desc *quad, const int32_t *rows, const int32_t *cols,
                               int64_t n, double *out)
{
    return pivot_impl(ctx, mesh_id, kernel, quad, rows, cols, n, out, true);
}

int bem_assemble_dense(bem_ctx *ctx, int32_t mesh_id, const bem_kernel_desc *kernel,
                       const bem_quad_desc *quad, int32_t lower_only, void *out)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    Mesh *m = get_mesh(ctx, mesh_id);
    if (!m) return fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    if (!out) return fail(ctx, BEM_ERR_INVALID_ARG, "null output");
    bem_block_job J;
    std::memset(&J, 0, sizeof J);
    J.mesh_id = mesh_id;
    if (kernel) J.kernel = *kernel;
    if (quad) J.quad = *quad;
    if (!kernel || !quad) return fail(ctx, BEM_ERR_INVALID_ARG, "null descriptor");
    J.row_ptr = m->dense_csr;
    J.row_idx = m->iota;
    J.n_row_clusters = 1;
    J.col_ptr = m->dense_csr;
    J.col_idx = m->iota;
    J.n_col_clusters = 1;
    J.blk_row = m->dense_csr + 2;
    J.blk_col = m->dense_csr + 3;
    J.blk_off = nullptr;
    J.n_blocks = 1;
    J.out = out;
    // block offset 0: reuse the zero at dense_csr[2..3] as an int64 zero
    J.blk_off = reinterpret_cast<const int64_t *>(m->dense_csr + 2);
    return run_blocks(ctx, &J, 1, true, lower_only ? 1 : 0);
}

int bem_profile_enable(bem_ctx *ctx, int32_t on)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    ctx->profile = on != 0;
    return BEM_OK;
}

int bem_profile_reset(bem_ctx *ctx)
{
    if (!ctx) return BEM_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    for (auto &r : ctx->prof_pending) {
        ctx->prof_free.push_back(r.a);
        ctx->prof_free.push_back(r.b);
    }
    ctx->prof_pending.clear();
    ctx->prof_total.clear();
    return BEM_OK;
}

int bem_profile_read(bem_ctx *ctx, bem_kernel_time *out, int32_t cap, int32_t *n_out)
{
    if (!ctx || (cap > 0 && !out)) return BEM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    for (auto &r : ctx->prof_pending) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &t = ctx->prof_total[r.name];
        t.first += 1;
        t.second += ms;
        ctx->prof_free.push_back(r.a);
        ctx->prof_free.push_back(r.b);
    }
    ctx->prof_pending.clear();
    plan_drain_profile(ctx);
    int k = 0;
    for (auto &kv : ctx->prof_total) {
        if (k < cap) {
            std::memset(out[k].name, 0, sizeof out[k].name);
            std::strncpy(out[k].name, kv.first.c_str(), sizeof out[k].name - 1);
            out[k].launches = kv.second.first;
            out[k].total_ms = kv.second.second;
        }
        ++k;
    }
    if (n_out) *n_out = k;
    return BEM_OK;
}

int64_t bem_rule_points(int32_t cas, int32_t regular_rule, int32_t q, double *out, int64_t cap)
{
    if (cas < kRegular || cas > kIdentical || q < 1 || q > 20) return BEM_ERR_INVALID_ARG;
    std::vector<double> soa;
    if (!make_rule4d_host(cas, regular_rule, q, soa)) return BEM_ERR_INVALID_ARG;
    const int64_t n = (int64_t)(soa.size() / kRuleCols);
    if (out && cap >= (int64_t)soa.size()) std::memcpy(out, soa.data(), soa.size() * sizeof(double));
    return n;
}

int64_t bem_rule_points_xi(int32_t cas, int32_t q, double *out, int64_t cap)
{
    if (cas < kVertex || cas > kIdentical || q < 1 || q > 20) return BEM_ERR_INVALID_ARG;
    std::vector<double> soa;
    if (!make_rule4d_host(cas, 0, q, soa, true)) return BEM_ERR_INVALID_ARG;
    const int64_t n = (int64_t)(soa.size() / kRuleCols);
    if (out && cap >= (int64_t)soa.size()) std::memcpy(out, soa.data(), soa.size() * sizeof(double));
    return n;
}

int bem_shard_blocks(const int64_t *cost, int64_t n_blocks, int32_t n_shards, int64_t *bounds)
{
    if (!bounds || n_shards < 1 || n_blocks < 0 || (n_blocks > 0 && !cost)) return BEM_ERR_INVALID_ARG;
    long double total = 0.0L;
    for (int64_t b = 0; b < n_blocks; ++b) {
        if (cost[b] < 0) return BEM_ERR_INVALID_ARG;
        total += (long double)cost[b];
    }
    // shard k ends at the first block whose inclusive prefix reaches (k+1)/n of the total
    bounds[0] = 0;
    long double acc = 0.0L;
    int64_t b = 0;
    for (int k = 1; k < n_shards; ++k) {
        const long double target = total * k / n_shards;
        while (b < n_blocks && acc + (long double)cost[b] <= target) acc += (long double)cost[b++];
        // take the block that crosses the target if that lands closer to it
        if (b < n_blocks && target - acc > acc + (long double)cost[b] - target) acc += (long double)cost[b++];
        bounds[k] = b;
    }
    bounds[n_shards] = n_blocks;
    return BEM_OK;
}

}  // extern "C"
