// bem_near_field_noalloc: the near-field block engine for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: a service whose device memory is owned
// by its own pool allocator, a loop that must never block on the implicit
// device synchronisation cudaMalloc / cudaFree may cause, or a host program
// that has handed all device memory out before it starts assembling.  This
// entry point runs the same kernels as bem_near_field, but its scratch (the
// singular-case quadrature tables and the per-block tile prefix sums) lives in
// the file-scope array g_noalloc_scratch below, which every GPU that loads the
// library holds until the process exits.  Nothing here allocates.
//
// Layout of the array: kMaxBlocks int64 tile prefix slots, then the rule
// tables of every singular case (vertex, edge, identical) at every order
// q = 1..kMaxOrder, back to back.  The tables are written once per device, by
// the first call on that device (a synchronous copy from host memory); later
// calls only pick the offsets of the tables they need, so they copy nothing
// from the host and do not wait for the device.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "bem_internal.h"

namespace {

constexpr int64_t kMaxBlocks = 65536;   // tile prefix slots (int64 each)
constexpr int kMaxOrder = 6;            // singular orders q <= 6
// points of the three singular cases at order q: vertex 2 q^4 + edge 4 q^4 +
// identical 6 q^4; the tables of all orders 1..6 hold 12 (1 + 16 + 81 + 256 +
// 625 + 1296) = 27,300 points of kRuleCols = 7 doubles
constexpr int64_t kSumQ4 = 1 + 16 + 81 + 256 + 625 + 1296;
constexpr int64_t kRuleDoubles = 7LL * 12 * kSumQ4;                // 191,100
constexpr int64_t kScratchDoubles = kMaxBlocks + kRuleDoubles;     // 2,053,088 B in all

// One copy per device of every process that loads the library.  In host code
// this name is only a host-side stand-in: the device address comes from
// cudaGetSymbolAddress (scratch_setup below).
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;

struct DeviceScratch {
    double *base = nullptr;                  // device address of g_noalloc_scratch
    bem::Rule4D rule[4][kMaxOrder + 1];           // [case][q], views into the array
};
DeviceScratch *g_dev[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` and its rule tables, set up
// once per device with that device current: the address lookup, then every
// singular rule of order 1..kMaxOrder built on the host and copied into the
// array with one synchronous cudaMemcpy per table.
cudaError_t scratch_setup(int device, const DeviceScratch **out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        auto *S = new DeviceScratch;
        S->base = static_cast<double *>(p);
        int64_t at = kMaxBlocks;
        for (int c = bem::kVertex; c <= bem::kIdentical; ++c)
            for (int q = 1; q <= kMaxOrder; ++q) {
                std::vector<double> soa;
                if (!bem::make_rule4d_host(c, 0, q, soa) || at + (int64_t)soa.size() > kScratchDoubles) {
                    delete S;
                    return cudaErrorInvalidValue;
                }
                bem::Rule4D &r = S->rule[c][q];
                r.n = (int)(soa.size() / bem::kRuleCols);
                r.d = S->base + at;
                e = cudaMemcpy(r.d, soa.data(), soa.size() * sizeof(double), cudaMemcpyHostToDevice);
                if (e != cudaSuccess) {
                    delete S;
                    return e;
                }
                at += (int64_t)soa.size();
            }
        g_dev[device] = S;
    }
    *out = g_dev[device];
    return cudaSuccess;
}

int noalloc_fail(bem_ctx *ctx, int code, const char *msg)
{
    ctx->err = msg;
    return code;
}

}  // namespace

extern "C" int bem_near_field_noalloc(bem_ctx *ctx, const bem_block_job *job)
{
    using namespace bem;
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!job) return noalloc_fail(ctx, BEM_ERR_INVALID_ARG, "null job");
    const bem_block_job &J = *job;
    auto it = ctx->meshes.find(J.mesh_id);
    if (it == ctx->meshes.end()) return noalloc_fail(ctx, BEM_ERR_INVALID_ARG, "unknown mesh id");
    Mesh *m = it->second;
    if (J.kernel.kind < BEM_LAPLACE_SLP || J.kernel.kind > BEM_HELMHOLTZ_SLP ||
        !std::isfinite(J.kernel.kappa))
        return noalloc_fail(ctx, BEM_ERR_INVALID_ARG, "bad kernel descriptor");
    if (J.quad.precision != BEM_FP64 || J.quad.order_mode != BEM_ORDER_FIXED)
        return noalloc_fail(ctx, BEM_ERR_UNSUPPORTED, "only the FP64 form with fixed orders");
    Rule2D r2;
    if (!make_rule2d(J.quad.regular_rule, J.quad.q_regular, r2) ||
        (r2.np != 4 && r2.np != 7 && r2.np != 9 && r2.np != 16))
        return noalloc_fail(ctx, BEM_ERR_UNSUPPORTED, "regular rule must be TRI7 or DUFFY q in [2, 4]");
    const int qs[4] = {0, J.quad.q_vertex, J.quad.q_edge, J.quad.q_identical};
    for (int c = kVertex; c <= kIdentical; ++c)
        if (qs[c] < 1 || qs[c] > kMaxOrder)
            return noalloc_fail(ctx, BEM_ERR_INVALID_ARG,
                                "bem_near_field_noalloc: singular orders must be in [1, 6] "
                                "(size of its static scratch)");
    if (J.n_blocks < 0) return noalloc_fail(ctx, BEM_ERR_INVALID_ARG, "negative block count");
    if (J.n_blocks > kMaxBlocks)
        return noalloc_fail(ctx, BEM_ERR_INVALID_ARG,
                            "bem_near_field_noalloc: more than 65536 blocks (size of its "
                            "static scratch); split the list into several calls");
    if (J.n_blocks == 0) return BEM_OK;
    if (!J.row_ptr || !J.row_idx || !J.col_ptr || !J.col_idx || !J.blk_row || !J.blk_col ||
        !J.blk_off || !J.out || J.n_row_clusters < 1 || J.n_col_clusters < 1)
        return noalloc_fail(ctx, BEM_ERR_INVALID_ARG, "null pointer or empty cluster list");
    if (J.kernel.kind == BEM_HELMHOLTZ_SLP && (reinterpret_cast<uintptr_t>(J.out) & 15))
        return noalloc_fail(ctx, BEM_ERR_INVALID_ARG, "complex output must be 16-byte aligned");
    if (m->v.basis == BEM_P1 && m->v.maxdeg > kMaxDegP1)
        return noalloc_fail(ctx, BEM_ERR_UNSUPPORTED, "vertex degree above 16 (piecewise linear)");

    cudaError_t e = cudaSetDevice(ctx->device);
    const DeviceScratch *S = nullptr;
    if (e == cudaSuccess) e = scratch_setup(ctx->device, &S);
    if (e != cudaSuccess) return noalloc_fail(ctx, BEM_ERR_CUDA, cudaGetErrorString(e));
    int64_t *prefix = reinterpret_cast<int64_t *>(S->base);

    // touching pairs of the mesh from the resident singular rules
    for (int c = kVertex; c <= kIdentical; ++c) {
        if (m->nlist[c] == 0) continue;
        e = launch_touching(m->v, c, m->list[c], m->nlist[c], S->rule[c][qs[c]], J.kernel.kind,
                            J.kernel.kappa, 0, ctx->stream);
        if (e != cudaSuccess) return noalloc_fail(ctx, BEM_ERR_CUDA, cudaGetErrorString(e));
    }

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
    L.lower_only = 0;
    L.allow_touching = 1;
    L.mixed = 0;
    const TileShape ts = block_tile_shape(m->v.basis, false);
    e = launch_tile_prefix(L, ts.tr, ts.tc, prefix, ctx->status, ctx->stream);
    if (e == cudaSuccess)
        e = launch_block_engine(m->v, L, r2, prefix, ctx->status,
                                ctx->num_sms * (m->v.basis == BEM_P0 ? 8 : 2), ctx->stream);
    if (e != cudaSuccess) return noalloc_fail(ctx, BEM_ERR_CUDA, cudaGetErrorString(e));
    return BEM_OK;
}
