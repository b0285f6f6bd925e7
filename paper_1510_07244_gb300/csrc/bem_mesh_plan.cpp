// Host planner of bem_mesh_upload and the host-only bem_touching_pairs.
//
// A pair of triangles touches when it shares vertex indices (Section 2.2: one
// shared index = common vertex, two = common edge, three = identical); every
// other pair is regular.  The vertex orders follow one convention, shared with
// the rules: the shared vertex first (common vertex); the shared edge as
// positions 0 -> 1 in the direction it has in a, b with the same two vertices
// in the same order (common edge); b in a's order (identical).  The orders
// decide which points a rule evaluates, so results are reproducible bit for
// bit only with the same orders.
#include "bem_mesh_plan.h"

#include <algorithm>
#include <array>
#include <climits>
#include <cstring>
#include <thread>
#include <vector>

#include "bem_internal.h"

namespace bem {

namespace {

int pos_in(const int32_t *B, int v) { return B[0] == v ? 0 : (B[1] == v ? 1 : 2); }

// The fans of a triangle's three vertices are ascending lists of triangles; a
// three-way merge visits every neighbour b once, in ascending order, and
// calls f(b, m) with bit k of m set when b is in the fan of the triangle's
// vertex k (so the bit count of m is the number of shared indices).
template <class F>
inline void for_each_neighbour(const int *vp, const int *vt, const int32_t *A, F &&f)
{
    int i[3], e[3];
    for (int k = 0; k < 3; ++k) {
        i[k] = vp[A[k]];
        e[k] = vp[A[k] + 1];
    }
    for (;;) {
        int b = INT32_MAX;
        for (int k = 0; k < 3; ++k)
            if (i[k] < e[k] && vt[i[k]] < b) b = vt[i[k]];
        if (b == INT32_MAX) return;
        int m = 0;
        for (int k = 0; k < 3; ++k)
            if (i[k] < e[k] && vt[i[k]] == b) {
                m |= 1 << k;
                ++i[k];
            }
        f(b, m);
    }
}

// Case of a pair from its mask of shared positions of a.
inline int mask_case(int m) { return m == 7 ? kIdentical : (m == 3 || m == 5 || m == 6 ? kEdge : kVertex); }

// Pass 1 over the triangles [lo, hi): neighbour counts per triangle (into
// cnt[a]) and per case for the range; flags two distinct triangles with the
// same three vertices.
struct RangeCount {
    int64_t per_case[4] = {0, 0, 0, 0};
    bool degenerate = false;
};

void count_range(const int32_t *tris, const TouchPlan &P, int64_t lo, int64_t hi, int *cnt,
                 RangeCount &C)
{
    const int *vp = P.vt_ptr.data(), *vt = P.vt_tri.data();
    for (int64_t a = lo; a < hi; ++a) {
        int n = 0;
        for_each_neighbour(vp, vt, tris + 3 * a, [&](int b, int m) {
            if (m == 7 && b != (int)a) C.degenerate = true;
            ++C.per_case[mask_case(m)];
            ++n;
        });
        cnt[a] = n;
    }
}

// Pass 2: the pairs of [lo, hi) at their final positions nb_ptr[a] ..., and
// their indices into the case lists from the range's offsets case_at[].
void fill_range(const int32_t *tris, TouchPlan &P, const int *perm2, int64_t lo, int64_t hi,
                int64_t case_at[4])
{
    const int *vp = P.vt_ptr.data(), *vt = P.vt_tri.data();
    for (int64_t a = lo; a < hi; ++a) {
        const int32_t *A = tris + 3 * a;
        int k = P.nb_ptr[(size_t)a];
        for_each_neighbour(vp, vt, A, [&](int b, int m) {
            const int32_t *B = tris + 3 * (int64_t)b;
            const int cas = mask_case(m);
            int o0, o1, p0, p1;   // a's order starts (o0, o1), b's (p0, p1)
            if (cas == kIdentical) {
                o0 = 0;
                o1 = 1;
                p0 = pos_in(B, A[0]);
                p1 = pos_in(B, A[1]);
            } else if (cas == kEdge) {
                // shared positions i0 < i1 of a; the edge starts at the one whose
                // cyclic successor is the other
                const int i0 = (m & 1) ? 0 : 1, i1 = (m & 4) ? 2 : 1;
                const int f = (i0 + 1) % 3 == i1 ? i0 : i1;
                o0 = f;
                o1 = (f + 1) % 3;
                p0 = pos_in(B, A[o0]);
                p1 = pos_in(B, A[o1]);
            } else {
                const int i0 = m == 1 ? 0 : (m == 2 ? 1 : 2);
                o0 = i0;
                o1 = (i0 + 1) % 3;
                p0 = pos_in(B, A[i0]);
                p1 = (p0 + 1) % 3;
            }
            P.lists[cas][(size_t)case_at[cas]++] = k;
            P.nb_tri[(size_t)k] = b;
            P.nb_src[(size_t)k] = (int)a;
            P.nb_case[(size_t)k] = (unsigned char)cas;
            P.nb_perm[(size_t)k] = (unsigned char)(perm2[o0 * 3 + o1] * 6 + perm2[p0 * 3 + p1]);
            ++k;
        });
    }
}

// Runs body(r) for r = 0 .. n-1, ranges 1.. on host threads and range 0 on
// the calling thread.
template <class F>
void run_ranges(int n, F &&body)
{
    std::vector<std::thread> pool;
    for (int r = 1; r < n; ++r) pool.emplace_back([&body, r] { body(r); });
    body(0);
    for (auto &t : pool) t.join();
}

}  // namespace

int plan_touching(const int32_t *tris, int64_t nt, int64_t nv, TouchPlan &P, const char **err)
{
    // vertex -> triangle adjacency by counting sort (ascending triangle ids)
    P.vt_ptr.assign((size_t)nv + 1, 0);
    P.vt_tri.resize((size_t)(3 * nt));
    for (int64_t k = 0; k < 3 * nt; ++k) P.vt_ptr[tris[k] + 1]++;
    for (int64_t v = 0; v < nv; ++v) P.vt_ptr[v + 1] += P.vt_ptr[v];
    {
        std::vector<int> fill(P.vt_ptr.begin(), P.vt_ptr.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 3; ++k) P.vt_tri[fill[tris[3 * t + k]]++] = (int)t;
    }
    P.maxdeg = 0;
    for (int64_t v = 0; v < nv; ++v) P.maxdeg = std::max(P.maxdeg, P.vt_ptr[v + 1] - P.vt_ptr[v]);

    // kPerm code of the permutation whose first two entries are (o0, o1)
    int perm2[9] = {};
    for (int c = 0; c < 6; ++c) perm2[kPerm[c][0] * 3 + kPerm[c][1]] = c;

    // Contiguous triangle ranges on host threads (one range below 4096
    // triangles).  Pass 1 counts, a prefix sum places every pair and every
    // case-list entry, pass 2 writes them: the result is the same for any
    // number of ranges.
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    const int n_ranges = (int)std::max<int64_t>(1, std::min<int64_t>({hw, 64, nt / 2048}));
    auto range_lo = [&](int r) { return nt * r / n_ranges; };
    P.nb_ptr.assign((size_t)nt + 1, 0);
    std::vector<RangeCount> C((size_t)n_ranges);
    run_ranges(n_ranges, [&](int r) {
        count_range(tris, P, range_lo(r), range_lo(r + 1), P.nb_ptr.data() + 1, C[(size_t)r]);
    });
    for (const auto &c : C)
        if (c.degenerate) {
            *err = "two triangles with the same vertices";
            return BEM_ERR_DEGENERATE;
        }
    for (int64_t a = 0; a < nt; ++a) {
        if ((int64_t)P.nb_ptr[(size_t)a] + P.nb_ptr[(size_t)a + 1] > (int64_t)INT32_MAX) {
            *err = "more than 2^31 touching pairs";
            return BEM_ERR_UNSUPPORTED;
        }
        P.nb_ptr[(size_t)a + 1] += P.nb_ptr[(size_t)a];
    }
    const size_t total = (size_t)P.nb_ptr[(size_t)nt];
    P.nb_tri.resize(total);
    P.nb_src.resize(total);
    P.nb_case.resize(total);
    P.nb_perm.resize(total);
    std::vector<std::array<int64_t, 4>> case_at((size_t)n_ranges);
    for (int c = 0; c < 4; ++c) {
        int64_t at = 0;
        for (int r = 0; r < n_ranges; ++r) {
            case_at[(size_t)r][c] = at;
            at += C[(size_t)r].per_case[c];
        }
        P.lists[c].resize((size_t)at);
    }
    run_ranges(n_ranges, [&](int r) {
        fill_range(tris, P, perm2, range_lo(r), range_lo(r + 1), case_at[(size_t)r].data());
    });
    return BEM_OK;
}

// Open addressing over the exact coordinate triples (linear probing, at most
// half full).  -0.0 and +0.0 are equal under == and hash alike (x + 0.0 maps
// -0.0 to +0.0); equal triples always probe the same chain, and a match is
// confirmed by == on the coordinates themselves.
int64_t find_duplicate_vertex(const double *verts, int64_t nv)
{
    size_t cap = 16;
    while (cap < 2 * (size_t)nv) cap <<= 1;
    std::vector<int64_t> slot(cap, -1);
    auto bits = [](double x) {
        x += 0.0;
        uint64_t u;
        std::memcpy(&u, &x, sizeof u);
        return u;
    };
    auto mix = [](uint64_t z) {   // splitmix64 finaliser
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    };
    for (int64_t v = 0; v < nv; ++v) {
        const double *p = verts + 3 * v;
        size_t k = (size_t)mix(bits(p[0]) ^ mix(bits(p[1]) ^ mix(bits(p[2])))) & (cap - 1);
        for (; slot[k] >= 0; k = (k + 1) & (cap - 1)) {
            const double *q = verts + 3 * slot[k];
            if (q[0] == p[0] && q[1] == p[1] && q[2] == p[2]) return v;
        }
        slot[k] = v;
    }
    return -1;
}

}  // namespace bem

extern "C" int bem_touching_pairs(const int32_t *tris, int64_t nt, int64_t nv, int32_t *src,
                                  int32_t *dst, int32_t *cas, int32_t *ord, int64_t cap,
                                  int64_t *n_pairs)
{
    using namespace bem;
    if (!tris || !n_pairs || nt < 1 || nv < 1 || cap < 0 ||
        (cap > 0 && (!src || !dst || !cas || !ord)))
        return BEM_ERR_INVALID_ARG;
    if (nt > (int64_t)1 << 28 || nv > (int64_t)1 << 30) return BEM_ERR_UNSUPPORTED;
    for (int64_t k = 0; k < 3 * nt; ++k)
        if (tris[k] < 0 || tris[k] >= nv) return BEM_ERR_INVALID_ARG;
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *T = tris + 3 * t;
        if (T[0] == T[1] || T[1] == T[2] || T[0] == T[2]) return BEM_ERR_DEGENERATE;
    }
    TouchPlan P;
    const char *err = nullptr;
    const int rc = plan_touching(tris, nt, nv, P, &err);
    if (rc != BEM_OK) return rc;
    const int64_t n = (int64_t)P.nb_tri.size();
    *n_pairs = n;
    for (int64_t k = 0; k < std::min(n, cap); ++k) {
        src[k] = P.nb_src[k];
        dst[k] = P.nb_tri[k];
        cas[k] = P.nb_case[k];
        const int pa = P.nb_perm[k] / 6, pb = P.nb_perm[k] % 6;
        for (int i = 0; i < 3; ++i) {
            ord[6 * k + i] = kPerm[pa][i];
            ord[6 * k + 3 + i] = kPerm[pb][i];
        }
    }
    return BEM_OK;
}
