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

#include "bem_internal.h"

namespace bem {

namespace {

// kPerm code of the permutation whose first two entries are (o0, o1)
int perm_code2(int o0, int o1)
{
    static const std::array<int, 9> table = [] {
        std::array<int, 9> t{};
        for (int c = 0; c < 6; ++c) t[kPerm[c][0] * 3 + kPerm[c][1]] = c;
        return t;
    }();
    return table[o0 * 3 + o1];
}

int pos_in(const int32_t *B, int v) { return B[0] == v ? 0 : (B[1] == v ? 1 : 2); }

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
    size_t bound = 0;     // sum over triangles of their vertices' degrees
    for (int64_t v = 0; v < nv; ++v) {
        const int d = P.vt_ptr[v + 1] - P.vt_ptr[v];
        P.maxdeg = std::max(P.maxdeg, d);
        bound += (size_t)d * d;
    }

    P.nb_ptr.assign((size_t)nt + 1, 0);
    for (auto *v : {&P.nb_tri, &P.nb_src}) {
        v->clear();
        v->reserve(bound);
    }
    P.nb_case.clear();
    P.nb_case.reserve(bound);
    P.nb_perm.clear();
    P.nb_perm.reserve(bound);
    for (auto &l : P.lists) l.clear();

    // For triangle a, walk the triangle fans of its three vertices: stamp[b] == a
    // marks b as collected, mask[b] has bit k set when a's vertex k is one of
    // b's (so the number of set bits is the number of shared indices).
    std::vector<int> stamp((size_t)nt, -1), cand;
    std::vector<unsigned char> mask((size_t)nt, 0);
    cand.reserve(64);
    for (int64_t a = 0; a < nt; ++a) {
        const int32_t *A = tris + 3 * a;
        cand.clear();
        for (int k = 0; k < 3; ++k) {
            const int v = A[k];
            for (int u = P.vt_ptr[v]; u < P.vt_ptr[v + 1]; ++u) {
                const int b = P.vt_tri[u];
                if (stamp[b] != (int)a) {
                    stamp[b] = (int)a;
                    mask[b] = 0;
                    cand.push_back(b);
                }
                mask[b] |= (unsigned char)(1 << k);
            }
        }
        // ascending b (a few dozen candidates: insertion sort)
        for (size_t i = 1; i < cand.size(); ++i) {
            const int x = cand[i];
            size_t j = i;
            for (; j > 0 && cand[j - 1] > x; --j) cand[j] = cand[j - 1];
            cand[j] = x;
        }
        for (const int b : cand) {
            const int32_t *B = tris + 3 * (int64_t)b;
            const int m = mask[b];
            int cas, o0, o1, p0, p1;   // a's order starts (o0, o1), b's (p0, p1)
            if (m == 7) {
                if (b != (int)a) {
                    *err = "two triangles with the same vertices";
                    return BEM_ERR_DEGENERATE;
                }
                cas = kIdentical;
                o0 = 0;
                o1 = 1;
                p0 = pos_in(B, A[0]);
                p1 = pos_in(B, A[1]);
            } else if (m == 3 || m == 5 || m == 6) {
                cas = kEdge;
                // shared positions i0 < i1 of a; the edge starts at the one whose
                // cyclic successor is the other
                const int i0 = (m & 1) ? 0 : 1, i1 = (m & 4) ? 2 : 1;
                const int f = (i0 + 1) % 3 == i1 ? i0 : i1;
                o0 = f;
                o1 = (f + 1) % 3;
                p0 = pos_in(B, A[o0]);
                p1 = pos_in(B, A[o1]);
            } else {
                cas = kVertex;
                const int i0 = m == 1 ? 0 : (m == 2 ? 1 : 2);
                o0 = i0;
                o1 = (i0 + 1) % 3;
                p0 = pos_in(B, A[i0]);
                p1 = (p0 + 1) % 3;
            }
            P.lists[cas].push_back((int)P.nb_tri.size());
            P.nb_tri.push_back(b);
            P.nb_src.push_back((int)a);
            P.nb_case.push_back((unsigned char)cas);
            P.nb_perm.push_back((unsigned char)(perm_code2(o0, o1) * 6 + perm_code2(p0, p1)));
        }
        P.nb_ptr[a + 1] = (int)P.nb_tri.size();
    }
    return BEM_OK;
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
