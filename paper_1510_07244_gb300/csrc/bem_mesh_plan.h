// Host planner of bem_mesh_upload (no device code): the vertex -> triangle
// adjacency and, for every triangle, its touching neighbours with their case
// and the vertex orders the Sauter-Schwab maps expect (Section 2.2; the case
// test of Algorithm 3, here done once per mesh).
#pragma once

#include <stdint.h>

#include <vector>

namespace bem {

struct TouchPlan {
    std::vector<int> vt_ptr, vt_tri;       // vertex -> triangles (CSR, ascending ids)
    int maxdeg = 0;                        // largest vertex degree
    // touching pairs, grouped by the first triangle a (CSR nb_ptr), each group
    // ascending in b; a == b (the identical pair) included
    std::vector<int> nb_ptr, nb_tri, nb_src;
    std::vector<unsigned char> nb_case;    // kVertex, kEdge or kIdentical
    std::vector<unsigned char> nb_perm;    // code_a * 6 + code_b (kPerm numbering)
    std::vector<int> lists[4];             // per case: indices into the pair arrays
};

// Fills P from the triangles tris (nt x 3, indices already checked to lie in
// [0, nv) and to be distinct within each triangle), on up to one host thread
// per hardware thread for contiguous triangle ranges (the result does not
// depend on their number).  Returns 0, or BEM_ERR_DEGENERATE with a message in
// *err when two triangles have the same three vertices.
int plan_touching(const int32_t *tris, int64_t nt, int64_t nv, TouchPlan &P, const char **err);

// The smallest vertex index v whose coordinates (verts[3v .. 3v+2], finite)
// equal, coordinate by coordinate under ==, those of a vertex u < v, or -1 if
// every vertex index has coordinates of its own.
int64_t find_duplicate_vertex(const double *verts, int64_t nv);

}  // namespace bem
