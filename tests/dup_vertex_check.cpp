// Host check of find_duplicate_vertex (the mesh upload's test for two vertex
// indices with equal coordinates) against a brute-force pairwise comparison,
// on seeded random vertex sets with planted duplicates, repeated values per
// coordinate, and signed zeros.  Built and run by tests/test_touching_pairs.py.
#include <cstdio>
#include <cstdint>
#include <random>
#include <vector>

#include "bem_mesh_plan.h"

static int64_t brute(const std::vector<double> &v)
{
    const int64_t n = (int64_t)v.size() / 3;
    for (int64_t b = 1; b < n; ++b)
        for (int64_t a = 0; a < b; ++a)
            if (v[3 * a] == v[3 * b] && v[3 * a + 1] == v[3 * b + 1] && v[3 * a + 2] == v[3 * b + 2])
                return b;
    return -1;
}

int main()
{
    std::mt19937_64 rng(151007244);
    int checked = 0, found = 0;
    for (int trial = 0; trial < 400; ++trial) {
        const int n = 1 + (int)(rng() % 300);
        // few distinct values per coordinate, so partial matches are common
        const int vals = 2 + (int)(rng() % 6);
        std::vector<double> v(3 * (size_t)n);
        for (auto &x : v) {
            const int k = (int)(rng() % vals);
            x = k == 0 ? ((rng() & 1) ? 0.0 : -0.0) : 0.25 * k - 0.5;
        }
        // mostly distinct points: perturb all but a planted few
        for (int i = 0; i < n; ++i)
            if (rng() % 4 != 0) v[3 * i] += 1e-3 * (double)(i + 1);
        const int64_t want = brute(v), got = bem::find_duplicate_vertex(v.data(), n);
        if (want != got) {
            std::printf("mismatch trial %d n %d: want %lld got %lld\n", trial, n, (long long)want,
                        (long long)got);
            return 1;
        }
        ++checked;
        found += want >= 0;
    }
    // no duplicates: a grid; one duplicate far apart; signed zero only
    std::vector<double> g;
    for (int i = 0; i < 20; ++i)
        for (int j = 0; j < 20; ++j)
            for (int k = 0; k < 20; ++k) g.insert(g.end(), {i * 0.1, j * 0.1, k * 0.1});
    if (bem::find_duplicate_vertex(g.data(), 8000) != -1) return 1;
    const std::vector<double> copy(g.begin() + 3 * 4321, g.begin() + 3 * 4322);   // an exact copy
    g.insert(g.end(), copy.begin(), copy.end());
    if (bem::find_duplicate_vertex(g.data(), 8001) != 8000) return 1;
    std::vector<double> z = {0.0, 1.0, -0.0, -0.0, 1.0, 0.0};
    if (bem::find_duplicate_vertex(z.data(), 2) != 1) return 1;
    std::printf("checked %d found %d\n", checked, found);
    return 0;
}
