// Host check of the level-by-level GCA driver (gca_pivots_levels) that
// bem_gca_pivots_device runs with its Green matrices from the device: here the
// producer writes every level's blocks as the device call lays them out
// (column-major rows x 2m at off[k], A_t+ columns then A_t- columns, factors
// sp = sqrt(w) and sm = sqrt(w) delta_t), from the host's own integrals with
// the same operations as bem_gca_pivots.  The pivots must then be those of
// bem_gca_pivots bit for bit.  Built and run by tests/test_gca_levels.py.
#include "bem_gca.cpp"

#include <cstdio>
#include <cstring>

int main(int argc, char **argv)
{
    if (argc != 2) return 2;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    // nv nt basis kappa g n_clusters | verts | tris | cl_ptr | cl_idx | cl_son
    int64_t hdr[6];
    double kappa;
    if (std::fread(hdr, 8, 3, f) != 3 || std::fread(&kappa, 8, 1, f) != 1 ||
        std::fread(hdr + 3, 8, 2, f) != 2)
        return 2;
    const int64_t nv = hdr[0], nt = hdr[1];
    const int basis = (int)hdr[2], g = (int)hdr[3], nc = (int)hdr[4];
    std::vector<double> v(3 * nv);
    std::vector<int32_t> t(3 * nt), ptr(nc + 1), son(2 * nc);
    bool ok = std::fread(v.data(), 8, v.size(), f) == v.size() &&
              std::fread(t.data(), 4, t.size(), f) == t.size() &&
              std::fread(ptr.data(), 4, ptr.size(), f) == ptr.size();
    std::vector<int32_t> idx(ok ? ptr[nc] : 0);
    ok = ok && std::fread(idx.data(), 4, idx.size(), f) == idx.size() &&
         std::fread(son.data(), 4, son.size(), f) == son.size();
    std::fclose(f);
    if (!ok) return 2;

    const int rank = 16;
    const double eps = 1e-6;
    std::vector<int32_t> pp_host(nc + 1), pi_host((size_t)nc * rank), pp_lev(nc + 1),
        pi_lev((size_t)nc * rank);
    int rc = bem_gca_pivots(v.data(), nv, t.data(), nt, basis, kappa, ptr.data(), idx.data(),
                            son.data(), nc, g, eps, rank, 0, pp_host.data(), pi_host.data(),
                            (int64_t)pi_host.size());
    if (rc != BEM_OK) return 3;

    // the host integrals of one level in the device layout
    HostMesh M;
    GcaRun R;
    rc = gca_setup(v.data(), nv, t.data(), nt, basis, kappa, ptr.data(), idx.data(), son.data(),
                   nc, g, eps, rank, 0, pp_lev.data(), pi_lev.data(), (int64_t)pi_lev.size(), R);
    if (rc != BEM_OK) return 3;
    int levels = 0;
    int64_t blocks = 0;
    auto produce = [&](const bem::GreenLevel &L, bool cplx_out, std::vector<double> &out) {
        ++levels;
        for (size_t k = 0; k + 1 < L.row_ptr.size(); ++k) {
            const int rn = L.row_ptr[k + 1] - L.row_ptr[k];
            const int p0 = L.pt_ptr[k], m = L.pt_ptr[k + 1] - p0;
            if (rn == 0 || m == 0) continue;
            ++blocks;
            BoxPoints Z;
            Z.m = m;
            for (int nu = 0; nu < m; ++nu) {
                Z.x.push_back(L.z[3 * (p0 + nu)]);
                Z.y.push_back(L.z[3 * (p0 + nu) + 1]);
                Z.z.push_back(L.z[3 * (p0 + nu) + 2]);
                Z.nx.push_back(L.nz[3 * (p0 + nu)]);
                Z.ny.push_back(L.nz[3 * (p0 + nu) + 1]);
                Z.nz.push_back(L.nz[3 * (p0 + nu) + 2]);
            }
            std::vector<cplx> gp(m), gm(m);
            for (int i = 0; i < rn; ++i) {
                basis_integrals(R.M, L.rows[L.row_ptr[k] + i], Z, gp.data(), gm.data());
                for (int nu = 0; nu < m; ++nu) {
                    const cplx a = L.sp[p0 + nu] * gp[nu], b = L.sm[p0 + nu] * gm[nu];
                    const size_t ep = (size_t)L.off[k] + i + (size_t)nu * rn;
                    const size_t em = (size_t)L.off[k] + i + (size_t)(m + nu) * rn;
                    if (cplx_out) {
                        out[2 * ep] = a.real();
                        out[2 * ep + 1] = a.imag();
                        out[2 * em] = b.real();
                        out[2 * em + 1] = b.imag();
                    } else {
                        out[ep] = a.real();
                        out[em] = b.real();
                    }
                }
            }
        }
        return BEM_OK;
    };
    rc = bem::gca_pivots_levels(v.data(), nv, t.data(), nt, basis, kappa, ptr.data(), idx.data(),
                                son.data(), nc, g, eps, rank, 0, produce, pp_lev.data(),
                                pi_lev.data(), (int64_t)pi_lev.size());
    if (rc != BEM_OK) return 4;
    const bool same = pp_host == pp_lev &&
                      std::equal(pi_host.begin(), pi_host.begin() + pp_host[nc], pi_lev.begin());
    std::printf("levels %d blocks %lld pivots %d same %d\n", levels, (long long)blocks,
                (int)pp_host[nc], (int)same);
    return same ? 0 : 1;
}
