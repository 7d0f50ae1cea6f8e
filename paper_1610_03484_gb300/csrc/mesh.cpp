// Hierarchic DOF map on a tetrahedral mesh (host).
//
// Entities (vertices, edges, faces) are numbered on the possibly folded vertex
// set: with the periodic BC every vertex on a max face of the box is replaced
// by its image on the opposite min face (Sec. 2, periodic fluctuation), so the
// fluctuation lives on a torus mesh and needs no constraint rows beyond the
// rigid translations.  Local vertex order of each tet is ascending folded id,
// which orients every edge function consistently across neighbouring tets and
// across periodic images.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "rve_internal.h"

namespace rve {
namespace {

struct Key3Hash {
    size_t operator()(const std::array<int64_t, 3>& k) const {
        uint64_t h = 1469598103934665603ull;
        for (auto v : k) {
            h ^= (uint64_t)v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        }
        return (size_t)h;
    }
};

}  // namespace

int build_dofmap(const double* xyz, int64_t nv, const int32_t* tets, int64_t nt, int p,
                 bool periodic, DofMap& out, std::string& err) {
    out = DofMap();
    out.periodic = periodic;
    out.p = p;
    out.nt = nt;
    for (int64_t t = 0; t < nt * 4; ++t)
        if (tets[t] < 0 || tets[t] >= nv) {
            err = "tet vertex index out of range";
            return RVE_ERR_BAD_MESH;
        }
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = 1e300;
        hi[a] = -1e300;
    }
    for (int64_t v = 0; v < nv; ++v)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], xyz[3 * v + a]);
            hi[a] = std::max(hi[a], xyz[3 * v + a]);
        }
    double L = 0;
    for (int a = 0; a < 3; ++a) L = std::max(L, hi[a] - lo[a]);
    const double tol = 1e-9 * L;

    // ---- periodic vertex folding
    std::vector<int64_t> master(nv);
    for (int64_t v = 0; v < nv; ++v) master[v] = v;
    if (periodic) {
        const double q = 1.0 / (1e-7 * L);   // quantisation for the coordinate hash
        std::unordered_map<std::array<int64_t, 3>, int64_t, Key3Hash> at;
        auto key = [&](const double* c) {
            return std::array<int64_t, 3>{(int64_t)std::llround((c[0] - lo[0]) * q),
                                          (int64_t)std::llround((c[1] - lo[1]) * q),
                                          (int64_t)std::llround((c[2] - lo[2]) * q)};
        };
        for (int64_t v = 0; v < nv; ++v) {
            const double* c = xyz + 3 * v;
            bool on_max = false;
            for (int a = 0; a < 3; ++a) on_max |= std::fabs(c[a] - hi[a]) <= tol;
            if (!on_max) at[key(c)] = v;
        }
        for (int64_t v = 0; v < nv; ++v) {
            double c[3];
            bool on_max = false;
            for (int a = 0; a < 3; ++a) {
                c[a] = xyz[3 * v + a];
                if (std::fabs(c[a] - hi[a]) <= tol) {
                    c[a] = lo[a];
                    on_max = true;
                }
            }
            if (!on_max) continue;
            auto it = at.find(key(c));
            if (it == at.end()) {
                err = "periodic BC: vertex on a max face has no image on the opposite face";
                return RVE_ERR_BAD_MESH;
            }
            master[v] = it->second;
        }
    }
    // compact folded vertex ids
    std::vector<int64_t> vid(nv, -1);
    int64_t V = 0;
    for (int64_t v = 0; v < nv; ++v)
        if (master[v] == v) vid[v] = V++;
    for (int64_t v = 0; v < nv; ++v) vid[v] = vid[master[v]];

    const int ne = n_local(p);
    out.lverts.resize(nt * 4);
    std::vector<int64_t> g(nt * 4);
    for (int64_t t = 0; t < nt; ++t) {
        std::array<std::pair<int64_t, int32_t>, 4> s;
        for (int a = 0; a < 4; ++a) s[a] = {vid[tets[4 * t + a]], tets[4 * t + a]};
        std::sort(s.begin(), s.end());
        for (int a = 0; a < 3; ++a)
            if (s[a].first == s[a + 1].first) {
                err = "tet has two vertices identified by the periodic fold (mesh needs >= 2 cells per direction)";
                return RVE_ERR_BAD_MESH;
            }
        for (int a = 0; a < 4; ++a) {
            g[4 * t + a] = s[a].first;
            out.lverts[4 * t + a] = s[a].second;
        }
    }
    // ---- edges and faces
    // Without folding an edge (face) is identified by its sorted vertex ids.
    // With the periodic fold two different edges of the torus can join the
    // same pair of folded vertices (a box only two cells thick), so entities
    // are identified by their midpoint / centroid folded into the box instead.
    static const int EL[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    static const int FL[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
    const double qpos = 1.0 / (1e-7 * L);
    auto folded_key = [&](const int32_t* vs, int n) {
        std::array<int64_t, 3> k;
        for (int a = 0; a < 3; ++a) {
            double c = 0;
            for (int i = 0; i < n; ++i) c += xyz[3 * (int64_t)vs[i] + a];
            c = c / n - lo[a];
            const double span = hi[a] - lo[a];
            if (c >= span - tol) c -= span;
            k[a] = (int64_t)std::llround(c * qpos);
        }
        return k;
    };
    std::unordered_map<std::array<int64_t, 3>, int64_t, Key3Hash> emap, fmap;
    emap.reserve(nt * 2);
    fmap.reserve(nt * 3);
    std::vector<int64_t> tedge(nt * 6), tface(nt * 4);
    std::vector<int32_t> fcount;
    std::vector<std::array<int64_t, 3>> fverts;
    for (int64_t t = 0; t < nt; ++t) {
        for (int e = 0; e < 6; ++e) {
            std::array<int64_t, 3> k{g[4 * t + EL[e][0]], g[4 * t + EL[e][1]], -1};
            if (periodic) {
                const int32_t vs[2] = {out.lverts[4 * t + EL[e][0]], out.lverts[4 * t + EL[e][1]]};
                k = folded_key(vs, 2);
            }
            auto it = emap.find(k);
            if (it == emap.end()) it = emap.emplace(k, (int64_t)emap.size()).first;
            tedge[6 * t + e] = it->second;
        }
        for (int f = 0; f < 4; ++f) {
            std::array<int64_t, 3> k{g[4 * t + FL[f][0]], g[4 * t + FL[f][1]], g[4 * t + FL[f][2]]};
            const std::array<int64_t, 3> kv = k;
            if (periodic) {
                const int32_t vs[3] = {out.lverts[4 * t + FL[f][0]], out.lverts[4 * t + FL[f][1]],
                                       out.lverts[4 * t + FL[f][2]]};
                k = folded_key(vs, 3);
            }
            auto it = fmap.find(k);
            if (it == fmap.end()) {
                it = fmap.emplace(k, (int64_t)fmap.size()).first;
                fcount.push_back(0);
                fverts.push_back(kv);
            }
            fcount[it->second]++;
            tface[4 * t + f] = it->second;
        }
    }
    const int64_t E = (int64_t)emap.size(), F = (int64_t)fmap.size();
    out.V = V;
    out.E = E;
    out.F = F;
    int64_t N = V;
    if (p >= 2) N += E;
    if (p >= 3) N += E + F;
    out.N = N;
    out.edofs.resize(nt * ne);
    for (int64_t t = 0; t < nt; ++t) {
        int32_t* d = &out.edofs[t * ne];
        for (int a = 0; a < 4; ++a) d[a] = (int32_t)g[4 * t + a];
        if (p >= 2)
            for (int e = 0; e < 6; ++e) d[4 + e] = (int32_t)(V + tedge[6 * t + e]);
        if (p >= 3) {
            for (int e = 0; e < 6; ++e) d[10 + e] = (int32_t)(V + E + tedge[6 * t + e]);
            for (int f = 0; f < 4; ++f) d[16 + f] = (int32_t)(V + 2 * E + tface[4 * t + f]);
        }
    }
    // ---- vertex DOFs back to an original vertex (for coordinates)
    out.dof_vertex.assign(N, -1);
    for (int64_t v = 0; v < nv; ++v)
        if (master[v] == v) out.dof_vertex[vid[v]] = (int32_t)v;
    // ---- topological boundary: faces owned by a single tet
    out.boundary.assign(N, 0);
    if (!periodic) {
        std::vector<uint8_t> bvert(V, 0);
        for (int64_t f = 0; f < F; ++f) {
            if (fcount[f] != 1) continue;
            for (int a = 0; a < 3; ++a) bvert[fverts[f][a]] = 1;
            if (p >= 3) out.boundary[V + 2 * E + f] = 1;
        }
        for (int64_t v = 0; v < V; ++v) out.boundary[v] = bvert[v];
        if (p >= 2) {
            // an edge is on the boundary iff it is an edge of a boundary face
            for (int64_t f = 0; f < F; ++f) {
                if (fcount[f] != 1) continue;
                for (int e = 0; e < 3; ++e) {
                    int a = e == 2 ? 1 : 0, b = e == 0 ? 1 : 2;
                    std::array<int64_t, 3> k{fverts[f][a], fverts[f][b], -1};
                    int64_t eid = emap.at(k);
                    out.boundary[V + eid] = 1;
                    if (p >= 3) out.boundary[V + E + eid] = 1;
                }
            }
        }
    }
    for (int64_t f = 0; f < F; ++f)
        if (fcount[f] > 2) {
            err = "non-manifold mesh: a face is shared by more than two tets";
            return RVE_ERR_BAD_MESH;
        }
    return RVE_OK;
}

}  // namespace rve
