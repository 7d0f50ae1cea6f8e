// Internal declarations shared by the host files of librve.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rve.h"

namespace rve {

// ------------------------------------------------------------------ basis
// Hierarchic H1 basis on a tetrahedron (Sec. 1 and Sec. 7 use Ainsworth-Coyle
// hierarchic functions of order p = 1..3).  Local vertex order is ascending
// global vertex id, so every edge/face function is globally consistent:
//   vertices  lam_a                                  (4)
//   edges     lam_a lam_b            (p >= 2)        (6, local edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3))
//   edges     lam_a lam_b (lam_b - lam_a)  (p = 3)   (6, same order, a < b)
//   faces     lam_a lam_b lam_c      (p = 3)         (4, faces (0,1,2),(0,1,3),(0,2,3),(1,2,3))
// The reference gradient of every function, d phi_j / d xi_k with
// xi = (lam_1, lam_2, lam_3), is a polynomial of degree p-1 and is stored as
// its coefficients on an L2-orthonormal basis psi_m of P_{p-1} (psi_0 = 1):
//   A[k][m][j] = (1/|T|) int_T (d phi_j / d xi_k) psi_m.
// With element-constant material and geometry, products of such expansions
// integrate exactly: int_T f g = |T| sum_m f_m g_m.
struct Basis {
    int p = 0;
    int ne = 0;   // local functions: 4, 10, 20
    int nm = 0;   // modes of P_{p-1}: 1, 4, 10
    std::vector<double> A;   // [3][nm][ne]
};
const Basis& basis(int p);
inline int n_local(int p) { return p == 1 ? 4 : (p == 2 ? 10 : 20); }
inline int n_modes(int p) { return p == 1 ? 1 : (p == 2 ? 4 : 10); }

// ----------------------------------------------------------------- DOF map
struct DofMap {
    bool periodic = false;
    int p = 1;
    int64_t nt = 0, V = 0, E = 0, F = 0, N = 0;   // N = scalar DOFs
    std::vector<int32_t> edofs;      // [nt][ne]
    std::vector<int32_t> lverts;     // [nt][4] original vertex ids in local order
    std::vector<uint8_t> boundary;   // [N] DOF lies on a boundary entity (unfolded maps)
    std::vector<int32_t> dof_vertex; // [N] original vertex id for vertex DOFs, -1 otherwise
};

// Builds the hierarchic DOF map.  Returns RVE_OK or RVE_ERR_BAD_MESH with a
// message in `err`.
int build_dofmap(const double* xyz, int64_t nv, const int32_t* tets, int64_t nt, int p,
                 bool periodic, DofMap& out, std::string& err);

// thread-local error detail
void set_error(const std::string& s);

}  // namespace rve
