// Launch wrappers for the librve device kernels (defined in kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rve {

// Column layout shared by every vector kernel.  A vector of one field holds
// n_rows = n_scalar_dofs * NC rows (NC = 3 for mechanics, 1 for the scalar
// fields) and ncols right-hand sides, stored row-major: v[row * ncols + col].
// Columns are grouped by RVE: RVE b owns columns [6b, 6b+6).  Mechanics uses
// the six unit strains; the scalar solve uses columns 0..2 for the thermal and
// 3..5 for the moisture unit gradients.
struct Launch {
    int ncols = 6;
    int cpb = 6;          // columns per block (divides ncols)
    int rows_per_block = 42;
    int nby = 1;          // grid.y of the 2-D launches (partials are [nby][ncols][...])
    int nby_op = 0;       // grid.y of the operator and rows of its energy partials (0: nby)
    int n_colour = 0;     // deterministic mode: element colours, one operator launch (and one
                          // block of op_rows() partial rows) per colour
    double* energy_acc = nullptr;   // fused iteration: the operator adds its per-column energy
                                    // here (FP64 atomics) instead of writing partial rows
    cudaStream_t stream = 0;
    int op_rows() const { return nby_op > 0 ? nby_op : nby; }
    int op_partials() const { return op_rows() * (n_colour > 0 ? n_colour : 1); }
};

template <typename T>
struct ElemView {
    int64_t nt = 0;
    const int32_t* edofs = nullptr;   // [nt][ne]
    const T* geo = nullptr;           // [nt][10]: Jinv (row k = grad xi_k), |T|
    const T* mat = nullptr;           // mech [nt][21] upper-triangular Voigt D; scalar [nt][12] k(6), d(6)
    const uint8_t* phase = nullptr;   // [nt]
    const T* scale = nullptr;         // [ncols][2] factor per column and phase
    // element list: the scatter kernels visit elist[0 .. nt) instead of 0 .. nt
    const int32_t* elist = nullptr;
    // deterministic mode (host side): the elements sorted by colour, no two elements of a
    // colour sharing a DOF; colour k is elist_all[coff[k] .. coff[k+1]).  The launchers run
    // one launch per colour, so every (DOF, column) entry receives one addition per
    // launch, in colour order: the sums are bit-reproducible.
    const int32_t* elist_all = nullptr;   // device
    const int64_t* coff = nullptr;        // host, [ncolour + 1]
    int ncolour = 0;
    // DOF nodes of the map (bound of edofs), used by the checking build only
    int64_t n_nodes = 0;
};

// Checking build (compiled with -DRVE_BOUNDS_CHECK=1): every element visited by the
// operator, the double-float residual and the diagonal has its DOF indices and its
// column checked before the gather; an element out of range is counted and skipped.
// Release builds compile the check out and report checking_build = 0.
bool bounds_check_built();
// violations since the last reset, and the (element, column) of the first one
int bounds_status(unsigned long long* count, long long* first_elem, int* first_col);
int bounds_reset();

// Per-row preconditioner / constraint data of one field.
template <typename T>
struct RowView {
    int64_t n_rows = 0;
    const T* diag = nullptr;          // [nfield][2 phases][n_rows], nfield = 1 (mech) or 2 (scalar)
    const uint8_t* mask = nullptr;    // [n_scalar_dofs] 1 = Dirichlet-constrained (or nullptr)
    const T* scale = nullptr;         // [ncols][2]
    int nfield = 1;
    int nc = 3;
    // constraint rows (periodic / Neumann), FP64
    int m = 0;                        // number of rows
    int64_t n_sup = 0;                // support entries (rows of the vector touched by C)
    const int64_t* sup_row = nullptr; // [n_sup] vector row
    const double* sup_coef = nullptr; // [n_sup][m]
    const int32_t* sup_of_row = nullptr;  // [n_rows] index into support or -1
};

// Per-column PCG state, FP64, each array [ncols] unless noted.
struct ColState {
    double* rz;       // current (r, z)
    double* rz0;      // initial (r, z)
    double* alpha;
    double* beta;
    double* mu;       // [m][ncols] constraint multipliers of the current residual
    double* schur;    // [ncols][m*m] Cholesky factor of C M^-1 C^T
    int32_t* active;  // 1 while the column iterates
    int32_t* iters;   // iterations taken
    int32_t* flags;   // [1] bit0: numeric error
    int32_t* list;    // [ncols] the active columns in ascending order (compacted)
    int32_t* n_list;  // [1] their number
    const double* tol;  // [1] relative tolerance on sqrt(rz / rz0), in device memory so that a
                        // captured iteration graph can be reused with another tolerance
    // fused iteration (no constraint rows, not deterministic): the operator adds its
    // per-column energies into pq_acc and the update its (r, z) into rz_acc with FP64
    // atomics, block y into slot y % ACC_SLOTS (fewer atomics per address); the
    // loop-control kernel sums the slots and clears them
    double* pq_acc = nullptr;   // [ACC_SLOTS][ncols]
    double* rz_acc = nullptr;   // [ACC_SLOTS][ncols]
};
constexpr int ACC_SLOTS = 8;

void upload_basis_tables();
// SMs of the current device (cached per device ordinal)
int sm_count();

// y += K x (+ macro load when macro != 0); energy partials x.Kx per column.
// active (optional, [ncols]): columns with active == 0 are skipped.
template <typename T>
// list / n_list (optional, single block column only): the block's threads are spread
// over the listed (active) columns only, so converged columns cost no lanes.
void launch_operator(int p, int nc, bool macro, const ElemView<T>& ev, const T* x, T* y,
                     double* energy_partial, const Launch& L, const int32_t* active = nullptr,
                     const int32_t* list = nullptr, const int32_t* n_list = nullptr);
// grid.y of the operator for a launch shape: one wave of the blocks that fit on the
// GPU at once (grid-stride over elements), at most L.nby
template <typename T>
int operator_grid_y(int p, int nc, const Launch& L, int64_t nt);
// list[0 .. n) = the columns with active != 0, ascending (one block)
void launch_compact_active(const int32_t* active, int ncols, int32_t* list, int32_t* n_list, cudaStream_t s);

template <typename T>
void launch_diag(int p, int nc, int64_t n_rows, const ElemView<T>& ev, T* diag, cudaStream_t s);

void launch_geometry(int64_t nt, const double* xyz, const int32_t* lverts, double* geo64,
                     float* geo32, int32_t* bad, cudaStream_t s);

struct MaterialConsts {
    double Em, num, km, dm;
    double E1, E2, G12, nu12, nu23, k1, k2, d1, d2;
    double ref_mech, ref_k, ref_d;   // internal scaling (outputs multiplied back)
};
void launch_materials(int64_t nt, const uint8_t* phase, const double* tangent,
                      const MaterialConsts& mc, double* matm64, float* matm32, double* mats64,
                      float* mats32, int32_t* bad, cudaStream_t s);

void launch_degradation(int64_t n, const double* T_C, const double* c_wt, const double* t_h,
                        double beta, double Tg_C, double c_sat, double* out, cudaStream_t s);

// column scales from per-RVE degradation factors
template <typename T>
void launch_column_scales(int nrve, const double* w, int apply_to_yarn, bool mech, T* scale,
                          cudaStream_t s);

// PCG pieces
template <typename T>
void launch_finalize_alpha(const double* energy_partial, ColState cs, const Launch& L);
// also accumulates the constraint products C M^-1 r into c_partial when given
template <typename T>
void launch_update(const RowView<T>& rv, T* x, T* r, const T* p, const T* q, ColState cs,
                   double* rz_partial, bool apply_update, const Launch& L, double* c_partial = nullptr);
template <typename T>
void launch_constraint_dot(const RowView<T>& rv, const T* r, double* c_partial, const Launch& L);
void launch_finalize_beta(int m, const double* rz_partial, const double* c_partial, ColState cs,
                          bool first, const Launch& L);
template <typename T>
void launch_pupdate(const RowView<T>& rv, T* r, T* p, T* q, ColState cs, bool first,
                    const Launch& L);
// per-column tolerances tolc [ncols] (after the initial finalisation): rz0 scaled by
// (tolc / tol)^2, columns with tolc >= 1 inactive
void launch_column_tol(int ncols, const double* tolc, ColState cs, cudaStream_t s);
void launch_constraint_multipliers(int m, const double* c_partial, ColState cs, const Launch& L);
// FP64 r projected in place; (r, M^-1 r) partials from the FP32 preconditioner view rv32
void launch_project_residual(const RowView<double>& rv, const RowView<float>& rv32, double* r, ColState cs,
                             double* rz_partial, const Launch& L);
template <typename T>
void launch_schur(const RowView<T>& rv, ColState cs, const Launch& L);

// reductions for the homogenised tensors
void launch_gram(int64_t n_rows, const double* b, const double* u, const double* r,
                 double* partial, const Launch& L);
// element data in T, the solution in TU (converted on load)
template <typename T, typename TU>
void launch_mean_stress(int p, int nc, const ElemView<T>& ev, const TU* u, double* partial,
                        const Launch& L);
void launch_reduce_partials(int nby, int width, const double* partial, double* out,
                            cudaStream_t s);

// batch gather of (T, c, t) and scatter of [B][55] results (C 36, K 9, D 9, status)
void launch_gather_states(int B, const int64_t* idx, const double* T, const double* c, const double* t,
                          double* out, cudaStream_t s);
void launch_scatter_results(int B, const int64_t* idx, const double* res, double* C, double* K, double* D,
                            int32_t* status, cudaStream_t s);

// previous solutions combined per column (warm starts); map and coef are [ncols][WARM_SOURCES]
constexpr int WARM_SOURCES = 8;
constexpr int WARM_GALERKIN = 3;   // previous solutions spanning the energy-optimal start
// the energy-optimal start's residual map holds two entries per source in a column's row
static_assert(2 * WARM_GALERKIN <= WARM_SOURCES, "WARM_SOURCES must hold 2 * WARM_GALERKIN entries");
template <typename TI, typename TO>
void launch_combine_columns(int64_t n_rows, int ncols, int src_cols, const int32_t* map, const double* coef,
                            const TI* src, TO* x, cudaStream_t s, bool accumulate = false);
// inner products of the energy-optimal warm start (ns <= WARM_GALERKIN sources of the
// previous batch, columns 6 src[p] + lc): out[split][lc][p][t] for t < ns x_p . Kc_t,
// t in [ns, 2 ns) x_p . Kc_{6 ns + (t - ns)} (Kc: [n_rows][12 ns], the degraded and the
// other phases' products), then x_p . Y_0 and x_p . Y_1
void launch_warm_gram(int64_t n_rows, int ns, const int32_t* src, int src_cols, const double* X,
                      const double* Kc, const double* Y, double* out, int splits, cudaStream_t s);

// r_hi + r_lo += -K32 (x_h + x_l + u_macro) in double-float arithmetic (FP32 element
// data; x_h = nullptr: x = 0); the caller adds r_lo (FP32) into r_hi (FP64) afterwards
void launch_residual_df(int p, int nc, const ElemView<float>& ev, const float* xh, const float* xl,
                        double* r_hi, float* r_lo, const Launch& L);
// x = x_h + x_l (two FP32 words per FP64 entry)
void launch_split_d2ff(int64_t n, const double* x, float* xh, float* xl, cudaStream_t s);

// the compaction above, plus the device-side PCG loop control: counter += 1;
// condition = any active && counter < max_iter
// Fused iteration: x += alpha p, r -= alpha q with alpha = rz / pq_acc formed by every
// thread for its column (no separate alpha kernel), (r, M^-1 r) added into rz_acc.
template <typename T>
void launch_update_fused(const RowView<T>& rv, T* x, T* r, const T* p, const T* q, ColState cs, const Launch& L);
// Fused iteration: beta, rz and convergence per column from rz_acc, both accumulators
// cleared, then the active list and the loop control (one block).
void launch_beta_compact_continue(ColState cs, int ncols, cudaGraphConditionalHandle h, int32_t* counter,
                                  int max_iter, bool ctl, cudaStream_t s);
void launch_compact_continue(const int32_t* active, int ncols, int32_t* list, int32_t* n_list,
                             cudaGraphConditionalHandle h, int32_t* counter, int max_iter, cudaStream_t s);

// right-hand sides of a batch from the per-phase macro loads y = [2][n_rows][6]:
// b = -(scale_0 y_0 + scale_1 y_1) per column (accumulate: b += that instead)
void launch_rhs_combine(int64_t n_rows, int nrve, const double* y, const double* scale, double* b,
                        cudaStream_t s, bool accumulate = false);

// elementwise helpers
void launch_cast_d2f(int64_t n, const double* a, float* b, cudaStream_t s);
void launch_axpy_f2d(int64_t n, const float* a, double* b, cudaStream_t s);
void launch_neg(int64_t n, double* a, cudaStream_t s);

// multiplier route of Eq. eq_homo_stress: vertex reactions of the total field
// u + X (macro load of each column) scattered to original vertex ids, r [nv][nc][ncols]
void launch_vertex_reactions(int p, int nc, const ElemView<double>& ev, const int32_t* lverts, const double* u,
                             double* r, int ncols, cudaStream_t s);
// out[i][col] = sum_k w[k][i][:] . r[vid[k]][:][col]
void launch_weighted_vertex_sum(int n, int ni, int nc, const int32_t* vid, const double* w, const double* r,
                                int ncols, double* out, cudaStream_t s);
// out[k][col] = sum_i coef[i][k] y[row[i]][col]
void launch_rows_dot(int64_t n_sup, int m, const int64_t* row, const double* coef, const double* y, int ncols,
                     double* out, cudaStream_t s);

// tensor-core operator of the mixed-precision inner solve (operator_tc.cu): mechanics, p = 2, 3
bool operator_tc_supported(int p, int nc);
int64_t element_matrix_floats(int p);   // packed FP32 floats per element (padded to 4)
int element_matrix_pairs(int p);        // packed entries per element: n (n + 1) / 2, n = 3 n_local(p)
// the packed element matrices ke [nt][element_matrix_floats(p)] from the FP64 element data;
// pairs_dev [element_matrix_pairs(p)] and ptab_dev [9 n_local(p)^2] are caller-owned scratch
cudaError_t build_element_matrices(int p, int64_t nt, const double* geo64, const double* matm64, float* ke,
                                   uint16_t* pairs_dev, double* ptab_dev, cudaStream_t s);
// sets the kernels' shared-memory limit; call once per device before the first launch
cudaError_t operator_tc_prepare(int p);
// y += s K x for the listed (or active) columns; energy partials [nby_total][ncols] like
// launch_operator's; err bit 2 set when a bounded device wait gave up
cudaError_t launch_operator_tc(int p, int64_t nt, const int32_t* edofs, const float* ke, const uint16_t* pairs,
                               const uint8_t* phase, const float* scale, const float* x, float* y, double* epart,
                               const int32_t* active, int ncols, const int32_t* list, const int32_t* n_list,
                               int nby_total, int32_t* err, cudaStream_t s);

// allocation-free entry point support (noalloc.cu)
int noalloc_max_cols();
int noalloc_max_blocks_y();
double* noalloc_scratch(int device, cudaError_t* err);
void launch_fill(int64_t n, double v, double* a, cudaStream_t s);
void launch_scale_cols(int64_t n_rows, int ncols, double f_lo, double f_hi, double* y, cudaStream_t s);

}  // namespace rve
