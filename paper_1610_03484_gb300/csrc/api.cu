// C ABI of librve: handles, mesh set-up, the multi-RHS projected PCG driver
// and the homogenised-tensor assembly.  Device work lives in kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "api_internal.h"

namespace rve {

static thread_local std::string g_last_error;
void set_error(const std::string& s) { g_last_error = s; }
const std::string& last_error() { return g_last_error; }

}  // namespace rve

using namespace rve;

namespace rve {
int check_ctx(rve_ctx c) {
    if (!c) {
        set_error("null context");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    cudaSetDevice(c->device);
    return RVE_OK;
}
}  // namespace rve

namespace {
int table_nonzeros(int p);

// ------------------------------------------------------------ geometry + map
// Greedy colouring of the elements over the current DOF map: elements in mesh
// order, each taking the smallest colour that none of its DOFs has met yet, so
// that no two elements of one colour share a DOF.  The elements are then sorted
// by colour (stable) for the deterministic launches.
int build_colouring(rve_mesh m) {
    const int ne = n_local(m->p);
    const int64_t nt = m->nt, N = m->map.N;
    constexpr int W = 4;   // colour bit sets of 256 colours
    std::vector<uint64_t> used((size_t)N * W, 0);
    std::vector<int32_t> colour(nt);
    int ncol = 0;
    for (int64_t e = 0; e < nt; ++e) {
        const int32_t* ed = &m->map.edofs[(size_t)e * ne];
        uint64_t seen[W] = {0, 0, 0, 0};
        for (int j = 0; j < ne; ++j) {
            if (ed[j] < 0 || ed[j] >= N) {
                set_error("DOF index out of range in the map");
                return RVE_ERR_BAD_MESH;
            }
            for (int w = 0; w < W; ++w) seen[w] |= used[(size_t)ed[j] * W + w];
        }
        int c = -1;
        for (int w = 0; w < W && c < 0; ++w)
            if (~seen[w]) c = 64 * w + __builtin_ctzll(~seen[w]);
        if (c < 0) {
            set_error("element colouring needs more than 256 colours");
            return RVE_ERR_BAD_MESH;
        }
        colour[e] = c;
        ncol = std::max(ncol, c + 1);
        for (int j = 0; j < ne; ++j) used[(size_t)ed[j] * W + c / 64] |= 1ull << (c % 64);
    }
    m->colour_off.assign(ncol + 1, 0);
    for (int64_t e = 0; e < nt; ++e) m->colour_off[colour[e] + 1]++;
    for (int k = 0; k < ncol; ++k) m->colour_off[k + 1] += m->colour_off[k];
    std::vector<int64_t> pos(m->colour_off.begin(), m->colour_off.end() - 1);
    std::vector<int32_t> order(nt);
    for (int64_t e = 0; e < nt; ++e) order[pos[colour[e]]++] = (int32_t)e;
    RVE_TRY(upload(m->d_colour_elems, order.data(), order.size(), m->ctx->stream));
    m->ncolour = ncol;
    return RVE_OK;
}

// Element-view fields common to every launch: the DOF-node bound of the checking
// build and, in deterministic mode (or when forced), the colouring.
template <typename T>
void set_view_extras(ElemView<T>& ev, rve_mesh m, bool force_colours = false) {
    ev.n_nodes = m->debug_node_bound > 0 ? m->debug_node_bound : m->map.N;
    if ((force_colours || m->ctx->opt.deterministic) && m->ncolour > 0) {
        ev.elist_all = m->d_colour_elems.as<int32_t>();
        ev.coff = m->colour_off.data();
        ev.ncolour = m->ncolour;
    }
}

// Checking build: the counter starts from zero at each checked call, and the
// violations counted during the call turn its result into RVE_ERR_BOUNDS (the
// counter keeps them for rve_debug_bounds).
void bounds_begin(cudaStream_t s) {
    if (!bounds_check_built()) return;
    cudaStreamSynchronize(s);
    bounds_reset();
}

int bounds_outcome(int rc, cudaStream_t s) {
    if (!bounds_check_built()) return rc;
    cudaStreamSynchronize(s);
    unsigned long long n = 0;
    long long fe = -1;
    int fc = -1;
    if (bounds_status(&n, &fe, &fc) != 0 || n == 0) return rc;
    set_error("bounds check: " + std::to_string(n) + " element visits out of range (first: element " +
              std::to_string(fe) + ", column " + std::to_string(fc) + "), skipped");
    return RVE_ERR_BOUNDS;
}

int rebuild_map(rve_mesh m) {
    cudaStream_t s = m->ctx->stream;
    std::string err;
    int rc = build_dofmap(m->xyz.data(), m->nv, m->tets.data(), m->nt, m->p,
                          m->bc == RVE_BC_PERIODIC, m->map, err);
    if (rc != RVE_OK) {
        set_error(err);
        return rc;
    }
    const int ne = n_local(m->p);
    RVE_TRY(upload(m->d_edofs, m->map.edofs.data(), (size_t)m->nt * ne, s));
    RVE_TRY(build_colouring(m));
    RVE_TRY(upload(m->d_lverts, m->map.lverts.data(), (size_t)m->nt * 4, s));
    RVE_TRY(m->d_geo64.ensure(sizeof(double) * m->nt * 10));
    RVE_TRY(m->d_geo32.ensure(sizeof(float) * m->nt * 10));
    RVE_TRY(m->d_flag.ensure(sizeof(int32_t) * 4));
    RVE_CUDA(cudaMemsetAsync(m->d_flag.p, 0, sizeof(int32_t) * 4, s));
    launch_geometry(m->nt, m->d_xyz.as<double>(), m->d_lverts.as<int32_t>(), m->d_geo64.as<double>(),
                    m->d_geo32.as<float>(), m->d_flag.as<int32_t>(), s);
    m->ctx->launches++;
    int32_t bad = 0;
    RVE_CUDA(cudaMemcpyAsync(&bad, m->d_flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    if (bad) {
        set_error("degenerate (zero-volume) tetrahedron");
        return RVE_ERR_BAD_MESH;
    }
    return RVE_OK;
}

// Constraint rows of the current BC (FP64), normalised per row.
int build_constraints(rve_mesh m, FieldDev& f, const std::vector<double>& geo) {
    cudaStream_t s = m->ctx->stream;
    const DofMap& M = m->map;
    const int nc = f.nc;
    const int64_t N = M.N;
    f.n_rows = N * nc;
    // Dirichlet mask
    std::vector<uint8_t> mask;
    if (m->bc == RVE_BC_DIRICHLET) mask = M.boundary;
    RVE_TRY(upload(f.mask, mask.data(), mask.size(), s));
    f.m = 0;
    f.n_sup = 0;
    // Periodic: the folded (torus) problem is singular only by rigid translations,
    // to which the right-hand side is orthogonal; PCG on this consistent system
    // converges without a projection, and translations change no strain, so no
    // constraint rows are needed.  Dirichlet: the mask is the whole constraint.
    if (m->bc == RVE_BC_DIRICHLET || m->bc == RVE_BC_PERIODIC) return RVE_OK;

    // vertex coordinates relative to the centroid (rotation rows)
    double cen[3] = {0, 0, 0};
    int64_t nvx = 0;
    for (int64_t d = 0; d < N; ++d)
        if (M.dof_vertex[d] >= 0) {
            for (int a = 0; a < 3; ++a) cen[a] += m->xyz[3 * M.dof_vertex[d] + a];
            ++nvx;
        }
    for (int a = 0; a < 3; ++a) cen[a] /= std::max<int64_t>(nvx, 1);
    // g_d = int_Omega grad phi_d (Neumann strain / flux rows), nonzero on boundary DOFs only
    std::vector<double> g;
    const bool neu = m->bc == RVE_BC_NEUMANN;
    if (neu) {
        g.assign(N * 3, 0.0);
        const Basis& B = basis(m->p);
        const int ne = B.ne, nm = B.nm;
        for (int64_t e = 0; e < m->nt; ++e) {
            const double* G = &geo[e * 10];
            for (int j = 0; j < ne; ++j) {
                double a[3];
                for (int k = 0; k < 3; ++k) a[k] = B.A[(k * nm + 0) * ne + j];
                const int64_t d = M.edofs[e * ne + j];
                for (int l = 0; l < 3; ++l)
                    g[d * 3 + l] += G[9] * (a[0] * G[l] + a[1] * G[3 + l] + a[2] * G[6 + l]);
            }
        }
    }
    const int m_rows = nc == 3 ? (neu ? 12 : 3) : (neu ? 4 : 1);
    f.m = m_rows;
    std::vector<int64_t> rows;
    std::vector<double> coef;
    for (int64_t d = 0; d < N; ++d) {
        const bool isv = M.dof_vertex[d] >= 0;
        const bool isb = neu && M.boundary[d];
        if (!isv && !isb) continue;
        double y[3] = {0, 0, 0};
        if (isv)
            for (int a = 0; a < 3; ++a) y[a] = m->xyz[3 * M.dof_vertex[d] + a] - cen[a];
        for (int c = 0; c < nc; ++c) {
            std::vector<double> cr(m_rows, 0.0);
            if (nc == 3) {
                if (isv) {
                    cr[c] = 1.0;   // translation c
                    if (neu) {
                        // rotation k: (e_k x y)_c
                        const double rot[3][3] = {{0, -y[2], y[1]}, {y[2], 0, -y[0]}, {-y[1], y[0], 0}};
                        for (int k = 0; k < 3; ++k) cr[3 + k] = rot[k][c];
                    }
                }
                if (isb) {
                    // strain rows: (E_k g_d)_c with E_k the Voigt basis of symmetric tensors
                    const double* gd = &g[d * 3];
                    static const int VI[6] = {0, 1, 2, 0, 1, 2}, VJ[6] = {0, 1, 2, 1, 2, 0};
                    for (int k = 0; k < 6; ++k) {
                        double v = 0;
                        if (c == VI[k]) v += gd[VJ[k]];
                        if (k >= 3 && c == VJ[k]) v += gd[VI[k]];
                        cr[6 + k] = v;
                    }
                }
            } else {
                if (isv) cr[0] = 1.0;
                if (isb)
                    for (int k = 0; k < 3; ++k) cr[1 + k] = g[d * 3 + k];
            }
            rows.push_back(d * nc + c);
            coef.insert(coef.end(), cr.begin(), cr.end());
        }
    }
    // normalise each constraint row
    std::vector<double> nrm(m_rows, 0.0);
    for (size_t i = 0; i < rows.size(); ++i)
        for (int k = 0; k < m_rows; ++k) nrm[k] += coef[i * m_rows + k] * coef[i * m_rows + k];
    for (int k = 0; k < m_rows; ++k) nrm[k] = nrm[k] > 0 ? 1.0 / std::sqrt(nrm[k]) : 0.0;
    for (size_t i = 0; i < rows.size(); ++i)
        for (int k = 0; k < m_rows; ++k) coef[i * m_rows + k] *= nrm[k];
    std::vector<int32_t> of_row(f.n_rows, -1);
    for (size_t i = 0; i < rows.size(); ++i) of_row[rows[i]] = (int32_t)i;
    f.n_sup = (int64_t)rows.size();
    f.h_sup_row = rows;
    f.h_sup_coef = coef;
    RVE_TRY(upload(f.sup_row, rows.data(), rows.size(), s));
    RVE_TRY(upload(f.sup_coef, coef.data(), coef.size(), s));
    RVE_TRY(upload(f.sup_of_row, of_row.data(), of_row.size(), s));
    RVE_CUDA(cudaStreamSynchronize(s));
    return RVE_OK;
}

int build_field_data(rve_mesh m) {
    cudaStream_t s = m->ctx->stream;
    std::vector<double> geo(m->nt * 10);
    RVE_CUDA(cudaMemcpyAsync(geo.data(), m->d_geo64.p, sizeof(double) * geo.size(),
                             cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    m->volume = 0;
    for (int64_t e = 0; e < m->nt; ++e) m->volume += geo[e * 10 + 9];
    m->mech.nc = 3;
    m->mech.nfield = 1;
    m->scal.nc = 1;
    m->scal.nfield = 2;
    RVE_TRY(build_constraints(m, m->mech, geo));
    RVE_TRY(build_constraints(m, m->scal, geo));
    return RVE_OK;
}

// Jacobi diagonals per phase (needs materials and the DOF map).
int build_diagonals(rve_mesh m) {
    cudaStream_t s = m->ctx->stream;
    m->ke_valid = false;   // the element matrices follow the map and the materials
    for (FieldDev* f : {&m->mech, &m->scal}) {
        const int64_t n = f->n_rows * 2 * f->nfield;
        RVE_TRY(f->diag64.ensure(sizeof(double) * n));
        RVE_TRY(f->diag32.ensure(sizeof(float) * n));
        RVE_CUDA(cudaMemsetAsync(f->diag64.p, 0, sizeof(double) * n, s));
        ElemView<double> ev;
        ev.nt = m->nt;
        ev.edofs = m->d_edofs.as<int32_t>();
        ev.geo = m->d_geo64.as<double>();
        ev.mat = (f->nc == 3 ? m->d_matm64 : m->d_mats64).as<double>();
        ev.phase = m->d_phase.as<uint8_t>();
        set_view_extras(ev, m, true);   // colour by colour: the diagonal is bit-reproducible
        launch_diag<double>(m->p, f->nc, f->n_rows, ev, f->diag64.as<double>(), s);
        launch_cast_d2f(n, f->diag64.as<double>(), f->diag32.as<float>(), s);
        m->ctx->launches += 2;
    }
    RVE_CUDA(cudaGetLastError());
    return RVE_OK;
}

// Packed FP32 element matrices of the mechanics for the tensor-core operator,
// formed in FP64 from the element data on first use after a change.
int ensure_element_matrices(rve_mesh m, cudaStream_t s) {
    if (m->ke_valid) return RVE_OK;
    const int p = m->p, ne = n_local(p);
    RVE_TRY(m->d_ke32.ensure((size_t)m->nt * element_matrix_floats(p) * sizeof(float)));
    RVE_TRY(m->d_kepairs.ensure((size_t)element_matrix_pairs(p) * sizeof(uint16_t)));
    RVE_TRY(m->d_keptab.ensure((size_t)9 * ne * ne * sizeof(double)));
    RVE_CUDA(operator_tc_prepare(p));
    RVE_CUDA(build_element_matrices(p, m->nt, m->d_geo64.as<double>(), m->d_matm64.as<double>(),
                                    m->d_ke32.as<float>(), m->d_kepairs.as<uint16_t>(), m->d_keptab.as<double>(), s));
    m->ctx->launches++;
    m->ke_valid = true;
    return RVE_OK;
}

// ------------------------------------------------------------- launch shape
Launch make_launch(int ncols, int64_t work, cudaStream_t s) {
    Launch L;
    L.ncols = ncols;
    const int B = ncols / 6;
    int gcd = 1;
    for (int d = 8; d >= 1; d >>= 1)
        if (B % d == 0) {
            gcd = d;
            break;
        }
    L.cpb = 6 * gcd;
    L.rows_per_block = 256 / L.cpb;
    const int gx = ncols / L.cpb;
    const int64_t want = (work + L.rows_per_block - 1) / L.rows_per_block;
    const int64_t cap = std::max<int64_t>(1, (sm_count() * 8) / gx);
    L.nby = (int)std::max<int64_t>(1, std::min(want, cap));
    L.stream = s;
    return L;
}

// ----------------------------------------------------------- the solver

// Starting data for a warm-started batch: the previous batch's solutions u_k
// (factors w_k) and, in mixed precision, their final projected FP64 residuals r_k.
// Column c starts from x0 = sum_k c_k u_k; because the modulus of the degrading
// phases is linear in w, its residual is
//   b(w) - K(w) x0 = sum_k c_k r_k - K_deg v - alpha K_deg u_macro,
//   v = sum_k c_k (w - w_k) u_k,   alpha = sum_k c_k (w - w_k),
// where K_deg is the operator over the degrading phases at unit modulus.  v is
// small (|w - w_k| |u|), so K_deg v is accurate in FP32; alpha is zero whenever
// the weights reproduce lines (two or three sources).
struct WarmStart {
    const double* x = nullptr;      // [n_rows][cols] previous solutions
    const double* r = nullptr;      // [n_rows][cols] their residuals (nullptr: recompute in FP64)
    int cols = 0;
    const int32_t* map = nullptr;   // [ncols][WARM_SOURCES] source columns
    const double* coef = nullptr;   // [ncols][WARM_SOURCES] c_k
    const double* dcoef = nullptr;  // [ncols][WARM_SOURCES] c_k (w - w_k)
    std::vector<double> alpha;      // [ncols]
    double degrade[2] = {0, 0};     // 1 for a phase whose modulus is proportional to w
    // energy-optimal combination: minus the degraded and the other phases' operator
    // applied to the sources (FP64, compact columns), and the column map and coefficients
    // (in dcoef) that form r0 = b(w) + their combination
    const double* nkx = nullptr;
    int kx_cols = 0;
    const int32_t* kx_map = nullptr;   // [ncols][WARM_SOURCES]
};

struct Solver {
    rve_mesh m;
    FieldDev& f;
    int B, ncols;
    int64_t n_rows;
    int fid;   // 0 mechanics, 1 scalar fields
    Launch L;
    cudaStream_t s;
    ColState cs64{};
    std::atomic<int64_t>* launches;

    Solver(rve_mesh mm, FieldDev& ff, int b)
        : m(mm), f(ff), B(b), ncols(6 * b), n_rows(ff.n_rows), fid(&ff == &mm->mech ? 0 : 1),
          s(mm->on_own_streams ? mm->stream : mm->ctx->stream), launches(&mm->ctx->launches) {
        L = make_launch(ncols, std::max<int64_t>(n_rows, mm->nt), s);
    }

    template <typename T>
    ElemView<T> ev(const DevBuf& scale) const {
        ElemView<T> e;
        e.nt = m->nt;
        e.edofs = m->d_edofs.as<int32_t>();
        if constexpr (sizeof(T) == 8) {
            e.geo = m->d_geo64.as<double>();
            e.mat = (f.nc == 3 ? m->d_matm64 : m->d_mats64).as<double>();
        } else {
            e.geo = m->d_geo32.as<float>();
            e.mat = (f.nc == 3 ? m->d_matm32 : m->d_mats32).as<float>();
        }
        e.phase = m->d_phase.as<uint8_t>();
        e.scale = scale.as<T>();
        set_view_extras(e, m);
        return e;
    }
    template <typename T>
    RowView<T> rv(const DevBuf& scale) const {
        RowView<T> r;
        r.n_rows = n_rows;
        r.diag = (sizeof(T) == 8 ? f.diag64 : f.diag32).as<T>();
        r.mask = m->bc == RVE_BC_DIRICHLET ? f.mask.as<uint8_t>() : nullptr;
        r.scale = scale.as<T>();
        r.nfield = f.nfield;
        r.nc = f.nc;
        r.m = f.m;
        r.n_sup = f.n_sup;
        r.sup_row = f.sup_row.as<int64_t>();
        r.sup_coef = f.sup_coef.as<double>();
        r.sup_of_row = f.sup_of_row.as<int32_t>();
        return r;
    }

    int alloc(bool mixed) {
        const size_t nv = (size_t)n_rows * ncols;
        if (nv >= ((size_t)1 << 31)) {   // the scatter kernels index vectors in 32 bits
            set_error("batch too large: a solve vector would exceed 2^31 entries");
            return RVE_ERR_INVALID_ARGUMENT;
        }
        RVE_TRY(m->x64f[fid].ensure(nv * 8));
        RVE_TRY(m->r64f[fid].ensure(nv * 8));
        RVE_TRY(m->b64.ensure(nv * 8));
        if (mixed) {
            RVE_TRY(m->x32.ensure(nv * 4));
            RVE_TRY(m->r32.ensure(nv * 4));
            RVE_TRY(m->p32.ensure(nv * 4));
            RVE_TRY(m->q32.ensure(nv * 4));
        } else {
            RVE_TRY(m->p64.ensure(nv * 8));
            RVE_TRY(m->q64.ensure(nv * 8));
        }
        const size_t np = (size_t)L.nby * ncols;
        // deterministic mode: one block of operator partials per colour
        RVE_TRY(m->epart.ensure(np * 8 * (m->ctx->opt.deterministic ? std::max(1, m->ncolour) : 1)));
        RVE_TRY(m->rzp.ensure(np * 8));
        RVE_TRY(m->cpart.ensure(np * 12 * 8));
        RVE_TRY(m->gpart.ensure(np * 12 * 8));
        RVE_TRY(m->mpart.ensure(np * 12 * 8));
        RVE_TRY(m->gsum.ensure((size_t)ncols * 12 * 8));
        RVE_TRY(m->msum.ensure((size_t)ncols * 12 * 8));
        // col state: rz, rz0, alpha, beta (4*ncols) + mu (12*ncols) + schur (144*ncols) + the fused
        // iteration's pq and rz accumulators (2*ACC_SLOTS*ncols) doubles,
        // then active, iters (ints) and flags
        const size_t nd = (size_t)ncols * (4 + 12 + 144 + 2 * ACC_SLOTS);
        RVE_TRY(m->colstate.ensure(nd * 8 + (size_t)ncols * 12 + 64));
        double* base = m->colstate.as<double>();
        cs64.rz = base;
        cs64.rz0 = base + ncols;
        cs64.alpha = base + 2 * ncols;
        cs64.beta = base + 3 * ncols;
        cs64.mu = base + 4 * ncols;
        cs64.schur = base + 16 * ncols;
        cs64.pq_acc = base + 160 * ncols;
        cs64.rz_acc = base + (160 + ACC_SLOTS) * ncols;
        int32_t* ib = reinterpret_cast<int32_t*>(base + nd);
        cs64.active = ib;
        cs64.iters = ib + ncols;
        cs64.flags = ib + 2 * ncols;            // [0] numeric flag, [1] loop counter
        cs64.n_list = ib + 2 * ncols + 4;
        cs64.list = ib + 2 * ncols + 16;
        cs64.tol = reinterpret_cast<const double*>(ib + 2 * ncols + 8);   // 8-byte aligned slot
        RVE_CUDA(cudaMemsetAsync(cs64.flags, 0, sizeof(int32_t), s));
        return RVE_OK;
    }

    // b = -K(s) u_macro for every column: the mesh keeps K_ph u_macro per phase at
    // unit modulus (two macro-load-only operator passes over 6 columns, once per
    // materials, boundary condition and precision), and each batch combines them
    // with its column scales.  FP64 mode uses the FP64 operator; mixed mode the
    // double-float evaluation of the FP32-data operator, so that its right-hand
    // side and true residual belong to one and the same discrete system.
    int rhs(double* b, bool mixed) {
        const int prec = mixed ? RVE_PREC_MIXED : RVE_PREC_FP64;
        if (!m->bph_valid[fid] || m->bph_prec[fid] != prec) {
            const size_t n6 = (size_t)n_rows * 6;
            RVE_TRY(m->bph[fid].ensure(2 * n6 * 8));
            RVE_CUDA(cudaMemsetAsync(m->bph[fid].p, 0, 2 * n6 * 8, s));
            const Launch L6 = make_launch(6, std::max<int64_t>(n_rows, m->nt), s);
            for (int ph = 0; ph < 2; ++ph) {
                double sc[12];
                float sc32[12];
                for (int c = 0; c < 6; ++c) {
                    sc[2 * c] = sc32[2 * c] = ph == 0 ? 1.0 : 0.0;
                    sc[2 * c + 1] = sc32[2 * c + 1] = ph == 1 ? 1.0 : 0.0;
                }
                double* y = m->bph[fid].as<double>() + ph * n6;
                if (mixed) {
                    // the double-float kernel returns -K u_macro: stored negated
                    float* lo = m->q32.as<float>();
                    RVE_TRY(upload(m->dscale32, sc32, 12, s));
                    RVE_CUDA(cudaMemsetAsync(lo, 0, n6 * 4, s));
                    launch_residual_df(m->p, f.nc, ev<float>(m->dscale32), nullptr, nullptr, y, lo, L6);
                    launch_axpy_f2d((int64_t)n6, lo, y, s);
                    launch_neg((int64_t)n6, y, s);
                    *launches += 3;
                } else {
                    RVE_TRY(upload(m->dscale64, sc, 12, s));
                    launch_operator<double>(m->p, f.nc, true, ev<double>(m->dscale64), nullptr, y, nullptr, L6);
                    *launches += 1;
                }
            }
            m->bph_valid[fid] = true;
            m->bph_prec[fid] = prec;
        }
        launch_rhs_combine(n_rows, B, m->bph[fid].as<double>(), m->scale64.as<double>(), b, s);
        *launches += 1;
        return RVE_OK;
    }

    // y = b - K x in mixed mode: the double-float evaluation of the FP32-data operator
    int residual_df(const double* x, double* y) {
        NvtxRange nvtx_("true residual, double-float, field %d, %d columns", fid, ncols);
        const bool prof = m->ctx->opt.profile != 0;
        auto& evs = m->ctx->ev;
        while (prof && evs.size() < 2) {
            cudaEvent_t e;
            RVE_CUDA(cudaEventCreate(&e));
            evs.push_back(e);
        }
        if (prof) RVE_CUDA(cudaEventRecord(evs[0], s));
        // FP32 scratch: x32 and p32 hold the split x, q32 the low words of r
        // (free between inner solves)
        const size_t nv = (size_t)n_rows * ncols;
        float* xh = m->x32.as<float>();
        float* xl = m->p32.as<float>();
        float* lo = m->q32.as<float>();
        RVE_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * nv, s));
        RVE_CUDA(cudaMemsetAsync(lo, 0, sizeof(float) * nv, s));
        launch_split_d2ff((int64_t)nv, x, xh, xl, s);
        launch_residual_df(m->p, f.nc, ev<float>(m->scale32), xh, xl, y, lo, L);
        launch_axpy_f2d((int64_t)nv, lo, y, s);
        *launches += 3;
        if (prof) {
            RVE_CUDA(cudaEventRecord(evs[1], s));
            RVE_CUDA(cudaEventSynchronize(evs[1]));
            float ms = 0;
            RVE_CUDA(cudaEventElapsedTime(&ms, evs[0], evs[1]));
            m->ctx->prof.res_ms += ms;
            m->ctx->prof.res_launches++;
        }
        return RVE_OK;
    }

    // y = -(K x + macro)  (FP64): the fluctuation residual b - K x
    int residual64(const double* x, double* y) {
        NvtxRange nvtx_("true residual, FP64, field %d, %d columns", fid, ncols);
        const bool prof = m->ctx->opt.profile != 0;
        auto& evs = m->ctx->ev;
        while (prof && evs.size() < 2) {
            cudaEvent_t e;
            RVE_CUDA(cudaEventCreate(&e));
            evs.push_back(e);
        }
        if (prof) RVE_CUDA(cudaEventRecord(evs[0], s));
        RVE_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n_rows * ncols, s));
        launch_operator<double>(m->p, f.nc, true, ev<double>(m->scale64), x, y, nullptr, L);
        launch_neg(n_rows * ncols, y, s);
        *launches += 2;
        if (prof) {
            RVE_CUDA(cudaEventRecord(evs[1], s));
            RVE_CUDA(cudaEventSynchronize(evs[1]));
            float ms = 0;
            RVE_CUDA(cudaEventElapsedTime(&ms, evs[0], evs[1]));
            m->ctx->prof.res_ms += ms;
            m->ctx->prof.res_launches++;
        }
        return RVE_OK;
    }

    template <typename T>
    int pcg(T* x, T* r, T* p, T* q, const DevBuf& scale, double tol, int max_iter, int& iters_out,
            bool& conv, const std::vector<double>* tolc = nullptr) {
        // profile mode launches one iteration at a time so that the byte and flop
        // counts follow the set of columns still iterating
        const bool prof = m->ctx->opt.profile != 0;
        // FP32 inner solve of the mechanics at p = 2, 3: the tensor-core operator
        int kern = m->ctx->opt.operator_kernel;
        if (kern == RVE_KERNEL_AUTO) kern = m->tuned_kernel != 0 ? m->tuned_kernel : RVE_KERNEL_CUDA_CORE;
        const bool det = m->ctx->opt.deterministic != 0;
        const bool use_tc =
            !det && sizeof(T) == 4 && operator_tc_supported(m->p, f.nc) && kern == RVE_KERNEL_TENSOR;
        if (use_tc) RVE_TRY(ensure_element_matrices(m, s));
        ColState cs = cs64;
        // the operator of the iteration runs one wave of resident blocks; its energy
        // partials (and the alpha reduction over them) have as many rows
        Launch Lop = L;
        Lop.nby_op = operator_grid_y<T>(m->p, f.nc, L, m->nt);
        Lop.n_colour = det ? m->ncolour : 0;
        // fused iteration (four kernels: operator, update, beta + loop control,
        // p-update): FP64 atomic accumulators replace the alpha and beta partial-row
        // reductions.  Not with constraint rows (their multipliers need the partial
        // rows), the tensor-core operator or the deterministic mode (atomic order).
        const bool fused = !det && !use_tc && f.m == 0;
        if (fused) {
            Lop.energy_acc = cs.pq_acc;
            RVE_CUDA(cudaMemsetAsync(cs.pq_acc, 0, sizeof(double) * 2 * ACC_SLOTS * ncols, s));   // pq_acc, rz_acc
        }
        const int kernels_per_iter = fused ? 4 : 6;
        RVE_CUDA(cudaMemcpyAsync(const_cast<double*>(cs.tol), &tol, sizeof(double), cudaMemcpyHostToDevice, s));
        RowView<T> rvw = rv<T>(scale);
        ElemView<T> evw = ev<T>(scale);
        launch_schur<T>(rvw, cs, L);
        launch_update<T>(rvw, x, r, p, q, cs, m->rzp.as<double>(), false, L, m->cpart.as<double>());
        launch_finalize_beta(f.m, m->rzp.as<double>(), m->cpart.as<double>(), cs, true, L);
        if (tolc) {
            RVE_TRY(upload(m->coltol, tolc->data(), tolc->size(), s));
            launch_column_tol(ncols, m->coltol.as<double>(), cs, s);
            *launches += 1;
        }
        launch_compact_active(cs.active, ncols, cs.list, cs.n_list, s);
        launch_pupdate<T>(rvw, r, p, q, cs, true, L);
        *launches += 6;
        std::vector<int32_t> act(ncols);
        conv = false;
        int n_act = ncols;
        auto read_active = [&]() -> int {
            RVE_CUDA(cudaMemcpyAsync(act.data(), cs.active, sizeof(int32_t) * ncols,
                                     cudaMemcpyDeviceToHost, s));
            RVE_CUDA(cudaStreamSynchronize(s));
            n_act = 0;
            for (int c = 0; c < ncols; ++c) n_act += act[c] != 0;
            return RVE_OK;
        };
        // profile mode: 6 events bracket the operator, alpha, update, beta and
        // p-update launches of an iteration
        if (prof && (int)m->ctx->ev.size() < 6) {
            for (int k = (int)m->ctx->ev.size(); k < 6; ++k) {
                cudaEvent_t e;
                RVE_CUDA(cudaEventCreate(&e));
                m->ctx->ev.push_back(e);
            }
        }
        auto evr = [&](int i, cudaStream_t st) {
            if (prof) cudaEventRecord(m->ctx->ev[i], st);
        };
        // in the graph body the compaction also runs the loop control
        bool loop_ctl = false;
        cudaGraphConditionalHandle loop_handle = 0;
        cudaError_t tc_err = cudaSuccess;
        auto iteration = [&](const Launch& Lx0) {
            Launch Lx = Lx0;
            Lx.nby_op = Lop.nby_op;
            Lx.n_colour = Lop.n_colour;
            Lx.energy_acc = Lop.energy_acc;
            double* epart_it = fused ? nullptr : m->epart.as<double>();
            evr(0, Lx.stream);
            if constexpr (sizeof(T) == 4) {
                if (use_tc) {
                    const cudaError_t e = launch_operator_tc(
                        m->p, m->nt, m->d_edofs.as<int32_t>(), m->d_ke32.as<float>(), m->d_kepairs.as<uint16_t>(),
                        m->d_phase.as<uint8_t>(), evw.scale, p, q, m->epart.as<double>(), cs.active, ncols, cs.list,
                        cs.n_list, Lx.op_rows(), cs.flags, Lx.stream);
                    if (e != cudaSuccess) tc_err = e;
                } else {
                    launch_operator<T>(m->p, f.nc, false, evw, p, q, epart_it, Lx, cs.active, cs.list, cs.n_list);
                }
            } else {
                launch_operator<T>(m->p, f.nc, false, evw, p, q, epart_it, Lx, cs.active, cs.list, cs.n_list);
            }
            evr(1, Lx.stream);
            if (!fused) launch_finalize_alpha<T>(m->epart.as<double>(), cs, Lx);
            evr(2, Lx.stream);
            if (fused)
                launch_update_fused<T>(rvw, x, r, p, q, cs, Lx);
            else
                launch_update<T>(rvw, x, r, p, q, cs, m->rzp.as<double>(), true, Lx, m->cpart.as<double>());
            evr(3, Lx.stream);
            if (fused) {
                launch_beta_compact_continue(cs, ncols, loop_handle, cs.flags + 1, max_iter, loop_ctl, Lx.stream);
            } else {
                launch_finalize_beta(f.m, m->rzp.as<double>(), m->cpart.as<double>(), cs, false, Lx);
                if (loop_ctl)
                    launch_compact_continue(cs.active, ncols, cs.list, cs.n_list, loop_handle, cs.flags + 1,
                                            max_iter, Lx.stream);
                else
                    launch_compact_active(cs.active, ncols, cs.list, cs.n_list, Lx.stream);
            }
            evr(4, Lx.stream);
            launch_pupdate<T>(rvw, r, p, q, cs, false, Lx);
            evr(5, Lx.stream);
        };
        if (!prof) {
            // The iterations run as one CUDA graph whose conditional WHILE node
            // repeats the iteration's six kernels; the compaction among them also
            // ends the loop on the device once no column is active or max_iter
            // iterations have run: no host round trip and no idle iterations.
            // The instantiated graph is kept per mesh, field and precision and
            // reused while every captured parameter is unchanged (the tolerance
            // lives in device memory).
            struct Key {
                int ncols, cpb, rows, nby, nby_op, p, nc, m, max_iter, tc, ncolour, fused;
                int64_t n_rows, n_sup, nt, n_nodes;
                const void* ptr[19];
            } key;
            std::memset(&key, 0, sizeof(key));
            key.ncols = L.ncols;
            key.cpb = L.cpb;
            key.rows = L.rows_per_block;
            key.nby = L.nby;
            key.nby_op = Lop.nby_op;
            key.p = m->p;
            key.nc = f.nc;
            key.m = rvw.m;
            key.max_iter = max_iter;
            key.n_rows = rvw.n_rows;
            key.n_sup = rvw.n_sup;
            key.nt = evw.nt;
            key.n_nodes = evw.n_nodes;
            key.tc = use_tc ? 1 : 0;
            key.ncolour = Lop.n_colour;
            key.fused = fused ? 1 : 0;
            const void* ptrs[19] = {x, r, p, q, m->epart.p, m->rzp.p, m->cpart.p, cs.rz, rvw.scale, rvw.diag,
                                    rvw.mask, rvw.sup_row, rvw.sup_coef, rvw.sup_of_row, evw.edofs, evw.geo,
                                    evw.mat, evw.phase, use_tc ? m->d_ke32.p : nullptr};
            std::memcpy(key.ptr, ptrs, sizeof(ptrs));
            auto& gc = m->graph_cache[fid][sizeof(T) == 4 ? 1 : 0];
            const unsigned char* kb = reinterpret_cast<const unsigned char*>(&key);
            const bool hit = gc.exec && gc.key.size() == sizeof(key) && std::memcmp(gc.key.data(), kb, sizeof(key)) == 0;
            if (!hit) {
                if (gc.exec) {
                    cudaGraphExecDestroy(gc.exec);
                    gc.exec = nullptr;
                }
                const auto g0 = std::chrono::steady_clock::now();
                cudaGraph_t graph = nullptr;
                RVE_CUDA(cudaGraphCreate(&graph, 0));
                struct GraphGuard {
                    cudaGraph_t g;
                    ~GraphGuard() { if (g) cudaGraphDestroy(g); }
                } gguard{graph};
                cudaGraphConditionalHandle handle;
                RVE_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
                cudaGraphNodeParams np = {};
                np.type = cudaGraphNodeTypeConditional;
                np.conditional.handle = handle;
                np.conditional.type = cudaGraphCondTypeWhile;
                np.conditional.size = 1;
                cudaGraphNode_t node;
                RVE_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
                cudaGraph_t body = np.conditional.phGraph_out[0];
                Launch Lc = L;
                Lc.stream = m->on_own_streams ? m->capture : m->ctx->capture;
                RVE_CUDA(cudaStreamBeginCaptureToGraph(Lc.stream, body, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal));
                loop_ctl = true;
                loop_handle = handle;
                iteration(Lc);
                loop_ctl = false;
                RVE_CUDA(cudaStreamEndCapture(Lc.stream, &body));
                if (tc_err != cudaSuccess) {
                    set_error(std::string("tensor-core operator launch: ") + cudaGetErrorString(tc_err));
                    return RVE_ERR_CUDA;
                }
                RVE_CUDA(cudaGraphInstantiate(&gc.exec, graph, 0));
                gc.key.assign(kb, kb + sizeof(key));
                std::lock_guard<std::mutex> lock(m->ctx->prof_mu);
                m->ctx->prof.graph_host_ms +=
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - g0).count();
                m->ctx->prof.graphs++;
            }
            cudaGraphExec_t exec = gc.exec;
            RVE_CUDA(cudaMemsetAsync(cs.flags + 1, 0, sizeof(int32_t), s));   // loop counter
            RVE_CUDA(cudaGraphLaunch(exec, s));
            RVE_CUDA(cudaGetLastError());
            int32_t loops = 0;
            RVE_CUDA(cudaMemcpyAsync(&loops, cs.flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            RVE_TRY(read_active());
            *launches += (int64_t)loops * kernels_per_iter;
            conv = n_act == 0;
        } else {
            RVE_TRY(read_active());
            for (int it = 0; it < max_iter && n_act > 0; ++it) {
                iteration(L);
                *launches += kernels_per_iter;
                RVE_CUDA(cudaGetLastError());
                if (tc_err != cudaSuccess) {
                    set_error(std::string("tensor-core operator launch: ") + cudaGetErrorString(tc_err));
                    return RVE_ERR_CUDA;
                }
                const int n_act_run = n_act;    // columns the iteration just run worked on
                RVE_TRY(read_active());
                // algorithmic bytes / flops of one operator launch of this solve:
                // vectors and flops of the columns still active, element data once
                const int ne = n_local(m->p), nmod = n_modes(m->p), nc = f.nc;
                const double sz = sizeof(T);
                const int na = n_act_run;
                const double bytes = 2.0 * n_rows * na * sz +
                                     (double)m->nt * (4.0 * ne + 10 * sz + (nc == 3 ? 21 : 6) * sz + 1);
                // FMAs per element and column: forward and backward contractions with the
                // non-zero entries of the edge/face table, plus per-mode gradient, stress
                // and back-mapping
                const double fma = 2.0 * table_nonzeros(m->p) * nc + nmod * (18.0 * nc + (nc == 3 ? 36 : 9));
                const double flops = 2.0 * fma * (double)m->nt * na;
                const double vb = (double)n_rows * na * sz;
                auto el = [&](int a2, int b2) {
                    float ms = 0;
                    return cudaEventElapsedTime(&ms, m->ctx->ev[a2], m->ctx->ev[b2]) == cudaSuccess ? (double)ms
                                                                                                    : 0.0;
                };
                ProfCounters& pc = m->ctx->prof;
                const double op_ms = el(0, 1);
                pc.op_ms += op_ms;
                pc.op_launches++;
                pc.op_bytes += bytes;
                pc.op_flops += flops;
                pc.op_cols += na;
                pc.op_cols_all += ncols;
                const int cl = 2 * (m->p - 1) + (nc == 3 ? 0 : 1);
                pc.cls_ms[cl] += op_ms;
                pc.cls_launches[cl]++;
                pc.cls_bytes[cl] += bytes;
                pc.cls_flops[cl] += flops;
                pc.cls_cols[cl] += na;
                pc.cls_cols_all[cl] += ncols;
                pc.fin_ms += el(1, 2) + el(3, 4);
                pc.upd_ms += el(2, 3);
                pc.upd_bytes += 6 * vb;
                pc.pup_ms += el(4, 5);
                pc.pup_bytes += 4 * vb;
            }
            conv = n_act == 0;
        }
        std::vector<int32_t> its(ncols);
        RVE_CUDA(cudaMemcpyAsync(its.data(), cs.iters, sizeof(int32_t) * ncols,
                                 cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
        iters_out = *std::max_element(its.begin(), its.end());
        return RVE_OK;
    }

    // Projects r in place (r <- r - C^T mu, the constraint-force part removed)
    // and returns per column rz = (r, M^-1 r) of the projected residual and the
    // worst relative value sqrt(rz / bnorm2).
    int rel_residual(double* r, const std::vector<double>& bnorm2, double& worst,
                     std::vector<double>* rz_out = nullptr) {
        ColState cs = cs64;
        RowView<double> rvw = rv<double>(m->scale64);
        if (f.m > 0) {
            launch_schur<double>(rvw, cs, L);
            launch_constraint_dot<double>(rvw, r, m->cpart.as<double>(), L);
            launch_constraint_multipliers(f.m, m->cpart.as<double>(), cs, L);
            *launches += 4;
        }
        launch_project_residual(rvw, rv<float>(m->scale32), r, cs, m->rzp.as<double>(), L);
        launch_reduce_partials(L.nby, ncols, m->rzp.as<double>(), m->gsum.as<double>(), s);
        *launches += 2;
        std::vector<double> rz(ncols);
        RVE_CUDA(cudaMemcpyAsync(rz.data(), m->gsum.p, sizeof(double) * ncols, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
        worst = 0;
        last_rel.assign(ncols, 0.0);
        for (int c = 0; c < ncols; ++c)
            if (bnorm2[c] > 0) {
                last_rel[c] = std::sqrt(std::max(rz[c], 0.0) / bnorm2[c]);
                worst = std::max(worst, last_rel[c]);
            }
        if (rz_out) *rz_out = rz;
        return RVE_OK;
    }

    // per-column relative residuals of the last rel_residual call
    std::vector<double> last_rel;

    // Per-column tolerances of an FP64 solve: a column already at rtol takes no part
    // (tolerance 1), the others are reduced by rtol / rel_c, so that no column whose
    // start is much better than the worst is driven down into rounding.
    std::vector<double> column_tolerances(double rtol) const {
        std::vector<double> t(ncols, 1.0);
        for (int c = 0; c < ncols && c < (int)last_rel.size(); ++c)
            if (last_rel[c] > rtol) t[c] = rtol / last_rel[c];
        return t;
    }

    // warm: optional starting data from the previous batch (see WarmStart).
    int run(int precision, SolveOut& out, const WarmStart* warm = nullptr) {
        NvtxRange nvtx_("cell solve, field %d, p = %d, %d columns, %s", fid, m->p, ncols,
                     precision == RVE_PREC_MIXED ? "mixed" : "fp64");
        const rve_options& o = m->ctx->opt;
        const bool mixed = precision == RVE_PREC_MIXED;
        RVE_TRY(alloc(mixed));
        const size_t nv = (size_t)n_rows * ncols;
        double* x64 = m->x64f[fid].as<double>();
        double* r64 = m->r64f[fid].as<double>();
        double* b64 = m->b64.as<double>();
        RVE_TRY(rhs(b64, mixed));
        // reference norms (b, P b); b is projected in place, which leaves the energy
        // reductions unchanged: (P b) . u = b . u for every admissible u
        std::vector<double> bn(ncols, 1.0);
        {
            double dummy;
            std::vector<double> ones(ncols, 1.0);
            RVE_TRY(rel_residual(b64, ones, dummy, &bn));
        }
        // A column whose projected right-hand side is rounding noise (a single-phase
        // RVE, whose exact fluctuation is zero) is solved by u = 0: its (b, P b)
        // is compared with the Voigt energy scale V <D>_jj of its unit load.
        std::vector<int> zero_cols;
        {
            std::vector<double> sc((size_t)ncols * 2);
            RVE_CUDA(cudaMemcpyAsync(sc.data(), m->scale64.p, sc.size() * 8, cudaMemcpyDeviceToHost, s));
            RVE_CUDA(cudaStreamSynchronize(s));
            for (int c = 0; c < ncols; ++c) {
                const int j = f.nc == 3 ? c % 6 : ((c % 6) < 3 ? 6 + c % 3 : 9 + c % 3);
                const double ev = sc[2 * c] * m->phase_voigt[0][j] + sc[2 * c + 1] * m->phase_voigt[1][j];
                if (bn[c] <= 1e-24 * ev) {
                    zero_cols.push_back(c);
                    bn[c] = 0.0;
                }
            }
        }
        auto zero_noise_columns = [&]() -> int {
            for (int c : zero_cols) {
                RVE_CUDA(cudaMemset2DAsync(r64 + c, (size_t)ncols * 8, 0, 8, (size_t)n_rows, s));
                RVE_CUDA(cudaMemset2DAsync(x64 + c, (size_t)ncols * 8, 0, 8, (size_t)n_rows, s));
            }
            return RVE_OK;
        };
        out.iterations = 0;
        out.sweeps = 0;
        out.converged = false;
        double rel = 1.0;
        if (warm) {
            launch_combine_columns<double, double>(n_rows, ncols, warm->cols, warm->map, warm->coef, warm->x, x64, s);
            *launches += 1;
            if (mixed && warm->nkx) {
                // energy-optimal start: r0 = b(w) - sum_k c_k (K_o + w K_d) x_k from the
                // sources' operator products (formed with the warm start, double-float)
                RVE_CUDA(cudaMemcpyAsync(r64, b64, nv * 8, cudaMemcpyDeviceToDevice, s));
                launch_combine_columns<double, double>(n_rows, ncols, warm->kx_cols, warm->kx_map, warm->dcoef,
                                                       warm->nkx, r64, s, true);
                *launches += 1;
            } else if (mixed && warm->r) {
                // the residual from the previous residuals (see WarmStart); a plain
                // FP32 b - K x0 would be too noisy to set the inner tolerance from
                launch_combine_columns<double, double>(n_rows, ncols, warm->cols, warm->map, warm->coef, warm->r, r64, s);
                *launches += 1;
                if (warm->degrade[0] != 0.0 || warm->degrade[1] != 0.0) {
                    float* v32 = m->x32.as<float>();
                    float* y32 = m->r32.as<float>();
                    launch_combine_columns<double, float>(n_rows, ncols, warm->cols, warm->map, warm->dcoef, warm->x, v32, s);
                    std::vector<float> sc32((size_t)ncols * 2);
                    for (int c = 0; c < ncols; ++c)
                        for (int ph = 0; ph < 2; ++ph) sc32[2 * c + ph] = (float)-warm->degrade[ph];
                    RVE_TRY(upload(m->dscale32, sc32.data(), sc32.size(), s));
                    RVE_CUDA(cudaMemsetAsync(y32, 0, nv * 4, s));
                    launch_operator<float>(m->p, f.nc, false, ev<float>(m->dscale32), v32, y32, nullptr, L);
                    launch_axpy_f2d((int64_t)nv, y32, r64, s);      // r0 -= K_deg v
                    *launches += 3;
                    bool any_alpha = false;
                    for (int c = 0; c < ncols; ++c)
                        for (int ph = 0; ph < 2; ++ph) {
                            sc32[2 * c + ph] = (float)(warm->alpha[c] * warm->degrade[ph]);
                            any_alpha |= sc32[2 * c + ph] != 0.0f;
                        }
                    if (any_alpha) {
                        // r0 -= alpha K_deg u_macro: the macro load of each phase at unit
                        // modulus is cached per mesh (the right-hand side's bph, formed by
                        // the same double-float operator), so this is a column combination
                        std::vector<double> sc64((size_t)ncols * 2);
                        for (int c = 0; c < ncols; ++c)
                            for (int ph = 0; ph < 2; ++ph) sc64[2 * c + ph] = warm->alpha[c] * warm->degrade[ph];
                        RVE_TRY(upload(m->dscale64, sc64.data(), sc64.size(), s));
                        launch_rhs_combine(n_rows, B, m->bph[fid].as<double>(), m->dscale64.as<double>(), r64, s,
                                           true);
                        *launches += 1;
                    }
                }
            } else {
                RVE_TRY(mixed ? residual_df(x64, r64) : residual64(x64, r64));
            }
            RVE_TRY(zero_noise_columns());
            RVE_TRY(rel_residual(r64, bn, rel));
        } else {
            RVE_CUDA(cudaMemcpyAsync(r64, b64, nv * 8, cudaMemcpyDeviceToDevice, s));
            RVE_CUDA(cudaMemsetAsync(x64, 0, nv * 8, s));
            RVE_TRY(zero_noise_columns());
            last_rel.assign(ncols, 1.0);
            for (int c : zero_cols) last_rel[c] = 0.0;
        }
        out.rel_res = rel;
        if (!mixed) {
            if (rel > o.rtol) {
                int its = 0;
                bool conv = false;
                const std::vector<double> tolc = column_tolerances(o.rtol);
                RVE_TRY(pcg<double>(x64, r64, m->p64.as<double>(), m->q64.as<double>(), m->scale64,
                                    o.rtol / rel, o.max_iter, its, conv, &tolc));
                out.iterations = its;
                RVE_TRY(residual64(x64, r64));
                RVE_TRY(zero_noise_columns());
                RVE_TRY(rel_residual(r64, bn, out.rel_res));
                out.converged = conv || out.rel_res <= o.rtol * 10;
            } else {
                out.converged = true;
            }
        } else {
            float* x32 = m->x32.as<float>();
            float* r32 = m->r32.as<float>();
            int total = 0;
            // Every sweep ends with the FP64 true residual, which alone decides
            // convergence and feeds the tensor reduction; a sweep whose starting
            // residual is already below rtol skips the FP32 inner solve.
            for (int sw = 0; sw < std::max(1, o.max_refine); ++sw) {
                if (out.rel_res > o.rtol) {
                    // reduce the residual only as far as the outer tolerance needs
                    // (half again for margin), never below what FP32 can resolve
                    const double inner = std::max(o.inner_rtol, 0.5 * o.rtol / out.rel_res);
                    launch_cast_d2f((int64_t)nv, r64, r32, s);
                    RVE_CUDA(cudaMemsetAsync(x32, 0, nv * 4, s));
                    *launches += 1;
                    int its = 0;
                    bool conv = false;
                    RVE_TRY(pcg<float>(x32, r32, m->p32.as<float>(), m->q32.as<float>(), m->scale32,
                                       std::min(inner, 0.5), o.max_iter, its, conv));
                    total += its;
                    launch_axpy_f2d((int64_t)nv, x32, x64, s);
                    *launches += 1;
                }
                RVE_TRY(residual_df(x64, r64));
                RVE_TRY(zero_noise_columns());
                RVE_TRY(rel_residual(r64, bn, out.rel_res));
                out.sweeps = sw + 1;
                out.converged = out.rel_res <= o.rtol;
                if (out.converged) break;
            }
            out.iterations = total;
        }
        // reductions for the tensors
        launch_gram(n_rows, b64, x64, r64, m->gpart.as<double>(), L);
        launch_reduce_partials(L.nby, ncols * 12, m->gpart.as<double>(), m->gsum.as<double>(), s);
        if (mixed) {
            // the volume-averaged stress is a diagnostic (Hill-Mandel): FP32 with
            // compensated sums, as the inner solve, on the FP32-rounded solution
            // (one conversion per entry instead of one per gathered value)
            float* u32 = m->x32.as<float>();
            launch_cast_d2f((int64_t)nv, x64, u32, s);
            launch_mean_stress<float, float>(m->p, f.nc, ev<float>(m->scale32), u32, m->mpart.as<double>(), L);
            *launches += 1;
        } else {
            launch_mean_stress<double, double>(m->p, f.nc, ev<double>(m->scale64), x64, m->mpart.as<double>(), L);
        }
        launch_reduce_partials(L.nby, ncols * 12, m->mpart.as<double>(), m->msum.as<double>(), s);
        *launches += 4;
        std::vector<double> Gs(ncols * 12), Ms(ncols * 12);
        int32_t flags = 0;
        RVE_CUDA(cudaMemcpyAsync(Gs.data(), m->gsum.p, Gs.size() * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaMemcpyAsync(Ms.data(), m->msum.p, Ms.size() * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaMemcpyAsync(&flags, cs64.flags, 4, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
        out.numeric = (flags & 1) != 0;
        out.timeout = (flags & 4) != 0;
        const double V = m->volume;
        out.tensor.assign((size_t)B * 36, 0.0);
        out.sig.assign((size_t)B * 36, 0.0);
        for (int b = 0; b < B; ++b)
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    const int ci = 6 * b + i, cj = 6 * b + j;
                    // V C_ij = V <D>_ij - b_i . u_j - u_i . r_j
                    const int irow = f.nc == 3 ? i : i % 3;   // flux component of the scalar fields
                    const double e = Ms[cj * 12 + 6 + irow] - Gs[ci * 12 + j] - Gs[ci * 12 + 6 + j];
                    out.tensor[b * 36 + i * 6 + j] = e / V;
                    out.sig[b * 36 + i * 6 + j] = Ms[cj * 12 + (f.nc == 3 ? i : i % 3)] / V;
                }
        return RVE_OK;
    }
};

// Non-zero entries of the edge/face part (j >= 4) of the basis table of order p.
int table_nonzeros(int p) {
    const Basis& B = basis(p);
    int n = 0;
    for (int k = 0; k < 3; ++k)
        for (int mm = 0; mm < B.nm; ++mm)
            for (int j = 4; j < B.ne; ++j)
                if (std::fabs(B.A[(k * B.nm + mm) * B.ne + j]) >= 1e-14) ++n;
    return n;
}

double rel_fro(const double* a, const double* b, int n) {
    double num = 0, den = 0;
    for (int i = 0; i < n; ++i) {
        num += (a[i] - b[i]) * (a[i] - b[i]);
        den += b[i] * b[i];
    }
    return den > 0 ? std::sqrt(num / den) : std::sqrt(num);
}

}  // namespace

// Starting guess for an RVE with degradation factor w from the solutions of the
// previous batch (factors pw): the polynomial in w through up to `order` of them.
// The nodes are the nearest factor, the farthest one and the one nearest the
// middle; a node closer than 1e-9 to another is dropped, and the order is lowered
// when w lies far outside the nodes (quadratic up to one node span beyond them,
// linear up to three), so that the coefficients stay small (at most about 8).
// Returns the number of sources written to src/coef.
static int warm_sources(const std::vector<double>& pw, double w, int order, int* src, double* coef) {
    const int n = (int)pw.size();
    int q0 = 0;
    for (int q = 1; q < n; ++q)
        if (std::fabs(pw[q] - w) < std::fabs(pw[q0] - w)) q0 = q;
    src[0] = q0;
    coef[0] = 1.0;
    if (order < 2 || n < 2) return 1;
    int q2 = q0;
    for (int q = 0; q < n; ++q)
        if (std::fabs(pw[q] - pw[q0]) > std::fabs(pw[q2] - pw[q0])) q2 = q;
    const double span = std::fabs(pw[q2] - pw[q0]);
    const double d = std::fabs(w - pw[q0]);
    if (span <= 1e-9 || d > 3.0 * span) return 1;
    int nodes[3] = {q0, q2, -1};
    int nn = 2;
    if (order >= 3 && d <= span && n >= 3) {
        const double mid = 0.5 * (pw[q0] + pw[q2]);
        int q1 = -1;
        for (int q = 0; q < n; ++q) {
            if (std::fabs(pw[q] - pw[q0]) <= 1e-9 || std::fabs(pw[q] - pw[q2]) <= 1e-9) continue;
            if (q1 < 0 || std::fabs(pw[q] - mid) < std::fabs(pw[q1] - mid)) q1 = q;
        }
        if (q1 >= 0 && std::fabs(pw[q1] - pw[q0]) > 0.25 * span && std::fabs(pw[q1] - pw[q2]) > 0.25 * span)
            nodes[nn++] = q1;
    }
    for (int i = 0; i < nn; ++i) {
        double l = 1.0;
        for (int j = 0; j < nn; ++j)
            if (j != i) l *= (w - pw[nodes[j]]) / (pw[nodes[i]] - pw[nodes[j]]);
        src[i] = nodes[i];
        coef[i] = l;
    }
    return nn;
}

// c = G^+ g for a small symmetric positive semi-definite G (n <= WARM_SOURCES):
// cyclic Jacobi rotations, eigenvalues at or below `rel` of the largest dropped (the
// sources are nearly parallel, so G is close to singular, and its entries carry the
// rounding of the double-float operator products).  False if G has no positive
// eigenvalue or a value is not finite.
static bool galerkin_solve(int n, const double* Gin, const double* g, double* c, double rel) {
    double A[WARM_SOURCES][WARM_SOURCES], V[WARM_SOURCES][WARM_SOURCES];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            A[i][j] = 0.5 * (Gin[i * n + j] + Gin[j * n + i]);
            V[i][j] = i == j ? 1.0 : 0.0;
            if (!std::isfinite(A[i][j])) return false;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i) {
            diag += A[i][i] * A[i][i];
            for (int j = i + 1; j < n; ++j) off += A[i][j] * A[i][j];
        }
        if (off <= 1e-30 * diag) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (A[p][q] == 0.0) continue;
                const double th = 0.5 * (A[q][q] - A[p][p]) / A[p][q];
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = cs * akp - sn * akq;
                    A[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = cs * apk - sn * aqk;
                    A[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {   // V <- V J
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = cs * vkp - sn * vkq;
                    V[k][q] = sn * vkp + cs * vkq;
                }
            }
    }
    double lmax = 0.0;
    for (int i = 0; i < n; ++i) lmax = std::max(lmax, A[i][i]);
    if (!(lmax > 0.0) || !std::isfinite(lmax)) return false;
    for (int i = 0; i < n; ++i) c[i] = 0.0;
    for (int k = 0; k < n; ++k) {
        if (!(A[k][k] > rel * lmax)) continue;
        double vg = 0.0;
        for (int i = 0; i < n; ++i) vg += V[i][k] * g[i];
        const double a = vg / A[k][k];
        for (int i = 0; i < n; ++i) c[i] += a * V[i][k];
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(c[i])) return false;
    return true;
}

int rve_debug_galerkin_solve(int n, const double* G, const double* g, double rel, double* c) {
    if (n < 1 || n > WARM_SOURCES || !G || !g || !c || !(rel >= 0.0)) {
        set_error("rve_debug_galerkin_solve: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    double out[WARM_SOURCES];
    if (!galerkin_solve(n, G, g, out, rel)) {
        set_error("rve_debug_galerkin_solve: non-finite entry or no positive eigenvalue");
        return RVE_ERR_NUMERIC;
    }
    for (int i = 0; i < n; ++i) c[i] = out[i];
    return RVE_OK;
}

// Energy-optimal warm start of the mechanics (warm_start >= 4).  With A(w) = K_o + w
// K_d (K_d: the degraded phases at unit modulus, K_o the others) and b(w) =
// -A(w) u_macro, the start for a column at w is x0 = sum_k c_k x_k over ns previous
// solutions of the same load case with G c = g, G_pk = x_p . A(w) x_k, g_p =
// x_p . b(w): the Galerkin projection onto their span (the energy minimisation of
// Sec. 2 restricted to it).  K_d x_k and K_o x_k come from one pass of the operator
// that defines the solve (double-float in mixed mode), so G is exact to rounding and
// its nearly singular directions (the extrapolation in w) survive; its residual
// r0 = b(w) - sum_k c_k (K_o + w K_d) x_k needs no further operator pass.
static int warm_galerkin(rve_mesh m, int B, const double* w_host, bool mixed, cudaStream_t s, WarmStart& ws,
                         bool& used) {
    used = false;
    const std::vector<double>& pw = m->warm_w[0];
    const int Bp = m->warm_cols[0] / 6;
    FieldDev& f = m->mech;
    if (Bp < 1 || (int)pw.size() != Bp || !m->bph_valid[0] || B < 1 || f.m != 0) return RVE_OK;
    const int64_t n_rows = f.n_rows;
    const double deg[2] = {ws.degrade[0], ws.degrade[1]};
    auto sph = [&](double w, int ph) { return deg[ph] != 0.0 ? w : 1.0; };
    // the operator of a mixed solve scales the phases by the FP32 column scales (the
    // right-hand side by the FP64 ones)
    auto wop = [&](double w) { return mixed ? (double)(float)w : w; };
    // sources: ns previous RVEs spread evenly over the previous batch's range of the
    // factor (its ends included), so that their span holds the line through the ends
    std::vector<int> ord(Bp);
    for (int q = 0; q < Bp; ++q) ord[q] = q;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return pw[a] < pw[b]; });
    const int ns = std::min(WARM_GALERKIN, Bp), kc = 6 * ns, k2 = 2 * kc;
    std::vector<int32_t> src(ns);
    for (int k = 0; k < ns; ++k) src[k] = ord[ns > 1 ? (int)std::lround((double)k * (Bp - 1) / (ns - 1)) : 0];
    // compact copy: columns h kc + 6 t + lc hold source t, load case lc, for h = 0 (the
    // degraded phases' product) and h = 1 (the other phases')
    std::vector<int32_t> omap((size_t)k2 * WARM_SOURCES, 0);
    std::vector<double> ocoef((size_t)k2 * WARM_SOURCES, 0.0);
    for (int h = 0; h < 2; ++h)
        for (int t = 0; t < ns; ++t)
            for (int lc = 0; lc < 6; ++lc) {
                omap[(size_t)(h * kc + 6 * t + lc) * WARM_SOURCES] = 6 * src[t] + lc;
                ocoef[(size_t)(h * kc + 6 * t + lc) * WARM_SOURCES] = 1.0;
            }
    RVE_TRY(upload(m->warm_src, src.data(), src.size(), s));
    RVE_TRY(upload(m->warm_omap, omap.data(), omap.size(), s));
    RVE_TRY(upload(m->warm_ocoef, ocoef.data(), ocoef.size(), s));
    RVE_TRY(m->warm_xs64.ensure((size_t)n_rows * k2 * 8));
    RVE_TRY(m->warm_xs.ensure((size_t)n_rows * k2 * 8));   // FP32 high and low words
    RVE_TRY(m->warm_kx.ensure((size_t)n_rows * k2 * 8));
    RVE_TRY(m->warm_klo.ensure((size_t)n_rows * k2 * 4));
    double* xs64 = m->warm_xs64.as<double>();
    float* xh = m->warm_xs.as<float>();
    float* xl = xh + (size_t)n_rows * k2;
    double* kx = m->warm_kx.as<double>();
    float* klo = m->warm_klo.as<float>();
    launch_combine_columns<double, double>(n_rows, k2, m->warm_cols[0], m->warm_omap.as<int32_t>(),
                                           m->warm_ocoef.as<double>(), m->warm[0].as<double>(), xs64, s);
    std::vector<float> sc((size_t)k2 * 2);
    std::vector<double> nsc((size_t)k2 * 2);
    for (int c = 0; c < k2; ++c)
        for (int ph = 0; ph < 2; ++ph) {
            const double v = c < kc ? deg[ph] : 1.0 - deg[ph];
            sc[2 * c + ph] = (float)v;
            nsc[2 * c + ph] = -v;
        }
    RVE_CUDA(cudaMemsetAsync(kx, 0, (size_t)n_rows * k2 * 8, s));
    Solver sk(m, f, 2 * ns);
    if (mixed) {
        // kx + klo = -K_part (x_t + u_macro) in double-float; then + K_part u_macro
        // from the cached per-phase loads (rhs_combine adds -(s0 y0 + s1 y1))
        launch_split_d2ff((int64_t)n_rows * k2, xs64, xh, xl, s);
        RVE_TRY(upload(m->warm_ksc, sc.data(), sc.size(), s));
        RVE_TRY(upload(m->warm_phs, nsc.data(), nsc.size(), s));
        RVE_CUDA(cudaMemsetAsync(klo, 0, (size_t)n_rows * k2 * 4, s));
        launch_residual_df(m->p, f.nc, sk.ev<float>(m->warm_ksc), xh, xl, kx, klo, sk.L);
        launch_axpy_f2d((int64_t)n_rows * k2, klo, kx, s);
        launch_rhs_combine(n_rows, 2 * ns, m->bph[0].as<double>(), m->warm_phs.as<double>(), kx, s, true);
    } else {
        // FP64 operator with the scales -K_part
        RVE_TRY(upload(m->warm_phs, nsc.data(), nsc.size(), s));
        launch_operator<double>(m->p, f.nc, false, sk.ev<double>(m->warm_phs), xs64, kx, nullptr, sk.L);
    }
    const int splits = 16, nout = 2 * ns + 2;
    RVE_TRY(m->warm_gram.ensure((size_t)splits * 6 * ns * nout * 8));
    launch_warm_gram(n_rows, ns, m->warm_src.as<int32_t>(), m->warm_cols[0], m->warm[0].as<double>(), kx,
                     m->bph[0].as<double>(), m->warm_gram.as<double>(), splits, s);
    m->ctx->launches += 7;
    std::vector<double> h((size_t)splits * 6 * ns * nout), P((size_t)6 * ns * nout, 0.0);
    RVE_CUDA(cudaMemcpyAsync(h.data(), m->warm_gram.p, h.size() * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    for (int sp = 0; sp < splits; ++sp)
        for (size_t i = 0; i < P.size(); ++i) P[i] += h[(size_t)sp * P.size() + i];
    const size_t n = (size_t)6 * B * WARM_SOURCES;
    std::vector<int32_t> cmap(n, 0), kmap(n, 0);
    std::vector<double> ccoef(n, 0.0), kcoef(n, 0.0);
    for (int b = 0; b < B; ++b) {
        const double w = w_host[b], wf = wop(w);
        for (int lc = 0; lc < 6; ++lc) {
            double G[WARM_GALERKIN * WARM_GALERKIN], g[WARM_GALERKIN], c[WARM_GALERKIN];
            for (int p = 0; p < ns; ++p) {
                const double* Pp = &P[((size_t)lc * ns + p) * nout];
                g[p] = -(sph(w, 0) * Pp[2 * ns] + sph(w, 1) * Pp[2 * ns + 1]);
                for (int t = 0; t < ns; ++t) G[p * ns + t] = -(Pp[ns + t] + wf * Pp[t]);   // x_p . (K_o + w K_d) x_t
            }
            // exact to rounding: directions below 1e-12 of the largest are noise
            if (!galerkin_solve(ns, G, g, c, 1e-12)) return RVE_OK;   // the caller falls back to the polynomial
            const int col = 6 * b + lc;
            for (int k = 0; k < ns; ++k) {
                const size_t i = (size_t)col * WARM_SOURCES + k;
                cmap[i] = 6 * src[k] + lc;
                ccoef[i] = c[k];
                // r0 = b(w) + sum_k c_k (-K_o x_k) + sum_k c_k w (-K_d x_k)
                kmap[i] = kc + 6 * k + lc;
                kcoef[i] = c[k];
                kmap[i + ns] = 6 * k + lc;
                kcoef[i + ns] = c[k] * wf;
            }
        }
    }
    RVE_TRY(upload(m->warm_map, cmap.data(), n, s));
    RVE_TRY(upload(m->warm_coef, ccoef.data(), n, s));
    RVE_TRY(upload(m->warm_kxmap, kmap.data(), n, s));
    RVE_TRY(upload(m->warm_dcoef, kcoef.data(), n, s));
    ws.x = m->warm[0].as<double>();
    ws.r = mixed ? m->warm_r[0].as<double>() : nullptr;
    ws.cols = m->warm_cols[0];
    ws.map = m->warm_map.as<int32_t>();
    ws.coef = m->warm_coef.as<double>();
    ws.dcoef = m->warm_dcoef.as<double>();
    ws.alpha.assign((size_t)6 * B, 0.0);
    ws.nkx = kx;
    ws.kx_cols = k2;
    ws.kx_map = m->warm_kxmap.as<int32_t>();
    used = true;
    return RVE_OK;
}

// Solve B RVEs of one mesh whose degradation factors are in d_w (device).
int rve::homogenise_batch(rve_mesh m, int B, const double* d_w, double* C, double* K, double* D,
                          rve_stats* st, const double* w_host) {
    NvtxRange nvtx_("homogenise batch of %d RVEs (%d tets, p = %d)", B, (int)m->nt, m->p);
    cudaStream_t s = m->on_own_streams ? m->stream : m->ctx->stream;
    const int ncols = 6 * B;
    RVE_TRY(m->scale64.ensure((size_t)ncols * 2 * 8));
    RVE_TRY(m->scale32.ensure((size_t)ncols * 2 * 4));
    const int prec = m->ctx->opt.precision;
    // mechanics
    launch_column_scales<double>(B, d_w, m->deg.apply_to_yarn, true, m->scale64.as<double>(), s);
    launch_column_scales<float>(B, d_w, m->deg.apply_to_yarn, true, m->scale32.as<float>(), s);
    m->ctx->launches += 2;
    SolveOut om, osc;
    // warm start from the mesh's previous batch (set up by macro_update_gauss_points)
    const bool mixed = prec == RVE_PREC_MIXED;
    auto warm_ready = [&](int f) { return w_host && m->warm_cols[f] > 0 && !m->warm_w[f].empty(); };
    auto build_warm = [&](int f, WarmStart& ws) -> int {
        const std::vector<double>& pw = m->warm_w[f];
        ws.degrade[0] = f == 0 ? 1.0 : 0.0;
        ws.degrade[1] = (f == 0 && m->deg.apply_to_yarn) ? 1.0 : 0.0;
        // a field that does not degrade has one solution for every w: the nearest will do
        const bool degrades = ws.degrade[0] != 0.0 || ws.degrade[1] != 0.0;
        if (f == 0 && degrades && m->ctx->opt.warm_start >= 4 && m->bph_prec[0] == prec) {
            bool used = false;
            RVE_TRY(warm_galerkin(m, B, w_host, mixed, s, ws, used));
            if (used) return RVE_OK;
        }
        const int order = degrades ? std::max(1, std::min(m->ctx->opt.warm_start, WARM_SOURCES)) : 1;
        const size_t n = (size_t)6 * B * WARM_SOURCES;
        std::vector<int32_t> cmap(n, 0);
        std::vector<double> ccoef(n, 0.0), dcoef(n, 0.0);
        ws.alpha.assign((size_t)6 * B, 0.0);
        for (int b = 0; b < B; ++b) {
            int src[WARM_SOURCES];
            double cf[WARM_SOURCES];
            const int ns = warm_sources(pw, w_host[b], order, src, cf);
            double al = 0.0;
            for (int k = 0; k < ns; ++k) al += cf[k] * (w_host[b] - pw[src[k]]);
            if (ns > 1) al = 0.0;   // the weights reproduce lines: zero up to rounding
            for (int c = 0; c < 6; ++c) {
                ws.alpha[6 * b + c] = al;
                for (int k = 0; k < ns; ++k) {
                    const size_t i = (size_t)(6 * b + c) * WARM_SOURCES + k;
                    cmap[i] = 6 * src[k] + c;
                    ccoef[i] = cf[k];
                    dcoef[i] = cf[k] * (w_host[b] - pw[src[k]]);
                }
            }
        }
        RVE_TRY(upload(m->warm_map, cmap.data(), n, s));
        RVE_TRY(upload(m->warm_coef, ccoef.data(), n, s));
        RVE_TRY(upload(m->warm_dcoef, dcoef.data(), n, s));
        ws.x = m->warm[f].as<double>();
        ws.r = mixed ? m->warm_r[f].as<double>() : nullptr;
        ws.cols = m->warm_cols[f];
        ws.map = m->warm_map.as<int32_t>();
        ws.coef = m->warm_coef.as<double>();
        ws.dcoef = m->warm_dcoef.as<double>();
        return RVE_OK;
    };
    auto keep_warm = [&](int f, FieldDev& fd) -> int {
        if (!w_host) return RVE_OK;
        const size_t nb = (size_t)fd.n_rows * 6 * B * 8;
        (void)nb;
        m->warm[f].swap(m->x64f[f]);
        if (mixed) m->warm_r[f].swap(m->r64f[f]);
        m->warm_cols[f] = 6 * B;
        m->warm_w[f].assign(w_host, w_host + B);
        return RVE_OK;
    };
    {
        Solver sv(m, m->mech, B);
        if (warm_ready(0)) {
            WarmStart ws;
            RVE_TRY(build_warm(0, ws));
            RVE_TRY(sv.run(prec, om, &ws));
        } else {
            RVE_TRY(sv.run(prec, om));
        }
        RVE_TRY(keep_warm(0, m->mech));
    }
    // thermal and moisture: transport is not degraded (Sec. 5), so these cell
    // problems are the same for every point of the mesh.  With transport_once
    // the batched call solves them once per mesh (one RVE, six columns) and
    // gives all of the mesh's points their tensors; otherwise every batch solves
    // them (warm-started from the previous batch's solutions).
    const bool reuse_scalar = w_host != nullptr && m->ctx->opt.transport_once != 0;
    if (reuse_scalar && m->scal_cached) {
        osc = m->scal_out;
        osc.iterations = 0;
        osc.sweeps = 0;
    } else {
        const int Bs = reuse_scalar ? 1 : B;
        launch_column_scales<double>(Bs, d_w, 0, false, m->scale64.as<double>(), s);
        launch_column_scales<float>(Bs, d_w, 0, false, m->scale32.as<float>(), s);
        m->ctx->launches += 2;
        Solver sv(m, m->scal, Bs);
        if (!reuse_scalar && warm_ready(1)) {
            WarmStart ws;
            RVE_TRY(build_warm(1, ws));
            RVE_TRY(sv.run(prec, osc, &ws));
        } else {
            RVE_TRY(sv.run(prec, osc));
        }
        if (reuse_scalar) {
            m->scal_out = osc;
            m->scal_cached = true;
        } else {
            RVE_TRY(keep_warm(1, m->scal));
        }
    }
    if (reuse_scalar) {
        // every RVE of the batch gets the mesh's scalar tensors
        const std::vector<double> t1 = osc.tensor, s1 = osc.sig;
        osc.tensor.resize((size_t)B * 36);
        osc.sig.resize((size_t)B * 36);
        for (int b = 0; b < B; ++b) {
            std::memcpy(&osc.tensor[(size_t)b * 36], t1.data(), 36 * sizeof(double));
            std::memcpy(&osc.sig[(size_t)b * 36], s1.data(), 36 * sizeof(double));
        }
    }
    double hm_m = 0, hm_s = 0;
    for (int b = 0; b < B; ++b) {
        double c[36], cs[36];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                const double* T = &om.tensor[b * 36];
                c[i * 6 + j] = 0.5 * (T[i * 6 + j] + T[j * 6 + i]) * m->mc.ref_mech;
                cs[i * 6 + j] = om.sig[b * 36 + i * 6 + j] * m->mc.ref_mech;
            }
        hm_m = std::max(hm_m, rel_fro(cs, c, 36));
        if (C) std::memcpy(C + 36 * b, c, sizeof(c));
        double k[9], d[9], ks[9];
        const double* T = &osc.tensor[b * 36];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                k[i * 3 + j] = 0.5 * (T[i * 6 + j] + T[j * 6 + i]) * m->mc.ref_k;
                d[i * 3 + j] = 0.5 * (T[(3 + i) * 6 + 3 + j] + T[(3 + j) * 6 + 3 + i]) * m->mc.ref_d;
                ks[i * 3 + j] = osc.sig[b * 36 + i * 6 + j] * m->mc.ref_k;
            }
        hm_s = std::max(hm_s, rel_fro(ks, k, 9));
        if (K) std::memcpy(K + 9 * b, k, sizeof(k));
        if (D) std::memcpy(D + 9 * b, d, sizeof(d));
    }
    if (st) {
        st->iterations_mech = std::max(st->iterations_mech, om.iterations);
        st->iterations_scalar = std::max(st->iterations_scalar, osc.iterations);
        st->refine_sweeps = std::max(st->refine_sweeps, std::max(om.sweeps, osc.sweeps));
        st->converged = st->converged && om.converged && osc.converged;
        st->rel_residual_mech = std::max(st->rel_residual_mech, om.rel_res);
        st->rel_residual_scalar = std::max(st->rel_residual_scalar, osc.rel_res);
        st->hill_mandel_mech = std::max(st->hill_mandel_mech, hm_m);
        st->hill_mandel_scalar = std::max(st->hill_mandel_scalar, hm_s);
    }
    if (om.timeout || osc.timeout) {
        set_error("a bounded wait inside the tensor-core operator gave up");
        return RVE_ERR_TIMEOUT;
    }
    if (om.numeric || osc.numeric) {
        set_error("non-finite or non-positive value in a PCG reduction");
        return RVE_ERR_NUMERIC;
    }
    if (!(om.converged && osc.converged)) {
        set_error("PCG did not reach rtol within max_iter");
        return RVE_ERR_NOT_CONVERGED;
    }
    return RVE_OK;
}

namespace {
bool finite_pos(double v) { return std::isfinite(v) && v > 0; }
}  // namespace

// =================================================================== C ABI
extern "C" {

const char* rve_strerror(int code) {
    switch (code) {
        case RVE_OK: return "ok";
        case RVE_ERR_INVALID_ARGUMENT: return "invalid argument";
        case RVE_ERR_BAD_MESH: return "bad mesh";
        case RVE_ERR_NOT_SPD: return "material not positive definite";
        case RVE_ERR_NOT_CONVERGED: return "not converged";
        case RVE_ERR_NUMERIC: return "numeric error (NaN/Inf)";
        case RVE_ERR_CUDA: return "CUDA error";
        case RVE_ERR_NO_DEVICE: return "no suitable CUDA device";
        case RVE_ERR_OUT_OF_MEMORY: return "out of device memory";
        case RVE_ERR_STATE: return "call order violated";
        case RVE_ERR_TIMEOUT: return "bounded device wait timed out";
        default: return "unknown error";
    }
}

const char* rve_last_error(void) { return g_last_error.c_str(); }

void rve_default_options(rve_options* o) {
    if (!o) return;
    o->device = 0;
    o->precision = RVE_PREC_FP64;
    o->rtol = 1e-10;
    o->max_iter = 20000;
    o->inner_rtol = 1e-6;
    o->max_refine = 4;
    o->check_every = 16;
    o->batch = 0;
    o->stream = nullptr;
    o->profile = 0;
    o->warm_start = 4;
    o->transport_once = 0;
    o->operator_kernel = 0;
    o->deterministic = 0;
}

int rve_create(rve_ctx* out, const rve_options* opts) {
    if (!out) {
        set_error("null output handle");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    *out = nullptr;
    rve_options o;
    rve_default_options(&o);
    if (opts) o = *opts;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        set_error("no CUDA device visible");
        return RVE_ERR_NO_DEVICE;
    }
    if (o.device < 0 || o.device >= n) {
        set_error("device ordinal out of range");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    cudaDeviceProp prop;
    RVE_CUDA(cudaGetDeviceProperties(&prop, o.device));
    if (!(prop.major == 10 && prop.minor == 3)) {
        set_error("librve is built for sm_103a (GB300); found compute capability " +
                  std::to_string(prop.major) + "." + std::to_string(prop.minor));
        return RVE_ERR_NO_DEVICE;
    }
    RVE_CUDA(cudaSetDevice(o.device));
    auto* c = new rve_ctx_s();
    c->opt = o;
    c->device = o.device;
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            set_error("cudaStreamCreate failed");
            return RVE_ERR_CUDA;
        }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        set_error("cudaStreamCreate failed");
        return RVE_ERR_CUDA;
    }
    upload_basis_tables();
    if (cudaGetLastError() != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        set_error("uploading basis tables failed");
        return RVE_ERR_CUDA;
    }
    *out = c;
    return RVE_OK;
}

int rve_destroy(rve_ctx c) {
    if (!c) return RVE_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (c->capture) cudaStreamDestroy(c->capture);
    delete c;
    return RVE_OK;
}

int rve_set_options(rve_ctx c, const rve_options* o) {
    RVE_TRY(check_ctx(c));
    if (!o || !(o->rtol > 0) || o->max_iter <= 0 || (o->precision != RVE_PREC_FP64 && o->precision != RVE_PREC_MIXED)) {
        set_error("invalid options");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    const void* keep_stream = c->opt.stream;
    const int keep_dev = c->opt.device;
    c->opt = *o;
    c->opt.stream = const_cast<void*>(keep_stream);
    c->opt.device = keep_dev;
    return RVE_OK;
}

int rve_get_options(rve_ctx c, rve_options* o) {
    RVE_TRY(check_ctx(c));
    if (!o) return RVE_ERR_INVALID_ARGUMENT;
    *o = c->opt;
    o->stream = c->stream;
    return RVE_OK;
}

int rve_mesh_load(rve_ctx c, const double* xyz, int64_t nv, const int32_t* tets, int64_t nt,
                  const uint8_t* phase, const double* fibre_dir, int p, rve_mesh* out) {
    RVE_TRY(check_ctx(c));
    if (!out || !xyz || !tets || nv < 4 || nt < 1 || p < 1 || p > 3 || nt > (int64_t)INT32_MAX / 20) {
        set_error("rve_mesh_load: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    *out = nullptr;
    auto m = std::make_unique<rve_mesh_s>();
    m->ctx = c;
    m->p = p;
    m->bc = RVE_BC_DIRICHLET;
    m->nv = nv;
    m->nt = nt;
    m->xyz.assign(xyz, xyz + 3 * nv);
    m->tets.assign(tets, tets + 4 * nt);
    m->phase.assign(nt, 0);
    if (phase)
        for (int64_t e = 0; e < nt; ++e) {
            if (phase[e] > 1) {
                set_error("phase must be 0 (matrix) or 1 (yarn)");
                return RVE_ERR_INVALID_ARGUMENT;
            }
            m->phase[e] = phase[e];
        }
    m->tangent.assign(3 * nt, 0.0);
    for (int64_t e = 0; e < nt; ++e) m->tangent[3 * e] = 1.0;
    if (fibre_dir) m->tangent.assign(fibre_dir, fibre_dir + 3 * nt);
    cudaStream_t s = c->stream;
    RVE_TRY(upload(m->d_xyz, m->xyz.data(), m->xyz.size(), s));
    RVE_TRY(upload(m->d_phase, m->phase.data(), m->phase.size(), s));
    RVE_TRY(upload(m->d_tangent, m->tangent.data(), m->tangent.size(), s));
    RVE_TRY(rebuild_map(m.get()));
    RVE_TRY(build_field_data(m.get()));
    *out = m.release();
    return RVE_OK;
}

int rve_mesh_free(rve_ctx c, rve_mesh m) {
    if (!m) return RVE_OK;
    if (c) cudaSetDevice(c->device);
    if (m->ctx) cudaStreamSynchronize(m->ctx->stream);
    delete m;
    return RVE_OK;
}

int rve_mesh_info(rve_ctx c, rve_mesh m, rve_mesh_stats* o) {
    RVE_TRY(check_ctx(c));
    if (!m || !o) return RVE_ERR_INVALID_ARGUMENT;
    o->n_vertices = m->map.V;
    o->n_edges = m->map.E;
    o->n_faces = m->map.F;
    o->n_tets = m->nt;
    o->n_scalar_dofs = m->map.N;
    int64_t nb = 0;
    if (m->bc == RVE_BC_DIRICHLET)
        for (auto b : m->map.boundary) nb += b;
    o->n_constrained = nb;
    o->p = m->p;
    o->bc = m->bc;
    o->volume = m->volume;
    return RVE_OK;
}

int rve_set_materials(rve_ctx c, rve_mesh m, const rve_matrix_props* mp, const rve_yarn_props* yp,
                      double T_C, double c_wt, double t_h, const rve_degradation* deg) {
    RVE_TRY(check_ctx(c));
    if (!m || !mp || !yp) {
        set_error("rve_set_materials: null argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    rve_degradation dg{-0.001682, 126.0, 1.5, 0};
    if (deg) dg = *deg;
    if (!std::isfinite(T_C) || !std::isfinite(c_wt) || !std::isfinite(t_h) || t_h < 0 ||
        !(T_C < dg.Tg_C) || T_C <= -273.15 || !finite_pos(dg.c_sat_wt) || !std::isfinite(dg.beta)) {
        set_error("degradation state out of range (need -273.15 < T < Tg, t >= 0)");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    // positive definiteness of the constituents
    bool ok = finite_pos(mp->E) && mp->nu > -1 && mp->nu < 0.5 && finite_pos(mp->k) && finite_pos(mp->d);
    ok = ok && finite_pos(yp->E1) && finite_pos(yp->E2) && finite_pos(yp->G12) && yp->nu23 > -1 &&
         yp->nu23 < 1 && finite_pos(yp->k1) && finite_pos(yp->k2) && finite_pos(yp->d1) &&
         finite_pos(yp->d2);
    // TI normal block: 1 - nu23 - 2 nu12^2 E2/E1 > 0 (with 1 + nu23 > 0)
    ok = ok && (1 - yp->nu23 - 2 * yp->nu12 * yp->nu12 * yp->E2 / yp->E1) > 0;
    if (!ok) {
        set_error("constituent properties are not positive definite");
        return RVE_ERR_NOT_SPD;
    }
    cudaStream_t s = c->stream;
    MaterialConsts mc;
    mc.Em = mp->E; mc.num = mp->nu; mc.km = mp->k; mc.dm = mp->d;
    mc.E1 = yp->E1; mc.E2 = yp->E2; mc.G12 = yp->G12; mc.nu12 = yp->nu12; mc.nu23 = yp->nu23;
    mc.k1 = yp->k1; mc.k2 = yp->k2; mc.d1 = yp->d1; mc.d2 = yp->d2;
    mc.ref_mech = mp->E;
    mc.ref_k = mp->k;
    mc.ref_d = mp->d;
    const int64_t nt = m->nt;
    RVE_TRY(m->d_matm64.ensure(nt * 21 * 8));
    RVE_TRY(m->d_matm32.ensure(nt * 21 * 4));
    RVE_TRY(m->d_mats64.ensure(nt * 12 * 8));
    RVE_TRY(m->d_mats32.ensure(nt * 12 * 4));
    RVE_CUDA(cudaMemsetAsync(m->d_flag.p, 0, sizeof(int32_t), s));
    launch_materials(nt, m->d_phase.as<uint8_t>(), m->d_tangent.as<double>(), mc,
                     m->d_matm64.as<double>(), m->d_matm32.as<float>(), m->d_mats64.as<double>(),
                     m->d_mats32.as<float>(), m->d_flag.as<int32_t>(), s);
    c->launches++;
    int32_t bad = 0;
    RVE_CUDA(cudaMemcpyAsync(&bad, m->d_flag.p, 4, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    if (bad) {
        set_error("yarn tangent is zero or TI tensor not invertible");
        return RVE_ERR_NOT_SPD;
    }
    {
        std::vector<double> geo(nt * 10), mm(nt * 21), ms(nt * 12);
        RVE_CUDA(cudaMemcpyAsync(geo.data(), m->d_geo64.p, geo.size() * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaMemcpyAsync(mm.data(), m->d_matm64.p, mm.size() * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaMemcpyAsync(ms.data(), m->d_mats64.p, ms.size() * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
        static const int diag21[6] = {0, 6, 11, 15, 18, 20};   // (i,i) in the upper-triangular Voigt layout
        for (int ph = 0; ph < 2; ++ph)
            for (int k = 0; k < 12; ++k) m->phase_voigt[ph][k] = 0.0;
        for (int64_t e = 0; e < nt; ++e) {
            const int ph = m->phase[e];
            const double v = geo[e * 10 + 9];
            for (int k = 0; k < 6; ++k) m->phase_voigt[ph][k] += v * mm[e * 21 + diag21[k]];
            for (int k = 0; k < 3; ++k) {
                m->phase_voigt[ph][6 + k] += v * ms[e * 12 + k];
                m->phase_voigt[ph][9 + k] += v * ms[e * 12 + 6 + k];
            }
        }
    }
    m->mc = mc;
    m->deg = dg;
    m->T_C = T_C;
    m->c_wt = c_wt;
    m->t_h = t_h;
    m->have_materials = true;
    m->bph_valid[0] = m->bph_valid[1] = false;
    RVE_TRY(build_diagonals(m));
    return RVE_OK;
}

int rve_set_bc(rve_ctx c, rve_mesh m, int bc) {
    RVE_TRY(check_ctx(c));
    if (!m || (bc != RVE_BC_DIRICHLET && bc != RVE_BC_PERIODIC && bc != RVE_BC_NEUMANN)) {
        set_error("rve_set_bc: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    m->bph_valid[0] = m->bph_valid[1] = false;
    const bool fold_changes = (bc == RVE_BC_PERIODIC) != (m->bc == RVE_BC_PERIODIC);
    const int old = m->bc;
    m->bc = bc;
    if (fold_changes) {
        int rc = rebuild_map(m);
        if (rc != RVE_OK) {
            m->bc = old;
            std::string keep = g_last_error;
            rebuild_map(m);
            build_field_data(m);
            if (m->have_materials) build_diagonals(m);
            set_error(keep);
            return rc;
        }
    }
    RVE_TRY(build_field_data(m));
    if (m->have_materials) RVE_TRY(build_diagonals(m));
    return RVE_OK;
}

// Profile counters accumulated between two snapshots, into the caller's stats.
static void fill_profile(const ProfCounters& a, const ProfCounters& b, rve_stats* st) {
    st->op_ms = b.op_ms - a.op_ms;
    st->op_launches = b.op_launches - a.op_launches;
    st->op_bytes = b.op_bytes - a.op_bytes;
    st->op_flops = b.op_flops - a.op_flops;
    st->update_ms = b.upd_ms - a.upd_ms;
    st->update_bytes = b.upd_bytes - a.upd_bytes;
    st->pupdate_ms = b.pup_ms - a.pup_ms;
    st->pupdate_bytes = b.pup_bytes - a.pup_bytes;
    st->finalize_ms = b.fin_ms - a.fin_ms;
    st->residual_ms = b.res_ms - a.res_ms;
    st->residual_launches = b.res_launches - a.res_launches;
    st->graph_host_ms = b.graph_host_ms - a.graph_host_ms;
    st->graphs = b.graphs - a.graphs;
    const double cols = b.op_cols_all - a.op_cols_all;
    st->op_active_frac = cols > 0 ? (b.op_cols - a.op_cols) / cols : 0.0;
    for (int k = 0; k < 6; ++k) {
        st->op_class_ms[k] = b.cls_ms[k] - a.cls_ms[k];
        st->op_class_launches[k] = b.cls_launches[k] - a.cls_launches[k];
        st->op_class_bytes[k] = b.cls_bytes[k] - a.cls_bytes[k];
        st->op_class_flops[k] = b.cls_flops[k] - a.cls_flops[k];
        const double cc = b.cls_cols_all[k] - a.cls_cols_all[k];
        st->op_class_active_frac[k] = cc > 0 ? (b.cls_cols[k] - a.cls_cols[k]) / cc : 0.0;
    }
}

static int weak_sigma(rve_mesh m, int fid, const double* d_w, std::vector<double>& sig);

int rve_homogenise_weak(rve_ctx c, rve_mesh m, double* C, double* K, double* D, double* C_energy,
                        double* K_energy, double* D_energy, rve_stats* st) {
    RVE_TRY(check_ctx(c));
    if (!m) return RVE_ERR_INVALID_ARGUMENT;
    const int rc = rve_homogenise(c, m, C_energy, K_energy, D_energy, st);
    if (rc != RVE_OK) return rc;
    cudaStream_t s = c->stream;
    double state[3] = {m->T_C, m->c_wt, m->t_h};
    DevBuf dstate;
    RVE_TRY(dstate.ensure(4 * 8));
    RVE_CUDA(cudaMemcpyAsync(dstate.p, state, sizeof(state), cudaMemcpyHostToDevice, s));
    double* d = dstate.as<double>();
    launch_degradation(1, d, d + 1, d + 2, m->deg.beta, m->deg.Tg_C, m->deg.c_sat_wt, d + 3, s);
    c->launches++;
    std::vector<double> sm, ss;
    RVE_TRY(weak_sigma(m, 0, d + 3, sm));
    RVE_TRY(weak_sigma(m, 1, d + 3, ss));
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J)
            if (C) C[I * 6 + J] = sm[I * 6 + J] * m->mc.ref_mech;
    for (int I = 0; I < 3; ++I)
        for (int J = 0; J < 3; ++J) {
            if (K) K[I * 3 + J] = ss[I * 6 + J] * m->mc.ref_k;
            if (D) D[I * 3 + J] = ss[I * 6 + 3 + J] * m->mc.ref_d;
        }
    return RVE_OK;
}

int rve_homogenise(rve_ctx c, rve_mesh m, double* C, double* K, double* D, rve_stats* st) {
    NvtxRange nvtx_("rve_homogenise");
    RVE_TRY(check_ctx(c));
    if (!m) return RVE_ERR_INVALID_ARGUMENT;
    if (!m->have_materials) {
        set_error("rve_set_materials must be called before rve_homogenise");
        return RVE_ERR_STATE;
    }
    auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = c->launches;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->converged = 1;
    }
    cudaStream_t s = c->stream;
    bounds_begin(s);
    double Th[1] = {m->T_C}, ch[1] = {m->c_wt}, th[1] = {m->t_h};
    DevBuf tmp;
    RVE_TRY(tmp.ensure(4 * 8));
    double* d = tmp.as<double>();
    RVE_CUDA(cudaMemcpyAsync(d, Th, 8, cudaMemcpyHostToDevice, s));
    RVE_CUDA(cudaMemcpyAsync(d + 1, ch, 8, cudaMemcpyHostToDevice, s));
    RVE_CUDA(cudaMemcpyAsync(d + 2, th, 8, cudaMemcpyHostToDevice, s));
    launch_degradation(1, d, d + 1, d + 2, m->deg.beta, m->deg.Tg_C, m->deg.c_sat_wt, d + 3, s);
    c->launches++;
    const ProfCounters pc0 = c->prof;
    int rc = homogenise_batch(m, 1, d + 3, C, K, D, st);
    RVE_CUDA(cudaStreamSynchronize(s));
    rc = bounds_outcome(rc, s);
    if (st) {
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        st->kernel_launches = c->launches - l0;
        fill_profile(pc0, c->prof, st);
    }
    return rc;
}

// sigma_bar = -D^T lambda / V (Eq. eq_homo_stress) of one field from the solution
// left by rve_homogenise (six columns), with the constraint rows C of the BC
// written out (Eqs. eq_RVE_disc_Eqs, eq_mat_C_and_D) and lambda recovered from
// the equilibrium K u + C^T lambda = 0 of the total field u = u_tilde + X:
//   Dirichlet: one row per boundary DOF, lambda = -(K u) there;
//   periodic:  one row u_s - u_master(s) per image DOF s of the unfolded mesh,
//              lambda_s = -(K u)_s (each image DOF sits in exactly one row);
//   Neumann:   the six (three) uniform-traction rows plus the rigid-mode rows,
//              lambda = -(C C^T)^-1 C K u (the rigid-mode multipliers vanish).
// D = C X, with X the nodal interpolant of the unit macro fields: in the
// hierarchic basis a linear field lives on the vertex functions alone, so only
// vertex rows carry D, and for Dirichlet and periodic only the vertex
// multipliers are formed (K u at vertices, from the element-mean stresses).
static int weak_sigma(rve_mesh m, int fid, const double* d_w, std::vector<double>& sig /* [ni][6] */) {
    cudaStream_t s = m->ctx->stream;
    FieldDev& f = fid == 0 ? m->mech : m->scal;
    const int nc = f.nc, ni = nc == 3 ? 6 : 3, ncols = 6;
    // this field's column scales at the RVE's degradation factor (transport does not degrade)
    DevBuf dscale;
    RVE_TRY(dscale.ensure((size_t)ncols * 2 * 8));
    launch_column_scales<double>(1, d_w, fid == 0 ? m->deg.apply_to_yarn : 0, fid == 0, dscale.as<double>(), s);
    m->ctx->launches++;
    ElemView<double> ev;
    ev.nt = m->nt;
    ev.edofs = m->d_edofs.as<int32_t>();
    ev.geo = m->d_geo64.as<double>();
    ev.mat = (nc == 3 ? m->d_matm64 : m->d_mats64).as<double>();
    ev.phase = m->d_phase.as<uint8_t>();
    ev.scale = dscale.as<double>();
    set_view_extras(ev, m);
    const double* u = m->x64f[fid].as<double>();
    // unit macro field of load case I at a point y (engineering shear: E_ab = E_ba = 1/2)
    auto Xval = [&](int I, const double* y, int c) -> double {
        if (nc == 1) return y[I];
        static const int VI[6] = {0, 1, 2, 0, 1, 2}, VJ[6] = {0, 1, 2, 1, 2, 0};
        if (I < 3) return c == I ? y[I] : 0.0;
        double v = 0.0;
        if (c == VI[I]) v += 0.5 * y[VJ[I]];
        if (c == VJ[I]) v += 0.5 * y[VI[I]];
        return v;
    };
    DevBuf dout;
    RVE_TRY(dout.ensure((size_t)12 * ncols * 8));
    std::vector<double> out((size_t)12 * ncols, 0.0);
    sig.assign((size_t)ni * ncols, 0.0);
    if (m->bc == RVE_BC_DIRICHLET || m->bc == RVE_BC_PERIODIC) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int64_t v = 0; v < m->nv; ++v)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], m->xyz[3 * v + a]);
                hi[a] = std::max(hi[a], m->xyz[3 * v + a]);
            }
        std::vector<int32_t> vid;
        std::vector<double> w;
        for (int64_t v = 0; v < m->nv; ++v) {
            const double* y = &m->xyz[3 * v];
            double dy[3] = {0, 0, 0};
            bool on = false;
            for (int a = 0; a < 3; ++a) {
                const double tol = 1e-9 * (hi[a] - lo[a]);
                const bool at_lo = std::fabs(y[a] - lo[a]) <= tol, at_hi = std::fabs(y[a] - hi[a]) <= tol;
                if (m->bc == RVE_BC_DIRICHLET) {
                    on = on || at_lo || at_hi;
                } else if (at_hi) {   // image of the vertex with this coordinate at the low face
                    on = true;
                    dy[a] = hi[a] - lo[a];
                }
            }
            if (!on) continue;
            if (m->bc == RVE_BC_DIRICHLET)
                for (int a = 0; a < 3; ++a) dy[a] = y[a];
            vid.push_back((int32_t)v);
            for (int I = 0; I < ni; ++I)
                for (int c = 0; c < nc; ++c) w.push_back(Xval(I, dy, c));
        }
        DevBuf dr, dvid, dw;
        RVE_TRY(dr.ensure((size_t)m->nv * nc * ncols * 8));
        RVE_CUDA(cudaMemsetAsync(dr.p, 0, (size_t)m->nv * nc * ncols * 8, s));
        RVE_TRY(upload(dvid, vid.data(), vid.size(), s));
        RVE_TRY(upload(dw, w.data(), w.size(), s));
        launch_vertex_reactions(m->p, nc, ev, m->d_lverts.as<int32_t>(), u, dr.as<double>(), ncols, s);
        // sigma_I = -(1/V) sum_rows D_I lambda = (1/V) sum_constrained-vertices X_I . (K u)
        launch_weighted_vertex_sum((int)vid.size(), ni, nc, dvid.as<int32_t>(), dw.as<double>(), dr.as<double>(),
                                   ncols, dout.as<double>(), s);
        m->ctx->launches += 2;
        RVE_CUDA(cudaGetLastError());
        RVE_CUDA(cudaMemcpyAsync(out.data(), dout.p, (size_t)ni * ncols * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < ni * ncols; ++i) sig[i] = out[i] / m->volume;
        return RVE_OK;
    }
    // Neumann: K u on every DOF, then C K u over the constraint rows
    const int mr = f.m;
    DevBuf dy;
    RVE_TRY(dy.ensure((size_t)f.n_rows * ncols * 8));
    RVE_CUDA(cudaMemsetAsync(dy.p, 0, (size_t)f.n_rows * ncols * 8, s));
    Launch L = make_launch(ncols, std::max<int64_t>(f.n_rows, m->nt), s);
    launch_operator<double>(m->p, nc, true, ev, u, dy.as<double>(), nullptr, L);
    launch_rows_dot(f.n_sup, mr, f.sup_row.as<int64_t>(), f.sup_coef.as<double>(), dy.as<double>(), ncols,
                    dout.as<double>(), s);
    m->ctx->launches += 2;
    RVE_CUDA(cudaGetLastError());
    RVE_CUDA(cudaMemcpyAsync(out.data(), dout.p, (size_t)mr * ncols * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    // C C^T and D = C X from the host copies of the rows
    std::vector<double> CC((size_t)mr * mr, 0.0), Dm((size_t)mr * ni, 0.0);
    const DofMap& M = m->map;
    for (size_t i = 0; i < f.h_sup_row.size(); ++i) {
        const double* cr = &f.h_sup_coef[i * mr];
        for (int a = 0; a < mr; ++a)
            for (int b = 0; b < mr; ++b) CC[a * mr + b] += cr[a] * cr[b];
        const int64_t row = f.h_sup_row[i], dof = row / nc;
        const int c = (int)(row % nc);
        if (M.dof_vertex[dof] < 0) continue;
        const double* y = &m->xyz[3 * (int64_t)M.dof_vertex[dof]];
        for (int I = 0; I < ni; ++I) {
            const double xv = Xval(I, y, c);
            for (int a = 0; a < mr; ++a) Dm[a * ni + I] += cr[a] * xv;
        }
    }
    // lambda = -(C C^T)^-1 C K u (Cholesky of the m x m Gram matrix)
    std::vector<double> Lc((size_t)mr * mr, 0.0);
    for (int j = 0; j < mr; ++j) {
        double d = CC[j * mr + j];
        for (int k = 0; k < j; ++k) d -= Lc[j * mr + k] * Lc[j * mr + k];
        if (!(d > 0)) {
            set_error("rve_homogenise_weak: constraint rows are linearly dependent");
            return RVE_ERR_NUMERIC;
        }
        Lc[j * mr + j] = std::sqrt(d);
        for (int r = j + 1; r < mr; ++r) {
            double t = CC[r * mr + j];
            for (int k = 0; k < j; ++k) t -= Lc[r * mr + k] * Lc[j * mr + k];
            Lc[r * mr + j] = t / Lc[j * mr + j];
        }
    }
    const int t0 = nc == 3 ? 6 : 1;   // first uniform-traction row (rigid-mode rows come first)
    for (int col = 0; col < ncols; ++col) {
        std::vector<double> z(mr);
        for (int a = 0; a < mr; ++a) {
            double t = -out[a * ncols + col];
            for (int k = 0; k < a; ++k) t -= Lc[a * mr + k] * z[k];
            z[a] = t / Lc[a * mr + a];
        }
        for (int a = mr - 1; a >= 0; --a) {
            double t = z[a];
            for (int k = a + 1; k < mr; ++k) t -= Lc[k * mr + a] * z[k];
            z[a] = t / Lc[a * mr + a];
        }
        for (int I = 0; I < ni; ++I) {
            double acc = 0.0;
            for (int a = t0; a < t0 + ni; ++a) acc += Dm[a * ni + I] * z[a];
            sig[I * ncols + col] = -acc / m->volume;
        }
    }
    return RVE_OK;
}

// RVEs per device pass for one mesh: enough columns to fill the GPU (about 16M
// vector entries per field), a multiple of 8, between 8 and 256.
static int auto_batch(rve_mesh m) {
    const double rows = (double)m->mech.n_rows;
    int B = (int)(16.0e6 / (rows * 6.0));
    B = std::max(8, std::min(256, B));
    return (B / 8) * 8;
}

// W_dev (optional, [G]): the degradation factor 1 - omega of each point, used in
// place of the degradation law at (T, c, t) (which are then not read).
static int macro_update_impl(rve_ctx c, const rve_mesh* meshes, int n_meshes, int64_t G,
                             const double* T_dev, const double* c_dev, const double* t_dev,
                             const int32_t* mesh_id, double* C_dev, double* K_dev, double* D_dev,
                             int32_t* status_dev, rve_stats* st, const double* W_dev = nullptr) {
    NvtxRange nvtx_("macro_update_gauss_points: %lld points on %d meshes", (long long)G, n_meshes);
    bounds_begin(c->stream);
    cudaStream_t s = c->stream;
    // group points by mesh
    std::vector<std::vector<int64_t>> groups(n_meshes);
    for (int64_t g = 0; g < G; ++g) {
        if (mesh_id[g] < 0 || mesh_id[g] >= n_meshes) {
            set_error("mesh_id out of range");
            return RVE_ERR_INVALID_ARGUMENT;
        }
        groups[mesh_id[g]].push_back(g);
    }
    std::vector<int> work;
    bool repeated = false;   // one mesh under two ids: its entries share state, so run in order
    for (int mi = 0; mi < n_meshes; ++mi) {
        if (groups[mi].empty()) continue;
        rve_mesh m = meshes[mi];
        if (!m || !m->have_materials) {
            set_error("mesh without materials in macro_update_gauss_points");
            return RVE_ERR_STATE;
        }
        for (int mj : work) repeated |= meshes[mj] == m;
        work.push_back(mi);
    }
    // host copy of the states (or of the factors), used only to order the points
    // of each mesh
    std::vector<double> hT_all(G), hc_all(G), ht_all(G), hW_all;
    if (G > 0 && W_dev) {
        hW_all.resize(G);
        RVE_CUDA(cudaMemcpyAsync(hW_all.data(), W_dev, G * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
        for (int64_t g = 0; g < G; ++g)
            if (!(hW_all[g] > 0.0 && hW_all[g] <= 1.0)) {
                set_error("macro_update_gauss_points_w: degradation factor outside (0, 1]");
                return RVE_ERR_INVALID_ARGUMENT;
            }
    } else if (G > 0) {
        RVE_CUDA(cudaMemcpyAsync(hT_all.data(), T_dev, G * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaMemcpyAsync(hc_all.data(), c_dev, G * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaMemcpyAsync(ht_all.data(), t_dev, G * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
    }
    // One mesh's points in warm-started batches, on stream sm; results scattered
    // into the caller's arrays (each point written by exactly one mesh).
    auto solve_mesh = [&](int mi, cudaStream_t sm, rve_stats* stm, std::string* err) -> int {
        auto& grp = groups[mi];
        rve_mesh m = meshes[mi];
        const int Bmax = c->opt.batch > 0 ? c->opt.batch : (m->tuned_batch > 0 ? m->tuned_batch : auto_batch(m));
        // order the points by degradation factor so that each batch starts from
        // the solutions of its neighbours in the previous batch; no solution is
        // carried over from an earlier call
        std::vector<double> wg(grp.size());
        {
            const rve_degradation& dg = m->deg;
            for (size_t i = 0; i < grp.size(); ++i) {
                const int64_t g = grp[i];
                if (W_dev) {
                    wg[i] = hW_all[g];
                    continue;
                }
                const double cn = std::min(std::max(hc_all[g] / dg.c_sat_wt, 0.0), 1.0);
                const double alpha = dg.beta * std::log(1.0 - (hT_all[g] + 273.15) / (dg.Tg_C + 273.15));
                wg[i] = std::exp(-cn * alpha * ht_all[g] / 24.0);
            }
            std::vector<size_t> order(grp.size());
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](size_t a2, size_t b2) { return wg[a2] < wg[b2]; });
            std::vector<int64_t> g2(grp.size());
            std::vector<double> w2(grp.size());
            for (size_t i = 0; i < grp.size(); ++i) {
                g2[i] = grp[order[i]];
                w2[i] = wg[order[i]];
            }
            grp.swap(g2);
            wg.swap(w2);
        }
        m->warm_cols[0] = m->warm_cols[1] = 0;
        m->warm_w[0].clear();
        m->warm_w[1].clear();
        m->scal_cached = false;
        DevBuf d_idx, d_tmp, d_res;
        std::vector<double> res;
        int rc_mesh = RVE_OK;
        auto fail = [&](int rc) {
            *err = last_error();
            return rc;
        };
        int rc0 = upload(d_idx, grp.data(), grp.size(), sm);
        if (rc0 != RVE_OK) return fail(rc0);
        for (size_t off = 0; off < grp.size(); off += Bmax) {
            const int B = (int)std::min<size_t>(Bmax, grp.size() - off);
            const int64_t* idx = d_idx.as<int64_t>() + off;
            rc0 = d_tmp.ensure((size_t)B * 4 * 8);
            if (rc0 != RVE_OK) return fail(rc0);
            double* st3 = d_tmp.as<double>();
            double* dw = st3 + 3 * B;
            if (W_dev) {
                // the factors themselves: gathered three times over, the first copy is the batch's w
                launch_gather_states(B, idx, W_dev, W_dev, W_dev, st3, sm);
                dw = st3;
                c->launches += 1;
            } else {
                launch_gather_states(B, idx, T_dev, c_dev, t_dev, st3, sm);
                launch_degradation(B, st3, st3 + B, st3 + 2 * B, m->deg.beta, m->deg.Tg_C, m->deg.c_sat_wt, dw,
                                   sm);
                c->launches += 2;
            }
            res.assign((size_t)B * 55, 0.0);
            std::vector<double> hC((size_t)B * 36), hK((size_t)B * 9), hD((size_t)B * 9);
            int rc = homogenise_batch(m, B, dw, hC.data(), hK.data(), hD.data(), stm,
                                      c->opt.warm_start ? &wg[off] : nullptr);
            if (rc != RVE_OK && rc != RVE_ERR_NOT_CONVERGED && rc != RVE_ERR_NUMERIC) return fail(rc);
            if (rc != RVE_OK) {
                rc_mesh = rc;
                *err = last_error();
            }
            for (int b = 0; b < B; ++b) {
                std::memcpy(&res[(size_t)b * 55], &hC[(size_t)b * 36], 36 * 8);
                std::memcpy(&res[(size_t)b * 55 + 36], &hK[(size_t)b * 9], 9 * 8);
                std::memcpy(&res[(size_t)b * 55 + 45], &hD[(size_t)b * 9], 9 * 8);
                res[(size_t)b * 55 + 54] = rc;
            }
            rc0 = upload(d_res, res.data(), res.size(), sm);
            if (rc0 != RVE_OK) return fail(rc0);
            launch_scatter_results(B, idx, d_res.as<double>(), C_dev, K_dev, D_dev, status_dev, sm);
            c->launches++;
            if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(sm) != cudaSuccess) {
                set_error("macro_update_gauss_points: a batch's kernels failed");
                return fail(RVE_ERR_CUDA);
            }
        }
        return rc_mesh;
    };
    // Meshes are independent: with more than one, each gets its own streams and host
    // thread so that one mesh's small kernels and host round trips overlap another's
    // work.  Profile mode keeps one stream (its event timings assume it).
    const bool parallel = work.size() > 1 && c->opt.profile == 0 && !repeated;
    if (!parallel) {
        int rc_all = RVE_OK;
        for (int mi : work) {
            std::string err;
            const int rc = solve_mesh(mi, s, st, &err);
            if (rc != RVE_OK && rc != RVE_ERR_NOT_CONVERGED && rc != RVE_ERR_NUMERIC) return rc;
            if (rc != RVE_OK) rc_all = rc;
        }
        return rc_all;
    }
    cudaEvent_t ready;
    RVE_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    struct EventGuard {
        cudaEvent_t e;
        ~EventGuard() { cudaEventDestroy(e); }
    } eg{ready};
    RVE_CUDA(cudaEventRecord(ready, s));
    for (int mi : work) {
        rve_mesh m = meshes[mi];
        if (!m->stream) RVE_CUDA(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
        if (!m->capture) RVE_CUDA(cudaStreamCreateWithFlags(&m->capture, cudaStreamNonBlocking));
        RVE_CUDA(cudaStreamWaitEvent(m->stream, ready, 0));
    }
    struct OwnStreams {   // back to the context's streams however this call ends
        const rve_mesh* ms;
        const std::vector<int>& w;
        ~OwnStreams() {
            for (int mi : w) ms[mi]->on_own_streams = false;
        }
    } own{meshes, work};
    for (int mi : work) meshes[mi]->on_own_streams = true;
    const size_t nw = work.size();
    std::vector<int> rcs(nw, RVE_OK);
    std::vector<std::string> errs(nw);
    std::vector<rve_stats> sts(nw);
    for (auto& x : sts) {
        std::memset(&x, 0, sizeof(x));
        x.converged = 1;
    }
    {
        std::vector<std::thread> threads;
        for (size_t k = 0; k < nw; ++k)
            threads.emplace_back([&, k]() {
                cudaSetDevice(c->device);
                rcs[k] = solve_mesh(work[k], meshes[work[k]]->stream, st ? &sts[k] : nullptr, &errs[k]);
            });
        for (auto& t : threads) t.join();
    }
    // the caller's stream continues after every mesh's work
    for (int mi : work) {
        rve_mesh m = meshes[mi];
        cudaEvent_t done;
        RVE_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        cudaEventRecord(done, m->stream);
        cudaStreamWaitEvent(s, done, 0);
        cudaEventDestroy(done);
    }
    if (st)
        for (const auto& x : sts) {
            st->iterations_mech = std::max(st->iterations_mech, x.iterations_mech);
            st->iterations_scalar = std::max(st->iterations_scalar, x.iterations_scalar);
            st->refine_sweeps = std::max(st->refine_sweeps, x.refine_sweeps);
            st->converged = st->converged && x.converged;
            st->rel_residual_mech = std::max(st->rel_residual_mech, x.rel_residual_mech);
            st->rel_residual_scalar = std::max(st->rel_residual_scalar, x.rel_residual_scalar);
            st->hill_mandel_mech = std::max(st->hill_mandel_mech, x.hill_mandel_mech);
            st->hill_mandel_scalar = std::max(st->hill_mandel_scalar, x.hill_mandel_scalar);
        }
    int rc_all = RVE_OK;
    for (size_t k = 0; k < nw; ++k) {
        if (rcs[k] == RVE_OK) continue;
        set_error(errs[k]);
        if (rcs[k] != RVE_ERR_NOT_CONVERGED && rcs[k] != RVE_ERR_NUMERIC) return rcs[k];
        rc_all = rcs[k];
    }
    return rc_all;
}

int macro_update_gauss_points_dev(rve_ctx c, const rve_mesh* meshes, int n_meshes, int64_t G,
                                  const double* T_dev, const double* c_dev, const double* t_dev,
                                  const int32_t* mesh_id_host, double* C_dev, double* K_dev,
                                  double* D_dev, int32_t* status_dev, int mode, rve_stats* st) {
    RVE_TRY(check_ctx(c));
    if (!meshes || n_meshes <= 0 || G < 0 || (G > 0 && (!T_dev || !c_dev || !t_dev || !mesh_id_host || !C_dev ||
        !K_dev || !D_dev || !status_dev)) || mode != RVE_MODE_PCG) {
        set_error("macro_update_gauss_points_dev: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = c->launches;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->converged = 1;
    }
    const ProfCounters pc0 = c->prof;
    int rc = macro_update_impl(c, meshes, n_meshes, G, T_dev, c_dev, t_dev, mesh_id_host, C_dev, K_dev,
                               D_dev, status_dev, st);
    rc = bounds_outcome(rc, c->stream);
    if (st) {
        cudaStreamSynchronize(c->stream);
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        st->kernel_launches = c->launches - l0;
        fill_profile(pc0, c->prof, st);
    }
    return rc;
}

int macro_update_gauss_points(rve_ctx c, const rve_mesh* meshes, int n_meshes, int64_t G,
                              const double* T_C, const double* c_wt, const double* t_h,
                              const int32_t* mesh_id, double* C, double* K, double* D,
                              int32_t* status, int mode, rve_stats* st) {
    RVE_TRY(check_ctx(c));
    if (G < 0 || (G > 0 && (!T_C || !c_wt || !t_h || !mesh_id || !C || !K || !D || !status))) {
        set_error("macro_update_gauss_points: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (G == 0) return RVE_OK;
    cudaStream_t s = c->stream;
    DevBuf in, outb;
    RVE_TRY(in.ensure((size_t)G * 3 * 8));
    RVE_TRY(outb.ensure((size_t)G * (36 + 9 + 9) * 8 + (size_t)G * 4));
    double* dT = in.as<double>();
    RVE_CUDA(cudaMemcpyAsync(dT, T_C, G * 8, cudaMemcpyHostToDevice, s));
    RVE_CUDA(cudaMemcpyAsync(dT + G, c_wt, G * 8, cudaMemcpyHostToDevice, s));
    RVE_CUDA(cudaMemcpyAsync(dT + 2 * G, t_h, G * 8, cudaMemcpyHostToDevice, s));
    double* dC = outb.as<double>();
    double* dK = dC + 36 * G;
    double* dD = dK + 9 * G;
    int32_t* dS = reinterpret_cast<int32_t*>(dD + 9 * G);
    int rc = macro_update_gauss_points_dev(c, meshes, n_meshes, G, dT, dT + G, dT + 2 * G, mesh_id,
                                           dC, dK, dD, dS, mode, st);
    if (rc != RVE_OK && rc != RVE_ERR_NOT_CONVERGED && rc != RVE_ERR_NUMERIC) return rc;
    RVE_CUDA(cudaMemcpyAsync(C, dC, G * 36 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(K, dK, G * 9 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(D, dD, G * 9 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(status, dS, G * 4, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int macro_update_gauss_points_w_dev(rve_ctx c, const rve_mesh* meshes, int n_meshes, int64_t G,
                                    const double* W_dev, const int32_t* mesh_id_host, double* C_dev,
                                    double* K_dev, double* D_dev, int32_t* status_dev, int mode, rve_stats* st) {
    RVE_TRY(check_ctx(c));
    if (!meshes || n_meshes <= 0 || G < 0 || (G > 0 && (!W_dev || !mesh_id_host || !C_dev || !K_dev || !D_dev ||
        !status_dev)) || mode != RVE_MODE_PCG) {
        set_error("macro_update_gauss_points_w_dev: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = c->launches;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->converged = 1;
    }
    const ProfCounters pc0 = c->prof;
    int rc = macro_update_impl(c, meshes, n_meshes, G, nullptr, nullptr, nullptr, mesh_id_host, C_dev, K_dev,
                               D_dev, status_dev, st, W_dev);
    rc = bounds_outcome(rc, c->stream);
    if (st) {
        cudaStreamSynchronize(c->stream);
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        st->kernel_launches = c->launches - l0;
        fill_profile(pc0, c->prof, st);
    }
    return rc;
}

int macro_update_gauss_points_w(rve_ctx c, const rve_mesh* meshes, int n_meshes, int64_t G, const double* W,
                                const int32_t* mesh_id, double* C, double* K, double* D, int32_t* status,
                                int mode, rve_stats* st) {
    RVE_TRY(check_ctx(c));
    if (G < 0 || (G > 0 && (!W || !mesh_id || !C || !K || !D || !status))) {
        set_error("macro_update_gauss_points_w: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (G == 0) return RVE_OK;
    cudaStream_t s = c->stream;
    DevBuf in, outb;
    RVE_TRY(in.ensure((size_t)G * 8));
    RVE_TRY(outb.ensure((size_t)G * (36 + 9 + 9) * 8 + (size_t)G * 4));
    double* dW = in.as<double>();
    RVE_CUDA(cudaMemcpyAsync(dW, W, G * 8, cudaMemcpyHostToDevice, s));
    double* dC = outb.as<double>();
    double* dK = dC + 36 * G;
    double* dD = dK + 9 * G;
    int32_t* dS = reinterpret_cast<int32_t*>(dD + 9 * G);
    int rc = macro_update_gauss_points_w_dev(c, meshes, n_meshes, G, dW, mesh_id, dC, dK, dD, dS, mode, st);
    if (rc != RVE_OK && rc != RVE_ERR_NOT_CONVERGED && rc != RVE_ERR_NUMERIC) return rc;
    RVE_CUDA(cudaMemcpyAsync(C, dC, G * 36 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(K, dK, G * 9 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(D, dD, G * 9 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(status, dS, G * 4, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int rve_autotune_batch(rve_ctx c, rve_mesh m, int64_t n, const double* T_C, const double* c_wt,
                       const double* t_h, const int32_t* candidates, int n_cand, int32_t* best,
                       double* rates) {
    RVE_TRY(check_ctx(c));
    if (!m || n <= 0 || !T_C || !c_wt || !t_h || !best || n_cand < 0 || (n_cand > 0 && !candidates)) {
        set_error("rve_autotune_batch: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (!m->have_materials) {
        set_error("rve_autotune_batch: materials not set");
        return RVE_ERR_STATE;
    }
    static const int32_t dflt[] = {8, 16, 32, 64, 128, 256};
    const int32_t* cand = n_cand > 0 ? candidates : dflt;
    const int nc = n_cand > 0 ? n_cand : 6;
    for (int k = 0; k < nc; ++k)
        if (cand[k] < 1) {
            set_error("rve_autotune_batch: candidate batch sizes must be positive");
            return RVE_ERR_INVALID_ARGUMENT;
        }
    std::vector<double> C((size_t)n * 36), K((size_t)n * 9), D((size_t)n * 9);
    std::vector<int32_t> st((size_t)n), mid((size_t)n, 0);
    const int saved = c->opt.batch;
    rve_mesh ms[1] = {m};
    auto run = [&](int B, double& secs) -> int {
        c->opt.batch = B;
        const auto t0 = std::chrono::steady_clock::now();
        int rc = macro_update_gauss_points(c, ms, 1, n, T_C, c_wt, t_h, mid.data(), C.data(), K.data(),
                                           D.data(), st.data(), RVE_MODE_PCG, nullptr);
        secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return rc;
    };
    // one untimed pass forms the per-mesh caches and the device buffers
    double secs = 0;
    int rc = run(cand[0], secs);
    double bestRate = 0;
    std::vector<double> rate_of(nc, 0.0);
    // each candidate is timed twice and its faster pass kept (a single pass of a
    // sample this size varies by several per cent)
    for (int k = 0; k < nc && (rc == RVE_OK || rc == RVE_ERR_NOT_CONVERGED); ++k) {
        double best_secs = 0;
        for (int rep = 0; rep < 2 && (rc == RVE_OK || rc == RVE_ERR_NOT_CONVERGED); ++rep) {
            rc = run(cand[k], secs);
            if (rc == RVE_OK && secs > 0 && (best_secs == 0 || secs < best_secs)) best_secs = secs;
        }
        rate_of[k] = (rc == RVE_OK && best_secs > 0) ? (double)n / best_secs : 0.0;
        if (rates) rates[k] = rate_of[k];
        bestRate = std::max(bestRate, rate_of[k]);
    }
    c->opt.batch = saved;
    if (rc != RVE_OK && rc != RVE_ERR_NOT_CONVERGED) return rc;
    // The mesh is timed alone, but a batched call runs several meshes at once,
    // which fill the GPU between them, so a larger batch gains less there than
    // alone: of the candidates within 6 % of the best rate the smallest batch is
    // taken.
    int bestB = 0;
    for (int k = 0; k < nc; ++k)
        if (rate_of[k] > 0 && rate_of[k] >= 0.94 * bestRate && (bestB == 0 || cand[k] < bestB)) bestB = cand[k];
    if (bestB == 0) {
        set_error("rve_autotune_batch: no candidate converged");
        return RVE_ERR_NOT_CONVERGED;
    }
    m->tuned_batch = bestB;
    *best = bestB;
    return RVE_OK;
}

int rve_autotune_schedule(rve_ctx c, rve_mesh m, int64_t n, const double* T_C, const double* c_wt,
                          const double* t_h, const int32_t* batches, int n_batch, const int32_t* kernels,
                          int n_kernel, int32_t* best_batch, int32_t* best_kernel, double* rates) {
    RVE_TRY(check_ctx(c));
    if (!m || n <= 0 || !T_C || !c_wt || !t_h || !best_batch || !best_kernel || n_batch < 1 || !batches ||
        n_kernel < 1 || !kernels) {
        set_error("rve_autotune_schedule: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    for (int k = 0; k < n_kernel; ++k)
        if (kernels[k] != RVE_KERNEL_CUDA_CORE && kernels[k] != RVE_KERNEL_TENSOR) {
            set_error("rve_autotune_schedule: kernel candidates are RVE_KERNEL_CUDA_CORE or RVE_KERNEL_TENSOR");
            return RVE_ERR_INVALID_ARGUMENT;
        }
    const int saved = c->opt.operator_kernel;
    std::vector<double> r((size_t)n_batch, 0.0), all((size_t)n_batch * n_kernel, 0.0);
    int rc = RVE_OK;
    for (int k = 0; k < n_kernel; ++k) {
        c->opt.operator_kernel = kernels[k];
        int32_t b = 0;
        rc = rve_autotune_batch(c, m, n, T_C, c_wt, t_h, batches, n_batch, &b, r.data());
        if (rc != RVE_OK) break;
        for (int j = 0; j < n_batch; ++j) all[(size_t)k * n_batch + j] = r[j];
    }
    c->opt.operator_kernel = saved;
    if (rc != RVE_OK) return rc;
    if (rates) std::memcpy(rates, all.data(), all.size() * sizeof(double));
    // as the batch tuner: of the pairs within 6 % of the best rate, the smallest
    // batch, and of those the faster kernel
    double top = 0;
    for (double v : all) top = std::max(top, v);
    int bk = -1, bb = 0;
    double bv = 0;
    for (int k = 0; k < n_kernel; ++k)
        for (int j = 0; j < n_batch; ++j) {
            const double v = all[(size_t)k * n_batch + j];
            if (!(v > 0) || v < 0.94 * top) continue;
            if (bk < 0 || batches[j] < bb || (batches[j] == bb && v > bv)) {
                bk = k;
                bb = batches[j];
                bv = v;
            }
        }
    if (bk < 0) {
        set_error("rve_autotune_schedule: no candidate converged");
        return RVE_ERR_NOT_CONVERGED;
    }
    m->tuned_batch = bb;
    m->tuned_kernel = kernels[bk];
    *best_batch = bb;
    *best_kernel = kernels[bk];
    return RVE_OK;
}

int rve_degradation_factor(rve_ctx c, int64_t n, const double* T_C, const double* c_wt,
                           const double* t_h, const rve_degradation* deg, double* out) {
    RVE_TRY(check_ctx(c));
    if (n < 0 || (n > 0 && (!T_C || !c_wt || !t_h || !out))) return RVE_ERR_INVALID_ARGUMENT;
    if (n == 0) return RVE_OK;
    rve_degradation dg{-0.001682, 126.0, 1.5, 0};
    if (deg) dg = *deg;
    cudaStream_t s = c->stream;
    DevBuf b;
    RVE_TRY(b.ensure((size_t)n * 4 * 8));
    double* d = b.as<double>();
    RVE_CUDA(cudaMemcpyAsync(d, T_C, n * 8, cudaMemcpyHostToDevice, s));
    RVE_CUDA(cudaMemcpyAsync(d + n, c_wt, n * 8, cudaMemcpyHostToDevice, s));
    RVE_CUDA(cudaMemcpyAsync(d + 2 * n, t_h, n * 8, cudaMemcpyHostToDevice, s));
    launch_degradation(n, d, d + n, d + 2 * n, dg.beta, dg.Tg_C, dg.c_sat_wt, d + 3 * n, s);
    c->launches++;
    RVE_CUDA(cudaGetLastError());
    RVE_CUDA(cudaMemcpyAsync(out, d + 3 * n, n * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    return RVE_OK;
}

int rve_mesh_get_tensors(rve_ctx c, rve_mesh m, double* stiff, double* cond, double* diff) {
    RVE_TRY(check_ctx(c));
    if (!m) return RVE_ERR_INVALID_ARGUMENT;
    if (!m->have_materials) return RVE_ERR_STATE;
    cudaStream_t s = c->stream;
    const int64_t nt = m->nt;
    std::vector<double> a(nt * 21), b(nt * 12);
    RVE_CUDA(cudaMemcpyAsync(a.data(), m->d_matm64.p, a.size() * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(b.data(), m->d_mats64.p, b.size() * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    auto u6 = [](int i, int j) {
        if (i > j) std::swap(i, j);
        return i * 6 - i * (i - 1) / 2 + (j - i);
    };
    auto sym3 = [](int i, int j) { return i == j ? i : ((i + j == 1) ? 3 : ((i + j == 3) ? 4 : 5)); };
    for (int64_t e = 0; e < nt; ++e) {
        if (stiff)
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) stiff[e * 36 + i * 6 + j] = a[e * 21 + u6(i, j)] * m->mc.ref_mech;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                if (cond) cond[e * 9 + i * 3 + j] = b[e * 12 + sym3(i, j)] * m->mc.ref_k;
                if (diff) diff[e * 9 + i * 3 + j] = b[e * 12 + 6 + sym3(i, j)] * m->mc.ref_d;
            }
    }
    return RVE_OK;
}

int rve_apply_operator(rve_ctx c, rve_mesh m, int field, int ncols, const double* x, double* y) {
    RVE_TRY(check_ctx(c));
    if (!m || !x || !y || field < 0 || field > 2 || ncols <= 0) return RVE_ERR_INVALID_ARGUMENT;
    if (!m->have_materials) return RVE_ERR_STATE;
    cudaStream_t s = c->stream;
    FieldDev& f = field == 0 ? m->mech : m->scal;
    // pad columns to a multiple of 6; select the scalar field through the column index
    const int cpad = 6 * ((ncols + 5) / 6);
    const int64_t n_rows = f.n_rows;
    std::vector<double> xp((size_t)n_rows * cpad, 0.0), yp((size_t)n_rows * cpad, 0.0);
    // scalar: thermal uses columns 0..2 of each group, moisture 3..5
    std::vector<int> colmap(ncols);
    for (int j = 0; j < ncols; ++j) colmap[j] = j;
    int cpad2 = cpad;
    if (field != 0) {
        cpad2 = 6 * ncols;   // one group per column, place it at 0 (thermal) or 3 (moisture)
        xp.assign((size_t)n_rows * cpad2, 0.0);
        yp.assign((size_t)n_rows * cpad2, 0.0);
        for (int j = 0; j < ncols; ++j) colmap[j] = 6 * j + (field == 2 ? 3 : 0);
    }
    for (int64_t r = 0; r < n_rows; ++r)
        for (int j = 0; j < ncols; ++j) xp[r * cpad2 + colmap[j]] = x[r * ncols + j];
    if (xp.size() >= ((size_t)1 << 31)) {
        set_error("rve_apply_operator: more than 2^31 vector entries");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    DevBuf dx, dy, sc;
    RVE_TRY(upload(dx, xp.data(), xp.size(), s));
    RVE_TRY(dy.ensure(yp.size() * 8));
    RVE_CUDA(cudaMemsetAsync(dy.p, 0, yp.size() * 8, s));
    std::vector<double> ones((size_t)cpad2 * 2, 1.0);
    RVE_TRY(upload(sc, ones.data(), ones.size(), s));
    ElemView<double> ev;
    ev.nt = m->nt;
    ev.edofs = m->d_edofs.as<int32_t>();
    ev.geo = m->d_geo64.as<double>();
    ev.mat = (f.nc == 3 ? m->d_matm64 : m->d_mats64).as<double>();
    ev.phase = m->d_phase.as<uint8_t>();
    ev.scale = sc.as<double>();
    set_view_extras(ev, m);
    Launch L = make_launch(cpad2, m->nt, s);
    launch_operator<double>(m->p, f.nc, false, ev, dx.as<double>(), dy.as<double>(), nullptr, L);
    c->launches++;
    RVE_CUDA(cudaGetLastError());
    RVE_CUDA(cudaMemcpyAsync(yp.data(), dy.p, yp.size() * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    const double ref = field == 0 ? m->mc.ref_mech : (field == 1 ? m->mc.ref_k : m->mc.ref_d);
    for (int64_t r = 0; r < n_rows; ++r)
        for (int j = 0; j < ncols; ++j) y[r * ncols + j] = yp[r * cpad2 + colmap[j]] * ref;
    return RVE_OK;
}

int rve_apply_operator_mixed(rve_ctx c, rve_mesh m, int kernel, int ncols, const double* x, const double* scale,
                             const int32_t* active, double* y, double* energy) {
    RVE_TRY(check_ctx(c));
    if (!m || !x || !y || ncols <= 0 || ncols % 6 != 0 || (kernel != 0 && kernel != 1)) {
        set_error("rve_apply_operator_mixed: invalid argument (kernel 0 or 1, ncols a positive multiple of 6)");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (!m->have_materials) return RVE_ERR_STATE;
    if (kernel == 0 && !operator_tc_supported(m->p, 3)) {
        set_error("rve_apply_operator_mixed: the tensor-core operator needs p = 2 or 3");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = c->stream;
    FieldDev& f = m->mech;
    const int64_t n_rows = f.n_rows;
    const size_t nv = (size_t)n_rows * ncols;
    if (nv >= ((size_t)1 << 31)) {
        set_error("rve_apply_operator_mixed: more than 2^31 vector entries");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    std::vector<float> x32(nv), sc32((size_t)ncols * 2, 1.f);
    for (size_t i = 0; i < nv; ++i) x32[i] = (float)x[i];
    if (scale)
        for (int i = 0; i < 2 * ncols; ++i) sc32[i] = (float)scale[i];
    std::vector<int32_t> act(ncols, 1);
    if (active)
        for (int i = 0; i < ncols; ++i) act[i] = active[i] != 0;
    Launch L = make_launch(ncols, std::max<int64_t>(n_rows, m->nt), s);
    DevBuf dx, dy, dsc, dact, dlist, dpart, dsum, dflag;
    RVE_TRY(upload(dx, x32.data(), nv, s));
    RVE_TRY(upload(dsc, sc32.data(), sc32.size(), s));
    RVE_TRY(upload(dact, act.data(), act.size(), s));
    RVE_TRY(dy.ensure(nv * 4));
    RVE_TRY(dlist.ensure((size_t)ncols * 4 + 64));
    RVE_TRY(dpart.ensure((size_t)L.nby * ncols * 8));
    RVE_TRY(dsum.ensure((size_t)ncols * 8));
    RVE_TRY(dflag.ensure(16));
    RVE_CUDA(cudaMemsetAsync(dy.p, 0, nv * 4, s));
    RVE_CUDA(cudaMemsetAsync(dpart.p, 0, (size_t)L.nby * ncols * 8, s));
    RVE_CUDA(cudaMemsetAsync(dflag.p, 0, 16, s));
    int32_t* list = dlist.as<int32_t>();
    int32_t* n_list = list + ncols;
    launch_compact_active(dact.as<int32_t>(), ncols, list, n_list, s);
    if (kernel == 0) {
        RVE_TRY(ensure_element_matrices(m, s));
        RVE_CUDA(launch_operator_tc(m->p, m->nt, m->d_edofs.as<int32_t>(), m->d_ke32.as<float>(),
                                    m->d_kepairs.as<uint16_t>(), m->d_phase.as<uint8_t>(), dsc.as<float>(),
                                    dx.as<float>(), dy.as<float>(), dpart.as<double>(), dact.as<int32_t>(), ncols,
                                    list, n_list, L.nby, dflag.as<int32_t>(), s));
    } else {
        ElemView<float> ev;
        ev.nt = m->nt;
        ev.edofs = m->d_edofs.as<int32_t>();
        ev.geo = m->d_geo32.as<float>();
        ev.mat = m->d_matm32.as<float>();
        ev.phase = m->d_phase.as<uint8_t>();
        ev.scale = dsc.as<float>();
        ev.n_nodes = m->debug_node_bound > 0 ? m->debug_node_bound : m->map.N;   // no colours: L.nby partial rows
        launch_operator<float>(m->p, 3, false, ev, dx.as<float>(), dy.as<float>(), dpart.as<double>(), L,
                               dact.as<int32_t>(), list, n_list);
    }
    launch_reduce_partials(L.nby, ncols, dpart.as<double>(), dsum.as<double>(), s);
    c->launches += 3;
    RVE_CUDA(cudaGetLastError());
    std::vector<float> y32(nv);
    std::vector<double> es(ncols);
    int32_t flag = 0;
    RVE_CUDA(cudaMemcpyAsync(y32.data(), dy.p, nv * 4, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(es.data(), dsum.p, (size_t)ncols * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(&flag, dflag.p, 4, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    if (flag & 4) {
        set_error("a bounded wait inside the tensor-core operator gave up");
        return RVE_ERR_TIMEOUT;
    }
    const double ref = m->mc.ref_mech;
    for (size_t i = 0; i < nv; ++i) y[i] = (double)y32[i] * ref;
    if (energy)
        for (int j = 0; j < ncols; ++j) energy[j] = act[j] ? es[j] * ref : 0.0;
    return RVE_OK;
}

int rve_operator_energy_noalloc(rve_ctx c, rve_mesh m, int field, int ncols, const double* x_dev,
                                double* y_dev, double* energy_dev) {
    RVE_TRY(check_ctx(c));
    if (!m || !x_dev || !y_dev || !energy_dev || (field != 0 && field != 1) || ncols <= 0 ||
        ncols % 6 != 0) {
        set_error("rve_operator_energy_noalloc: invalid argument (field 0 or 1, ncols a positive multiple of 6)");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (ncols > noalloc_max_cols()) {
        set_error("rve_operator_energy_noalloc: ncols exceeds the static scratch limit of " +
                  std::to_string(noalloc_max_cols()) + " columns");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (!m->have_materials) {
        set_error("rve_set_materials must be called first");
        return RVE_ERR_STATE;
    }
    cudaError_t e = cudaSuccess;
    double* scratch = noalloc_scratch(c->device, &e);
    if (!scratch) {
        set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return RVE_ERR_CUDA;
    }
    cudaStream_t s = c->stream;
    FieldDev& f = field == 0 ? m->mech : m->scal;
    if ((size_t)f.n_rows * ncols >= ((size_t)1 << 31)) {
        set_error("rve_operator_energy_noalloc: more than 2^31 vector entries");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    Launch L = make_launch(ncols, std::max<int64_t>(f.n_rows, m->nt), s);
    L.nby = std::min(L.nby, noalloc_max_blocks_y());
    double* partial = scratch;                                                   // [nby][ncols]
    double* scale = scratch + (size_t)noalloc_max_blocks_y() * noalloc_max_cols(); // [ncols][2]
    launch_fill((int64_t)ncols * 2, 1.0, scale, s);   // unit scales: the materials as set
    RVE_CUDA(cudaMemsetAsync(y_dev, 0, sizeof(double) * f.n_rows * ncols, s));
    ElemView<double> ev;
    ev.nt = m->nt;
    ev.edofs = m->d_edofs.as<int32_t>();
    ev.geo = m->d_geo64.as<double>();
    ev.mat = (f.nc == 3 ? m->d_matm64 : m->d_mats64).as<double>();
    ev.phase = m->d_phase.as<uint8_t>();
    ev.scale = scale;
    ev.n_nodes = m->debug_node_bound > 0 ? m->debug_node_bound : m->map.N;   // no colours: fixed partial rows
    launch_operator<double>(m->p, f.nc, false, ev, x_dev, y_dev, partial, L);
    launch_reduce_partials(L.nby, ncols, partial, energy_dev, s);
    const double lo = field == 0 ? m->mc.ref_mech : m->mc.ref_k;
    const double hi = field == 0 ? m->mc.ref_mech : m->mc.ref_d;
    launch_scale_cols(f.n_rows, ncols, lo, hi, y_dev, s);
    launch_scale_cols(1, ncols, lo, hi, energy_dev, s);
    c->launches += 5;
    RVE_CUDA(cudaGetLastError());
    return RVE_OK;
}

int rve_mesh_get_dofmap(rve_ctx c, rve_mesh m, int32_t* edofs, int32_t* lverts) {
    RVE_TRY(check_ctx(c));
    if (!m) return RVE_ERR_INVALID_ARGUMENT;
    if (edofs) std::memcpy(edofs, m->map.edofs.data(), m->map.edofs.size() * 4);
    if (lverts) std::memcpy(lverts, m->map.lverts.data(), m->map.lverts.size() * 4);
    return RVE_OK;
}

int rve_mesh_get_colouring(rve_ctx c, rve_mesh m, int32_t* colour_of, int32_t* n_colours) {
    RVE_TRY(check_ctx(c));
    if (!m || !n_colours) return RVE_ERR_INVALID_ARGUMENT;
    *n_colours = m->ncolour;
    if (colour_of) {
        std::vector<int32_t> order(m->nt);
        if (m->nt > 0) {
            RVE_CUDA(cudaMemcpy(order.data(), m->d_colour_elems.p, order.size() * 4, cudaMemcpyDeviceToHost));
        }
        for (int k = 0; k < m->ncolour; ++k)
            for (int64_t i = m->colour_off[k]; i < m->colour_off[k + 1]; ++i) colour_of[order[i]] = k;
    }
    return RVE_OK;
}

int rve_debug_bounds(rve_ctx c, int32_t* checking_build, int64_t* violations, int64_t* first_element,
                     int32_t* first_column, int reset) {
    RVE_TRY(check_ctx(c));
    RVE_CUDA(cudaStreamSynchronize(c->stream));
    unsigned long long n = 0;
    long long fe = -1;
    int fc = -1;
    if (bounds_status(&n, &fe, &fc) != 0) {
        set_error("rve_debug_bounds: reading the device counters failed");
        return RVE_ERR_CUDA;
    }
    if (checking_build) *checking_build = bounds_check_built() ? 1 : 0;
    if (violations) *violations = (int64_t)n;
    if (first_element) *first_element = fe;
    if (first_column) *first_column = fc;
    if (reset && bounds_reset() != 0) return RVE_ERR_CUDA;
    return RVE_OK;
}

int rve_debug_set_node_bound(rve_ctx c, rve_mesh m, int64_t n_nodes) {
    RVE_TRY(check_ctx(c));
    if (!m || n_nodes < 0) return RVE_ERR_INVALID_ARGUMENT;
    m->debug_node_bound = n_nodes;
    return RVE_OK;
}

}  // extern "C"
