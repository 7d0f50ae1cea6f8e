// Coupled macro time step on the GPU (Secs. 3, 4, 5): heat and moisture
// transport on a linear-tetrahedron macro mesh with the homogenised tensors
// (Eq. Eq_field discretised as Eq. Eq_field_disc, one backward-Euler step), then
// the degradation field 1 - omega at the macro Gauss points by backward Euler of
// the rate form (Eq. Eq_Model_RateForm) and the equivalent exposure time that
// hands each Gauss point to the RVE path (macro_update_gauss_points[_dev] or the
// surrogate) as (T, c, t_eq).
//
// Both fields are solved together as two columns of one matrix-free operator:
// vectors v[node * 2 + field], field 0 temperature [C], field 1 moisture [wt%].
//
// The macro mechanical problem of the fully nested FE^2 step (Sec. 5) uses the
// same mesh: linear elasticity with the homogenised stiffness C_bar of every
// macro Gauss point, vectors u[node * 3 + component], solved by the same Jacobi
// PCG with one field and a per-DOF held mask.
// Everything here is FP64: the macro mesh is small next to the RVE batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"

struct rve_macro_s {
    rve_ctx ctx = nullptr;
    int64_t nv = 0, nt = 0;
    rve::DevBuf tets, geo, mask, hold, diag, x, b, r, z, p, q, acc, gp, W, flags;
    std::vector<double> vol_h, grad_h;    // host copies of the geometry
    std::vector<int32_t> tets_h;
    std::vector<uint8_t> mask_h;
    double KT[6] = {}, Dc[6] = {};          // symmetric (xx, yy, zz, xy, yz, zx)
    double rho_cp = 0;
    bool have_transport = false, have_face = false, have_state = false;
    double diag_dt = -1;                    // dt [s] the diagonal was formed for
    // macro mechanics: held DOFs and their values, traction load, Jacobi
    // diagonal, displacement, per-tet mean stiffness [nt][36], Gauss-point
    // stiffness staged from the host [nt*4][36] and stresses [nt*4][6]
    rve::DevBuf mfix, mval, mload, mdiag, mu, cm, cgp, msig;
    bool have_mech_bc = false, have_mech_load = false, have_mech_u = false, have_mech_sig = false;
};

namespace rve {
namespace {

constexpr double kKelvin = 273.15;

__device__ __forceinline__ double sym3(const double* k, int i, int j) {
    if (i == j) return k[i];
    const int s = i + j;   // (0,1) -> 3, (1,2) -> 4, (0,2) -> 5
    return k[s == 1 ? 3 : (s == 3 ? 4 : 5)];
}

struct MacroParams {
    double KT[6], Dc[6];
    double capT, capC;   // capacity / dt of each field (0: stiffness only)
    int stiff;           // 0: capacity part only
};

// y += (C/dt + K) x over both fields, one element per thread, FP64 atomics.
__global__ void k_macro_apply(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ geo,
                              const double* __restrict__ x, double* __restrict__ y, MacroParams prm) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        int v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = tets[e * 4 + a];
        const double vol = geo[e * 13];
        const double* g = geo + e * 13 + 1;   // grad lambda_a, [4][3]
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            double xa[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xa[a] = x[(int64_t)v[a] * 2 + f];
            const double* Kf = f == 0 ? prm.KT : prm.Dc;
            const double cap = f == 0 ? prm.capT : prm.capC;
            double gr[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) gr[i] += g[a * 3 + i] * xa[a];
            double fl[3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                fl[i] = sym3(Kf, i, 0) * gr[0] + sym3(Kf, i, 1) * gr[1] + sym3(Kf, i, 2) * gr[2];
            const double sum = xa[0] + xa[1] + xa[2] + xa[3];
            const double cm = cap * vol / 20.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                double ya = cm * (sum + xa[a]);
                if (prm.stiff) ya += vol * (g[a * 3] * fl[0] + g[a * 3 + 1] * fl[1] + g[a * 3 + 2] * fl[2]);
                atomicAdd(y + (int64_t)v[a] * 2 + f, ya);
            }
        }
    }
}

// block sum of two values per thread, added atomically to out[0..1]
__device__ __forceinline__ void block_add2(double a0, double a1, double* out) {
    __shared__ double s0[256], s1[256];
    s0[threadIdx.x] = a0;
    s1[threadIdx.x] = a1;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s0[threadIdx.x] += s0[threadIdx.x + w];
            s1[threadIdx.x] += s1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(out, s0[0]);
        atomicAdd(out + 1, s1[0]);
    }
}

// r = b - y on free rows (0 on held rows), z = r / diag, acc[0..1] += (r, z)
// and acc[14..15] += (b, M^-1 b) over the free rows (the reference norm)
// (Vector kernels: nf interleaved fields per row group, field of row i is
// i % nf; the held mask is indexed by i / mdiv: 2 for the per-node mask of the
// transport pair, 1 for the per-DOF mask of the mechanics.)
__global__ void __launch_bounds__(256) k_macro_residual(int64_t n, int nf, int mdiv, const double* __restrict__ b,
                                                        const double* __restrict__ y,
                                                        const uint8_t* __restrict__ mask,
                                                        const double* __restrict__ diag, double* __restrict__ r,
                                                        double* __restrict__ z, double* __restrict__ acc) {
    double a[2] = {0, 0}, bb[2] = {0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = nf == 2 ? (int)(i & 1) : 0;
        const bool held = mask[i / mdiv] != 0;
        const double ri = held ? 0.0 : b[i] - y[i];
        const double zi = ri / diag[i];
        r[i] = ri;
        z[i] = zi;
        a[f] += ri * zi;
        if (!held) bb[f] += b[i] * b[i] / diag[i];
    }
    block_add2(a[0], a[1], acc);
    block_add2(bb[0], bb[1], acc + 14);
}

// acc[2..3] += (p, q) per field
__global__ void __launch_bounds__(256) k_macro_dot(int64_t n, int nf, const double* __restrict__ p,
                                                   const double* __restrict__ q, double* __restrict__ acc) {
    double a[2] = {0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[nf == 2 ? (int)(i & 1) : 0] += p[i] * q[i];
    block_add2(a[0], a[1], acc + 2);
}

// Per-field scalars, one thread.  acc: [0..1] (r,z) new, [2..3] (p,q),
// [4..5] (r,z) of the previous iteration, [6..7] the reference max((b, M^-1 b), (r0, M^-1 r0)),
// [8..9] alpha, [10..11] beta, [12..13] active flags (as doubles).
__global__ void k_macro_alpha(double* acc) {
    for (int f = 0; f < 2; ++f) {
        const double pq = acc[2 + f];
        const bool ok = acc[12 + f] != 0.0 && pq > 0.0;
        acc[8 + f] = ok ? acc[4 + f] / pq : 0.0;
        acc[2 + f] = 0.0;
        acc[f] = 0.0;                       // for the (r, z) of this iteration
    }
}
__global__ void k_macro_beta(double* acc, double tol2) {
    for (int f = 0; f < 2; ++f) {
        const double rz = acc[f];
        if (acc[12 + f] != 0.0) {
            acc[10 + f] = acc[4 + f] > 0.0 ? rz / acc[4 + f] : 0.0;
            acc[4 + f] = rz;
            if (!(rz > tol2 * acc[6 + f])) acc[12 + f] = 0.0;   // converged (or not finite)
        }
    }
}

// x += alpha p, r -= alpha q (held rows stay 0), z = r / diag, acc[0..1] += (r, z)
__global__ void __launch_bounds__(256) k_macro_update(int64_t n, int nf, int mdiv, const uint8_t* __restrict__ mask,
                                                     const double* __restrict__ diag, double* __restrict__ x,
                                                     double* __restrict__ r, double* __restrict__ z,
                                                     const double* __restrict__ p, const double* __restrict__ q,
                                                     double* __restrict__ acc) {
    const double al[2] = {acc[8], acc[9]};
    double a[2] = {0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = nf == 2 ? (int)(i & 1) : 0;
        double ri = r[i];
        if (al[f] != 0.0) {
            x[i] += al[f] * p[i];
            ri = mask[i / mdiv] ? 0.0 : ri - al[f] * q[i];
            r[i] = ri;
        }
        const double zi = ri / diag[i];
        z[i] = zi;
        a[f] += ri * zi;
    }
    block_add2(a[0], a[1], acc);
}

// p = z + beta p for active fields; q = 0
__global__ void __launch_bounds__(256) k_macro_pupdate(int64_t n, int nf, const double* __restrict__ z,
                                                      double* __restrict__ p, double* __restrict__ q,
                                                      const double* __restrict__ acc, int first) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = nf == 2 ? (int)(i & 1) : 0;
        if (first)
            p[i] = z[i];
        else if (acc[12 + f] != 0.0)
            p[i] = z[i] + acc[10 + f] * p[i];
        q[i] = 0.0;
    }
}

// held rows take their prescribed values (hold[node * 2 + field])
__global__ void k_macro_hold(int64_t nv, const uint8_t* __restrict__ mask, const double* __restrict__ hold,
                             double* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i]) {
            x[i * 2] = hold[i * 2];
            x[i * 2 + 1] = hold[i * 2 + 1];
        }
}

// grad psi of one field per tetrahedron (constant on a linear element)
__global__ void k_macro_gradient(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ geo,
                                 const double* __restrict__ x, int field, double* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        const double* g = geo + e * 13 + 1;
        double gr[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double v = x[(int64_t)tets[e * 4 + a] * 2 + field];
#pragma unroll
            for (int i = 0; i < 3; ++i) gr[i] += g[a * 3 + i] * v;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) out[e * 3 + i] = gr[i];
    }
}

__global__ void k_macro_fill(int64_t nv, double T, double c, double* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        x[i * 2] = T;
        x[i * 2 + 1] = c;
    }
}

// Gauss-point states: gp[k][e*4 + g] for k = T, c, W, t_eq.  W is advanced by
// backward Euler of Eq. Eq_Model_RateForm at the new T and c; t_eq [h] solves
// the closed form for that W.  Where there is no moisture now (lambda = 0: the
// capacity-consistent transport undershoots slightly ahead of the front) t_eq = 0
// hands the point over as undegraded; such points with W < 1 are counted in
// bad[0] and the largest 1 - W among them (the hand-over error) is kept in
// errbits as the bit pattern of a non-negative double.
__global__ void k_macro_gauss(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ x,
                              double* __restrict__ Wst, double* __restrict__ gp, double dt_h, double beta,
                              double Tg_C, double c_sat, int advance, int* __restrict__ bad,
                              unsigned long long* __restrict__ errbits) {
    const double A = 0.5854101966249685, Bc = 0.1381966011250105;
    const int64_t n = nt * 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / 4;
        const int g = (int)(i % 4);
        double T = 0, c = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double N = a == g ? A : Bc;
            const int v = tets[e * 4 + a];
            T += N * x[(int64_t)v * 2];
            c += N * x[(int64_t)v * 2 + 1];
        }
        const double cn = fmin(fmax(c / c_sat, 0.0), 1.0);
        const double lam = cn * beta * log(1.0 - (T + kKelvin) / (Tg_C + kKelvin));
        double W = Wst[i];
        if (advance) {
            W = W / (1.0 + dt_h / 24.0 * lam);
            Wst[i] = W;
        }
        double teq = 0.0;
        if (lam > 0.0) {
            teq = -24.0 * log(W) / lam;
        } else if (W < 1.0) {
            atomicAdd(bad, 1);
            atomicMax(errbits, (unsigned long long)__double_as_longlong(1.0 - W));
        }
        gp[i] = T;
        gp[n + i] = c;
        gp[2 * n + i] = W;
        gp[3 * n + i] = teq;
    }
}

// ---------------------------------------------------------- macro mechanics
// Voigt order [xx, yy, zz, xy, yz, zx] with engineering shear, as C_bar of the
// RVE path.  On a linear tetrahedron the strain is constant, so the 4-point
// Gauss rule of K = sum_g |T| / 4 B^T C_g B collapses to |T| B^T (mean_g C_g) B.

// Voigt strain from the displacement gradient H_ij = du_i / dx_j
__device__ __forceinline__ void mech_strain(const double* g, const double* ua, double eps[6]) {
    double H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) H[i][j] += ua[a * 3 + i] * g[a * 3 + j];
    eps[0] = H[0][0];
    eps[1] = H[1][1];
    eps[2] = H[2][2];
    eps[3] = H[0][1] + H[1][0];
    eps[4] = H[1][2] + H[2][1];
    eps[5] = H[2][0] + H[0][2];
}

// B^T sigma for node a with gradient (gx, gy, gz)
__device__ __forceinline__ void mech_bt(double gx, double gy, double gz, const double* sg, double f[3]) {
    f[0] = gx * sg[0] + gy * sg[3] + gz * sg[5];
    f[1] = gy * sg[1] + gx * sg[3] + gz * sg[4];
    f[2] = gz * sg[2] + gy * sg[4] + gx * sg[5];
}

// Per tetrahedron: cm = mean over its Gauss points of the symmetric part of C_g,
// and the Jacobi diagonal |T| b^T cm b of each of its 12 DOFs (b the DOF's
// column of B), added atomically into diag.
__global__ void k_mech_material(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ geo,
                                const double* __restrict__ Cgp, double* __restrict__ cm,
                                double* __restrict__ diag) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        double C[36];
#pragma unroll
        for (int k = 0; k < 36; ++k) C[k] = 0.0;
        for (int q = 0; q < 4; ++q) {
            const double* Cq = Cgp + (e * 4 + q) * 36;
#pragma unroll
            for (int J = 0; J < 6; ++J)
#pragma unroll
                for (int K = 0; K < 6; ++K) C[J * 6 + K] += 0.125 * (Cq[J * 6 + K] + Cq[K * 6 + J]);
        }
#pragma unroll
        for (int k = 0; k < 36; ++k) cm[e * 36 + k] = C[k];
        const double vol = geo[e * 13];
        const double* g = geo + e * 13 + 1;
        for (int a = 0; a < 4; ++a) {
            const double gx = g[a * 3], gy = g[a * 3 + 1], gz = g[a * 3 + 2];
            const int v = tets[e * 4 + a];
            for (int i = 0; i < 3; ++i) {
                double b[6] = {0, 0, 0, 0, 0, 0};
                if (i == 0) { b[0] = gx; b[3] = gy; b[5] = gz; }
                if (i == 1) { b[1] = gy; b[3] = gx; b[4] = gz; }
                if (i == 2) { b[2] = gz; b[4] = gy; b[5] = gx; }
                double d = 0.0;
#pragma unroll
                for (int J = 0; J < 6; ++J)
#pragma unroll
                    for (int K = 0; K < 6; ++K) d += b[J] * C[J * 6 + K] * b[K];
                atomicAdd(diag + (int64_t)v * 3 + i, vol * d);
            }
        }
    }
}

// y += K x: per tetrahedron eps = B x_T, sigma = cm eps, y_a += |T| B_a^T sigma
__global__ void k_mech_apply(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ geo,
                             const double* __restrict__ cm, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        int v[4];
        double ua[12];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            v[a] = tets[e * 4 + a];
#pragma unroll
            for (int i = 0; i < 3; ++i) ua[a * 3 + i] = x[(int64_t)v[a] * 3 + i];
        }
        const double vol = geo[e * 13];
        const double* g = geo + e * 13 + 1;
        double eps[6], sg[6];
        mech_strain(g, ua, eps);
        const double* C = cm + e * 36;
#pragma unroll
        for (int J = 0; J < 6; ++J) {
            double t = 0.0;
#pragma unroll
            for (int K = 0; K < 6; ++K) t += C[J * 6 + K] * eps[K];
            sg[J] = vol * t;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            double f[3];
            mech_bt(g[a * 3], g[a * 3 + 1], g[a * 3 + 2], sg, f);
#pragma unroll
            for (int i = 0; i < 3; ++i) atomicAdd(y + (int64_t)v[a] * 3 + i, f[i]);
        }
    }
}

// Consistent nodal forces of a uniform traction t on every tetrahedron face
// whose three vertices are all marked: t |F| / 3 on each, with the face area
// |F_a| = 3 |T| |grad lambda_a| of the face opposite vertex a.
__global__ void k_mech_traction(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ geo,
                                const uint8_t* __restrict__ face, double tx, double ty, double tz,
                                double* __restrict__ f) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        int v[4];
        bool on[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            v[a] = tets[e * 4 + a];
            on[a] = face[v[a]] != 0;
        }
        const double vol = geo[e * 13];
        const double* g = geo + e * 13 + 1;
        for (int a = 0; a < 4; ++a) {
            bool all = true;
            for (int k = 0; k < 4; ++k)
                if (k != a) all = all && on[k];
            if (!all) continue;
            const double gx = g[a * 3], gy = g[a * 3 + 1], gz = g[a * 3 + 2];
            const double third = vol * sqrt(gx * gx + gy * gy + gz * gz);   // |F_a| / 3
            for (int k = 0; k < 4; ++k)
                if (k != a) {
                    atomicAdd(f + (int64_t)v[k] * 3, tx * third);
                    atomicAdd(f + (int64_t)v[k] * 3 + 1, ty * third);
                    atomicAdd(f + (int64_t)v[k] * 3 + 2, tz * third);
                }
        }
    }
}

// held DOFs take their prescribed values
__global__ void k_mech_hold(int64_t n, const uint8_t* __restrict__ fix, const double* __restrict__ val,
                            double* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (fix[i]) x[i] = val[i];
}

// sigma_g = sym(C_g) B u_T at every Gauss point [nt*4][6]
__global__ void k_mech_stress(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ geo,
                              const double* __restrict__ Cgp, const double* __restrict__ u,
                              double* __restrict__ sig) {
    const int64_t n = nt * 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / 4;
        double ua[12];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) ua[a * 3 + k] = u[(int64_t)tets[e * 4 + a] * 3 + k];
        double eps[6];
        mech_strain(geo + e * 13 + 1, ua, eps);
        const double* C = Cgp + i * 36;
#pragma unroll
        for (int J = 0; J < 6; ++J) {
            double t = 0.0;
#pragma unroll
            for (int K = 0; K < 6; ++K) t += 0.5 * (C[J * 6 + K] + C[K * 6 + J]) * eps[K];
            sig[i * 6 + J] = t;
        }
    }
}

unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 4));
}

bool sym_pos_def(const double k[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (std::fabs(k[i * 3 + j] - k[j * 3 + i]) > 1e-12 * (std::fabs(k[i * 3 + j]) + std::fabs(k[j * 3 + i])))
                return false;
    const double d1 = k[0];
    const double d2 = k[0] * k[4] - k[1] * k[3];
    const double d3 = k[0] * (k[4] * k[8] - k[5] * k[7]) - k[1] * (k[3] * k[8] - k[5] * k[6]) +
                      k[2] * (k[3] * k[7] - k[4] * k[6]);
    return d1 > 0 && d2 > 0 && d3 > 0;
}

void to_sym6(const double k[9], double out[6]) {
    out[0] = k[0];
    out[1] = k[4];
    out[2] = k[8];
    out[3] = k[1];
    out[4] = k[5];
    out[5] = k[2];
}

// Jacobi diagonal of C/dt + K per node and field (host, FP64).
int build_diag(rve_macro m, double dt_s) {
    std::vector<double> d((size_t)m->nv * 2, 0.0);
    double K6[2][6];
    std::memcpy(K6[0], m->KT, sizeof(K6[0]));
    std::memcpy(K6[1], m->Dc, sizeof(K6[1]));
    const double cap[2] = {m->rho_cp / dt_s, 1.0 / dt_s};
    for (int64_t e = 0; e < m->nt; ++e) {
        const double vol = m->vol_h[e];
        const double* g = &m->grad_h[(size_t)e * 12];
        for (int a = 0; a < 4; ++a) {
            const int v = m->tets_h[e * 4 + a];
            for (int f = 0; f < 2; ++f) {
                const double* k = K6[f];
                const double gx = g[a * 3], gy = g[a * 3 + 1], gz = g[a * 3 + 2];
                const double kgg = gx * (k[0] * gx + k[3] * gy + k[5] * gz) + gy * (k[3] * gx + k[1] * gy + k[4] * gz) +
                                   gz * (k[5] * gx + k[4] * gy + k[2] * gz);
                d[(size_t)v * 2 + f] += vol * kgg + cap[f] * vol / 10.0;
            }
        }
    }
    RVE_TRY(upload(m->diag, d.data(), d.size(), m->ctx->stream));
    m->diag_dt = dt_s;
    return RVE_OK;
}

// Jacobi PCG on the macro mesh over nf (1 or 2) interleaved fields of n rows in
// all.  On entry x holds the start (held rows at their values) and b the
// right-hand side; apply(in, out) adds the operator times in to out.  A field
// has converged when (r, M^-1 r) <= rtol^2 max((b, M^-1 b), (r0, M^-1 r0)) over
// the free rows.  Returns the iterations and final relative residuals per field.
template <class Apply>
int macro_pcg(rve_macro mm, int64_t n, int nf, int mdiv, const uint8_t* mask, const double* diag, double* x,
              const double* b, Apply apply, double rtol, int max_iter, int its[2], double rel[2], bool& conv) {
    cudaStream_t s = mm->ctx->stream;
    double* r = mm->r.as<double>();
    double* z = mm->z.as<double>();
    double* p = mm->p.as<double>();
    double* q = mm->q.as<double>();
    double* acc = mm->acc.as<double>();
    const unsigned gv = grid_for(n);
    // r = b - A x, z = M^-1 r, (r, z)
    RVE_CUDA(cudaMemsetAsync(q, 0, n * 8, s));
    RVE_CUDA(cudaMemsetAsync(acc, 0, 16 * 8, s));
    apply(x, q);
    k_macro_residual<<<gv, 256, 0, s>>>(n, nf, mdiv, b, q, mask, diag, r, z, acc);
    const double tol2 = rtol * rtol;
    double h[16];
    RVE_CUDA(cudaMemcpyAsync(h, acc, 16 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    // convergence is relative to the larger of the right-hand side and the
    // initial residual (which carries the held values): a field already at
    // rest (rounding-level residual) needs no iteration
    for (int f = 0; f < 2; ++f) {
        h[4 + f] = h[f];                                  // current (r, z)
        h[6 + f] = std::max(h[14 + f], h[f]);             // reference
        h[12 + f] = h[f] > tol2 * h[6 + f] ? 1.0 : 0.0;   // active
    }
    h[0] = h[1] = h[2] = h[3] = 0.0;
    RVE_CUDA(cudaMemcpyAsync(acc, h, 16 * 8, cudaMemcpyHostToDevice, s));
    k_macro_pupdate<<<gv, 256, 0, s>>>(n, nf, z, p, q, acc, 1);
    int it = 0;
    its[0] = its[1] = 0;
    bool active[2] = {h[12] != 0.0, h[13] != 0.0};
    while ((active[0] || active[1]) && it < max_iter) {
        const int chunk = std::min(8, max_iter - it);
        for (int k = 0; k < chunk; ++k) {
            apply(p, q);
            k_macro_dot<<<gv, 256, 0, s>>>(n, nf, p, q, acc);
            k_macro_alpha<<<1, 1, 0, s>>>(acc);
            k_macro_update<<<gv, 256, 0, s>>>(n, nf, mdiv, mask, diag, x, r, z, p, q, acc);
            k_macro_beta<<<1, 1, 0, s>>>(acc, tol2);
            k_macro_pupdate<<<gv, 256, 0, s>>>(n, nf, z, p, q, acc, 0);
        }
        RVE_CUDA(cudaGetLastError());
        it += chunk;
        RVE_CUDA(cudaMemcpyAsync(h, acc, 16 * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
        for (int f = 0; f < 2; ++f) {
            if (active[f]) its[f] = it;
            active[f] = h[12 + f] != 0.0;
        }
    }
    conv = !(active[0] || active[1]);
    rel[0] = h[6] > 0 ? std::sqrt(std::max(h[4], 0.0) / h[6]) : 0.0;
    rel[1] = h[7] > 0 ? std::sqrt(std::max(h[5], 0.0) / h[7]) : 0.0;
    return RVE_OK;
}

}  // namespace
}  // namespace rve

using namespace rve;

extern "C" {

int rve_macro_create(rve_ctx c, const double* xyz, int64_t nv, const int32_t* tets, int64_t nt, rve_macro* out) {
    RVE_TRY(check_ctx(c));
    if (!xyz || !tets || !out || nv < 4 || nt < 1) {
        set_error("rve_macro_create: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    rve_macro m = new rve_macro_s();
    m->ctx = c;
    m->nv = nv;
    m->nt = nt;
    m->tets_h.assign(tets, tets + nt * 4);
    m->vol_h.resize(nt);
    m->grad_h.resize((size_t)nt * 12);
    std::vector<double> geo((size_t)nt * 13);
    for (int64_t e = 0; e < nt; ++e) {
        const double* X[4];
        for (int a = 0; a < 4; ++a) {
            const int32_t v = tets[e * 4 + a];
            if (v < 0 || v >= nv) {
                delete m;
                set_error("rve_macro_create: vertex index out of range");
                return RVE_ERR_BAD_MESH;
            }
            X[a] = xyz + (int64_t)v * 3;
        }
        double J[3][3];   // rows: edges from vertex 0
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) J[r][k] = X[r + 1][k] - X[0][k];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(det > 0)) {
            delete m;
            set_error("rve_macro_create: non-positive tetrahedron volume");
            return RVE_ERR_BAD_MESH;
        }
        // inverse of J: grad lambda_{r+1} is row r of inv(J)^T, i.e. column r of inv(J)
        double inv[3][3];
        inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        double g[4][3];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) g[r + 1][k] = inv[k][r];
        for (int k = 0; k < 3; ++k) g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
        m->vol_h[e] = det / 6.0;
        geo[(size_t)e * 13] = det / 6.0;
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < 3; ++k) {
                geo[(size_t)e * 13 + 1 + a * 3 + k] = g[a][k];
                m->grad_h[(size_t)e * 12 + a * 3 + k] = g[a][k];
            }
    }
    cudaStream_t s = c->stream;
    int rc = upload(m->tets, tets, (size_t)nt * 4, s);
    if (rc == RVE_OK) rc = upload(m->geo, geo.data(), geo.size(), s);
    const size_t n2 = (size_t)nv * 2;
    for (DevBuf* bfr : {&m->x, &m->b, &m->r, &m->z, &m->p, &m->q})
        if (rc == RVE_OK) rc = bfr->ensure(n2 * 8);
    if (rc == RVE_OK) rc = m->acc.ensure(16 * 8);
    if (rc == RVE_OK) rc = m->gp.ensure((size_t)nt * 4 * 4 * 8);
    if (rc == RVE_OK) rc = m->W.ensure((size_t)nt * 4 * 8);
    if (rc == RVE_OK) rc = m->flags.ensure(16);
    if (rc == RVE_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("rve_macro_create: upload failed");
        rc = RVE_ERR_CUDA;
    }
    if (rc != RVE_OK) {
        delete m;
        return rc;
    }
    *out = m;
    return RVE_OK;
}

int rve_macro_free(rve_ctx c, rve_macro m) {
    RVE_TRY(check_ctx(c));
    if (m) cudaStreamSynchronize(c->stream);
    delete m;
    return RVE_OK;
}

int rve_macro_set_transport(rve_ctx c, rve_macro m, const double K_T[9], double rho_cp, const double D_c[9]) {
    RVE_TRY(check_ctx(c));
    if (!m || !K_T || !D_c || !(rho_cp > 0)) {
        set_error("rve_macro_set_transport: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (!sym_pos_def(K_T) || !sym_pos_def(D_c)) {
        set_error("rve_macro_set_transport: conductivity or diffusivity not symmetric positive definite");
        return RVE_ERR_NOT_SPD;
    }
    to_sym6(K_T, m->KT);
    to_sym6(D_c, m->Dc);
    m->rho_cp = rho_cp;
    m->have_transport = true;
    m->diag_dt = -1;
    return RVE_OK;
}

int rve_macro_set_face(rve_ctx c, rve_macro m, const uint8_t* node_mask, double T_C, double c_wt) {
    RVE_TRY(check_ctx(c));
    if (!m || !node_mask) {
        set_error("rve_macro_set_face: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    std::vector<double> hold((size_t)m->nv * 2);
    for (int64_t i = 0; i < m->nv; ++i) {
        hold[(size_t)i * 2] = T_C;
        hold[(size_t)i * 2 + 1] = c_wt;
    }
    return rve_macro_set_held(c, m, node_mask, hold.data());
}

int rve_macro_set_held(rve_ctx c, rve_macro m, const uint8_t* node_mask, const double* values) {
    RVE_TRY(check_ctx(c));
    if (!m || !node_mask || !values) {
        set_error("rve_macro_set_held: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    m->mask_h.assign(node_mask, node_mask + m->nv);
    for (auto& v : m->mask_h) v = v ? 1 : 0;
    RVE_TRY(upload(m->mask, m->mask_h.data(), m->mask_h.size(), c->stream));
    RVE_TRY(upload(m->hold, values, (size_t)m->nv * 2, c->stream));
    RVE_CUDA(cudaStreamSynchronize(c->stream));
    m->have_face = true;
    return RVE_OK;
}

int rve_macro_reset(rve_ctx c, rve_macro m, double T0_C, double c0_wt) {
    RVE_TRY(check_ctx(c));
    if (!m) {
        set_error("rve_macro_reset: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = c->stream;
    k_macro_fill<<<grid_for(m->nv), 256, 0, s>>>(m->nv, T0_C, c0_wt, m->x.as<double>());
    std::vector<double> ones((size_t)m->nt * 4, 1.0);
    RVE_TRY(upload(m->W, ones.data(), ones.size(), s));
    RVE_CUDA(cudaGetLastError());
    RVE_CUDA(cudaStreamSynchronize(s));
    m->have_state = true;
    return RVE_OK;
}

// One implicit transport solve over both fields: (C/dt + K) x' = C/dt x with the
// held rows at their values; dt_s = infinity gives the steady problem K x = 0.
// Returns the iterations and final relative residuals per field.
static int transport_solve(rve_macro mm, double dt_s, double rtol, int max_iter, int its[2], double rel[2],
                           bool& conv) {
    cudaStream_t s = mm->ctx->stream;
    if (mm->diag_dt != dt_s) RVE_TRY(build_diag(mm, dt_s));
    const int64_t n = mm->nv * 2;
    double* x = mm->x.as<double>();
    double* b = mm->b.as<double>();
    const uint8_t* mask = mm->mask.as<uint8_t>();
    const unsigned ge = grid_for(mm->nt);
    MacroParams prm;
    std::memcpy(prm.KT, mm->KT, sizeof(prm.KT));
    std::memcpy(prm.Dc, mm->Dc, sizeof(prm.Dc));
    prm.capT = mm->rho_cp / dt_s;
    prm.capC = 1.0 / dt_s;
    // b = C/dt x^n; start from x^n with the held values in place
    MacroParams mass = prm;
    mass.stiff = 0;
    prm.stiff = 1;
    RVE_CUDA(cudaMemsetAsync(b, 0, n * 8, s));
    k_macro_apply<<<ge, 256, 0, s>>>(mm->nt, mm->tets.as<int32_t>(), mm->geo.as<double>(), x, b, mass);
    k_macro_hold<<<grid_for(mm->nv), 256, 0, s>>>(mm->nv, mask, mm->hold.as<double>(), x);
    auto apply = [&](const double* in, double* out) {
        k_macro_apply<<<ge, 256, 0, s>>>(mm->nt, mm->tets.as<int32_t>(), mm->geo.as<double>(), in, out, prm);
    };
    return macro_pcg(mm, n, 2, 2, mask, mm->diag.as<double>(), x, b, apply, rtol, max_iter, its, rel, conv);
}

int rve_macro_step(rve_ctx c, rve_macro m, double dt_h, const rve_degradation* deg, double rtol, int max_iter,
                   rve_macro_stats* st) {
    NvtxRange nvtx_("macro transport and degradation step");
    RVE_TRY(check_ctx(c));
    if (!m || !(dt_h > 0) || !(rtol > 0) || max_iter < 1) {
        set_error("rve_macro_step: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (!m->have_transport || !m->have_face || !m->have_state) {
        set_error("rve_macro_step: set transport, face and initial state first");
        return RVE_ERR_STATE;
    }
    const auto t0 = std::chrono::steady_clock::now();
    rve_degradation dg{-0.001682, 126.0, 1.5, 0};
    if (deg) dg = *deg;
    const double dt_s = dt_h * 3600.0;
    int its[2] = {0, 0};
    double rel[2] = {0, 0};
    bool conv = false;
    RVE_TRY(transport_solve(m, dt_s, rtol, max_iter, its, rel, conv));
    cudaStream_t s = c->stream;
    double* x = m->x.as<double>();
    // Gauss-point states and the degradation update
    RVE_CUDA(cudaMemsetAsync(m->flags.p, 0, 16, s));
    k_macro_gauss<<<grid_for(m->nt * 4), 256, 0, s>>>(m->nt, m->tets.as<int32_t>(), x, m->W.as<double>(),
                                                      m->gp.as<double>(), dt_h, dg.beta, dg.Tg_C, dg.c_sat_wt, 1,
                                                      m->flags.as<int>(),
                                                      reinterpret_cast<unsigned long long*>(m->flags.as<char>() + 8));
    int bad = 0;
    double herr = 0.0;
    RVE_CUDA(cudaMemcpyAsync(&bad, m->flags.p, 4, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaMemcpyAsync(&herr, m->flags.as<char>() + 8, 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    RVE_CUDA(cudaGetLastError());
    if (st) {
        st->iterations_T = its[0];
        st->iterations_c = its[1];
        st->rel_residual_T = rel[0];
        st->rel_residual_c = rel[1];
        st->converged = conv ? 1 : 0;
        st->gauss_points_unencodable = bad;
        st->handover_max_err = herr;
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!conv) {
        set_error("rve_macro_step: PCG did not reach rtol within max_iter");
        return RVE_ERR_NOT_CONVERGED;
    }
    return RVE_OK;
}

int rve_macro_set_state(rve_ctx c, rve_macro m, const double* T_nodal, const double* c_nodal, const double* W_gp,
                        const rve_degradation* deg) {
    RVE_TRY(check_ctx(c));
    if (!m || !T_nodal || !c_nodal || !W_gp) {
        set_error("rve_macro_set_state: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    const int64_t n = m->nt * 4;
    for (int64_t i = 0; i < n; ++i)
        if (!(W_gp[i] > 0.0 && W_gp[i] <= 1.0)) {
            set_error("rve_macro_set_state: 1 - omega outside (0, 1]");
            return RVE_ERR_INVALID_ARGUMENT;
        }
    std::vector<double> x((size_t)m->nv * 2);
    for (int64_t i = 0; i < m->nv; ++i) {
        if (!std::isfinite(T_nodal[i]) || !std::isfinite(c_nodal[i])) {
            set_error("rve_macro_set_state: non-finite nodal value");
            return RVE_ERR_INVALID_ARGUMENT;
        }
        x[(size_t)i * 2] = T_nodal[i];
        x[(size_t)i * 2 + 1] = c_nodal[i];
    }
    rve_degradation dg{-0.001682, 126.0, 1.5, 0};
    if (deg) dg = *deg;
    cudaStream_t s = c->stream;
    RVE_TRY(upload(m->x, x.data(), x.size(), s));
    RVE_TRY(upload(m->W, W_gp, (size_t)n, s));
    // the Gauss-point T, c and t_eq of the restored state; 1 - omega is not advanced
    RVE_CUDA(cudaMemsetAsync(m->flags.p, 0, 16, s));
    k_macro_gauss<<<grid_for(n), 256, 0, s>>>(m->nt, m->tets.as<int32_t>(), m->x.as<double>(), m->W.as<double>(),
                                              m->gp.as<double>(), 0.0, dg.beta, dg.Tg_C, dg.c_sat_wt, 0,
                                              m->flags.as<int>(),
                                              reinterpret_cast<unsigned long long*>(m->flags.as<char>() + 8));
    RVE_CUDA(cudaGetLastError());
    RVE_CUDA(cudaStreamSynchronize(s));
    m->have_state = true;
    return RVE_OK;
}

int rve_macro_gauss_dev(rve_ctx c, rve_macro m, const double** T_gp, const double** c_gp, const double** W_gp,
                        const double** t_eq_gp) {
    RVE_TRY(check_ctx(c));
    if (!m) {
        set_error("rve_macro_gauss_dev: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    const double* g = m->gp.as<double>();
    const int64_t n = m->nt * 4;
    if (T_gp) *T_gp = g;
    if (c_gp) *c_gp = g + n;
    if (W_gp) *W_gp = g + 2 * n;
    if (t_eq_gp) *t_eq_gp = g + 3 * n;
    return RVE_OK;
}

int rve_macro_solve_steady(rve_ctx c, rve_macro m, double rtol, int max_iter, rve_macro_stats* st) {
    NvtxRange nvtx_("macro steady transport solve");
    RVE_TRY(check_ctx(c));
    if (!m || !(rtol > 0) || max_iter < 1) {
        set_error("rve_macro_solve_steady: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (!m->have_transport || !m->have_face || !m->have_state) {
        set_error("rve_macro_solve_steady: set transport, held values and initial state first");
        return RVE_ERR_STATE;
    }
    const auto t0 = std::chrono::steady_clock::now();
    int its[2] = {0, 0};
    double rel[2] = {0, 0};
    bool conv = false;
    RVE_TRY(transport_solve(m, HUGE_VAL, rtol, max_iter, its, rel, conv));
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->iterations_T = its[0];
        st->iterations_c = its[1];
        st->rel_residual_T = rel[0];
        st->rel_residual_c = rel[1];
        st->converged = conv ? 1 : 0;
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!conv) {
        set_error("rve_macro_solve_steady: PCG did not reach rtol within max_iter");
        return RVE_ERR_NOT_CONVERGED;
    }
    return RVE_OK;
}

int rve_macro_gradients(rve_ctx c, rve_macro m, int field, double* grad) {
    RVE_TRY(check_ctx(c));
    if (!m || !grad || (field != 0 && field != 1)) {
        set_error("rve_macro_gradients: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = c->stream;
    DevBuf g;
    RVE_TRY(g.ensure((size_t)m->nt * 3 * 8));
    k_macro_gradient<<<grid_for(m->nt), 256, 0, s>>>(m->nt, m->tets.as<int32_t>(), m->geo.as<double>(),
                                                     m->x.as<double>(), field, g.as<double>());
    RVE_CUDA(cudaGetLastError());
    RVE_CUDA(cudaMemcpyAsync(grad, g.p, (size_t)m->nt * 3 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    return RVE_OK;
}

int rve_fibre_directions(rve_ctx c, const double* xyz, int64_t nv, const int32_t* tets, int64_t nt,
                         const int32_t* yarn_of_tet, int n_yarn, const int32_t* yarn_axis, double rtol,
                         double* dir) {
    NvtxRange nvtx_("yarn directions (potential flow)");
    RVE_TRY(check_ctx(c));
    if (!xyz || !tets || !yarn_of_tet || !yarn_axis || !dir || nv < 4 || nt < 1 || n_yarn < 0 || !(rtol > 0)) {
        set_error("rve_fibre_directions: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    for (int y = 0; y < n_yarn; ++y)
        if (yarn_axis[y] < 0 || yarn_axis[y] > 2) {
            set_error("rve_fibre_directions: yarn axis must be 0, 1 or 2");
            return RVE_ERR_INVALID_ARGUMENT;
        }
    for (int y = 0; y < n_yarn; ++y) {
        // the yarn's own tetrahedra, nodes renumbered
        std::vector<int64_t> sel;
        for (int64_t e = 0; e < nt; ++e)
            if (yarn_of_tet[e] == y) sel.push_back(e);
        if (sel.empty()) continue;
        std::vector<int32_t> local(nv, -1), sub_tets(sel.size() * 4);
        std::vector<double> sub_xyz;
        int32_t nn = 0;
        for (size_t i = 0; i < sel.size(); ++i)
            for (int a = 0; a < 4; ++a) {
                const int32_t v = tets[sel[i] * 4 + a];
                if (v < 0 || v >= nv) {
                    set_error("rve_fibre_directions: vertex index out of range");
                    return RVE_ERR_BAD_MESH;
                }
                if (local[v] < 0) {
                    local[v] = nn++;
                    sub_xyz.insert(sub_xyz.end(), xyz + (int64_t)v * 3, xyz + (int64_t)v * 3 + 3);
                }
                sub_tets[i * 4 + a] = local[v];
            }
        // inlet (phi = 0) and outlet (phi = 1): the yarn's ends along its axis
        const int ax = yarn_axis[y];
        double lo = HUGE_VAL, hi = -HUGE_VAL;
        for (int32_t k = 0; k < nn; ++k) {
            lo = std::min(lo, sub_xyz[(size_t)k * 3 + ax]);
            hi = std::max(hi, sub_xyz[(size_t)k * 3 + ax]);
        }
        const double tol = 1e-9 * std::max(1.0, hi - lo);
        std::vector<uint8_t> held(nn, 0);
        std::vector<double> vals((size_t)nn * 2, 0.0);
        for (int32_t k = 0; k < nn; ++k) {
            const double sk = sub_xyz[(size_t)k * 3 + ax];
            if (sk <= lo + tol || sk >= hi - tol) {
                held[k] = 1;
                vals[(size_t)k * 2] = sk >= hi - tol ? 1.0 : 0.0;
            }
        }
        rve_macro m = nullptr;
        RVE_TRY(rve_macro_create(c, sub_xyz.data(), nn, sub_tets.data(), (int64_t)sel.size(), &m));
        static const double eye[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        int rc = rve_macro_set_transport(c, m, eye, 1.0, eye);
        if (rc == RVE_OK) rc = rve_macro_set_held(c, m, held.data(), vals.data());
        if (rc == RVE_OK) rc = rve_macro_reset(c, m, 0.0, 0.0);
        if (rc == RVE_OK) rc = rve_macro_solve_steady(c, m, rtol, 20000, nullptr);
        std::vector<double> g(sel.size() * 3);
        if (rc == RVE_OK) rc = rve_macro_gradients(c, m, 0, g.data());
        rve_macro_free(c, m);
        if (rc != RVE_OK) return rc;
        for (size_t i = 0; i < sel.size(); ++i) {
            const double* gi = &g[i * 3];
            const double nrm = std::sqrt(gi[0] * gi[0] + gi[1] * gi[1] + gi[2] * gi[2]);
            if (nrm > 0)
                for (int k = 0; k < 3; ++k) dir[sel[i] * 3 + k] = gi[k] / nrm;
        }
    }
    return RVE_OK;
}

int rve_macro_get(rve_ctx c, rve_macro m, double* T_nodal, double* c_nodal, double* T_gp, double* c_gp, double* W_gp,
                  double* t_eq_gp) {
    RVE_TRY(check_ctx(c));
    if (!m) {
        set_error("rve_macro_get: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = c->stream;
    if (T_nodal || c_nodal) {
        std::vector<double> x((size_t)m->nv * 2);
        RVE_CUDA(cudaMemcpyAsync(x.data(), m->x.p, x.size() * 8, cudaMemcpyDeviceToHost, s));
        RVE_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < m->nv; ++i) {
            if (T_nodal) T_nodal[i] = x[(size_t)i * 2];
            if (c_nodal) c_nodal[i] = x[(size_t)i * 2 + 1];
        }
    }
    const int64_t n = m->nt * 4;
    double* outs[4] = {T_gp, c_gp, W_gp, t_eq_gp};
    for (int k = 0; k < 4; ++k)
        if (outs[k]) RVE_CUDA(cudaMemcpyAsync(outs[k], m->gp.as<double>() + k * n, n * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    return RVE_OK;
}

// ---------------------------------------------------------- macro mechanics

int rve_macro_mech_set_bc(rve_ctx c, rve_macro m, const uint8_t* fixed, const double* values) {
    RVE_TRY(check_ctx(c));
    if (!m || !fixed) {
        set_error("rve_macro_mech_set_bc: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    const size_t n = (size_t)m->nv * 3;
    std::vector<uint8_t> f(n);
    std::vector<double> v(n, 0.0);
    for (size_t i = 0; i < n; ++i) {
        f[i] = fixed[i] ? 1 : 0;
        if (f[i] && values) {
            if (!std::isfinite(values[i])) {
                set_error("rve_macro_mech_set_bc: non-finite prescribed value");
                return RVE_ERR_INVALID_ARGUMENT;
            }
            v[i] = values[i];
        }
    }
    cudaStream_t s = c->stream;
    RVE_TRY(upload(m->mfix, f.data(), n, s));
    RVE_TRY(upload(m->mval, v.data(), n, s));
    if (!m->have_mech_u) {
        RVE_TRY(m->mu.ensure(n * 8));
        RVE_CUDA(cudaMemsetAsync(m->mu.p, 0, n * 8, s));
    }
    RVE_CUDA(cudaStreamSynchronize(s));
    m->have_mech_u = true;
    m->have_mech_bc = true;
    return RVE_OK;
}

int rve_macro_mech_set_u(rve_ctx c, rve_macro m, const double* u) {
    RVE_TRY(check_ctx(c));
    if (!m) {
        set_error("rve_macro_mech_set_u: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    const size_t n = (size_t)m->nv * 3;
    cudaStream_t s = c->stream;
    if (u) {
        RVE_TRY(upload(m->mu, u, n, s));
    } else {
        RVE_TRY(m->mu.ensure(n * 8));
        RVE_CUDA(cudaMemsetAsync(m->mu.p, 0, n * 8, s));
    }
    RVE_CUDA(cudaStreamSynchronize(s));
    m->have_mech_u = true;
    return RVE_OK;
}

int rve_macro_mech_set_traction(rve_ctx c, rve_macro m, const uint8_t* face_nodes, const double t[3], int add) {
    RVE_TRY(check_ctx(c));
    if (!m || !face_nodes || !t || !std::isfinite(t[0]) || !std::isfinite(t[1]) || !std::isfinite(t[2])) {
        set_error("rve_macro_mech_set_traction: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    const size_t n = (size_t)m->nv * 3;
    std::vector<uint8_t> mk(face_nodes, face_nodes + m->nv);
    for (auto& x : mk) x = x ? 1 : 0;
    cudaStream_t s = c->stream;
    DevBuf fm;
    RVE_TRY(upload(fm, mk.data(), mk.size(), s));
    if (!add || !m->have_mech_load) {
        RVE_TRY(m->mload.ensure(n * 8));
        RVE_CUDA(cudaMemsetAsync(m->mload.p, 0, n * 8, s));
    }
    k_mech_traction<<<grid_for(m->nt), 256, 0, s>>>(m->nt, m->tets.as<int32_t>(), m->geo.as<double>(),
                                                    fm.as<uint8_t>(), t[0], t[1], t[2], m->mload.as<double>());
    RVE_CUDA(cudaGetLastError());
    RVE_CUDA(cudaStreamSynchronize(s));
    m->have_mech_load = true;
    return RVE_OK;
}

int rve_macro_mech_solve(rve_ctx c, rve_macro m, const double* C_gp, int C_on_device, double rtol, int max_iter,
                         rve_macro_mech_stats* st) {
    NvtxRange nvtx_("macro elastic solve");
    RVE_TRY(check_ctx(c));
    if (!m || !C_gp || !(rtol > 0) || max_iter < 1) {
        set_error("rve_macro_mech_solve: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if (!m->have_mech_bc || !m->have_mech_load) {
        set_error("rve_macro_mech_solve: set the held DOFs and the traction first");
        return RVE_ERR_STATE;
    }
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = c->stream;
    const int64_t n = m->nv * 3;
    const double* Cg = C_gp;
    if (!C_on_device) {
        RVE_TRY(upload(m->cgp, C_gp, (size_t)m->nt * 4 * 36, s));
        Cg = m->cgp.as<double>();
    }
    for (DevBuf* bfr : {&m->b, &m->r, &m->z, &m->p, &m->q, &m->mdiag}) RVE_TRY(bfr->ensure((size_t)n * 8));
    RVE_TRY(m->cm.ensure((size_t)m->nt * 36 * 8));
    RVE_TRY(m->msig.ensure((size_t)m->nt * 4 * 6 * 8));
    RVE_CUDA(cudaMemsetAsync(m->mdiag.p, 0, n * 8, s));
    const unsigned ge = grid_for(m->nt);
    const int32_t* tets = m->tets.as<int32_t>();
    const double* geo = m->geo.as<double>();
    k_mech_material<<<ge, 256, 0, s>>>(m->nt, tets, geo, Cg, m->cm.as<double>(), m->mdiag.as<double>());
    double* b = m->b.as<double>();
    double* u = m->mu.as<double>();
    RVE_CUDA(cudaMemcpyAsync(b, m->mload.p, n * 8, cudaMemcpyDeviceToDevice, s));
    k_mech_hold<<<grid_for(n), 256, 0, s>>>(n, m->mfix.as<uint8_t>(), m->mval.as<double>(), u);
    const double* cm = m->cm.as<double>();
    auto apply = [&](const double* in, double* out) {
        k_mech_apply<<<ge, 256, 0, s>>>(m->nt, tets, geo, cm, in, out);
    };
    int its[2] = {0, 0};
    double rel[2] = {0, 0};
    bool conv = false;
    RVE_TRY(macro_pcg(m, n, 1, 1, m->mfix.as<uint8_t>(), m->mdiag.as<double>(), u, b, apply, rtol, max_iter, its,
                      rel, conv));
    k_mech_stress<<<grid_for(m->nt * 4), 256, 0, s>>>(m->nt, tets, geo, Cg, u, m->msig.as<double>());
    RVE_CUDA(cudaGetLastError());
    RVE_CUDA(cudaStreamSynchronize(s));
    m->have_mech_sig = true;
    if (st) {
        st->iterations = its[0];
        st->converged = conv ? 1 : 0;
        st->rel_residual = rel[0];
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!conv) {
        set_error("rve_macro_mech_solve: PCG did not reach rtol within max_iter");
        return RVE_ERR_NOT_CONVERGED;
    }
    return RVE_OK;
}

int rve_macro_mech_get(rve_ctx c, rve_macro m, double* u, double* stress_gp, double* load) {
    RVE_TRY(check_ctx(c));
    if (!m) {
        set_error("rve_macro_mech_get: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    if ((u && !m->have_mech_u) || (stress_gp && !m->have_mech_sig) || (load && !m->have_mech_load)) {
        set_error("rve_macro_mech_get: nothing of that kind has been set or solved yet");
        return RVE_ERR_STATE;
    }
    cudaStream_t s = c->stream;
    const size_t n = (size_t)m->nv * 3;
    if (u) RVE_CUDA(cudaMemcpyAsync(u, m->mu.p, n * 8, cudaMemcpyDeviceToHost, s));
    if (load) RVE_CUDA(cudaMemcpyAsync(load, m->mload.p, n * 8, cudaMemcpyDeviceToHost, s));
    if (stress_gp)
        RVE_CUDA(cudaMemcpyAsync(stress_gp, m->msig.p, (size_t)m->nt * 4 * 6 * 8, cudaMemcpyDeviceToHost, s));
    RVE_CUDA(cudaStreamSynchronize(s));
    return RVE_OK;
}

}  // extern "C"
