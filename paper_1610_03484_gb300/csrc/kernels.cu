// Device kernels of librve (sm_103a).
//
// Vector layout (all vector kernels): v[row * ncols + col], row = dof * NC + comp.
// 2-D launches: grid = (ncols / cpb, nby), block = cpb * rows_per_block threads;
// thread (cl, r) owns column blockIdx.x * cpb + cl and strides over rows
// (or elements) starting at blockIdx.y * rows_per_block + r.  Every reduction
// writes one FP64 partial per (blockIdx.y, column), summed by a finalize kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>

#include "kernels.h"
#include "rve_internal.h"

namespace rve {

// Number of SMs of the current device, queried once per device ordinal; grid caps
// of the grid-stride kernels are multiples of it.
int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

// ------------------------------------------------------ checking build
#ifndef RVE_BOUNDS_CHECK
#define RVE_BOUNDS_CHECK 0
#endif
__device__ unsigned long long g_bounds_count;
__device__ long long g_bounds_first[2];   // element, column of the first violation

// True (and counted) when element e, its DOF indices or column col lie outside
// the arrays the kernel is about to index; always false in release builds.
template <int NE, typename T>
__device__ __forceinline__ bool elem_out_of_bounds(const ElemView<T>& ev, int64_t e, int col, int ncols) {
#if RVE_BOUNDS_CHECK
    // (a listed element comes from a colouring the host validated against the mesh)
    bool bad = e < 0 || (ev.elist == nullptr && e >= ev.nt) || col < 0 || col >= ncols;
    if (!bad)
        for (int j = 0; j < NE; ++j) {
            const int d = ev.edofs[e * NE + j];
            bad = bad || d < 0 || (ev.n_nodes > 0 && (int64_t)d >= ev.n_nodes);
        }
    if (bad && atomicAdd(&g_bounds_count, 1ull) == 0ull) {
        g_bounds_first[0] = (long long)e;
        g_bounds_first[1] = col;
    }
    return bad;
#else
    (void)ev;
    (void)e;
    (void)col;
    (void)ncols;
    return false;
#endif
}

bool bounds_check_built() { return RVE_BOUNDS_CHECK != 0; }

int bounds_status(unsigned long long* count, long long* first_elem, int* first_col) {
    unsigned long long c = 0;
    long long f[2] = {-1, -1};
    if (cudaMemcpyFromSymbol(&c, g_bounds_count, sizeof c) != cudaSuccess) return -1;
    if (c && cudaMemcpyFromSymbol(f, g_bounds_first, sizeof f) != cudaSuccess) return -1;
    if (count) *count = c;
    if (first_elem) *first_elem = c ? f[0] : -1;
    if (first_col) *first_col = c ? (int)f[1] : -1;
    return 0;
}

int bounds_reset() {
    const unsigned long long z = 0;
    return cudaMemcpyToSymbol(g_bounds_count, &z, sizeof z) == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------ basis tables
// A[k][m][j] of the hierarchic basis (see rve_internal.h), per order p.
__constant__ double cA64[3][3 * 10 * 20];
__constant__ float cA32[3][3 * 10 * 20];

void upload_basis_tables() {
    static double h64[3][3 * 10 * 20];
    static float h32[3][3 * 10 * 20];
    for (int p = 1; p <= 3; ++p) {
        const Basis& B = basis(p);
        for (size_t i = 0; i < B.A.size(); ++i) {
            h64[p - 1][i] = B.A[i];
            h32[p - 1][i] = (float)B.A[i];
        }
    }
    cudaMemcpyToSymbol(cA64, h64, sizeof(h64));
    cudaMemcpyToSymbol(cA32, h32, sizeof(h32));
}

template <typename T>
struct Tab;
template <>
struct Tab<double> {
    __device__ __forceinline__ static double a(int p, int i) { return cA64[p - 1][i]; }
};
template <>
struct Tab<float> {
    __device__ __forceinline__ static float a(int p, int i) { return cA32[p - 1][i]; }
};

// Compile-time copies of the same tables (generated at build time from
// basis.cpp): inside fully unrolled loops every entry is a literal, so the
// structurally zero entries drop out of the operator's arithmetic.
#include "basis_tables.inc"

template <int P, typename T>
__device__ __forceinline__ T basis_a(int i) {
    if constexpr (sizeof(T) == 4) {
        if constexpr (P == 1) return ctab::A1f[i];
        else if constexpr (P == 2) return ctab::A2f[i];
        else return ctab::A3f[i];
    } else {
        if constexpr (P == 1) return ctab::A1[i];
        else if constexpr (P == 2) return ctab::A2[i];
        else return ctab::A3[i];
    }
}

template <int P>
struct Order {
    static constexpr int NE = P == 1 ? 4 : (P == 2 ? 10 : 20);
    static constexpr int NM = P == 1 ? 1 : (P == 2 ? 4 : 10);
};

// Upper-triangular index of a symmetric 6x6 stored row by row.
__host__ __device__ constexpr int ut6(int i, int j) {
    return i <= j ? (i * 6 - i * (i - 1) / 2 + (j - i)) : (j * 6 - j * (j - 1) / 2 + (i - j));
}
// Symmetric 3x3 stored as (xx, yy, zz, xy, yz, zx).
__host__ __device__ constexpr int s3(int i, int j) {
    return i == j ? i : ((i + j == 1) ? 3 : ((i + j == 3) ? 4 : 5));
}

// ------------------------------------------------------- partial-sum type
// Per-thread partial sums: FP64 for the FP64 path; for the FP32 path a
// compensated (Kahan) FP32 sum, because FP64 arithmetic runs at a small
// fraction of the FP32 rate on this GPU.  Either way the block and grid level
// reductions that follow are FP64.
template <typename T>
struct PartialSum;
template <>
struct PartialSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct PartialSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---------------------------------------------------- block column reduction
// Reduce `nacc` per-thread values over the rows of the block for each column
// and store them to out[(blockIdx.y * ncols + col) * nacc + a].
template <int NACC>
__device__ __forceinline__ void block_column_reduce(const double (&acc)[NACC], double* out,
                                                    int ncols, int cpb, int col, double* atomic_out = nullptr) {
    __shared__ double buf[256];
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, r = threadIdx.x / cpb;
#pragma unroll 1
    for (int a = 0; a < NACC; ++a) {
        buf[threadIdx.x] = acc[a];
        __syncthreads();
        if (r == 0) {
            double s = 0.0;
            for (int q = 0; q < rows; ++q) s += buf[q * cpb + cl];
            if (atomic_out)   // fused iteration: one FP64 accumulator per column
                atomicAdd(atomic_out + (int64_t)col * NACC + a, s);
            else
                out[((int64_t)blockIdx.y * ncols + col) * NACC + a] = s;
        }
        __syncthreads();
    }
}

// Sum of one value per thread over the whole block (blockDim a multiple of 32,
// at most 1024); the result is valid in every thread.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double warp_part[32];
    __shared__ double total;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) warp_part[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? warp_part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) total = t;
    }
    __syncthreads();
    return total;
}

// Index of (DOF node d, component c, column col) in an n_rows x ncols vector, in
// 32-bit arithmetic (the hosts keep every vector of a solve below 2^31 entries).
template <int NC>
__device__ __forceinline__ uint32_t vix(int d, int c, int ncols, int col) {
    return ((uint32_t)d * (uint32_t)NC + (uint32_t)c) * (uint32_t)ncols + (uint32_t)col;
}

// ------------------------------------------------------------- the operator
// y += sum_e A_e^T K_e A_e x  for every column, matrix-free (Eq. RVE_Eq_var_final):
// per element, the reference gradient of the field is expanded on the
// orthonormal modes of P_{p-1}; each mode is mapped to the physical gradient
// by J^{-1}, turned into a stress (s * D : eps) or flux (s * k grad), mapped
// back and contracted with the same table, then scatter-added.  With MACRO
// the unit macro strain / gradient of the column is added to the constant mode,
// so -y is the fluctuation problem's residual b - K x.
template <int P, int NC, typename T, bool MACRO>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && P == 1) ? 4 : ((sizeof(T) == 4 && P == 2) ? 2 : 1)) k_operator(ElemView<T> ev, const T* __restrict__ x,
                                                  T* __restrict__ y, double* __restrict__ epart,
                                                  const int32_t* __restrict__ active, int ncols,
                                                  int cpb, const int32_t* __restrict__ list,
                                                  const int32_t* __restrict__ n_list,
                                                  double* __restrict__ eacc) {
    constexpr int NE = Order<P>::NE;
    constexpr int NM = Order<P>::NM;
    // With a column list the block's threads are spread over the listed (active)
    // columns only: rows per block grow as columns converge, and no lane is spent
    // on a converged column.  Otherwise thread (cl, rr) owns column blockIdx.x * cpb
    // + cl and converged columns skip the element loop (their step length is zero).
    int cpb_e = cpb, col;
    bool live;
    if (list != nullptr) {
        const int na = *n_list;
        cpb_e = na > 0 ? na : 1;
        live = na > 0 && (int)(threadIdx.x / cpb_e) < (int)(blockDim.x / cpb_e);
        col = live ? list[threadIdx.x % cpb_e] : 0;
    } else {
        col = blockIdx.x * cpb + threadIdx.x % cpb;
        live = !(active && !active[col]);
    }
    const int rows = blockDim.x / cpb_e;
    const int rr = threadIdx.x / cpb_e;
    const int field = (col % 6) >= 3 ? 1 : 0;   // scalar solve: thermal / moisture
    const int macro_id = NC == 3 ? (col % 6) : ((col % 6) % 3);
    PartialSum<T> energy;
    const int64_t e_end = live ? ev.nt : 0;

    for (int64_t ei = (int64_t)blockIdx.y * rows + rr; ei < e_end; ei += (int64_t)gridDim.y * rows) {
        const int64_t e = ev.elist ? (int64_t)__ldg(ev.elist + ei) : ei;
        if (elem_out_of_bounds<NE>(ev, e, col, ncols)) continue;
        const int32_t* ed = ev.edofs + e * NE;
        // ---- forward: reference-gradient modes V[m][k][c] = sum_j A[k][m][j] x_j,c.
        // Each gathered value is used for every mode at once and then dropped.
        // Without x (macro load only) every mode starts at zero.
        T V[NM][3][NC];
        if (MACRO && x == nullptr) {
#pragma unroll
            for (int m = 0; m < NM; ++m)
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c) V[m][k][c] = T(0);
        } else {
            const int d0 = __ldg(ed);
            T x0[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) x0[c] = x[vix<NC>(d0, c, ncols, col)];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int dk = __ldg(ed + k + 1);
#pragma unroll
                for (int c = 0; c < NC; ++c) V[0][k][c] = x[vix<NC>(dk, c, ncols, col)] - x0[c];
            }
#pragma unroll
            for (int m = 1; m < NM; ++m)
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int c = 0; c < NC; ++c) V[m][k][c] = T(0);
        }
        if (!(MACRO && x == nullptr)) {
#pragma unroll
        for (int j = 4; j < NE; ++j) {
            const int dj = __ldg(ed + j);
            T xj[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) xj[c] = x[vix<NC>(dj, c, ncols, col)];
#pragma unroll
            for (int m = 0; m < NM; ++m)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const T a = basis_a<P, T>((k * NM + m) * NE + j);
                    if (a != T(0))
#pragma unroll
                        for (int c = 0; c < NC; ++c) V[m][k][c] = fma(a, xj[c], V[m][k][c]);
                }
        }
        }
        // ---- element data; s * |T| folded into the material
        T G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) G[i] = __ldg(ev.geo + e * 10 + i);
        const T sv = __ldg(ev.scale + col * 2 + __ldg(ev.phase + e)) * __ldg(ev.geo + e * 10 + 9);
        constexpr int NMAT = NC == 3 ? 21 : 6;
        T Dm[NMAT];
#pragma unroll
        for (int i = 0; i < NMAT; ++i)
            Dm[i] = sv * __ldg(ev.mat + e * (NC == 3 ? 21 : 12) + (NC == 3 ? 0 : 6 * field) + i);
        // ---- per mode: gradient -> stress/flux -> W = J^-1 S, overwriting V
        // (macro load only: the higher modes are zero and stay zero)
        T e_elem = T(0);
        const int nm_live = (MACRO && x == nullptr) ? 1 : NM;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            if (m >= nm_live) break;
            T H[NC][3];
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int l = 0; l < 3; ++l)
                    H[c][l] = V[m][0][c] * G[l] + V[m][1][c] * G[3 + l] + V[m][2][c] * G[6 + l];
            if (MACRO && m == 0) {
                if constexpr (NC == 3) {
                    if (macro_id < 3) {
                        H[macro_id][macro_id] += T(1);
                    } else {
                        const int a = macro_id == 3 ? 0 : (macro_id == 4 ? 1 : 2);
                        const int b = macro_id == 3 ? 1 : (macro_id == 4 ? 2 : 0);
                        H[a][b] += T(0.5);
                        H[b][a] += T(0.5);
                    }
                } else {
                    H[0][macro_id] += T(1);
                }
            }
            T S[NC][3];
            if constexpr (NC == 3) {
                const T ev6[6] = {H[0][0], H[1][1], H[2][2], H[0][1] + H[1][0], H[1][2] + H[2][1],
                                  H[2][0] + H[0][2]};
                T sg[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    T t = T(0);
#pragma unroll
                    for (int jj = 0; jj < 6; ++jj) t = fma(Dm[ut6(i, jj)], ev6[jj], t);
                    sg[i] = t;
                }
                S[0][0] = sg[0]; S[0][1] = sg[3]; S[0][2] = sg[5];
                S[1][0] = sg[3]; S[1][1] = sg[1]; S[1][2] = sg[4];
                S[2][0] = sg[5]; S[2][1] = sg[4]; S[2][2] = sg[2];
            } else {
#pragma unroll
                for (int l = 0; l < 3; ++l)
                    S[0][l] = Dm[s3(l, 0)] * H[0][0] + Dm[s3(l, 1)] * H[0][1] + Dm[s3(l, 2)] * H[0][2];
            }
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const T w = G[3 * k] * S[c][0] + G[3 * k + 1] * S[c][1] + G[3 * k + 2] * S[c][2];
                    if (!MACRO) e_elem = fma(V[m][k][c], w, e_elem);   // x.Kx = sum V.W
                    V[m][k][c] = w;
                }
        }
        if ((epart || eacc) && !MACRO) energy.add(e_elem);
        // ---- backward and scatter: y_j,c = sum_m sum_k A[k][m][j] W[m][k][c]
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const T w0 = V[0][0][c], w1 = V[0][1][c], w2 = V[0][2][c];
            atomicAdd(y + vix<NC>(__ldg(ed), c, ncols, col), -(w0 + w1 + w2));
            atomicAdd(y + vix<NC>(__ldg(ed + 1), c, ncols, col), w0);
            atomicAdd(y + vix<NC>(__ldg(ed + 2), c, ncols, col), w1);
            atomicAdd(y + vix<NC>(__ldg(ed + 3), c, ncols, col), w2);
        }
#pragma unroll
        for (int j = 4; j < NE; ++j) {
            T yj[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) yj[c] = T(0);
#pragma unroll
            for (int m = 0; m < NM; ++m)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const T a = basis_a<P, T>((k * NM + m) * NE + j);
                    if (a != T(0))
#pragma unroll
                        for (int c = 0; c < NC; ++c) yj[c] = fma(a, V[m][k][c], yj[c]);
                }
            const int dj = __ldg(ed + j);
#pragma unroll
            for (int c = 0; c < NC; ++c) atomicAdd(y + vix<NC>(dj, c, ncols, col), yj[c]);
        }
    }
    if (epart || eacc) {
        double acc[1] = {energy.value()};
        block_column_reduce<1>(acc, epart, ncols, cpb_e, col,
                               eacc ? eacc + (size_t)(blockIdx.y % ACC_SLOTS) * ncols : nullptr);
    }
}

template <typename T>
int operator_grid_y(int p, int nc, const Launch& L, int64_t nt) {
    const int threads = L.cpb * L.rows_per_block;
    int per_sm = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define RVE_OCC_CASE(PP, NCC)                                                                           \
    if (p == PP && nc == NCC)                                                                           \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_operator<PP, NCC, T, false>, threads, 0);
    RVE_OCC_CASE(1, 3) RVE_OCC_CASE(2, 3) RVE_OCC_CASE(3, 3) RVE_OCC_CASE(1, 1) RVE_OCC_CASE(2, 1) RVE_OCC_CASE(3, 1)
#undef RVE_OCC_CASE
    if (e != cudaSuccess || per_sm < 1) return L.nby;
    const int gx = L.ncols / L.cpb;
    const int64_t want = (nt + L.rows_per_block - 1) / L.rows_per_block;
    const int64_t wave = std::max<int64_t>(1, (int64_t)per_sm * sm_count() / gx);
    return (int)std::max<int64_t>(1, std::min<int64_t>({want, wave, (int64_t)L.nby}));
}
template int operator_grid_y<float>(int, int, const Launch&, int64_t);
template int operator_grid_y<double>(int, int, const Launch&, int64_t);

template <typename T>
void launch_operator(int p, int nc, bool macro, const ElemView<T>& ev, const T* x, T* y,
                     double* energy_partial, const Launch& L, const int32_t* active, const int32_t* list,
                     const int32_t* n_list) {
    if (ev.ncolour > 0 && ev.coff && ev.elist_all) {
        // deterministic: one launch per colour, each with its own rows of partials
        Launch Lc = L;
        Lc.n_colour = 0;
        for (int k = 0; k < ev.ncolour; ++k) {
            ElemView<T> evk = ev;
            evk.ncolour = 0;
            evk.elist = ev.elist_all + ev.coff[k];
            evk.nt = ev.coff[k + 1] - ev.coff[k];
            double* ep = energy_partial ? energy_partial + (size_t)k * L.op_rows() * L.ncols : nullptr;
            launch_operator<T>(p, nc, macro, evk, x, y, ep, Lc, active, list, n_list);
        }
        return;
    }
    dim3 grid(L.ncols / L.cpb, L.op_rows()), block(L.cpb * L.rows_per_block);
    if (grid.x != 1) list = n_list = nullptr;   // the list maps one block column
#define RVE_OP_CASE(PP, NCC, MM)                                                                \
    if (p == PP && nc == NCC && macro == MM) {                                                  \
        k_operator<PP, NCC, T, MM><<<grid, block, 0, L.stream>>>(ev, x, y, energy_partial,      \
                                                                 active, L.ncols, L.cpb, list, \
                                                                 n_list, L.energy_acc);        \
        return;                                                                                 \
    }
    RVE_OP_CASE(1, 3, false) RVE_OP_CASE(2, 3, false) RVE_OP_CASE(3, 3, false)
    RVE_OP_CASE(1, 1, false) RVE_OP_CASE(2, 1, false) RVE_OP_CASE(3, 1, false)
    RVE_OP_CASE(1, 3, true) RVE_OP_CASE(2, 3, true) RVE_OP_CASE(3, 3, true)
    RVE_OP_CASE(1, 1, true) RVE_OP_CASE(2, 1, true) RVE_OP_CASE(3, 1, true)
#undef RVE_OP_CASE
}
template void launch_operator<float>(int, int, bool, const ElemView<float>&, const float*, float*,
                                     double*, const Launch&, const int32_t*, const int32_t*, const int32_t*);
template void launch_operator<double>(int, int, bool, const ElemView<double>&, const double*,
                                      double*, double*, const Launch&, const int32_t*, const int32_t*,
                                      const int32_t*);

// list[0 .. n) = the columns with active != 0 in ascending order: each warp ballots
// 32 flags, the warp counts are scanned in shared memory, lanes write in order.
// With CTL it is also the loop control of the device-side PCG loop (the body of a
// conditional WHILE graph node): it counts the iteration and keeps the loop going
// while some column is active and fewer than max_iter iterations have run; one
// thread sets the condition, whose value the node reads when the body ends.
template <bool CTL>
__device__ __forceinline__ void compact_and_control(const int32_t* __restrict__ active, int ncols,
                                                    int32_t* __restrict__ list, int32_t* __restrict__ n_list,
                                                    cudaGraphConditionalHandle h, int32_t* __restrict__ counter,
                                                    int max_iter) {
    __shared__ int counts[8];
    __shared__ int base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < ncols; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const bool a = c < ncols && active[c] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, a);
        if (lane == 0) counts[warp] = __popc(m);
        __syncthreads();
        int off = base;
        for (int w = 0; w < warp; ++w) off += counts[w];
        if (a) list[off + __popc(m & ((1u << lane) - 1u))] = c;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) base += counts[w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *n_list = base;
        if constexpr (CTL) {
            const int n = *counter + 1;
            *counter = n;
            cudaGraphSetConditional(h, (base > 0 && n < max_iter) ? 1u : 0u);
        }
    }
}

template <bool CTL>
__global__ void __launch_bounds__(256) k_compact_active(const int32_t* __restrict__ active, int ncols,
                                                        int32_t* __restrict__ list, int32_t* __restrict__ n_list,
                                                        cudaGraphConditionalHandle h, int32_t* __restrict__ counter,
                                                        int max_iter) {
    compact_and_control<CTL>(active, ncols, list, n_list, h, counter, max_iter);
}

// Fused iteration, one block: per active column rz from the update's accumulator,
// beta = rz / rz_old, the convergence test (the general path's beta kernel without
// constraint rows); both accumulators cleared for the next iteration; then the
// active list and, with CTL, the loop control.
template <bool CTL>
__global__ void __launch_bounds__(256) k_beta_compact(ColState cs, int ncols, cudaGraphConditionalHandle h,
                                                      int32_t* __restrict__ counter, int max_iter) {
    const double tol = *cs.tol;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        if (cs.active[c]) {
            double rz = 0.0;
            for (int k = 0; k < ACC_SLOTS; ++k) rz += cs.rz_acc[(size_t)k * ncols + c];
            if (!isfinite(rz)) {
                atomicOr(cs.flags, 1);
                cs.active[c] = 0;
            } else {
                cs.beta[c] = rz / cs.rz[c];
                cs.rz[c] = rz;
                if (rz <= tol * tol * cs.rz0[c]) cs.active[c] = 0;
            }
        }
        for (int k = 0; k < ACC_SLOTS; ++k) {
            cs.rz_acc[(size_t)k * ncols + c] = 0.0;
            cs.pq_acc[(size_t)k * ncols + c] = 0.0;
        }
    }
    __syncthreads();
    compact_and_control<CTL>(cs.active, ncols, cs.list, cs.n_list, h, counter, max_iter);
}

void launch_beta_compact_continue(ColState cs, int ncols, cudaGraphConditionalHandle h, int32_t* counter,
                                  int max_iter, bool ctl, cudaStream_t s) {
    if (ctl)
        k_beta_compact<true><<<1, 256, 0, s>>>(cs, ncols, h, counter, max_iter);
    else
        k_beta_compact<false><<<1, 256, 0, s>>>(cs, ncols, 0, nullptr, 0);
}

void launch_compact_active(const int32_t* active, int ncols, int32_t* list, int32_t* n_list, cudaStream_t s) {
    k_compact_active<false><<<1, 256, 0, s>>>(active, ncols, list, n_list, 0, nullptr, 0);
}

void launch_compact_continue(const int32_t* active, int ncols, int32_t* list, int32_t* n_list,
                             cudaGraphConditionalHandle h, int32_t* counter, int max_iter, cudaStream_t s) {
    k_compact_active<true><<<1, 256, 0, s>>>(active, ncols, list, n_list, h, counter, max_iter);
}

// ------------------------------------- double-float residual (mixed precision)
// r += -K32 (x + u_macro), where K32 is the operator with exactly the FP32
// element data and tables of the FP32 kernel above, evaluated in double-float
// arithmetic: every FP32 x FP32 product is split exactly (p + e = a b with
// e = fma(a, b, -p)) and every sum carries its rounding error in a second FP32
// word (Knuth's two-sum).  Relative accuracy is about 2^-44 per stage, against
// 2^-53 in FP64 at 1/64 of the FP32 arithmetic rate on this GPU.  x enters split
// beforehand into two FP32 words x_h + x_l (x_h = nullptr: x = 0; the FP64
// remainder below 2^-48 |x| is dropped).  The high word of each result goes to
// r_hi with an FP64 atomic, the low word to r_lo with an FP32 atomic (its own
// rounding is 2^-24 of a word already 2^-24 below the high one); the caller adds
// r_lo into r_hi afterwards.  No FP64 arithmetic runs per element.

// s += a * (bh + bl) for an exact FP32 a; the low word collects the error terms.
// The _rn intrinsics keep the compiler from contracting a product and a sum into
// one FMA, which would break the exact error terms.
__device__ __forceinline__ void df_mac(float& sh, float& sl, float a, float bh, float bl) {
    const float ph = __fmul_rn(a, bh);
    const float pl = fmaf(a, bh, -ph);
    const float t = __fadd_rn(sh, ph);
    const float bb = __fsub_rn(t, sh);
    const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(ph, bb));
    sh = t;
    sl += e + fmaf(a, bl, pl);
}
// s += (bh + bl)
__device__ __forceinline__ void df_add(float& sh, float& sl, float bh, float bl) {
    const float t = __fadd_rn(sh, bh);
    const float bb = __fsub_rn(t, sh);
    const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(bh, bb));
    sh = t;
    sl += e + bl;
}
// (h, l) <- (h + l) renormalised so that |l| <= ulp(h) / 2
__device__ __forceinline__ void df_norm(float& h, float& l) {
    const float t = __fadd_rn(h, l);
    l = __fsub_rn(l, __fsub_rn(t, h));
    h = t;
}
__device__ __forceinline__ void df_split(double v, float& h, float& l) {
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
}

// True when local function j (>= 4) has a nonzero table entry in modes [M0, M1).
template <int P, int M0, int M1>
__host__ __device__ constexpr bool df_group_touches(int j) {
    constexpr int NE = Order<P>::NE, NM = Order<P>::NM;
    for (int m = M0; m < M1; ++m)
        for (int k = 0; k < 3; ++k)
            if (basis_a<P, float>((k * NM + m) * NE + j) != 0.f) return true;
    return false;
}

// The contribution of the reference-gradient modes [M0, M1) of every element: the
// modes are independent until the scatter (the stress of mode m depends on mode m
// alone), so the kernel runs once per group of modes and the groups' scatters
// add up.  Fewer modes per pass keep the double-float state of a thread small
// enough for two resident blocks per SM.
template <int P, int NC, int M0, int M1>
__global__ void __launch_bounds__(256, 2) k_residual_df(ElemView<float> ev, const float* __restrict__ xh,
                                                        const float* __restrict__ xl, double* __restrict__ r,
                                                        float* __restrict__ rlo, int ncols, int cpb) {
    constexpr int NE = Order<P>::NE;
    constexpr int NM = Order<P>::NM;
    constexpr int G_ = M1 - M0;
    constexpr bool HAS0 = M0 == 0;
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, rr = threadIdx.x / cpb;
    const int col = blockIdx.x * cpb + cl;
    const int field = (col % 6) >= 3 ? 1 : 0;
    const int macro_id = NC == 3 ? (col % 6) : ((col % 6) % 3);
    for (int64_t ei = (int64_t)blockIdx.y * rows + rr; ei < ev.nt; ei += (int64_t)gridDim.y * rows) {
        const int64_t e = ev.elist ? (int64_t)__ldg(ev.elist + ei) : ei;
        if (elem_out_of_bounds<NE>(ev, e, col, ncols)) continue;
        const int32_t* ed = ev.edofs + e * NE;
        float Vh[G_][3][NC], Vl[G_][3][NC];
#pragma unroll
        for (int m = 0; m < G_; ++m)
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) Vh[m][k][c] = Vl[m][k][c] = 0.f;
        if (xh != nullptr) {
            if constexpr (HAS0) {
                const int d0 = __ldg(ed);
                float x0h[NC], x0l[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const uint32_t i0 = vix<NC>(d0, c, ncols, col);
                    x0h[c] = -xh[i0];
                    x0l[c] = -xl[i0];
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int dk = __ldg(ed + k + 1);
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const uint32_t ik = vix<NC>(dk, c, ncols, col);
                        Vh[0][k][c] = xh[ik];
                        Vl[0][k][c] = xl[ik];
                        df_add(Vh[0][k][c], Vl[0][k][c], x0h[c], x0l[c]);
                    }
                }
            }
#pragma unroll
            for (int j = 4; j < NE; ++j) {
                if (!df_group_touches<P, M0, M1>(j)) continue;
                const int dj = __ldg(ed + j);
                float vh[NC], vl[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const uint32_t ij = vix<NC>(dj, c, ncols, col);
                    vh[c] = xh[ij];
                    vl[c] = xl[ij];
                }
#pragma unroll
                for (int m = 0; m < G_; ++m)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float a = basis_a<P, float>((k * NM + M0 + m) * NE + j);
                        if (a != 0.f)
#pragma unroll
                            for (int c = 0; c < NC; ++c) df_mac(Vh[m][k][c], Vl[m][k][c], a, vh[c], vl[c]);
                    }
            }
        }
#pragma unroll
        for (int m = 0; m < G_; ++m)
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) df_norm(Vh[m][k][c], Vl[m][k][c]);
        // element data exactly as the FP32 kernel forms it
        float G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) G[i] = __ldg(ev.geo + e * 10 + i);
        const float sv = __ldg(ev.scale + col * 2 + __ldg(ev.phase + e)) * __ldg(ev.geo + e * 10 + 9);
        constexpr int NMAT = NC == 3 ? 21 : 6;
        float Dm[NMAT];
#pragma unroll
        for (int i = 0; i < NMAT; ++i)
            Dm[i] = sv * __ldg(ev.mat + e * (NC == 3 ? 21 : 12) + (NC == 3 ? 0 : 6 * field) + i);
#pragma unroll
        for (int m = 0; m < G_; ++m) {
            float Hh[NC][3], Hl[NC][3];
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    Hh[c][l] = Hl[c][l] = 0.f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) df_mac(Hh[c][l], Hl[c][l], G[3 * k + l], Vh[m][k][c], Vl[m][k][c]);
                }
            if (HAS0 && m == 0) {
                // the column's unit macro gradient, added entry by entry with
                // compile-time indices (keeps H in registers)
                const int ma = NC == 3 ? (macro_id < 3 ? macro_id : (macro_id == 3 ? 0 : (macro_id == 4 ? 1 : 2))) : 0;
                const int mb = NC == 3 ? (macro_id < 3 ? macro_id : (macro_id == 3 ? 1 : (macro_id == 4 ? 2 : 0)))
                                       : macro_id;
                const float v = (NC == 3 && macro_id >= 3) ? 0.5f : 1.f;
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int l = 0; l < 3; ++l)
                        if ((c == ma && l == mb) || (NC == 3 && macro_id >= 3 && c == mb && l == ma))
                            df_add(Hh[c][l], Hl[c][l], v, 0.f);
            }
            float Sh[NC][3], Sl[NC][3];
            if constexpr (NC == 3) {
                float eh[6] = {Hh[0][0], Hh[1][1], Hh[2][2], Hh[0][1], Hh[1][2], Hh[2][0]};
                float el[6] = {Hl[0][0], Hl[1][1], Hl[2][2], Hl[0][1], Hl[1][2], Hl[2][0]};
                df_add(eh[3], el[3], Hh[1][0], Hl[1][0]);
                df_add(eh[4], el[4], Hh[2][1], Hl[2][1]);
                df_add(eh[5], el[5], Hh[0][2], Hl[0][2]);
#pragma unroll
                for (int i = 0; i < 6; ++i) df_norm(eh[i], el[i]);
                float gh[6], gl[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    gh[i] = gl[i] = 0.f;
#pragma unroll
                    for (int jj = 0; jj < 6; ++jj) df_mac(gh[i], gl[i], Dm[ut6(i, jj)], eh[jj], el[jj]);
                }
                const int vi[3][3] = {{0, 3, 5}, {3, 1, 4}, {5, 4, 2}};
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        Sh[a][b] = gh[vi[a][b]];
                        Sl[a][b] = gl[vi[a][b]];
                    }
            } else {
#pragma unroll
                for (int q = 0; q < 3; ++q) df_norm(Hh[0][q], Hl[0][q]);
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    Sh[0][l] = Sl[0][l] = 0.f;
#pragma unroll
                    for (int q = 0; q < 3; ++q) df_mac(Sh[0][l], Sl[0][l], Dm[s3(l, q)], Hh[0][q], Hl[0][q]);
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int l = 0; l < 3; ++l) df_norm(Sh[c][l], Sl[c][l]);
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    float wh = 0.f, wl = 0.f;
#pragma unroll
                    for (int l = 0; l < 3; ++l) df_mac(wh, wl, G[3 * k + l], Sh[c][l], Sl[c][l]);
                    df_norm(wh, wl);
                    Vh[m][k][c] = wh;
                    Vl[m][k][c] = wl;
                }
        }
        // backward and scatter of -(K (x + u_macro)) for these modes
        if constexpr (HAS0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float sh = Vh[0][0][c], sl = Vl[0][0][c];
                df_add(sh, sl, Vh[0][1][c], Vl[0][1][c]);
                df_add(sh, sl, Vh[0][2][c], Vl[0][2][c]);
                const uint32_t i0 = vix<NC>(__ldg(ed), c, ncols, col);
                atomicAdd(r + i0, (double)sh);
                atomicAdd(rlo + i0, sl);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const uint32_t ik = vix<NC>(__ldg(ed + k + 1), c, ncols, col);
                    atomicAdd(r + ik, (double)-Vh[0][k][c]);
                    atomicAdd(rlo + ik, -Vl[0][k][c]);
                }
            }
        }
#pragma unroll
        for (int j = 4; j < NE; ++j) {
            if (!df_group_touches<P, M0, M1>(j)) continue;
            float yh[NC], yl[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) yh[c] = yl[c] = 0.f;
#pragma unroll
            for (int m = 0; m < G_; ++m)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float a = basis_a<P, float>((k * NM + M0 + m) * NE + j);
                    if (a != 0.f)
#pragma unroll
                        for (int c = 0; c < NC; ++c) df_mac(yh[c], yl[c], a, Vh[m][k][c], Vl[m][k][c]);
                }
            const int dj = __ldg(ed + j);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const uint32_t ij = vix<NC>(dj, c, ncols, col);
                atomicAdd(r + ij, (double)-yh[c]);
                atomicAdd(rlo + ij, -yl[c]);
            }
        }
    }
}

// x = x_h + x_l, two FP32 words per FP64 entry (the double-float kernel's input)
__global__ void k_split_d2ff(int64_t n, const double* __restrict__ x, float* __restrict__ xh,
                             float* __restrict__ xl) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        df_split(x[i], h, l);
        xh[i] = h;
        xl[i] = l;
    }
}

void launch_split_d2ff(int64_t n, const double* x, float* xh, float* xl, cudaStream_t s) {
    int64_t b = (n + 255) / 256;
    if (b > sm_count() * 16) b = sm_count() * 16;
    if (b < 1) b = 1;
    k_split_d2ff<<<(unsigned)b, 256, 0, s>>>(n, x, xh, xl);
}

void launch_residual_df(int p, int nc, const ElemView<float>& ev, const float* xh, const float* xl,
                        double* r, float* rlo, const Launch& L) {
    if (ev.ncolour > 0 && ev.coff && ev.elist_all) {
        for (int k = 0; k < ev.ncolour; ++k) {
            ElemView<float> evk = ev;
            evk.ncolour = 0;
            evk.elist = ev.elist_all + ev.coff[k];
            evk.nt = ev.coff[k + 1] - ev.coff[k];
            launch_residual_df(p, nc, evk, xh, xl, r, rlo, L);
        }
        return;
    }
    dim3 grid(L.ncols / L.cpb, L.nby), block(L.cpb * L.rows_per_block);
    // mode groups: p = 1 has one mode, p = 2 four (two passes of two), p = 3 ten
    // (passes of four, three and three)
#define RVE_DF_RUN(PP, NCC, A, B) \
    k_residual_df<PP, NCC, A, B><<<grid, block, 0, L.stream>>>(ev, xh, xl, r, rlo, L.ncols, L.cpb);
    if (p == 1) {
        if (nc == 3) { RVE_DF_RUN(1, 3, 0, 1) } else { RVE_DF_RUN(1, 1, 0, 1) }
    } else if (p == 2) {
        if (nc == 3) { RVE_DF_RUN(2, 3, 0, 2) RVE_DF_RUN(2, 3, 2, 4) }
        else { RVE_DF_RUN(2, 1, 0, 4) }
    } else if (p == 3) {
        if (nc == 3) { RVE_DF_RUN(3, 3, 0, 4) RVE_DF_RUN(3, 3, 4, 7) RVE_DF_RUN(3, 3, 7, 10) }
        else { RVE_DF_RUN(3, 1, 0, 5) RVE_DF_RUN(3, 1, 5, 10) }
    }
#undef RVE_DF_RUN
}

// ------------------------------------------------------ Jacobi diagonal (K6)
// diag[field][phase][row] = unscaled diagonal of K restricted to one phase.
template <int P, int NC, typename T>
__global__ void k_diag(ElemView<T> ev, int64_t n_rows, T* __restrict__ diag) {
    constexpr int NE = Order<P>::NE;
    constexpr int NM = Order<P>::NM;
    const int64_t ei = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ei >= ev.nt) return;
    const int64_t e = ev.elist ? (int64_t)ev.elist[ei] : ei;
    if (elem_out_of_bounds<NE>(ev, e, 0, 1)) return;
    double G[9];
    for (int i = 0; i < 9; ++i) G[i] = ev.geo[e * 10 + i];
    const double vol = ev.geo[e * 10 + 9];
    const int ph = ev.phase[e];
    const int nfield = NC == 3 ? 1 : 2;
    for (int f = 0; f < nfield; ++f) {
        double Dm[21];
        const int nmat = NC == 3 ? 21 : 6;
        for (int i = 0; i < nmat; ++i) Dm[i] = ev.mat[e * (NC == 3 ? 21 : 12) + 6 * f + i];
        for (int j = 0; j < NE; ++j) {
            const int dof = ev.edofs[e * NE + j];
            double d[NC];
            for (int c = 0; c < NC; ++c) d[c] = 0.0;
            for (int m = 0; m < NM; ++m) {
                double a[3];
                for (int k = 0; k < 3; ++k) {
                    if (j < 4)
                        a[k] = (m == 0) ? ((j == k + 1) ? 1.0 : (j == 0 ? -1.0 : 0.0)) : 0.0;
                    else
                        a[k] = Tab<double>::a(P, (k * NM + m) * NE + j);
                }
                double g[3];
                for (int l = 0; l < 3; ++l) g[l] = a[0] * G[l] + a[1] * G[3 + l] + a[2] * G[6 + l];
                if (NC == 3) {
                    for (int c = 0; c < 3; ++c) {
                        // Voigt strain of e_c (x) g
                        double ev6[6] = {0, 0, 0, 0, 0, 0};
                        ev6[c] = g[c];
                        if (c == 0) { ev6[3] = g[1]; ev6[5] = g[2]; }
                        if (c == 1) { ev6[3] = g[0]; ev6[4] = g[2]; }
                        if (c == 2) { ev6[4] = g[1]; ev6[5] = g[0]; }
                        double en = 0;
                        for (int i = 0; i < 6; ++i)
                            for (int jj = 0; jj < 6; ++jj) en += ev6[i] * Dm[ut6(i, jj)] * ev6[jj];
                        d[c % NC] += vol * en;
                    }
                } else {
                    double en = 0;
                    for (int l = 0; l < 3; ++l)
                        for (int l2 = 0; l2 < 3; ++l2) en += g[l] * Dm[s3(l, l2)] * g[l2];
                    d[0] += vol * en;
                }
            }
            for (int c = 0; c < NC; ++c)
                atomicAdd(diag + ((int64_t)(f * 2 + ph)) * n_rows + (int64_t)dof * NC + c, (T)d[c]);
        }
    }
}

template <typename T>
void launch_diag(int p, int nc, int64_t n_rows, const ElemView<T>& ev, T* diag, cudaStream_t s) {
    if (ev.ncolour > 0 && ev.coff && ev.elist_all) {
        for (int k = 0; k < ev.ncolour; ++k) {
            ElemView<T> evk = ev;
            evk.ncolour = 0;
            evk.elist = ev.elist_all + ev.coff[k];
            evk.nt = ev.coff[k + 1] - ev.coff[k];
            if (evk.nt > 0) launch_diag<T>(p, nc, n_rows, evk, diag, s);
        }
        return;
    }
    const int bs = 128;
    const int64_t nb = (ev.nt + bs - 1) / bs;
#define RVE_DG_CASE(PP, NCC)                                                                  \
    if (p == PP && nc == NCC) {                                                               \
        k_diag<PP, NCC, T><<<(unsigned)nb, bs, 0, s>>>(ev, n_rows, diag);                     \
        return;                                                                               \
    }
    RVE_DG_CASE(1, 3) RVE_DG_CASE(2, 3) RVE_DG_CASE(3, 3)
    RVE_DG_CASE(1, 1) RVE_DG_CASE(2, 1) RVE_DG_CASE(3, 1)
#undef RVE_DG_CASE
}
template void launch_diag<double>(int, int, int64_t, const ElemView<double>&, double*, cudaStream_t);

// ------------------------------------------------------------ geometry (K2)
__global__ void k_geometry(int64_t nt, const double* __restrict__ xyz,
                           const int32_t* __restrict__ lverts, double* __restrict__ geo64,
                           float* __restrict__ geo32, int32_t* bad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt) return;
    double v[4][3];
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) v[a][i] = xyz[3 * (int64_t)lverts[4 * e + a] + i];
    double a[3], b[3], c[3];
    for (int i = 0; i < 3; ++i) {
        a[i] = v[1][i] - v[0][i];
        b[i] = v[2][i] - v[0][i];
        c[i] = v[3][i] - v[0][i];
    }
    double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    double ca[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
    double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    const double det = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
    const double scale = fmax(fmax(fabs(a[0]) + fabs(a[1]) + fabs(a[2]), fabs(b[0]) + fabs(b[1]) + fabs(b[2])),
                              fabs(c[0]) + fabs(c[1]) + fabs(c[2]));
    if (!(fabs(det) > 1e-12 * scale * scale * scale)) {
        atomicExch(bad, 1);
        return;
    }
    double g[10];
    for (int i = 0; i < 3; ++i) {
        g[i] = bc[i] / det;       // grad xi_1
        g[3 + i] = ca[i] / det;   // grad xi_2
        g[6 + i] = ab[i] / det;   // grad xi_3
    }
    g[9] = fabs(det) / 6.0;
    for (int i = 0; i < 10; ++i) {
        geo64[e * 10 + i] = g[i];
        geo32[e * 10 + i] = (float)g[i];
    }
}

void launch_geometry(int64_t nt, const double* xyz, const int32_t* lverts, double* geo64,
                     float* geo32, int32_t* bad, cudaStream_t s) {
    const int bs = 128;
    k_geometry<<<(unsigned)((nt + bs - 1) / bs), bs, 0, s>>>(nt, xyz, lverts, geo64, geo32, bad);
}

// ----------------------------------------------------------- materials (K1)
// Isotropic matrix; transversely isotropic yarn built in the fibre frame and
// rotated with the Bond stress matrix M: D_global = M D_local M^T (Sec. 6).
__global__ void k_materials(int64_t nt, const uint8_t* __restrict__ phase,
                            const double* __restrict__ tangent, MaterialConsts mc,
                            double* __restrict__ m64, float* __restrict__ m32,
                            double* __restrict__ s64, float* __restrict__ s32, int32_t* bad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt) return;
    double D[6][6] = {};
    double kt[3][3] = {}, dt[3][3] = {};
    if (phase[e] == 0) {
        const double E = mc.Em, nu = mc.num;
        const double lam = E * nu / ((1 + nu) * (1 - 2 * nu)), mu = E / (2 * (1 + nu));
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) D[i][j] = lam;
            D[i][i] += 2 * mu;
            D[3 + i][3 + i] = mu;
            kt[i][i] = mc.km;
            dt[i][i] = mc.dm;
        }
    } else {
        double t[3] = {tangent[3 * e], tangent[3 * e + 1], tangent[3 * e + 2]};
        const double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        if (!(tn > 0)) {
            atomicExch(bad, 1);
            return;
        }
        for (int i = 0; i < 3; ++i) t[i] /= tn;
        double h[3] = {0, 0, 1};
        if (fabs(t[2]) >= 0.9) { h[0] = 1; h[2] = 0; }
        const double th = t[0] * h[0] + t[1] * h[1] + t[2] * h[2];
        double a[3] = {h[0] - th * t[0], h[1] - th * t[1], h[2] - th * t[2]};
        const double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int i = 0; i < 3; ++i) a[i] /= an;
        double b[3] = {t[1] * a[2] - t[2] * a[1], t[2] * a[0] - t[0] * a[2], t[0] * a[1] - t[1] * a[0]};
        double R[3][3];   // columns = local axes (fibre, a, b) in global coordinates
        for (int i = 0; i < 3; ++i) {
            R[i][0] = t[i];
            R[i][1] = a[i];
            R[i][2] = b[i];
        }
        // local stiffness: invert the normal compliance block, shear moduli direct
        const double S11 = 1 / mc.E1, S22 = 1 / mc.E2, S12 = -mc.nu12 / mc.E1, S23 = -mc.nu23 / mc.E2;
        double Sn[3][3] = {{S11, S12, S12}, {S12, S22, S23}, {S12, S23, S22}};
        double cof[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
                cof[i][j] = Sn[i1][j1] * Sn[i2][j2] - Sn[i1][j2] * Sn[i2][j1];
            }
        const double det = Sn[0][0] * cof[0][0] + Sn[0][1] * cof[0][1] + Sn[0][2] * cof[0][2];
        if (!(det > 0)) {
            atomicExch(bad, 1);
            return;
        }
        double Dl[6][6] = {};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Dl[i][j] = cof[j][i] / det;
        Dl[3][3] = mc.G12;                          // 12
        Dl[5][5] = mc.G12;                          // 31
        Dl[4][4] = mc.E2 / (2 * (1 + mc.nu23));     // 23
        static const int VI[6] = {0, 1, 2, 0, 1, 2}, VJ[6] = {0, 1, 2, 1, 2, 0};
        double M[6][6];
        for (int I = 0; I < 6; ++I)
            for (int J = 0; J < 6; ++J) {
                const int i = VI[I], j = VJ[I], p = VI[J], q = VJ[J];
                M[I][J] = (J < 3) ? R[i][p] * R[j][p] : R[i][p] * R[j][q] + R[i][q] * R[j][p];
            }
        double MD[6][6];
        for (int I = 0; I < 6; ++I)
            for (int J = 0; J < 6; ++J) {
                double sacc = 0;
                for (int K = 0; K < 6; ++K) sacc += M[I][K] * Dl[K][J];
                MD[I][J] = sacc;
            }
        for (int I = 0; I < 6; ++I)
            for (int J = 0; J < 6; ++J) {
                double sacc = 0;
                for (int K = 0; K < 6; ++K) sacc += MD[I][K] * M[J][K];
                D[I][J] = sacc;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                kt[i][j] = (i == j ? mc.k2 : 0.0) + (mc.k1 - mc.k2) * t[i] * t[j];
                dt[i][j] = (i == j ? mc.d2 : 0.0) + (mc.d1 - mc.d2) * t[i] * t[j];
            }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
            const double v = 0.5 * (D[i][j] + D[j][i]) / mc.ref_mech;
            m64[e * 21 + ut6(i, j)] = v;
            m32[e * 21 + ut6(i, j)] = (float)v;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            const double vk = kt[i][j] / mc.ref_k, vd = dt[i][j] / mc.ref_d;
            s64[e * 12 + s3(i, j)] = vk;
            s32[e * 12 + s3(i, j)] = (float)vk;
            s64[e * 12 + 6 + s3(i, j)] = vd;
            s32[e * 12 + 6 + s3(i, j)] = (float)vd;
        }
}

void launch_materials(int64_t nt, const uint8_t* phase, const double* tangent,
                      const MaterialConsts& mc, double* matm64, float* matm32, double* mats64,
                      float* mats32, int32_t* bad, cudaStream_t s) {
    const int bs = 128;
    k_materials<<<(unsigned)((nt + bs - 1) / bs), bs, 0, s>>>(nt, phase, tangent, mc, matm64,
                                                              matm32, mats64, mats32, bad);
}

// --------------------------------------------------------- degradation (K1)
// 1 - omega = exp(-c alpha(T) t), alpha(T) = beta ln(1 - T/Tg) in kelvin,
// c = clamp(c_wt / c_sat), t in days (Sec. 4, Eqs. alphaT and Model_final1).
__global__ void k_degradation(int64_t n, const double* __restrict__ T_C,
                              const double* __restrict__ c_wt, const double* __restrict__ t_h,
                              double beta, double Tg_C, double c_sat, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = fmin(fmax(c_wt[i] / c_sat, 0.0), 1.0);
    const double alpha = beta * log(1.0 - (T_C[i] + 273.15) / (Tg_C + 273.15));
    out[i] = exp(-c * alpha * (t_h[i] / 24.0));
}

void launch_degradation(int64_t n, const double* T_C, const double* c_wt, const double* t_h,
                        double beta, double Tg_C, double c_sat, double* out, cudaStream_t s) {
    if (n <= 0) return;
    const int bs = 128;
    k_degradation<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(n, T_C, c_wt, t_h, beta, Tg_C,
                                                               c_sat, out);
}

template <typename T>
__global__ void k_column_scales(int nrve, const double* __restrict__ w, int apply_to_yarn,
                                int mech, T* __restrict__ scale) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= nrve * 6) return;
    const double f = mech ? w[col / 6] : 1.0;
    scale[2 * col + 0] = (T)f;
    scale[2 * col + 1] = (T)((mech && apply_to_yarn) ? f : 1.0);
}

template <typename T>
void launch_column_scales(int nrve, const double* w, int apply_to_yarn, bool mech, T* scale,
                          cudaStream_t s) {
    const int bs = 128;
    k_column_scales<T><<<(nrve * 6 + bs - 1) / bs, bs, 0, s>>>(nrve, w, apply_to_yarn, mech ? 1 : 0,
                                                               scale);
}
template void launch_column_scales<float>(int, const double*, int, bool, float*, cudaStream_t);
template void launch_column_scales<double>(int, const double*, int, bool, double*, cudaStream_t);

// ------------------------------------------------------------- PCG pieces
// Jacobi preconditioner entry of one row for one column: the per-phase diagonals
// combined with the column's phase scales (an explicit FMA, so that every kernel
// forms exactly the same value), zero on Dirichlet-masked rows.
template <typename T>
__device__ __forceinline__ T jacobi_inv(T s0, T d0, T s1, T d1) {
    T d;
    if constexpr (sizeof(T) == 4) {
        d = fmaf(s0, d0, __fmul_rn(s1, d1));
        return d > 0.f ? __frcp_rn(d) : 0.f;   // correctly rounded reciprocal
    } else {
        d = fma(s0, d0, __dmul_rn(s1, d1));
        return d > 0.0 ? 1.0 / d : 0.0;
    }
}

template <typename T>
__device__ __forceinline__ T inv_diag(const RowView<T>& rv, int64_t row, int col, int ncols) {
    const int64_t dof = row / rv.nc;
    if (rv.mask && rv.mask[dof]) return T(0);
    const int f = (rv.nfield == 2 && (col % 6) >= 3) ? 1 : 0;
    return jacobi_inv<T>(rv.scale[2 * col], rv.diag[(int64_t)(2 * f) * rv.n_rows + row], rv.scale[2 * col + 1],
                         rv.diag[(int64_t)(2 * f + 1) * rv.n_rows + row]);
}

// The same for a fixed column, with its scales and diagonal rows held in registers.
template <typename T, int NC>
struct ColJacobi {
    const T* d0;
    const T* d1;
    const uint8_t* mask;
    T s0, s1;
    __device__ __forceinline__ ColJacobi(const RowView<T>& rv, int col) {
        const int f = (rv.nfield == 2 && (col % 6) >= 3) ? 1 : 0;
        d0 = rv.diag + (int64_t)(2 * f) * rv.n_rows;
        d1 = d0 + rv.n_rows;
        mask = rv.mask;
        s0 = rv.scale[2 * col];
        s1 = rv.scale[2 * col + 1];
    }
    __device__ __forceinline__ T inv(int64_t row) const {
        if (mask && mask[row / NC]) return T(0);
        return jacobi_inv<T>(s0, __ldg(d0 + row), s1, __ldg(d1 + row));
    }
};

// One block per column: alpha = (r, z) / (p, K p) with (p, K p) summed in parallel.
__global__ void __launch_bounds__(256) k_finalize_alpha(const double* __restrict__ ep, int nby, int ncols,
                                                        ColState cs) {
    const int col = blockIdx.x;
    // a bounded wait in the operator gave up (flag bit 2): every column stops, so
    // the device-side loop ends at the next compaction
    if (!cs.active[col] || (cs.flags[0] & 4)) {
        if (threadIdx.x == 0) {
            cs.alpha[col] = 0.0;
            cs.active[col] = 0;
        }
        return;
    }
    double v = 0.0;
    for (int b = threadIdx.x; b < nby; b += blockDim.x) v += ep[(int64_t)b * ncols + col];
    const double pq = block_sum(v);
    if (threadIdx.x != 0) return;
    double a = cs.rz[col] / pq;
    if (!(pq > 0.0) || !isfinite(a)) {
        atomicOr(cs.flags, 1);
        a = 0.0;
        cs.active[col] = 0;
    }
    cs.alpha[col] = a;
    cs.iters[col] += 1;
}

template <typename T>
void launch_finalize_alpha(const double* energy_partial, ColState cs, const Launch& L) {
    k_finalize_alpha<<<L.ncols, 256, 0, L.stream>>>(energy_partial, L.op_partials(), L.ncols, cs);
}
template void launch_finalize_alpha<float>(const double*, ColState, const Launch&);
template void launch_finalize_alpha<double>(const double*, ColState, const Launch&);

// x += alpha p, r -= alpha q (when apply), partial (r, M^-1 r) per column and,
// on constraint-support rows (HAS_C), the partial constraint products C M^-1 r
// (m <= 12 rows), written to cp[(blockIdx.y * m + k) * ncols + col].  Instances
// without constraint rows carry no constraint accumulators (fewer registers,
// more resident warps for this memory-bound pass).
template <typename T, int NC, bool HAS_C>
__global__ void __launch_bounds__(256) k_update(RowView<T> rv, T* __restrict__ x, T* __restrict__ r,
                                                const T* __restrict__ p, const T* __restrict__ q,
                                                ColState cs, double* __restrict__ rzp,
                                                double* __restrict__ cp, int ncols, int cpb, int apply) {
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, rr = threadIdx.x / cpb;
    const int col = blockIdx.x * cpb + cl;
    const T a = apply ? (T)cs.alpha[col] : T(0);
    const ColJacobi<T, NC> jac(rv, col);
    PartialSum<T> acc;
    PartialSum<T> cacc[HAS_C ? 12 : 1];
    const int m = HAS_C ? rv.m : 0;
    // a converged column keeps x and r; its partials stay zero
    const int64_t i_end = (apply && !cs.active[col]) ? 0 : rv.n_rows;
    const int64_t stride = (int64_t)gridDim.y * rows;
    for (int64_t i = (int64_t)blockIdx.y * rows + rr; i < i_end; i += stride) {
        const int64_t idx = i * ncols + col;
        T rv_ = r[idx];
        if (a != T(0)) {
            const T pv = p[idx], qv = q[idx], xv = x[idx];
            x[idx] = fma(a, pv, xv);
            rv_ = fma(-a, qv, rv_);
            r[idx] = rv_;
        }
        const T w = jac.inv(i) * rv_;
        acc.add(rv_ * w);
        if constexpr (HAS_C) {
            const int32_t sidx = rv.sup_of_row[i];
            if (sidx >= 0) {
#pragma unroll
                for (int k = 0; k < 12; ++k)
                    if (k < m) cacc[k].add((T)rv.sup_coef[(int64_t)sidx * m + k] * w);
            }
        }
    }
    double accs[1] = {acc.value()};
    block_column_reduce<1>(accs, rzp, ncols, cpb, col);
    if constexpr (HAS_C) {
        if (cp) {
            __shared__ double buf[256];
            for (int k = 0; k < m; ++k) {
                buf[threadIdx.x] = cacc[k].value();
                __syncthreads();
                if (rr == 0) {
                    double sacc = 0.0;
                    for (int qq = 0; qq < rows; ++qq) sacc += buf[qq * cpb + cl];
                    cp[((int64_t)blockIdx.y * m + k) * ncols + col] = sacc;
                }
                __syncthreads();
            }
        }
    }
}

// p = M^-1 r + beta p ; q = 0.  FP32, no constraint rows, column count a
// multiple of 4 per block: each thread handles four adjacent columns of a row
// with 16-byte loads and stores, four times the bytes in flight per instruction
// of the one-column form (this pass is bound by memory latency).  Thread
// (c4, rr) of a block covers columns blockIdx.x * cpb + 4 c4 .. + 3.  The same
// treatment of the x/r update pass was slower: its four per-column partial sums
// raise the register count and cut the occupancy below what hides the latency.
template <int NC>
__global__ void __launch_bounds__(256) k_pupdate_v4(RowView<float> rv, const float* __restrict__ r,
                                                    float* __restrict__ p, float* __restrict__ q, ColState cs,
                                                    int ncols, int cpb, int first) {
    const int t4 = cpb / 4;
    const int rows = blockDim.x / t4;
    const int c4 = threadIdx.x % t4, rr = threadIdx.x / t4;
    if (rr >= rows) return;
    const int col0 = blockIdx.x * cpb + 4 * c4;
    float beta[4], s0[4], s1[4];
    const float* d0[4];
    const float* d1[4];
    bool act[4];
    bool touch = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int col = col0 + k;
        act[k] = cs.active[col] != 0;
        touch |= act[k] || first;
        beta[k] = first ? 0.f : (float)cs.beta[col];
        const int f = (rv.nfield == 2 && (col % 6) >= 3) ? 1 : 0;
        d0[k] = rv.diag + (int64_t)(2 * f) * rv.n_rows;
        d1[k] = d0[k] + rv.n_rows;
        s0[k] = rv.scale[2 * col];
        s1[k] = rv.scale[2 * col + 1];
    }
    // converged columns are left alone, except on the first pass, which clears
    // p and q of columns with b = 0
    const int64_t i_end = touch ? rv.n_rows : 0;
    const int64_t stride = (int64_t)gridDim.y * rows;
    for (int64_t i = (int64_t)blockIdx.y * rows + rr; i < i_end; i += stride) {
        const int64_t idx = i * ncols + col0;
        const float4 r4 = *reinterpret_cast<const float4*>(r + idx);
        const float4 p4 = first ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(p + idx);
        const float rk[4] = {r4.x, r4.y, r4.z, r4.w}, pk[4] = {p4.x, p4.y, p4.z, p4.w};
        const bool masked = rv.mask && rv.mask[i / NC];
        float out[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float inv = masked ? 0.f : jacobi_inv<float>(s0[k], __ldg(d0[k] + i), s1[k], __ldg(d1[k] + i));
            const float z = inv * rk[k];
            out[k] = act[k] ? (first ? z : fmaf(beta[k], pk[k], z)) : (first ? 0.f : pk[k]);
        }
        *reinterpret_cast<float4*>(p + idx) = make_float4(out[0], out[1], out[2], out[3]);
        *reinterpret_cast<float4*>(q + idx) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <typename T>
void launch_update(const RowView<T>& rv, T* x, T* r, const T* p, const T* q, ColState cs,
                   double* rz_partial, bool apply_update, const Launch& L, double* c_partial) {
    dim3 grid(L.ncols / L.cpb, L.nby), block(L.cpb * L.rows_per_block);
    const int ap = apply_update ? 1 : 0;
#define RVE_UPD_CASE(NCC, HC)                                                                           \
    if (rv.nc == NCC && (rv.m > 0) == HC) {                                                             \
        k_update<T, NCC, HC><<<grid, block, 0, L.stream>>>(rv, x, r, p, q, cs, rz_partial, c_partial,   \
                                                           L.ncols, L.cpb, ap);                        \
        return;                                                                                         \
    }
    RVE_UPD_CASE(3, false) RVE_UPD_CASE(3, true) RVE_UPD_CASE(1, false) RVE_UPD_CASE(1, true)
#undef RVE_UPD_CASE
}
template void launch_update<float>(const RowView<float>&, float*, float*, const float*, const float*,
                                   ColState, double*, bool, const Launch&, double*);
template void launch_update<double>(const RowView<double>&, double*, double*, const double*,
                                    const double*, ColState, double*, bool, const Launch&, double*);

// Fused iteration (no constraint rows): every thread forms its column's step
// alpha = rz / pq from the operator's accumulated energy itself (the separate
// alpha kernel of the general path is dropped), then x += alpha p, r -= alpha q
// and (r, M^-1 r) into rz_acc.  Block (x, 0), row 0 records alpha and the
// iteration, and deactivates a column whose pq is not positive or alpha not
// finite; every other block reaches the same alpha = 0 for it on its own.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_update_fused(RowView<T> rv, T* __restrict__ x, T* __restrict__ r,
                                                      const T* __restrict__ p, const T* __restrict__ q,
                                                      ColState cs, int ncols, int cpb) {
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, rr = threadIdx.x / cpb;
    const int col = blockIdx.x * cpb + cl;
    // the block's first row of threads forms alpha for its columns (one FP64
    // division per column and block: FP64 runs at a small fraction of the FP32 rate)
    __shared__ double s_alpha[256];
    __shared__ int s_state[256];
    if (rr == 0) {
        const bool act = cs.active[col] != 0 && !(cs.flags[0] & 4);
        double a = 0.0;
        int st = act ? 1 : 0;
        if (act) {
            double pq = 0.0;
#pragma unroll
            for (int k = 0; k < ACC_SLOTS; ++k) pq += cs.pq_acc[(size_t)k * ncols + col];
            a = cs.rz[col] / pq;
            if (!(pq > 0.0) || !isfinite(a)) {
                a = 0.0;
                st = 2;
            }
        }
        s_alpha[cl] = a;
        s_state[cl] = st;
    }
    __syncthreads();
    const double a64 = s_alpha[cl];
    const bool was_active = s_state[cl] != 0, bad = s_state[cl] == 2;
    if (blockIdx.y == 0 && rr == 0) {
        if (was_active && !bad) {
            cs.alpha[col] = a64;
            cs.iters[col] += 1;
        } else {
            cs.alpha[col] = 0.0;
            if (bad) atomicOr(cs.flags, 1);
            if (cs.active[col]) cs.active[col] = 0;
        }
    }
    const T a = (T)a64;
    const ColJacobi<T, NC> jac(rv, col);
    PartialSum<T> acc;
    const int64_t i_end = (was_active && !bad) ? rv.n_rows : 0;
    const int64_t stride = (int64_t)gridDim.y * rows;
    for (int64_t i = (int64_t)blockIdx.y * rows + rr; i < i_end; i += stride) {
        const int64_t idx = i * ncols + col;
        const T pv = p[idx], qv = q[idx], xv = x[idx];
        T rv_ = r[idx];
        x[idx] = fma(a, pv, xv);
        rv_ = fma(-a, qv, rv_);
        r[idx] = rv_;
        const T w = jac.inv(i) * rv_;
        acc.add(rv_ * w);
    }
    double accs[1] = {acc.value()};
    block_column_reduce<1>(accs, nullptr, ncols, cpb, col, cs.rz_acc + (size_t)(blockIdx.y % ACC_SLOTS) * ncols);
}

template <typename T>
void launch_update_fused(const RowView<T>& rv, T* x, T* r, const T* p, const T* q, ColState cs, const Launch& L) {
    dim3 grid(L.ncols / L.cpb, L.nby), block(L.cpb * L.rows_per_block);
    if (rv.nc == 3)
        k_update_fused<T, 3><<<grid, block, 0, L.stream>>>(rv, x, r, p, q, cs, L.ncols, L.cpb);
    else
        k_update_fused<T, 1><<<grid, block, 0, L.stream>>>(rv, x, r, p, q, cs, L.ncols, L.cpb);
}
template void launch_update_fused<float>(const RowView<float>&, float*, float*, const float*, const float*, ColState,
                                         const Launch&);
template void launch_update_fused<double>(const RowView<double>&, double*, double*, const double*, const double*,
                                          ColState, const Launch&);

// partial C M^-1 r over the constraint support (m <= 12 rows)
template <typename T>
__global__ void __launch_bounds__(256) k_constraint_dot(RowView<T> rv, const T* __restrict__ r,
                                                        double* __restrict__ cp, int ncols, int cpb) {
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, rr = threadIdx.x / cpb;
    const int col = blockIdx.x * cpb + cl;
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0;
    const int m = rv.m;
    for (int64_t s = (int64_t)blockIdx.y * rows + rr; s < rv.n_sup; s += (int64_t)gridDim.y * rows) {
        const int64_t row = rv.sup_row[s];
        const double w = (double)(inv_diag(rv, row, col, ncols) * r[row * ncols + col]);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            if (k < m) acc[k] += rv.sup_coef[s * m + k] * w;
    }
    __shared__ double buf[256];
    for (int k = 0; k < m; ++k) {
        buf[threadIdx.x] = acc[k];
        __syncthreads();
        if (rr == 0) {
            double sacc = 0.0;
            for (int q = 0; q < rows; ++q) sacc += buf[q * cpb + cl];
            cp[((int64_t)blockIdx.y * m + k) * ncols + col] = sacc;
        }
        __syncthreads();
    }
}

template <typename T>
void launch_constraint_dot(const RowView<T>& rv, const T* r, double* c_partial, const Launch& L) {
    if (rv.m == 0) return;
    dim3 grid(L.ncols / L.cpb, L.nby), block(L.cpb * L.rows_per_block);
    k_constraint_dot<T><<<grid, block, 0, L.stream>>>(rv, r, c_partial, L.ncols, L.cpb);
}
template void launch_constraint_dot<float>(const RowView<float>&, const float*, double*, const Launch&);
template void launch_constraint_dot<double>(const RowView<double>&, const double*, double*,
                                            const Launch&);

// mu = S^-1 w, rz = (r, M^-1 r) - w . mu, beta, convergence.
// first: 0 = iteration, 1 = initial residual, 2 = multipliers only (no state change).
// One block per column: the partial sums are reduced in parallel, then thread 0
// solves the m x m Schur system for mu and updates rz, beta and convergence.
__global__ void __launch_bounds__(256) k_finalize_beta(int m, const double* __restrict__ rzp,
                                                       const double* __restrict__ cp, int nby,
                                                       int ncols, ColState cs, int first) {
    const int col = blockIdx.x;
    if (first == 0 && !cs.active[col]) return;
    double v = 0.0;
    if (first != 2)
        for (int b = threadIdx.x; b < nby; b += blockDim.x) v += rzp[(int64_t)b * ncols + col];
    double rz = block_sum(v);
    __shared__ double w[12];
    for (int k = 0; k < m; ++k) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nby; b += blockDim.x) t += cp[((int64_t)b * m + k) * ncols + col];
        t = block_sum(t);
        if (threadIdx.x == 0) w[k] = t;
    }
    if (threadIdx.x != 0) return;
    double mu[12];
    if (m > 0) {
        const double* Lc = cs.schur + (int64_t)col * m * m;
        for (int i2 = 0; i2 < m; ++i2) {   // forward
            double t = w[i2];
            for (int j2 = 0; j2 < i2; ++j2) t -= Lc[i2 * m + j2] * mu[j2];
            mu[i2] = t / Lc[i2 * m + i2];
        }
        for (int i2 = m - 1; i2 >= 0; --i2) {   // backward
            double t = mu[i2];
            for (int j2 = i2 + 1; j2 < m; ++j2) t -= Lc[j2 * m + i2] * mu[j2];
            mu[i2] = t / Lc[i2 * m + i2];
        }
        for (int k = 0; k < m; ++k) {
            rz -= w[k] * mu[k];
            cs.mu[(int64_t)k * ncols + col] = mu[k];
        }
    }
    if (first == 2) return;
    if (!isfinite(rz)) {
        atomicOr(cs.flags, 1);
        cs.active[col] = 0;
        return;
    }
    if (first) {
        cs.rz0[col] = rz;
        cs.rz[col] = rz;
        cs.beta[col] = 0.0;
        cs.iters[col] = 0;
        cs.active[col] = rz > 0.0 ? 1 : 0;
        return;
    }
    cs.beta[col] = rz / cs.rz[col];
    cs.rz[col] = rz;
    const double tol = *cs.tol;
    if (rz <= tol * tol * cs.rz0[col]) cs.active[col] = 0;
}

void launch_finalize_beta(int m, const double* rz_partial, const double* c_partial, ColState cs,
                          bool first, const Launch& L) {
    k_finalize_beta<<<L.ncols, 256, 0, L.stream>>>(m, rz_partial, c_partial, L.nby, L.ncols, cs,
                                                   first ? 1 : 0);
}

// Per-column tolerances: column c stops once rz <= tolc[c]^2 rz0, which the
// convergence tests (rz <= tol^2 rz0 with the scalar tol) see through rz0 scaled
// by (tolc[c] / tol)^2; a column with tolc[c] >= 1 has converged already and starts
// inactive.  Runs after the initial residual's finalisation.
__global__ void k_column_tol(int ncols, const double* __restrict__ tolc, ColState cs) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const double t = tolc[c] / *cs.tol;
    cs.rz0[c] *= t * t;
    if (tolc[c] >= 1.0) cs.active[c] = 0;
}

void launch_column_tol(int ncols, const double* tolc, ColState cs, cudaStream_t s) {
    k_column_tol<<<(ncols + 127) / 128, 128, 0, s>>>(ncols, tolc, cs);
}

void launch_constraint_multipliers(int m, const double* c_partial, ColState cs, const Launch& L) {
    if (m == 0) return;
    k_finalize_beta<<<L.ncols, 256, 0, L.stream>>>(m, c_partial, c_partial, L.nby, L.ncols, cs, 2);
}

// Residual reset r <- r - C^T mu on the constraint support (the part of the
// residual that the constraint forces carry), and partial (r, M^-1 r) of the
// projected residual, computed without cancellation.
// r <- r - C^T mu on the constraint support (FP64), and per column the partial
// (r, M^-1 r) of the result.  The norm only steers the stopping test, so it is
// formed from the FP32 preconditioner and FP32-rounded r with compensated FP32
// sums (relative accuracy ~1e-7), which keeps this FP64-vector pass off the
// FP64 pipe apart from one conversion per entry.
template <int NC, bool HAS_C>
__global__ void __launch_bounds__(256) k_project_residual(RowView<double> rv, RowView<float> rv32,
                                                          double* __restrict__ r, ColState cs,
                                                          double* __restrict__ rzp, int ncols, int cpb) {
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, rr = threadIdx.x / cpb;
    const int col = blockIdx.x * cpb + cl;
    const int m = HAS_C ? rv.m : 0;
    const ColJacobi<float, NC> jac(rv32, col);
    PartialSum<float> acc;
    for (int64_t i = (int64_t)blockIdx.y * rows + rr; i < rv.n_rows; i += (int64_t)gridDim.y * rows) {
        const int64_t idx = i * ncols + col;
        double v = r[idx];
        if constexpr (HAS_C) {
            const int32_t sidx = rv.sup_of_row[i];
            if (sidx >= 0) {
                double corr = 0.0;
                for (int k = 0; k < m; ++k)
                    corr += rv.sup_coef[(int64_t)sidx * m + k] * cs.mu[(int64_t)k * ncols + col];
                v -= corr;
                r[idx] = v;
            }
        }
        const float vf = (float)v;
        acc.add(vf * (jac.inv(i) * vf));
    }
    double accs[1] = {acc.value()};
    block_column_reduce<1>(accs, rzp, ncols, cpb, col);
}

void launch_project_residual(const RowView<double>& rv, const RowView<float>& rv32, double* r, ColState cs,
                             double* rz_partial, const Launch& L) {
    dim3 grid(L.ncols / L.cpb, L.nby), block(L.cpb * L.rows_per_block);
#define RVE_PR_CASE(NCC, HC)                                                                          \
    if (rv.nc == NCC && (rv.m > 0) == HC) {                                                           \
        k_project_residual<NCC, HC><<<grid, block, 0, L.stream>>>(rv, rv32, r, cs, rz_partial, L.ncols, \
                                                                  L.cpb);                             \
        return;                                                                                       \
    }
    RVE_PR_CASE(3, false) RVE_PR_CASE(3, true) RVE_PR_CASE(1, false) RVE_PR_CASE(1, true)
#undef RVE_PR_CASE
}

// p = M^-1 (r - C^T mu) + beta p ; q = 0
template <typename T, int NC, bool HAS_C>
__global__ void __launch_bounds__(256) k_pupdate(RowView<T> rv, T* __restrict__ r,
                                                 T* __restrict__ p, T* __restrict__ q, ColState cs,
                                                 int ncols, int cpb, int first) {
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, rr = threadIdx.x / cpb;
    const int col = blockIdx.x * cpb + cl;
    const bool act = cs.active[col] != 0;
    const T beta = first ? T(0) : (T)cs.beta[col];
    const ColJacobi<T, NC> jac(rv, col);
    const int m = HAS_C ? rv.m : 0;
    // converged columns are left alone (the operator and update skip them too),
    // except on the first pass, which clears p and q of columns with b = 0
    const int64_t i_end = (!act && !first) ? 0 : rv.n_rows;
    const int64_t stride = (int64_t)gridDim.y * rows;
    for (int64_t i = (int64_t)blockIdx.y * rows + rr; i < i_end; i += stride) {
        const int64_t idx = i * ncols + col;
        q[idx] = T(0);
        if (!act) {
            p[idx] = T(0);
            continue;
        }
        T rr_ = r[idx];
        const T pold = first ? T(0) : p[idx];
        if constexpr (HAS_C) {
            const int32_t sidx = rv.sup_of_row[i];
            if (sidx >= 0) {
                T corr = T(0);
                for (int k = 0; k < m; ++k)
                    corr = fma((T)rv.sup_coef[(int64_t)sidx * m + k], (T)cs.mu[(int64_t)k * ncols + col], corr);
                rr_ -= corr;
                r[idx] = rr_;   // residual reset: keeps r in the projected space
            }
        }
        const T z = jac.inv(i) * rr_;
        p[idx] = first ? z : fma(beta, pold, z);
    }
}

template <typename T>
void launch_pupdate(const RowView<T>& rv, T* r, T* p, T* q, ColState cs, bool first,
                    const Launch& L) {
    dim3 grid(L.ncols / L.cpb, L.nby), block(L.cpb * L.rows_per_block);
    const int fi = first ? 1 : 0;
    if constexpr (sizeof(T) == 4) {
        if (rv.m == 0 && L.cpb % 4 == 0) {
            const int t4 = L.cpb / 4;
            dim3 b4(t4 * (256 / t4));
            if (rv.nc == 3)
                k_pupdate_v4<3><<<grid, b4, 0, L.stream>>>(rv, r, p, q, cs, L.ncols, L.cpb, fi);
            else
                k_pupdate_v4<1><<<grid, b4, 0, L.stream>>>(rv, r, p, q, cs, L.ncols, L.cpb, fi);
            return;
        }
    }
#define RVE_PUP_CASE(NCC, HC)                                                                           \
    if (rv.nc == NCC && (rv.m > 0) == HC) {                                                             \
        k_pupdate<T, NCC, HC><<<grid, block, 0, L.stream>>>(rv, r, p, q, cs, L.ncols, L.cpb, fi);       \
        return;                                                                                         \
    }
    RVE_PUP_CASE(3, false) RVE_PUP_CASE(3, true) RVE_PUP_CASE(1, false) RVE_PUP_CASE(1, true)
#undef RVE_PUP_CASE
}
template void launch_pupdate<float>(const RowView<float>&, float*, float*, float*, ColState, bool,
                                    const Launch&);
template void launch_pupdate<double>(const RowView<double>&, double*, double*, double*, ColState,
                                     bool, const Launch&);

// S = C M^-1 C^T per column (one block per (column, row k)), then Cholesky.
template <typename T>
__global__ void k_schur_rows(RowView<T> rv, double* __restrict__ S, int ncols) {
    const int col = blockIdx.x, k = blockIdx.y, m = rv.m;
    double acc[12];
    for (int l = 0; l < 12; ++l) acc[l] = 0.0;
    for (int64_t s = threadIdx.x; s < rv.n_sup; s += blockDim.x) {
        const int64_t row = rv.sup_row[s];
        const double w = (double)inv_diag(rv, row, col, ncols) * rv.sup_coef[s * m + k];
        for (int l = 0; l < m; ++l) acc[l] += w * rv.sup_coef[s * m + l];
    }
    __shared__ double buf[256];
    for (int l = 0; l < m; ++l) {
        buf[threadIdx.x] = acc[l];
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) buf[threadIdx.x] += buf[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) S[((int64_t)col * m + k) * m + l] = buf[0];
        __syncthreads();
    }
}

__global__ void k_cholesky(int m, int ncols, double* __restrict__ S, int32_t* flags) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    double* A = S + (int64_t)col * m * m;
    for (int j = 0; j < m; ++j) {
        double s = A[j * m + j];
        for (int k = 0; k < j; ++k) s -= A[j * m + k] * A[j * m + k];
        if (!(s > 0)) {
            atomicOr(flags, 2);
            s = 1e-300;
        }
        const double d = sqrt(s);
        A[j * m + j] = d;
        for (int i = j + 1; i < m; ++i) {
            double t = A[i * m + j];
            for (int k = 0; k < j; ++k) t -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = t / d;
        }
        for (int i = 0; i < j; ++i) A[i * m + j] = 0.0;
    }
}

template <typename T>
void launch_schur(const RowView<T>& rv, ColState cs, const Launch& L) {
    if (rv.m == 0) return;
    dim3 grid(L.ncols, rv.m);
    k_schur_rows<T><<<grid, 256, 0, L.stream>>>(rv, cs.schur, L.ncols);
    k_cholesky<<<(L.ncols + 127) / 128, 128, 0, L.stream>>>(rv.m, L.ncols, cs.schur, cs.flags);
}
template void launch_schur<float>(const RowView<float>&, ColState, const Launch&);
template void launch_schur<double>(const RowView<double>&, ColState, const Launch&);

// ------------------------------------------------- homogenisation reductions
// Per column i of RVE b: sum_rows b_i u_j and u_i r_j, j over the RVE's six
// columns (FP64).  Used for the energy form
//   V C_ij = V <D>_ij - b_i . u_j - u_i . r_j      (r = b - K u).
__global__ void __launch_bounds__(256) k_gram(int64_t n_rows, const double* __restrict__ b,
                                              const double* __restrict__ u,
                                              const double* __restrict__ r,
                                              double* __restrict__ part, int ncols, int cpb) {
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, rr = threadIdx.x / cpb;
    const int col = blockIdx.x * cpb + cl;
    const int base = (col / 6) * 6;
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.y * rows + rr; i < n_rows; i += (int64_t)gridDim.y * rows) {
        const double bi = b[i * ncols + col], ui = u[i * ncols + col];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            acc[j] += bi * u[i * ncols + base + j];
            acc[6 + j] += ui * r[i * ncols + base + j];
        }
    }
    block_column_reduce<12>(acc, part, ncols, cpb, col);
}

void launch_gram(int64_t n_rows, const double* b, const double* u, const double* r,
                 double* partial, const Launch& L) {
    dim3 grid(L.ncols / L.cpb, L.nby), block(L.cpb * L.rows_per_block);
    k_gram<<<grid, block, 0, L.stream>>>(n_rows, b, u, r, partial, L.ncols, L.cpb);
}

// Volume integrals per column: int sigma(eps_bar + eps(u)) (Eq. macro_stress)
// and int sigma(eps_bar) (the Voigt term), 6 + 6 values (3 + 3 for scalars).
// Only the constant gradient mode enters an element mean (the higher modes
// integrate to zero).  T = float keeps per-thread compensated sums.
template <int P, int NC, typename T, typename TU>
__global__ void __launch_bounds__(256) k_mean_stress(ElemView<T> ev, const TU* __restrict__ u,
                                                     double* __restrict__ part, int ncols, int cpb) {
    constexpr int NE = Order<P>::NE;
    constexpr int NM = Order<P>::NM;
    const int rows = blockDim.x / cpb;
    const int cl = threadIdx.x % cpb, rr = threadIdx.x / cpb;
    const int col = blockIdx.x * cpb + cl;
    const int field = (col % 6) >= 3 ? 1 : 0;
    const int macro_id = NC == 3 ? (col % 6) : ((col % 6) % 3);
    PartialSum<T> acc[12];
    for (int64_t e = (int64_t)blockIdx.y * rows + rr; e < ev.nt; e += (int64_t)gridDim.y * rows) {
        const int32_t* ed = ev.edofs + e * NE;
        T G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) G[i] = __ldg(ev.geo + e * 10 + i);
        const T vol = __ldg(ev.geo + e * 10 + 9);
        const T sc = __ldg(ev.scale + col * 2 + __ldg(ev.phase + e));
        T V[3][NC];
        const int d0 = __ldg(ed);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int dk = __ldg(ed + k + 1);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                V[k][c] = (T)(u[((int64_t)dk * NC + c) * ncols + col] - u[((int64_t)d0 * NC + c) * ncols + col]);
        }
#pragma unroll
        for (int j = 4; j < NE; ++j) {
            const int dj = __ldg(ed + j);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T a = basis_a<P, T>((k * NM + 0) * NE + j);
                if (a != T(0))
#pragma unroll
                    for (int c = 0; c < NC; ++c) V[k][c] = fma(a, (T)u[((int64_t)dj * NC + c) * ncols + col], V[k][c]);
            }
        }
        T H[NC][3];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int l = 0; l < 3; ++l) H[c][l] = V[0][c] * G[l] + V[1][c] * G[3 + l] + V[2][c] * G[6 + l];
        const T sv = sc * vol;
        if constexpr (NC == 3) {
            T ev6[6] = {H[0][0], H[1][1], H[2][2], H[0][1] + H[1][0], H[1][2] + H[2][1], H[2][0] + H[0][2]};
            ev6[macro_id] += T(1);   // unit engineering macro strain of this column
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                T t = T(0);
#pragma unroll
                for (int j = 0; j < 6; ++j) t = fma(__ldg(ev.mat + e * 21 + ut6(i, j)), ev6[j], t);
                acc[i].add(sv * t);
                acc[6 + i].add(sv * __ldg(ev.mat + e * 21 + ut6(i, macro_id)));
            }
        } else {
            const T* Km = ev.mat + e * 12 + 6 * field;
            T g[3] = {H[0][0], H[0][1], H[0][2]};
            g[macro_id] += T(1);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                acc[l].add(sv * (__ldg(Km + s3(l, 0)) * g[0] + __ldg(Km + s3(l, 1)) * g[1] +
                                 __ldg(Km + s3(l, 2)) * g[2]));
                acc[6 + l].add(sv * __ldg(Km + s3(l, macro_id)));
            }
        }
    }
    double out[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = acc[k].value();
    block_column_reduce<12>(out, part, ncols, cpb, col);
}

template <typename T, typename TU>
void launch_mean_stress(int p, int nc, const ElemView<T>& ev, const TU* u, double* partial,
                        const Launch& L) {
    dim3 grid(L.ncols / L.cpb, L.nby), block(L.cpb * L.rows_per_block);
#define RVE_MS_CASE(PP, NCC)                                                                      \
    if (p == PP && nc == NCC) {                                                                   \
        k_mean_stress<PP, NCC, T, TU><<<grid, block, 0, L.stream>>>(ev, u, partial, L.ncols, L.cpb); \
        return;                                                                                   \
    }
    RVE_MS_CASE(1, 3) RVE_MS_CASE(2, 3) RVE_MS_CASE(3, 3)
    RVE_MS_CASE(1, 1) RVE_MS_CASE(2, 1) RVE_MS_CASE(3, 1)
#undef RVE_MS_CASE
}
template void launch_mean_stress<double, double>(int, int, const ElemView<double>&, const double*, double*,
                                                 const Launch&);
template void launch_mean_stress<float, double>(int, int, const ElemView<float>&, const double*, double*,
                                                const Launch&);
template void launch_mean_stress<float, float>(int, int, const ElemView<float>&, const float*, double*,
                                               const Launch&);

// ------------------------------------------- multiplier route (Eq. eq_homo_stress)
// Vertex reactions of the total field u = u_tilde + X (X the unit macro field of
// the column): every vertex function has a constant gradient, so its entry of
// K u on element e is |T| s grad(lam_a) . sigma_e with sigma_e the element-mean
// stress (flux); it is scattered to the ORIGINAL vertex id of local vertex a,
// i.e. onto the unfolded mesh, where the constraint rows of the BC live.
template <int P, int NC>
__global__ void __launch_bounds__(256) k_vertex_reactions(ElemView<double> ev, const int32_t* __restrict__ lverts,
                                                          const double* __restrict__ u, double* __restrict__ r,
                                                          int ncols) {
    constexpr int NE = Order<P>::NE;
    constexpr int NM = Order<P>::NM;
    const int64_t n = ev.nt * ncols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / ncols;
        const int col = (int)(i % ncols);
        const int field = (col % 6) >= 3 ? 1 : 0;
        const int macro_id = NC == 3 ? (col % 6) : ((col % 6) % 3);
        const int32_t* ed = ev.edofs + e * NE;
        double G[9];
        for (int q = 0; q < 9; ++q) G[q] = ev.geo[e * 10 + q];
        const double sv = ev.scale[col * 2 + ev.phase[e]] * ev.geo[e * 10 + 9];
        double V[3][NC];
        const int d0 = ed[0];
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < NC; ++c)
                V[k][c] = u[((int64_t)ed[k + 1] * NC + c) * ncols + col] - u[((int64_t)d0 * NC + c) * ncols + col];
        for (int j = 4; j < NE; ++j)
            for (int k = 0; k < 3; ++k) {
                const double a = basis_a<P, double>((k * NM + 0) * NE + j);
                if (a != 0.0)
                    for (int c = 0; c < NC; ++c) V[k][c] += a * u[((int64_t)ed[j] * NC + c) * ncols + col];
            }
        double H[NC][3];
        for (int c = 0; c < NC; ++c)
            for (int l = 0; l < 3; ++l) H[c][l] = V[0][c] * G[l] + V[1][c] * G[3 + l] + V[2][c] * G[6 + l];
        double S[NC][3];
        if constexpr (NC == 3) {
            double ev6[6] = {H[0][0], H[1][1], H[2][2], H[0][1] + H[1][0], H[1][2] + H[2][1], H[2][0] + H[0][2]};
            ev6[macro_id] += 1.0;
            double sg[6];
            for (int a = 0; a < 6; ++a) {
                double t = 0.0;
                for (int b = 0; b < 6; ++b) t += ev.mat[e * 21 + ut6(a, b)] * ev6[b];
                sg[a] = sv * t;
            }
            S[0][0] = sg[0]; S[0][1] = sg[3]; S[0][2] = sg[5];
            S[1][0] = sg[3]; S[1][1] = sg[1]; S[1][2] = sg[4];
            S[2][0] = sg[5]; S[2][1] = sg[4]; S[2][2] = sg[2];
        } else {
            const double* Km = ev.mat + e * 12 + 6 * field;
            double g[3] = {H[0][0], H[0][1], H[0][2]};
            g[macro_id] += 1.0;
            for (int l = 0; l < 3; ++l) S[0][l] = sv * (Km[s3(l, 0)] * g[0] + Km[s3(l, 1)] * g[1] + Km[s3(l, 2)] * g[2]);
        }
        for (int a = 0; a < 4; ++a) {
            double gl[3];
            for (int l = 0; l < 3; ++l) gl[l] = a == 0 ? -(G[l] + G[3 + l] + G[6 + l]) : G[3 * (a - 1) + l];
            const int64_t v = lverts[e * 4 + a];
            for (int c = 0; c < NC; ++c)
                atomicAdd(r + (v * NC + c) * ncols + col, gl[0] * S[c][0] + gl[1] * S[c][1] + gl[2] * S[c][2]);
        }
    }
}

void launch_vertex_reactions(int p, int nc, const ElemView<double>& ev, const int32_t* lverts, const double* u,
                             double* r, int ncols, cudaStream_t s) {
    const int64_t n = ev.nt * ncols;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16));
#define RVE_VR_CASE(PP, NCC)                                                                      \
    if (p == PP && nc == NCC) {                                                                   \
        k_vertex_reactions<PP, NCC><<<grid, 256, 0, s>>>(ev, lverts, u, r, ncols);                 \
        return;                                                                                   \
    }
    RVE_VR_CASE(1, 3) RVE_VR_CASE(2, 3) RVE_VR_CASE(3, 3)
    RVE_VR_CASE(1, 1) RVE_VR_CASE(2, 1) RVE_VR_CASE(3, 1)
#undef RVE_VR_CASE
}

// out[i][col] = sum_k sum_c w[k][i][c] r[vid[k]][c][col]: one block per (i, col)
__global__ void __launch_bounds__(256) k_weighted_vertex_sum(int n, int ni, int nc, const int32_t* __restrict__ vid,
                                                             const double* __restrict__ w,
                                                             const double* __restrict__ r, int ncols,
                                                             double* __restrict__ out) {
    const int i = blockIdx.x / ncols, col = blockIdx.x % ncols;
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        for (int c = 0; c < nc; ++c)
            v += w[((int64_t)k * ni + i) * nc + c] * r[((int64_t)vid[k] * nc + c) * ncols + col];
    v = block_sum(v);
    if (threadIdx.x == 0) out[i * ncols + col] = v;
}

void launch_weighted_vertex_sum(int n, int ni, int nc, const int32_t* vid, const double* w, const double* r,
                                int ncols, double* out, cudaStream_t s) {
    k_weighted_vertex_sum<<<ni * ncols, 256, 0, s>>>(n, ni, nc, vid, w, r, ncols, out);
}

// out[k][col] = sum_i coef[i][k] y[row[i]][col] (constraint rows applied to y): one block per (k, col)
__global__ void __launch_bounds__(256) k_rows_dot(int64_t n_sup, int m, const int64_t* __restrict__ row,
                                                  const double* __restrict__ coef, const double* __restrict__ y,
                                                  int ncols, double* __restrict__ out) {
    const int k = blockIdx.x / ncols, col = blockIdx.x % ncols;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < n_sup; i += blockDim.x) v += coef[i * m + k] * y[row[i] * ncols + col];
    v = block_sum(v);
    if (threadIdx.x == 0) out[k * ncols + col] = v;
}

void launch_rows_dot(int64_t n_sup, int m, const int64_t* row, const double* coef, const double* y, int ncols,
                     double* out, cudaStream_t s) {
    k_rows_dot<<<m * ncols, 256, 0, s>>>(n_sup, m, row, coef, y, ncols, out);
}

// out[w] = sum_b part[b][w]: one block per output value (up to 128 outputs per
// block row are handled by grid-striding over w).
__global__ void __launch_bounds__(256) k_reduce_partials(int nby, int width, const double* __restrict__ part,
                                                         double* __restrict__ out) {
    for (int w = blockIdx.x; w < width; w += gridDim.x) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nby; b += blockDim.x) v += part[(int64_t)b * width + w];
        v = block_sum(v);
        if (threadIdx.x == 0) out[w] = v;
    }
}

void launch_reduce_partials(int nby, int width, const double* partial, double* out, cudaStream_t s) {
    k_reduce_partials<<<width < 4096 ? width : 4096, 256, 0, s>>>(nby, width, partial, out);
}

// ------------------------------------------------------ batch gather/scatter
// states of the batch: out[b] = in[idx[b]] for T, c, t
__global__ void k_gather_states(int B, const int64_t* __restrict__ idx, const double* __restrict__ T,
                                const double* __restrict__ c, const double* __restrict__ t,
                                double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int64_t g = idx[b];
    out[b] = T[g];
    out[B + b] = c[g];
    out[2 * B + b] = t[g];
}

void launch_gather_states(int B, const int64_t* idx, const double* T, const double* c, const double* t,
                          double* out, cudaStream_t s) {
    k_gather_states<<<(B + 127) / 128, 128, 0, s>>>(B, idx, T, c, t, out);
}

// results of the batch [B][36 + 9 + 9 + 1 status] -> per-point outputs
__global__ void k_scatter_results(int B, const int64_t* __restrict__ idx, const double* __restrict__ res,
                                  double* __restrict__ C, double* __restrict__ K, double* __restrict__ D,
                                  int32_t* __restrict__ status) {
    const int b = blockIdx.x;
    const int64_t g = idx[b];
    const double* r = res + (int64_t)b * 55;
    for (int i = threadIdx.x; i < 54; i += blockDim.x) {
        if (i < 36) C[g * 36 + i] = r[i];
        else if (i < 45) K[g * 9 + i - 36] = r[i];
        else D[g * 9 + i - 45] = r[i];
    }
    if (threadIdx.x == 0) status[g] = (int32_t)r[54];
}

void launch_scatter_results(int B, const int64_t* idx, const double* res, double* C, double* K, double* D,
                            int32_t* status, cudaStream_t s) {
    k_scatter_results<<<B, 64, 0, s>>>(B, idx, res, C, K, D, status);
}

// x[:, col] = sum_k coef[col][k] src[:, map[col][k]] over WARM_SOURCES previous
// solutions (warm starts: a polynomial in the degradation factor through them, or
// their energy-optimal combination), read as TI and stored as TO
template <typename TI, typename TO>
__global__ void k_combine_columns(int64_t n_rows, int ncols, int src_cols, const int32_t* __restrict__ map,
                                  const double* __restrict__ coef, const TI* __restrict__ src,
                                  TO* __restrict__ x, int accumulate) {
    const int64_t n = n_rows * ncols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / ncols;
        const int col = (int)(i % ncols);
        double v = 0.0;
#pragma unroll
        for (int k = 0; k < WARM_SOURCES; ++k) {
            const double c = coef[col * WARM_SOURCES + k];
            if (c != 0.0) v = fma(c, (double)src[row * src_cols + map[col * WARM_SOURCES + k]], v);
        }
        x[i] = accumulate ? (TO)((double)x[i] + v) : (TO)v;
    }
}

template <typename TI, typename TO>
void launch_combine_columns(int64_t n_rows, int ncols, int src_cols, const int32_t* map, const double* coef,
                            const TI* src, TO* x, cudaStream_t s, bool accumulate) {
    int64_t b = (n_rows * ncols + 255) / 256;
    if (b > sm_count() * 16) b = sm_count() * 16;
    if (b < 1) b = 1;
    k_combine_columns<TI, TO><<<(unsigned)b, 256, 0, s>>>(n_rows, ncols, src_cols, map, coef, src, x,
                                                          accumulate ? 1 : 0);
}
template void launch_combine_columns<double, double>(int64_t, int, int, const int32_t*, const double*,
                                                     const double*, double*, cudaStream_t, bool);
template void launch_combine_columns<double, float>(int64_t, int, int, const int32_t*, const double*,
                                                    const double*, float*, cudaStream_t, bool);

// Inner products of the energy-optimal warm start, per load case lc and source p
// (ns sources, the columns 6 src[p] + lc of the previous batch): x_p . k_t and
// x_p . k'_t (t < ns; k_t, k'_t minus the degraded and the other phases' operator on
// source t, FP64, compact [n_rows][12 ns] with the k' columns from 6 ns on) and
// x_p . y_ph (the unit-modulus macro load of phase ph, [2][n_rows][6]).
// Block (lc * ns + p, split) sums its rows; out[split][lc][p][2 ns + 2].
__global__ void __launch_bounds__(256) k_warm_gram(int64_t n_rows, int ns, const int32_t* __restrict__ src,
                                                   int src_cols, const double* __restrict__ X,
                                                   const double* __restrict__ Kc, const double* __restrict__ Y,
                                                   double* __restrict__ out) {
    const int lc = blockIdx.x / ns, p = blockIdx.x % ns;
    const int nout = 2 * ns + 2, kst = 12 * ns;
    double am[WARM_GALERKIN], ay[WARM_GALERKIN], ay0 = 0.0, ay1 = 0.0;
#pragma unroll
    for (int t = 0; t < WARM_GALERKIN; ++t) am[t] = ay[t] = 0.0;
    const int cp = 6 * src[p] + lc;
    for (int64_t row = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; row < n_rows;
         row += (int64_t)gridDim.y * blockDim.x) {
        const double xp = X[row * src_cols + cp];
#pragma unroll
        for (int t = 0; t < WARM_GALERKIN; ++t)
            if (t < ns) {
                am[t] = fma(xp, Kc[row * kst + 6 * t + lc], am[t]);
                ay[t] = fma(xp, Kc[row * kst + 6 * ns + 6 * t + lc], ay[t]);
            }
        ay0 = fma(xp, Y[row * 6 + lc], ay0);
        ay1 = fma(xp, Y[n_rows * 6 + row * 6 + lc], ay1);
    }
    double* o = out + ((int64_t)blockIdx.y * 6 * ns + blockIdx.x) * nout;
#pragma unroll
    for (int t = 0; t < WARM_GALERKIN; ++t)
        if (t < ns) {
            const double a = block_sum(am[t]);
            const double b = block_sum(ay[t]);
            if (threadIdx.x == 0) {
                o[t] = a;
                o[ns + t] = b;
            }
        }
    const double y0 = block_sum(ay0);
    const double y1 = block_sum(ay1);
    if (threadIdx.x == 0) {
        o[2 * ns] = y0;
        o[2 * ns + 1] = y1;
    }
}

void launch_warm_gram(int64_t n_rows, int ns, const int32_t* src, int src_cols, const double* X, const double* Kc,
                      const double* Y, double* out, int splits, cudaStream_t s) {
    dim3 grid(6 * ns, splits);
    k_warm_gram<<<grid, 256, 0, s>>>(n_rows, ns, src, src_cols, X, Kc, Y, out);
}

// b[row][6r + c] = -(s0 y0[row][c] + s1 y1[row][c]) with the column's phase scales
__global__ void k_rhs_combine(int64_t n_rows, int nrve, const double* __restrict__ y,
                              const double* __restrict__ scale, double* __restrict__ b, int accumulate) {
    const int ncols = 6 * nrve;
    const int64_t n = n_rows * ncols;
    const double* y1 = y + n_rows * 6;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / ncols;
        const int col = (int)(i % ncols);
        const int c = col % 6;
        const double v = -(scale[2 * col] * y[row * 6 + c] + scale[2 * col + 1] * y1[row * 6 + c]);
        b[i] = accumulate ? b[i] + v : v;
    }
}

void launch_rhs_combine(int64_t n_rows, int nrve, const double* y, const double* scale, double* b,
                        cudaStream_t s, bool accumulate) {
    int64_t blocks = (n_rows * 6 * nrve + 255) / 256;
    if (blocks > sm_count() * 16) blocks = sm_count() * 16;
    if (blocks < 1) blocks = 1;
    k_rhs_combine<<<(unsigned)blocks, 256, 0, s>>>(n_rows, nrve, y, scale, b, accumulate ? 1 : 0);
}

// ---------------------------------------------------------- elementwise
__global__ void k_cast_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
__global__ void k_axpy_f2d(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] += (double)a[i];
}
__global__ void k_neg(int64_t n, double* __restrict__ a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = -a[i];
}
static unsigned ew_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (unsigned)(b > sm_count() * 16 ? sm_count() * 16 : (b < 1 ? 1 : b));
}
void launch_cast_d2f(int64_t n, const double* a, float* b, cudaStream_t s) {
    k_cast_d2f<<<ew_blocks(n), 256, 0, s>>>(n, a, b);
}
void launch_axpy_f2d(int64_t n, const float* a, double* b, cudaStream_t s) {
    k_axpy_f2d<<<ew_blocks(n), 256, 0, s>>>(n, a, b);
}
void launch_neg(int64_t n, double* a, cudaStream_t s) { k_neg<<<ew_blocks(n), 256, 0, s>>>(n, a); }

}  // namespace rve
