// Tensor-core operator of the mixed-precision inner solve (sm_103a, tcgen05).
//
// The operator of Eq. RVE_Eq_var_final, y += sum_e s(col, phase_e) K_e x_e, as a
// dense product per element on the 5th-generation tensor cores.  Degradation
// scales the matrix modulus only (Sec. 5), so within a batch every column sees
// the same reference element matrix K_e up to the scalar s(col, phase_e): one
// element is one MMA problem
//
//     D [128 columns x NP] = X_e^T [128 columns x NP] * K_e [NP x NP]
//
// with the element's NP = 32 (p = 2) or 64 (p = 3) local DOFs (3 NE padded with
// zeros).  Thread t of the 128-thread CTA owns column slot t: it gathers its
// column's element vector into TMEM lane t (the A operand sits in tensor
// memory), reads the product back from the accumulator lane t and scatters it
// with coalesced reductions (lanes are consecutive columns).  K_e is formed once
// per mesh and materials in FP64 and stored packed (upper triangle, FP32); each
// CTA expands it into a 128B-swizzled K-major SMEM tile (the B operand).
//
// FP32 accuracy on TF32 units: both operands are split into a TF32 high part
// and a TF32 low part (a = a_h + a_l, |a_l| <= 2^-11 |a|) and three MMAs
// accumulate a_h b_h + a_h b_l + a_l b_h in FP32 (the dropped a_l b_l term and
// the rounding of the low parts are about 2^-21 relative).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "kernels.h"
#include "rve_internal.h"

namespace rve {
namespace {

template <int P>
struct TcShape {
    static constexpr int NE = P == 1 ? 4 : (P == 2 ? 10 : 20);
    static constexpr int N = 3 * NE;                 // element DOFs (mechanics)
    static constexpr int NP = (N + 15) / 16 * 16;    // MMA N = K (multiple of 16)
    static constexpr int KS = NP / 8;                // K-steps of 8 TF32 values
    static constexpr int PACK = N * (N + 1) / 2;     // packed upper triangle
    static constexpr int PACKP = (PACK + 3) / 4 * 4;
    static constexpr int TILE = NP * NP * 4;         // bytes of one B tile
    static constexpr int ATOM = NP * 128;            // bytes of one 32-wide K atom
    static constexpr uint32_t TCOLS = 3 * NP <= 128 ? 128 : 256;   // A_hi, A_lo, D
    // operand prefetch ring depth and resident CTAs per SM (shared memory bound)
    static constexpr int STAGES = 3;
    static constexpr int CTAS_PER_SM = P == 2 ? 3 : 1;
    static constexpr int KE_BYTES = PACKP * 4;            // one packed element matrix
    static constexpr int XS_BYTES = N * 128 * 4;          // one element's values, 128 column slots
    // shared-memory layout (byte offsets from a 1024-aligned base)
    static constexpr int OFF_BHI = 0;
    static constexpr int OFF_BLO = TILE;
    static constexpr int OFF_KE = 2 * TILE;
    static constexpr int OFF_XS = OFF_KE + STAGES * KE_BYTES;
    static constexpr int OFF_OFFS = OFF_XS + STAGES * XS_BYTES;
    static constexpr int OFF_ED = OFF_OFFS + (PACK * 4 + 15) / 16 * 16;
    static constexpr int OFF_PH = OFF_ED + (STAGES * NE * 4 + 15) / 16 * 16;
    static constexpr int OFF_BAR = OFF_PH + 16;
    static constexpr int BYTES = OFF_BAR + 32;
};

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return u;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on a phase of an mbarrier: false after `ns` nanoseconds of the
// global timer, or after `max_polls` polls should the timer not advance (each
// poll may suspend the thread for a short system-dependent time).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity, uint64_t ns, int max_polls) {
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < max_polls; ++i) {
        if (mbar_try_wait(a, parity)) return true;
        if (global_ns() - t0 > ns) return false;
    }
    return false;
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
// D (TMEM) (+)= A (TMEM) * B (SMEM descriptor), kind::tf32, FP32 accumulate.
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout (rows of 128 bytes, 8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // swizzle: 128 bytes
    return d;
}
// Byte offset of element (n, k) of a K-major tile of NP rows stored as 32-wide
// K atoms with the 128-byte swizzle (16-byte chunk index XOR row mod 8).
template <int NP>
__device__ __forceinline__ uint32_t sw128_offset(int n, int k) {
    const int atom = k >> 5, kk = k & 31;
    const uint32_t chunk = (uint32_t)((kk >> 2) ^ (n & 7));
    return (uint32_t)(atom * NP * 128 + n * 128) + (chunk << 4) + (uint32_t)((kk & 3) << 2);
}

__host__ __device__ constexpr int ut6i(int i, int j) {
    return i <= j ? (i * 6 - i * (i - 1) / 2 + (j - i)) : (j * 6 - j * (j - 1) / 2 + (i - j));
}
__host__ __device__ constexpr int voigt(int c, int l) {
    return c == l ? c : ((c + l == 1) ? 3 : ((c + l == 3) ? 4 : 5));
}

// ------------------------------------------------- element matrices (setup)
// K_e[(j,c),(j',c')] = |T| sum_{k,k'} M[(k,c),(k',c')] P[k][k'][j][j'],
// M[(k,c),(k',c')] = sum_{l,l'} G[k][l] D[v(c,l)][v(c',l')] G[k'][l'] and
// P[k][k'][j][j'] = sum_m A[k][m][j] A[k'][m][j'] (reference gradient modes,
// vertex functions included): the matrix-free operator's arithmetic written as
// one matrix, in FP64, stored as FP32.  One CTA per element.
template <int P>
__global__ void __launch_bounds__(128) k_element_matrices(int64_t nt, const double* __restrict__ geo,
                                                          const double* __restrict__ mat,
                                                          const double* __restrict__ ptab,
                                                          const uint16_t* __restrict__ pairs,
                                                          float* __restrict__ ke) {
    using S = TcShape<P>;
    __shared__ double G[9], Dv[21], Ms[81];
    __shared__ double vol;
    for (int64_t e = blockIdx.x; e < nt; e += gridDim.x) {
        const int t = threadIdx.x;
        if (t < 9) G[t] = geo[e * 10 + t];
        if (t == 9) vol = geo[e * 10 + 9];
        if (t >= 32 && t < 53) Dv[t - 32] = mat[e * 21 + (t - 32)];
        __syncthreads();
        if (t < 81) {
            const int a = t / 9, b = t % 9;
            const int k = a / 3, c = a % 3, k2 = b / 3, c2 = b % 3;
            double s = 0.0;
            for (int l = 0; l < 3; ++l)
                for (int l2 = 0; l2 < 3; ++l2)
                    s += G[k * 3 + l] * Dv[ut6i(voigt(c, l), voigt(c2, l2))] * G[k2 * 3 + l2];
            Ms[t] = vol * s;
        }
        __syncthreads();
        for (int q = t; q < S::PACKP; q += blockDim.x) {
            float out = 0.f;
            if (q < S::PACK) {
                const int i = pairs[q] >> 8, j = pairs[q] & 255;
                const int ji = i / 3, ci = i % 3, jj = j / 3, cj = j % 3;
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int k2 = 0; k2 < 3; ++k2)
                        s += Ms[(k * 3 + ci) * 9 + k2 * 3 + cj] * ptab[((k * 3 + k2) * S::NE + ji) * S::NE + jj];
                out = (float)s;
            }
            ke[e * S::PACKP + q] = out;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- the operator kernel
struct TcView {
    int64_t nt;
    const int32_t* edofs;   // [nt][NE]
    const float* ke;        // [nt][PACKP] packed upper triangle, FP32
    const uint16_t* pairs;  // [PACK] (row << 8) | col of each packed entry
    const uint8_t* phase;   // [nt]
    const float* scale;     // [ncols][2]
};

constexpr uint64_t WAIT_NS = 1000000000ull;   // 1 s: one MMA group takes microseconds
constexpr int WAIT_POLLS = 1 << 26;

template <int NE>
__device__ __forceinline__ void tc_load_ed(const TcView& v, int64_t e, int64_t e1, int (&ed)[NE]) {
#pragma unroll
    for (int j = 0; j < NE; ++j) ed[j] = e < e1 ? __ldg(v.edofs + e * NE + j) : 0;
}

// Operands of element e into ring stage s: the packed matrix and this thread's
// column of the gathered values; one cp.async group per call (empty past the
// chunk end).  Each thread copies exactly the packed entries it expands later
// (q = t + 128 k) and the values it reads, so its own cp.async wait covers them.
template <int P>
__device__ __forceinline__ void tc_issue_loads(const TcView& v, const float* __restrict__ x, int64_t e, int64_t e1,
                                               int s, const int (&ed)[TcShape<P>::NE], uint32_t ke_s0,
                                               uint32_t xs_s0, int32_t* ed_ring, uint8_t* ph_ring, bool live,
                                               int col, int ncols, int t) {
    using S = TcShape<P>;
    if (e < e1) {
        const float* src = v.ke + e * S::PACKP;
        for (int q = t; q < S::PACK; q += 128) cp_async4(ke_s0 + s * S::KE_BYTES + q * 4, src + q);
        const uint32_t xs = xs_s0 + s * S::XS_BYTES;
        if (live) {
#pragma unroll
            for (int q = 0; q < S::N; ++q)
                cp_async4(xs + (q * 128 + t) * 4, x + ((int64_t)ed[q / 3] * 3 + q % 3) * ncols + col);
        }
        if (t == 0) {
#pragma unroll
            for (int j = 0; j < S::NE; ++j) ed_ring[s * S::NE + j] = ed[j];
            ph_ring[s] = v.phase[e];
        }
    }
    cp_async_commit();
}

// One CTA of 128 threads: thread t owns column slot t (TMEM lane t) of a
// 128-column tile and walks a contiguous chunk of elements.  Per element: the
// B tiles are expanded from the packed matrix, the A operand is written to TMEM
// from the gathered values, one thread issues the 3 x KS MMAs, one lane per warp
// waits for their completion and every thread scatters its lane of the product.  The
// operands of the next STAGES elements (packed matrix, this column's gathered
// values) stream into a shared-memory ring with cp.async while the current one
// is multiplied, so the per-element chain sees no global-memory latency.
template <int P>
__global__ void __launch_bounds__(128, TcShape<P>::CTAS_PER_SM)
    k_operator_tc(TcView v, const float* __restrict__ x, float* __restrict__ y, double* __restrict__ epart,
                  const int32_t* __restrict__ active, int ncols, const int32_t* __restrict__ list,
                  const int32_t* __restrict__ n_list, int nby_total, int32_t* __restrict__ err) {
    using S = TcShape<P>;
    constexpr int NE = S::NE, N = S::N, NP = S::NP, ST = S::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* Bhi = base + S::OFF_BHI;
    uint8_t* Blo = base + S::OFF_BLO;
    uint32_t* offs = reinterpret_cast<uint32_t*>(base + S::OFF_OFFS);   // swizzled (i,j) | (j,i) << 16
    int32_t* ed_ring = reinterpret_cast<int32_t*>(base + S::OFF_ED);
    uint8_t* ph_ring = base + S::OFF_PH;
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + S::OFF_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const uint32_t ke_s0 = smem_u32(base + S::OFF_KE), xs_s0 = smem_u32(base + S::OFF_XS);

    const int t = threadIdx.x, warp = t >> 5;
    const int n_act = list ? *n_list : ncols;
    if ((int)blockIdx.x * 128 >= n_act) return;   // whole CTA: no column of this tile is active
    const int slot = blockIdx.x * 128 + t;
    bool live = slot < n_act;
    int col = 0;
    if (live) {
        col = list ? list[slot] : slot;
        if (!list && active && !active[col]) live = false;
    }
    const float sc0 = live ? v.scale[col * 2] : 0.f, sc1 = live ? v.scale[col * 2 + 1] : 0.f;
    const int64_t e0 = v.nt * blockIdx.y / gridDim.y, e1 = v.nt * (blockIdx.y + 1) / gridDim.y;

    // setup: swizzled offsets of the packed entries, zero B tiles (the padding
    // rows and columns stay zero), the MMA completion barrier, tensor memory
    for (int q = t; q < S::PACK; q += 128) {
        const int i = v.pairs[q] >> 8, j = v.pairs[q] & 255;
        offs[q] = sw128_offset<NP>(i, j) | (sw128_offset<NP>(j, i) << 16);
    }
    for (int w = t; w < 2 * S::TILE / 16; w += 128) reinterpret_cast<float4*>(base)[w] = make_float4(0, 0, 0, 0);
    if (t == 0) {
        mbar_init(smem_u32(bar), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), S::TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t tAh = tmem, tAl = tmem + NP, tD = tmem + 2 * NP;
    // kind::tf32, D FP32, A and B TF32, both K-major, N = NP, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t bar_a = smem_u32(bar);

    // operand prefetch: element e into ring stage s (one cp.async group per call,
    // empty past the chunk), its DOF indices from registers
    int ed_next[NE];
    tc_load_ed<NE>(v, e0, e1, ed_next);
#pragma unroll
    for (int k = 0; k < ST; ++k) {
        tc_issue_loads<P>(v, x, e0 + k, e1, k, ed_next, ke_s0, xs_s0, ed_ring, ph_ring, live, col, ncols, t);
        tc_load_ed<NE>(v, e0 + k + 1, e1, ed_next);
    }
    __syncthreads();   // the ring's index entries of the first stages

    float esum = 0.f, ecomp = 0.f;   // compensated energy sum of this column
    uint32_t parity = 0;
    bool issued_pending = false, local_abort = false;
    int s = 0;
    for (int64_t e = e0; e < e1; ++e) {
        // this thread's copies of element e have landed; the ring's index entries were
        // written at least one CTA barrier ago (before the MMA issue of an earlier element)
        cp_async_wait<ST - 1>();
        int ed[NE];
#pragma unroll
        for (int j = 0; j < NE; ++j) ed[j] = ed_ring[s * NE + j];
        const float sc = ph_ring[s] ? sc1 : sc0;
        // after a timed-out wait this thread writes no operand (an MMA may still read them)
        if (!local_abort) {
            // ---- B: K_e expanded into the swizzled tiles, split into TF32 high and low parts
            const float* kes = reinterpret_cast<const float*>(base + S::OFF_KE + s * S::KE_BYTES);
            for (int q = t; q < S::PACK; q += 128) {
                const float val = kes[q];
                const uint32_t h = to_tf32(val);
                const uint32_t l = to_tf32(val - __uint_as_float(h));
                const uint32_t o = offs[q], o1 = o & 0xFFFFu, o2 = o >> 16;
                *reinterpret_cast<uint32_t*>(Bhi + o1) = h;
                *reinterpret_cast<uint32_t*>(Blo + o1) = l;
                *reinterpret_cast<uint32_t*>(Bhi + o2) = h;
                *reinterpret_cast<uint32_t*>(Blo + o2) = l;
            }
            // ---- A: this column's element vector into TMEM lane t, high and low parts
            const float* xs = reinterpret_cast<const float*>(base + S::OFF_XS + s * S::XS_BYTES);
#pragma unroll
            for (int ch = 0; ch < NP / 16; ++ch) {
                uint32_t hv[16], lv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int q = ch * 16 + u;
                    const float xv = (q < N && live) ? xs[q * 128 + t] : 0.f;
                    hv[u] = to_tf32(xv);
                    lv[u] = to_tf32(xv - __uint_as_float(hv[u]));
                }
                tmem_st16(tAh + lane + ch * 16, hv);
                tmem_st16(tAl + lane + ch * 16, lv);
            }
        }
        tmem_wait_st();
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (*abort_flag) break;
        // ---- issue: 3 MMAs per K-step (hi*hi, hi*lo, lo*hi), completion to the barrier
        if (t == 0) {
            tc_fence_after();
            const uint32_t bh0 = smem_u32(Bhi), bl0 = smem_u32(Blo);
#pragma unroll
            for (int ks = 0; ks < S::KS; ++ks) {
                const uint32_t off = (uint32_t)((ks >> 2) * S::ATOM + (ks & 3) * 32);
                const uint64_t dh = smem_desc_sw128(bh0 + off), dl = smem_desc_sw128(bl0 + off);
                tc_mma_tf32(tD, tAh + ks * 8, dh, idesc, ks > 0 ? 1u : 0u);
                tc_mma_tf32(tD, tAh + ks * 8, dl, idesc, 1u);
                tc_mma_tf32(tD, tAl + ks * 8, dh, idesc, 1u);
            }
            tc_commit(bar_a);
        }
        issued_pending = true;
        // one lane per warp polls the barrier; the others wait at the warp barrier
        bool ok = true;
        if ((t & 31) == 0) ok = mbar_wait_bounded(bar_a, parity, WAIT_NS, WAIT_POLLS);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        const int s_cur = s;
        s = s + 1 == ST ? 0 : s + 1;
        if (!ok) {
            if (err) atomicOr(err, 4);
            *abort_flag = 1;
            local_abort = true;
            continue;   // the next barrier ends the loop for the whole CTA
        }
        issued_pending = false;
        parity ^= 1u;
        tc_fence_after();
        // ---- epilogue: y += s K_e x_e for this column, energy s x_e . K_e x_e (x_e
        // from the ring stage, still this element's)
        const float* xs = reinterpret_cast<const float*>(base + S::OFF_XS + s_cur * S::XS_BYTES);
        float en = 0.f;
#pragma unroll
        for (int ch = 0; ch < NP / 16; ++ch) {
            uint32_t dv[16];
            tmem_ld16(tD + lane + ch * 16, dv);
            tmem_wait_ld();
            if (live) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int q = ch * 16 + u;
                    if (q < N) {
                        const float yv = __uint_as_float(dv[u]);
                        en = fmaf(xs[q * 128 + t], yv, en);
                        atomicAdd(y + ((int64_t)ed[q / 3] * 3 + q % 3) * ncols + col, sc * yv);
                    }
                }
            }
        }
        {
            const float yk = sc * en - ecomp;
            const float tk = esum + yk;
            ecomp = (tk - esum) - yk;
            esum = tk;
        }
        tc_fence_before();
        // ---- refill the consumed ring stage with the element STAGES ahead (its
        // last reader, this thread's energy sum, is done; the packed entries and
        // gathered values of a thread are its own copies; the shared index
        // entries are next read behind the MMA-issue barrier of a later element)
        tc_issue_loads<P>(v, x, e + ST, e1, s_cur, ed_next, ke_s0, xs_s0, ed_ring, ph_ring, live, col, ncols, t);
        tc_load_ed<NE>(v, e + ST + 1, e1, ed_next);
    }
    // teardown: copies still in flight land before the CTA exits; an MMA still in
    // flight after a timeout gets one more bounded wait
    cp_async_wait<0>();
    tc_fence_before();
    __syncthreads();
    if (t == 0 && *abort_flag && issued_pending) mbar_wait_bounded(bar_a, parity, WAIT_NS, WAIT_POLLS);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, S::TCOLS);
    }
    if (epart && live) {
        epart[(int64_t)blockIdx.y * ncols + col] = (double)esum - (double)ecomp;
        if (blockIdx.y == 0)
            for (int b = gridDim.y; b < nby_total; ++b) epart[(int64_t)b * ncols + col] = 0.0;
    }
}

template <int P>
constexpr size_t tc_smem_bytes() {
    using S = TcShape<P>;
    const size_t used = 1024 + (size_t)S::BYTES;
    // pad so that no more CTAs fit on an SM than intended (tensor memory and registers)
    const size_t cap = (size_t)(232448 / (S::CTAS_PER_SM + 1)) + 1024;
    return used > cap ? used : cap;
}

// P[k][k'][j][j'] of order p (FP64), vertex functions written out as in the
// matrix-free operator: mode 0 carries x_{k+1} - x_0, higher modes none.
std::vector<double> reference_ptab(int p) {
    const Basis& B = basis(p);
    const int ne = B.ne, nm = B.nm;
    auto a = [&](int k, int m, int j) -> double {
        if (j < 4) {
            if (m != 0) return 0.0;
            if (j == 0) return -1.0;
            return (j - 1 == k) ? 1.0 : 0.0;
        }
        return B.A[((size_t)k * nm + m) * ne + j];
    };
    std::vector<double> out((size_t)9 * ne * ne, 0.0);
    for (int k = 0; k < 3; ++k)
        for (int k2 = 0; k2 < 3; ++k2)
            for (int j = 0; j < ne; ++j)
                for (int j2 = 0; j2 < ne; ++j2) {
                    double s = 0.0;
                    for (int m = 0; m < nm; ++m) s += a(k, m, j) * a(k2, m, j2);
                    out[(((size_t)k * 3 + k2) * ne + j) * ne + j2] = s;
                }
    return out;
}

std::vector<uint16_t> packed_pairs(int n) {
    std::vector<uint16_t> out;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) out.push_back((uint16_t)((i << 8) | j));
    return out;
}

}  // namespace

bool operator_tc_supported(int p, int nc) { return nc == 3 && (p == 2 || p == 3); }

cudaError_t operator_tc_prepare(int p) {
    if (p == 2)
        return cudaFuncSetAttribute(k_operator_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tc_smem_bytes<2>());
    if (p == 3)
        return cudaFuncSetAttribute(k_operator_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tc_smem_bytes<3>());
    return cudaErrorInvalidValue;
}

int64_t element_matrix_floats(int p) {
    return p == 2 ? TcShape<2>::PACKP : (p == 3 ? TcShape<3>::PACKP : 0);
}

int element_matrix_pairs(int p) { return p == 2 ? TcShape<2>::PACK : (p == 3 ? TcShape<3>::PACK : 0); }

cudaError_t build_element_matrices(int p, int64_t nt, const double* geo64, const double* matm64, float* ke,
                                   uint16_t* pairs_dev, double* ptab_dev, cudaStream_t s) {
    const int ne = n_local(p);
    const std::vector<double> pt = reference_ptab(p);
    const std::vector<uint16_t> pr = packed_pairs(3 * ne);
    cudaError_t e = cudaMemcpyAsync(pairs_dev, pr.data(), pr.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(ptab_dev, pt.data(), pt.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<int64_t>(nt, (int64_t)sm_count() * 16);
    if (p == 2)
        k_element_matrices<2><<<grid, 128, 0, s>>>(nt, geo64, matm64, ptab_dev, pairs_dev, ke);
    else if (p == 3)
        k_element_matrices<3><<<grid, 128, 0, s>>>(nt, geo64, matm64, ptab_dev, pairs_dev, ke);
    else
        return cudaErrorInvalidValue;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);   // the host tables above must outlive the copies
}

cudaError_t launch_operator_tc(int p, int64_t nt, const int32_t* edofs, const float* ke, const uint16_t* pairs,
                               const uint8_t* phase, const float* scale, const float* x, float* y, double* epart,
                               const int32_t* active, int ncols, const int32_t* list, const int32_t* n_list,
                               int nby_total, int32_t* err, cudaStream_t s) {
    TcView v{nt, edofs, ke, pairs, phase, scale};
    const int tiles = (ncols + 127) / 128;
    auto go = [&](auto kernel, size_t smem, int per_sm) -> cudaError_t {
        int by = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * per_sm / tiles, nt));
        if (by > nby_total) by = nby_total;
        dim3 grid(tiles, by);
        kernel<<<grid, 128, smem, s>>>(v, x, y, epart, active, ncols, list, n_list, nby_total, err);
        return cudaGetLastError();
    };
    if (p == 2) return go(k_operator_tc<2>, tc_smem_bytes<2>(), TcShape<2>::CTAS_PER_SM);
    if (p == 3) return go(k_operator_tc<3>, tc_smem_bytes<3>(), TcShape<3>::CTAS_PER_SM);
    return cudaErrorInvalidValue;
}

}  // namespace rve
