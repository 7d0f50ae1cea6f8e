// Learned surrogate of the RVE homogenisation (no counterpart in the paper).
//
// An ensemble of MLPs maps 8 features of a macro Gauss point to the 33
// Cholesky-factor entries of its normalised C (21), K (6) and D (6):
//   h_{l+1} = silu(h_l W_l + b_l), l = 0..3 (width 256), z = h_4 W_4 + b_4,
//   L = tril(z) with softplus on the diagonal, tensor = L L^T (always SPD).
// Weights and activations are BF16, every product accumulates in FP32 on the
// 5th-generation tensor cores (tcgen05.mma kind::f16, accumulator in tensor
// memory), master weights and Adam moments are FP32.
//
// GEMM convention: C[M][N] = A[M][K] * B, with A row-major and B supplied as
// Bt[N][K] row-major (K contiguous in both), M a multiple of 64, N 64 or a
// multiple of 128, K a multiple of 64.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "surrogate.h"

namespace rve {

namespace {

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// a sigmoid(a) with the fast reciprocal division (a / inf -> 0 for very negative a)
__device__ __forceinline__ float silu_f(float a) { return __fdividef(a, 1.f + __expf(-a)); }
__device__ __forceinline__ float dsilu_f(float a) {
    const float s = 1.f / (1.f + __expf(-a));
    return s * (1.f + a * (1.f - s));
}

}  // namespace

// ------------------------------------------------ tcgen05 GEMM (sm_103a)
// C tile [128 rows x NT] = A [128 x K] * Bt [NT x K]^T on the 5th-generation tensor
// cores: BF16 operands staged by cp.async into 128-byte-swizzled K-major shared
// memory tiles (64 K values = 128 bytes per row), two K stages in flight, one
// thread issuing kind::f16 MMAs (M = 128, N = NT, K = 16) into an FP32 TMEM
// accumulator, thread t reading back row t for the epilogue.  Rows past M are
// zero-filled on load and not stored.
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gl_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool bar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait (1 s of the global timer, or a poll cap should the timer not advance)
__device__ __forceinline__ bool bar_wait(uint32_t a, uint32_t parity) {
    if (bar_try(a, parity)) return true;
    const uint64_t t0 = gl_ns();
    for (int i = 0; i < (1 << 26); ++i) {
        if (bar_try(a, parity)) return true;
        if (gl_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_f16_tmem(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16x(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ int g_gemm_timeout;   // set when a bounded wait of the GEMM gave up

}  // namespace

// epilogue: 0 = store FP32 only, 1 = bias + silu -> BF16 (pre-activation to Cf if non-null),
//           2 = bias, FP32 out, 3 = accumulate FP32 into Cf (C += A B),
//           4 = bias, FP32 out transposed (Cf[col * M + row])
//
// Persistent and warp-specialised: each CTA walks the output tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... (the N tiles of one row block are
// neighbours, so the A rows are read from L2 once per row block).
//   warp 0   TMA producer: K steps of 64 values of A and Bt into a ring of
//            GemmShape::S stages (128-byte swizzle; rows past M zero-filled by the
//            tensor map's bounds), each stage a "full" barrier counting its bytes;
//   warp 1   MMA issuer: kind::f16 MMAs into one of two FP32 TMEM accumulators,
//            releasing each stage through an "empty" barrier and each finished
//            tile through "tmem full";
//   warps 2.. epilogue (NT / 8 of them): a warp reads 32 rows (its TMEM lane
//            quarter) x 32 columns of the finished accumulator, hands it back through
//            "tmem empty" and runs bias / SiLU / conversion and the stores while
//            the MMAs of the next tile fill the other accumulator.
// Every wait is bounded; a role that gives up sets g_gemm_timeout and leaves its
// loop, after which the producer waits for its copies in flight and the MMA
// issuer for its MMAs, so the tensor memory is idle when it is freed.
template <int NT>
struct GemmShape {
    static constexpr int S = NT == 128 ? 6 : 8;
    static constexpr int A_BYTES = 128 * 128, B_BYTES = NT * 128, STAGE = A_BYTES + B_BYTES;
    // epilogue warps: four lane quarters x column groups of 32
    static constexpr int EPI_WARPS = 4 * (NT / 32), THREADS = 64 + 32 * EPI_WARPS;
    static constexpr int NBAR = 2 * S + 5;
    // bias vector staged in shared memory (N <= BIAS_MAX) behind the barriers
    static constexpr int BIAS_OFF = ((8 * NBAR + 16 + 15) / 16) * 16, BIAS_MAX = 256;
};

template <int NT>
__global__ void __launch_bounds__(GemmShape<NT>::THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
              uint32_t stage_tx, const float* __restrict__ bias, int epilogue, __nv_bfloat16* __restrict__ Cb,
              float* __restrict__ Cf) {
    using G = GemmShape<NT>;
    constexpr int S = G::S;
    extern __shared__ uint8_t gsm_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + S * G::STAGE);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;    // [2]
    uint64_t* tempty = tfull + 2;   // [2]
    uint64_t* done = tempty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    float* sbias = reinterpret_cast<float*>(base + S * G::STAGE + G::BIAS_OFF);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int KB = K / 64, n_tn = N / NT, n_tiles = ((M + 127) / 128) * n_tn;
    const bool bias_smem = bias != nullptr && (epilogue == 1 || epilogue == 2 || epilogue == 4) && N <= G::BIAS_MAX;
    if (bias_smem)
        for (int i = t; i < N; i += blockDim.x) sbias[i] = __ldg(bias + i);
    if (t == 0) {
        for (int k = 0; k < G::NBAR; ++k) {
            const uint32_t cnt = (k == 2 * S + 2 || k == 2 * S + 3) ? (uint32_t)G::EPI_WARPS : 1u;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(full + k)), "r"(cnt) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"((uint32_t)(2 * NT))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                const int m0 = (tile / n_tn) * 128, n0 = (tile % n_tn) * NT;
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % S;
                    if (it >= S && !bar_wait(smem_addr(empty + s), ((it / S) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = smem_addr(base + s * G::STAGE), sb = sa + G::A_BYTES, fb = smem_addr(full + s);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(stage_tx)
                                 : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                        "%3}], [%4];" ::"r"(sa),
                        "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(kb * 64), "r"(m0), "r"(fb)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                        "%3}], [%4];" ::"r"(sb),
                        "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(kb * 64), "r"(n0), "r"(fb)
                        : "memory");
                }
            }
            if (!ok) atomicOr(&g_gemm_timeout, 1);
            // the copies of the last min(S, it) steps may still be in flight
            for (int k = it - 1; k >= 0 && k >= it - S; --k)
                if (!bar_wait(smem_addr(full + k % S), (k / S) & 1)) atomicOr(&g_gemm_timeout, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: kind::f16, D FP32, A and B BF16, both K-major, N = NT, M = 128
            const uint32_t idesc =
                (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) | ((128u >> 4) << 24);
            int it = 0, i = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++i) {
                const int acc = i & 1;
                if (i >= 2 && !bar_wait(smem_addr(tempty + acc), ((i >> 1) & 1) ^ 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * NT);
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % S;
                    if (!bar_wait(smem_addr(full + s), (it / S) & 1)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_addr(base + s * G::STAGE), sb = sa + G::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_f16_tmem(d, desc_sw128(sa + kk * 32), desc_sw128(sb + kk * 32), idesc,
                                     (kb > 0 || kk > 0) ? 1u : 0u);
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_addr(empty + s))
                        : "memory");
                }
                if (ok)
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_addr(tfull + acc))
                        : "memory");
            }
            if (!ok) atomicOr(&g_gemm_timeout, 1);
            // every MMA issued has completed once this commit arrives
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(done))
                         : "memory");
            if (!bar_wait(smem_addr(done), 0)) atomicOr(&g_gemm_timeout, 1);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, column group (w - 2) / 4
        const int q = warp & 3, h = (warp - 2) >> 2;
        constexpr int HC = 32;
        int i = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
            __syncwarp();
            const int acc = i & 1;
            const int m0 = (tile / n_tn) * 128, n0 = (tile % n_tn) * NT;
            bool w = true;
            if (lane == 0) w = bar_wait(smem_addr(tfull + acc), (i >> 1) & 1);
            w = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
            if (!w) {
                if (lane == 0) atomicOr(&g_gemm_timeout, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[HC];
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * NT + h * HC);
#pragma unroll
            for (int c = 0; c < HC; c += 16) tmem_ld16x(ta + c, *reinterpret_cast<uint32_t(*)[16]>(v + c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(tempty + acc)) : "memory");
            const int row = m0 + 32 * q + lane;
            if (row >= M) continue;   // (rows past M hold the zero fill or, for M < 128, stale data)
            const int col0 = n0 + h * HC;
            const int64_t o = (int64_t)row * N + col0;
#pragma unroll
            for (int c = 0; c < HC; c += 16) {
                float f[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) f[u] = __uint_as_float(v[c + u]);
                if (epilogue == 3) {
#pragma unroll
                    for (int u = 0; u < 16; u += 4) {
                        float4* ptr = reinterpret_cast<float4*>(Cf + o + c + u);
                        float4 a = *ptr;
                        a.x += f[u]; a.y += f[u + 1]; a.z += f[u + 2]; a.w += f[u + 3];
                        *ptr = a;
                    }
                    continue;
                }
                if (bias_smem) {
#pragma unroll
                    for (int u = 0; u < 16; u += 4) {
                        const float4 b4 = *reinterpret_cast<const float4*>(sbias + col0 + c + u);
                        f[u] += b4.x;
                        f[u + 1] += b4.y;
                        f[u + 2] += b4.z;
                        f[u + 3] += b4.w;
                    }
                } else if (bias && epilogue != 0 && epilogue != 3) {
#pragma unroll
                    for (int u = 0; u < 16; u += 4) {
                        const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + col0 + c + u));
                        f[u] += b4.x;
                        f[u + 1] += b4.y;
                        f[u + 2] += b4.z;
                        f[u + 3] += b4.w;
                    }
                }
                if (epilogue == 4) {   // bias, FP32, transposed: Cf[col][row] (rows adjacent across lanes)
#pragma unroll
                    for (int u = 0; u < 16; ++u) Cf[(int64_t)(col0 + c + u) * M + row] = f[u];
                    continue;
                }
                if (epilogue == 1) {
                    if (Cf)
#pragma unroll
                        for (int u = 0; u < 16; u += 4)
                            *reinterpret_cast<float4*>(Cf + o + c + u) = make_float4(f[u], f[u + 1], f[u + 2], f[u + 3]);
                    uint32_t pk[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        pk[u] = pack_bf16(__float2bfloat16(silu_f(f[2 * u])), __float2bfloat16(silu_f(f[2 * u + 1])));
                    *reinterpret_cast<uint4*>(Cb + o + c) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4*>(Cb + o + c + 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                } else {
#pragma unroll
                    for (int u = 0; u < 16; u += 4)
                        *reinterpret_cast<float4*>(Cf + o + c + u) = make_float4(f[u], f[u + 1], f[u + 2], f[u + 3]);
                }
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * NT))
                     : "memory");
    }
}

// ------------------------------------------- fused ensemble inference (sm_103a)
// The whole network of up to MLP_MAXM members for 128-row tiles of features, with
// the activations kept in shared memory between the layers (only the features come
// in and the last layer's z goes out).  Per layer: kind::f16 MMAs (M = 128, N = 256
// or 64, K = 16) from the activation tile (A: 128-byte-swizzled K-major chunks of 64
// values, written by the epilogue in that layout) and a weight chunk W^T [N][64] (B,
// streamed by TMA through a two-stage ring from L2) into an FP32 accumulator of 256
// tensor-memory columns; the epilogue adds the bias, applies SiLU and writes the BF16
// activations back over the tile it came from (its layer's MMAs have completed), or,
// after the last layer, stores z transposed (zT[member][col][row]) for the head.
//
// Work items are (tile, member) pairs, walked persistently.  Two items are in flight
// per CTA, one per slot (own feature tile, activation tile and accumulator): the MMA
// warp alternates between the slots layer by layer, so that one slot's MMAs run while
// the other slot's epilogue works.  Warp 0 issues the TMA copies in the MMA's order,
// warp 1 the MMAs, and epilogue warps 2-9 serve slot 0 and 10-17 slot 1 (lane quarter
// w % 4, 128-column half).  Every wait is bounded.
constexpr int MLP_MAXM = 4, MLP_EPI = 16, MLP_THREADS = 64 + 32 * MLP_EPI;
constexpr int MLP_NL = 5;
constexpr int MLP_OFF_ACT = 0,        // [2][64 KB]
    MLP_OFF_X = 131072,               // [2][16 KB]
    MLP_OFF_W = 163840,               // [2][32 KB]
    MLP_OFF_BAR = 229376, MLP_SMEM = 1024 + MLP_OFF_BAR + 128;

struct MlpParams {
    CUtensorMap x;                       // features [M][64] BF16, box {64, x_rows}
    CUtensorMap w[MLP_MAXM][MLP_NL];     // member e, layer l: W^T [N_l][K_l] BF16, box {64, N_l}
    const float* bias[MLP_MAXM][MLP_NL];
    float* zT;                           // [members][64][ldz]
    int M, ldz, members;
    uint32_t x_tx;                       // bytes of one feature tile (x_rows x 128)
};

__device__ __forceinline__ int mlp_k(int l) { return l == 0 ? 64 : 256; }
__device__ __forceinline__ int mlp_n(int l) { return l == 4 ? 64 : 256; }

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(MLP_THREADS, 1) k_mlp_fused(const __grid_constant__ MlpParams P) {
    extern __shared__ uint8_t msm_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(msm_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + MLP_OFF_BAR);
    // per slot s: xfull[s], xempty[s], accfull[s], epidone[s]; the ring's wfull[2], wempty[2]; done
    auto B = [&](int k) { return smem_addr(bars + k); };
    const uint32_t b_xfull = B(0), b_xempty = B(2), b_acc = B(4), b_epi = B(6), b_wfull = B(8), b_wempty = B(10),
                   b_done = B(12);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 13);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int n_items = ((P.M + 127) / 128) * P.members;
    // this CTA's items k = 0 .. n_cta - 1 are blockIdx.x + k gridDim.x; slot s takes k = s (mod 2)
    const int n_cta = blockIdx.x < n_items ? (n_items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int ns0 = (n_cta + 1) / 2, ns1 = n_cta / 2;
    if (t == 0) {
        for (int k = 0; k < 13; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + k)),
                         "r"((k == 6 || k == 7) ? (uint32_t)(MLP_EPI / 2) : 1u)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t s_act = smem_addr(base + MLP_OFF_ACT), s_x = smem_addr(base + MLP_OFF_X),
                   s_w = smem_addr(base + MLP_OFF_W);

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer, in the MMA's order: round r gives slot 0, then slot 1,
            // layer r % 5 of its item r / 5; a layer-0 step also loads the item's features
            int wit = 0;
            bool ok = true;
            for (int r = 0; ok && r / 5 < ns0; ++r)
                for (int sl = 0; sl < 2 && ok; ++sl) {
                    const int idx = r / 5, l = r % 5;
                    if (idx >= (sl ? ns1 : ns0)) continue;
                    const int item = blockIdx.x + (2 * idx + sl) * gridDim.x;
                    const int tile = item / P.members, e = item % P.members;
                    if (l == 0) {
                        if (idx >= 1 && !bar_wait(b_xempty + 8 * sl, (idx - 1) & 1)) {
                            ok = false;
                            break;
                        }
                        bar_expect(b_xfull + 8 * sl, P.x_tx);
                        tma_2d(s_x + sl * 16384, &P.x, 0, tile * 128, b_xfull + 8 * sl);
                    }
                    for (int kc = 0; kc < mlp_k(l) / 64; ++kc, ++wit) {
                        const int st = wit & 1;
                        if (wit >= 2 && !bar_wait(b_wempty + 8 * st, ((wit >> 1) & 1) ^ 1)) {
                            ok = false;
                            break;
                        }
                        bar_expect(b_wfull + 8 * st, (uint32_t)mlp_n(l) * 128u);
                        tma_2d(s_w + st * 32768, &P.w[e][l], kc * 64, 0, b_wfull + 8 * st);
                    }
                }
            if (!ok) atomicOr(&g_gemm_timeout, 1);
            // copies that may still be in flight: each slot's last feature tile and the
            // last weight chunks
            for (int sl = 0; sl < 2; ++sl) {
                const int n = sl ? ns1 : ns0;
                if (n >= 1 && !bar_wait(b_xfull + 8 * sl, (n - 1) & 1)) atomicOr(&g_gemm_timeout, 1);
            }
            for (int k = wit - 1; k >= 0 && k >= wit - 2; --k)
                if (!bar_wait(b_wfull + 8 * (k & 1), (k >> 1) & 1)) atomicOr(&g_gemm_timeout, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: the same round order as the producer.  A slot's step waits
            // for the epilogue of the slot's previous step, which both freed the slot's
            // accumulator and wrote this step's input activations.
            int wit = 0, ks[2] = {0, 0};
            bool ok = true;
            for (int r = 0; ok && r / 5 < ns0; ++r)
                for (int sl = 0; sl < 2 && ok; ++sl) {
                    const int idx = r / 5, l = r % 5;
                    if (idx >= (sl ? ns1 : ns0)) continue;
                    if (l == 0 && !bar_wait(b_xfull + 8 * sl, idx & 1)) {
                        ok = false;
                        break;
                    }
                    if (ks[sl] >= 1 && !bar_wait(b_epi + 8 * sl, (ks[sl] - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a_base = l == 0 ? s_x + sl * 16384 : s_act + sl * 65536;
                    const uint32_t d = tmem + (uint32_t)(256 * sl);
                    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                           ((uint32_t)(mlp_n(l) >> 3) << 17) | ((128u >> 4) << 24);
                    for (int kc = 0; kc < mlp_k(l) / 64; ++kc, ++wit) {
                        const int st = wit & 1;
                        if (!bar_wait(b_wfull + 8 * st, (wit >> 1) & 1)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t a = a_base + kc * 16384, b = s_w + st * 32768;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_f16_tmem(d, desc_sw128(a + kk * 32), desc_sw128(b + kk * 32), idesc,
                                         (kc > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(b_wempty + 8 * st);
                    }
                    if (!ok) break;
                    if (l == 0) mma_commit(b_xempty + 8 * sl);
                    mma_commit(b_acc + 8 * sl);
                    ++ks[sl];
                }
            if (!ok) atomicOr(&g_gemm_timeout, 1);
            // every MMA issued has completed once this commit arrives
            mma_commit(b_done);
            if (!bar_wait(b_done, 0)) atomicOr(&g_gemm_timeout, 1);
        }
    } else {
        // ---- epilogue: warps 2-9 serve slot 0, 10-17 slot 1; lane quarter q, column half h
        const int sl = (warp - 2) >> 3, q = warp & 3, h = ((warp - 2) >> 2) & 1;
        const int r = 32 * q + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(256 * sl);
        uint8_t* act = base + MLP_OFF_ACT + sl * 65536;
        const int n_slot = sl ? ns1 : ns0;
        int ks = 0;
        bool ok = true;
        for (int idx = 0; idx < n_slot && ok; ++idx) {
            const int item = blockIdx.x + (2 * idx + sl) * gridDim.x;
            const int tile = item / P.members, e = item % P.members;
            const int grow = tile * 128 + r;
            for (int l = 0; l < MLP_NL; ++l, ++ks) {
                __syncwarp();
                bool w = true;
                if (lane == 0) w = bar_wait(b_acc + 8 * sl, ks & 1);
                w = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
                if (!w) {
                    if (lane == 0) atomicOr(&g_gemm_timeout, 1);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float* bias = P.bias[e][l];
                if (l < MLP_NL - 1) {
                    // columns 128 h + 64 j .. + 63: activation chunk 2 h + j
#pragma unroll 1
                    for (int j = 0; j < 2; ++j) {
                        const int c0 = 128 * h + 64 * j;
                        uint32_t v[64];
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj)
                            tmem_ld16x(lane_base + (uint32_t)(c0 + 16 * jj),
                                       *reinterpret_cast<uint32_t(*)[16]>(v + 16 * jj));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        uint8_t* out = act + (c0 / 64) * 16384 + r * 128;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float4 b0 = __ldg(reinterpret_cast<const float4*>(bias + c0 + 8 * u));
                            const float4 b1 = __ldg(reinterpret_cast<const float4*>(bias + c0 + 8 * u + 4));
                            const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                            uint32_t pk[4];
#pragma unroll
                            for (int hh = 0; hh < 4; ++hh)
                                pk[hh] = pack_bf16(
                                    __float2bfloat16(silu_f(__uint_as_float(v[8 * u + 2 * hh]) + bb[2 * hh])),
                                    __float2bfloat16(silu_f(__uint_as_float(v[8 * u + 2 * hh + 1]) + bb[2 * hh + 1])));
                            // 128-byte swizzle of the K-major operand layout: 16-byte unit u of row r
                            *reinterpret_cast<uint4*>(out + ((u ^ (r & 7)) << 4)) =
                                make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        }
                    }
                    // the next layer's MMAs read these writes through the async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                } else {
                    // N = 64: columns 32 h .. + 31
                    uint32_t v[32];
                    tmem_ld16x(lane_base + (uint32_t)(32 * h), *reinterpret_cast<uint32_t(*)[16]>(v));
                    tmem_ld16x(lane_base + (uint32_t)(32 * h + 16), *reinterpret_cast<uint32_t(*)[16]>(v + 16));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (grow < P.M) {
                        float* zt = P.zT + ((int64_t)e * 64 + 32 * h) * P.ldz + grow;
#pragma unroll
                        for (int u = 0; u < 32; ++u)
                            zt[(int64_t)u * P.ldz] = __uint_as_float(v[u]) + __ldg(bias + 32 * h + u);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b_epi + 8 * sl) : "memory");
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

template <int NT>
static size_t gemm_smem() {
    return 1024 + (size_t)GemmShape<NT>::S * GemmShape<NT>::STAGE + GemmShape<NT>::BIAS_OFF +
           4 * GemmShape<NT>::BIAS_MAX;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D BF16 row-major matrix [rows][cols] (cols contiguous), box of 64 columns x box_rows
// rows with the 128-byte swizzle; rows past `rows` read as zero
static bool make_map(CUtensorMap* m, const __nv_bfloat16* base, int rows, int cols, int box_rows) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void gemm_tc_prepare() {
    cudaFuncSetAttribute(k_gemm_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<128>());
    cudaFuncSetAttribute(k_gemm_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<64>());
    cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM);
}

int mlp_fused_max_members() { return MLP_MAXM; }

// The fused inference of `members` networks on M feature rows (M a multiple of 64):
// weights of member e at wt[e] + w_off[l] (W^T [N_l][K_l] BF16), biases bias[e * 5 + l].
cudaError_t launch_mlp_fused(int M, int members, const __nv_bfloat16* X, const __nv_bfloat16* const* wt,
                             const int64_t* w_off, const float* const* bias, float* zT, int ldz, cudaStream_t s) {
    if (M <= 0 || M % 64 || members < 1 || members > MLP_MAXM || ldz < M) return cudaErrorInvalidValue;
    static const int KL[MLP_NL] = {64, 256, 256, 256, 256}, NL[MLP_NL] = {256, 256, 256, 256, 64};
    MlpParams P;
    std::memset(&P, 0, sizeof(P));
    const int x_rows = M < 128 ? M : 128;
    if (!make_map(&P.x, X, M, 64, x_rows)) return cudaErrorInvalidValue;
    for (int e = 0; e < members; ++e)
        for (int l = 0; l < MLP_NL; ++l) {
            if (!make_map(&P.w[e][l], wt[e] + w_off[l], NL[l], KL[l], NL[l])) return cudaErrorInvalidValue;
            P.bias[e][l] = bias[e * MLP_NL + l];
        }
    P.zT = zT;
    P.M = M;
    P.ldz = ldz;
    P.members = members;
    P.x_tx = (uint32_t)x_rows * 128u;
    const int items = ((M + 127) / 128) * members;
    const int grid = std::min(items, sm_count());
    k_mlp_fused<<<grid, MLP_THREADS, MLP_SMEM, s>>>(P);
    return cudaGetLastError();
}

int gemm_tc_timed_out() {
    int v = 0;
    cudaMemcpyFromSymbol(&v, g_gemm_timeout, sizeof(int));
    return v;
}

// M a multiple of 64 (rows past a 128-row tile are zero-filled), N 64 or a
// multiple of 128, K a multiple of 64; A and Bt 16-byte aligned.  One CTA per
// SM (at most one per tile), two accumulators of NT TMEM columns each.
cudaError_t launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Bt,
                             const float* bias, int epilogue, __nv_bfloat16* Cb, float* Cf, cudaStream_t s) {
    const int NT = N == 64 ? 64 : 128;
    if (M <= 0 || M % 64 || K <= 0 || K % 64 || (N != 64 && N % 128)) return cudaErrorInvalidValue;
    // with M = 64 the A box is 64 rows and the MMA's rows 64..127 are never stored
    const int a_rows = M < 128 ? M : 128;
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, M, K, a_rows) || !make_map(&tb, Bt, N, K, NT)) return cudaErrorInvalidValue;
    const uint32_t tx = (uint32_t)(a_rows + NT) * 128u;
    const int tiles = (N / NT) * ((M + 127) / 128);
    const int grid = std::min(tiles, sm_count());
    if (NT == 64)
        k_gemm_tc<64><<<grid, GemmShape<64>::THREADS, gemm_smem<64>(), s>>>(ta, tb, M, N, K, tx, bias, epilogue, Cb,
                                                                            Cf);
    else
        k_gemm_tc<128><<<grid, GemmShape<128>::THREADS, gemm_smem<128>(), s>>>(ta, tb, M, N, K, tx, bias, epilogue,
                                                                              Cb, Cf);
    return cudaGetLastError();
}

// out[c][r] = in[r][c] (BF16), rows x cols
__global__ void k_transpose_bf16(int rows, int cols, const __nv_bfloat16* __restrict__ in,
                                 __nv_bfloat16* __restrict__ out) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = by + j, c = bx + threadIdx.x;
        tile[j][threadIdx.x] = (r < rows && c < cols) ? in[(int64_t)r * cols + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int c = bx + j, r = by + threadIdx.x;
        if (c < cols && r < rows) out[(int64_t)c * rows + r] = tile[threadIdx.x][j];
    }
}

void launch_transpose_bf16(int rows, int cols, const __nv_bfloat16* in, __nv_bfloat16* out, cudaStream_t s) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    k_transpose_bf16<<<grid, block, 0, s>>>(rows, cols, in, out);
}

// g = dY * silu'(Z)  (FP32 in, BF16 out), n elements
__global__ void k_silu_backward(int64_t n, const float* __restrict__ dY, const float* __restrict__ Z,
                                __nv_bfloat16* __restrict__ g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = __float2bfloat16(dY[i] * dsilu_f(Z[i]));
}

void launch_silu_backward(int64_t n, const float* dY, const float* Z, __nv_bfloat16* g, cudaStream_t s) {
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    k_silu_backward<<<(unsigned)b, 256, 0, s>>>(n, dY, Z, g);
}

// Output head loss: z [M][NOUTP] (FP32), target [M][33], sigma [33]; rows >= m_valid ignored.
// dz = d loss / d z (BF16, padded columns zero); loss partial per block.
__global__ void k_head_loss(int M, int m_valid, int noutp, const float* __restrict__ z,
                            const float* __restrict__ target, const float* __restrict__ sigma,
                            const uint8_t* __restrict__ diag, __nv_bfloat16* __restrict__ dz,
                            float* __restrict__ loss_acc) {
    float local = 0.f;
    const float inv = 1.f / ((float)m_valid * 33.f);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)M * noutp;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(i / noutp), c = (int)(i % noutp);
        float g = 0.f;
        if (row < m_valid && c < 33) {
            const float zz = z[i];
            const float L = diag[c] ? (zz > 20.f ? zz : log1pf(__expf(zz))) : zz;
            const float r = (L - target[(int64_t)row * 33 + c]) / sigma[c];
            local += r * r * inv;
            g = 2.f * r / sigma[c] * inv;
            if (diag[c]) g *= 1.f / (1.f + __expf(-zz));
        }
        dz[i] = __float2bfloat16(g);
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, local);
}

void launch_head_loss(int M, int m_valid, int noutp, const float* z, const float* target, const float* sigma,
                      const uint8_t* diag, __nv_bfloat16* dz, float* loss_acc, cudaStream_t s) {
    k_head_loss<<<(M * noutp + 255) / 256 < 2048 ? (M * noutp + 255) / 256 : 2048, 256, 0, s>>>(
        M, m_valid, noutp, z, target, sigma, diag, dz, loss_acc);
}

// column sums: out[c] = sum_r in[r][c] (FP32 accumulate of BF16), for bias gradients
__global__ void k_colsum_bf16(int rows, int cols, const __nv_bfloat16* __restrict__ in, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += __bfloat162float(in[(int64_t)r * cols + c]);
    out[c] = s;
}

void launch_colsum_bf16(int rows, int cols, const __nv_bfloat16* in, float* out, cudaStream_t s) {
    k_colsum_bf16<<<(cols + 127) / 128, 128, 0, s>>>(rows, cols, in, out);
}

// Adam on FP32 master weights W [K][N] with gradient G given transposed [N][K]
// (dW^T from the GEMM); refreshes both BF16 layouts Wt [N][K] and Wn [K][N].
__global__ void k_adam(int K, int N, float* __restrict__ W, const float* __restrict__ Gt, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, float b1, float b2, float c1, float c2, float eps,
                       __nv_bfloat16* __restrict__ Wt, __nv_bfloat16* __restrict__ Wn, int n_valid_out) {
    const int64_t n = (int64_t)K * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / N), c = (int)(i % N);
        float g = Gt[(int64_t)c * K + k];
        if (c >= n_valid_out) g = 0.f;
        const float a = b1 * m1[i] + (1.f - b1) * g;
        const float v = b2 * m2[i] + (1.f - b2) * g * g;
        m1[i] = a;
        m2[i] = v;
        float w = W[i];
        if (c < n_valid_out) w -= lr * (a / c1) / (sqrtf(v / c2) + eps);
        W[i] = w;
        Wt[(int64_t)c * K + k] = __float2bfloat16(w);
        Wn[i] = __float2bfloat16(w);
    }
}

__global__ void k_adam_bias(int N, float* __restrict__ b, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, float lr, float b1, float b2, float c1, float c2, float eps,
                            int n_valid_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float gg = i < n_valid_out ? g[i] : 0.f;
    const float a = b1 * m1[i] + (1.f - b1) * gg;
    const float v = b2 * m2[i] + (1.f - b2) * gg * gg;
    m1[i] = a;
    m2[i] = v;
    if (i < n_valid_out) b[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

void launch_adam(int K, int N, float* W, const float* Gt, float* m1, float* m2, float lr, int step,
                 __nv_bfloat16* Wt, __nv_bfloat16* Wn, int n_valid_out, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    const int64_t n = (int64_t)K * N;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_adam<<<(unsigned)blocks, 256, 0, s>>>(K, N, W, Gt, m1, m2, lr, b1, b2, c1, c2, eps, Wt, Wn, n_valid_out);
}

void launch_adam_bias(int N, float* b, const float* g, float* m1, float* m2, float lr, int step, int n_valid_out,
                      cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam_bias<<<(N + 127) / 128, 128, 0, s>>>(N, b, g, m1, m2, lr, b1, b2, c1, c2, eps, n_valid_out);
}

// features [n][8] (FP64) -> normalised BF16 rows of width kin (padded with zeros), rows up to M
__global__ void k_features(int n, int M, int kin, const double* __restrict__ feat, const float* __restrict__ mean,
                           const float* __restrict__ inv_std, __nv_bfloat16* __restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * kin) return;
    const int r = (int)(i / kin), c = (int)(i % kin);
    float v = 0.f;
    if (r < n && c < 8) v = ((float)feat[(int64_t)r * 8 + c] - mean[c]) * inv_std[c];
    X[i] = __float2bfloat16(v);
}

void launch_features(int n, int M, int kin, const double* feat, const float* mean, const float* inv_std,
                     __nv_bfloat16* X, cudaStream_t s) {
    const int64_t tot = (int64_t)M * kin;
    k_features<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, M, kin, feat, mean, inv_std, X);
}

// L L^T of one lower-triangular factor of size NN stored row-major from L[OFF]
// into out[(OO + i NN + j) * n] (compile-time indices keep L in registers).
template <int NN, int OFF, int OO>
__device__ __forceinline__ void head_block_t(const float (&L)[33], float* __restrict__ out, int n) {
#pragma unroll
    for (int i = 0; i < NN; ++i)
#pragma unroll
        for (int j = 0; j < NN; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q <= (i < j ? i : j); ++q)
                acc = fmaf(L[OFF + i * (i + 1) / 2 + q], L[OFF + j * (j + 1) / 2 + q], acc);
            out[(int64_t)(OO + i * NN + j) * n] = acc;
        }
}

// Head: zT [noutp][ldz] (the last layer's output, transposed) of member e ->
// factor entries (softplus diagonals), member tensors L L^T into TeT [54][n]
// (C 36, K 9, D 9; transposed, so that adjacent threads touch adjacent words).
// FP32 arithmetic (the network itself is BF16 with FP32 accumulation; FP64 runs
// at a small fraction of the FP32 rate on this GPU).
__global__ void k_head_tensors(int n, int ldz, const float* __restrict__ zT, const uint8_t* __restrict__ diag,
                               float* __restrict__ TeT) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float L[33];
#pragma unroll
    for (int c = 0; c < 33; ++c) {
        const float zz = zT[(int64_t)c * ldz + r];
        L[c] = diag[c] ? (zz > 20.f ? zz : log1pf(expf(zz))) : zz;
    }
    float* out = TeT + r;
    head_block_t<6, 0, 0>(L, out, n);
    head_block_t<3, 21, 36>(L, out, n);
    head_block_t<3, 27, 45>(L, out, n);
}

void launch_head_tensors(int n, int ldz, const float* zT, const uint8_t* diag, float* TeT, cudaStream_t s) {
    k_head_tensors<<<(n + 127) / 128, 128, 0, s>>>(n, ldz, zT, diag, TeT);
}

// Mean over the members of entries [LO, HI) of point r (member tensors T
// [members][54][n], transposed) into the block's staging rows, and the largest
// relative member deviation max_e ||T_e - mean|| / ||mean|| over them.
constexpr int ENS_BLOCK = 64, ENS_LD = 55;
template <int LO, int HI>
__device__ __forceinline__ float ensemble_block(int n, int r, int members, const float* __restrict__ T,
                                                double* __restrict__ stage) {
    float mean[HI - LO];
    const float inv = 1.f / (float)members;
#pragma unroll
    for (int c = 0; c < HI - LO; ++c) {
        // up to four members in independent loads; more in a second loop
        float sacc = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (e < members) sacc += __ldg(T + ((int64_t)e * 54 + LO + c) * n + r);
        for (int e = 4; e < members; ++e) sacc += __ldg(T + ((int64_t)e * 54 + LO + c) * n + r);
        mean[c] = sacc * inv;
        stage[LO + c] = (double)mean[c];
    }
    float den = 0.f;
#pragma unroll
    for (int c = 0; c < HI - LO; ++c) den = fmaf(mean[c], mean[c], den);
    float worst = 0.f;
    for (int e = 0; e < members; ++e) {
        float num = 0.f;
#pragma unroll
        for (int c = 0; c < HI - LO; ++c) {
            const float d = __ldg(T + ((int64_t)e * 54 + LO + c) * n + r) - mean[c];
            num = fmaf(d, d, num);
        }
        const float q = den > 0.f ? sqrtf(num / den) : 0.f;
        worst = q > worst ? q : worst;
    }
    return worst;
}

// Ensemble mean and spread: C [n][36], K [n][9], D [n][9] = mean over the members
// times the reference scales (SI units, FP64), spread[n] = max over the three tensors
// of max_e ||T_e - mean||_F / ||mean||_F.  The means of a block's points are staged
// in shared memory and each output is stored as one contiguous run of rows.
__global__ void __launch_bounds__(ENS_BLOCK) k_ensemble(int n, int members, const float* __restrict__ T, double rc,
                                                        double rk, double rd, double* __restrict__ C,
                                                        double* __restrict__ K, double* __restrict__ D,
                                                        double* __restrict__ spread) {
    __shared__ double stage[ENS_BLOCK * ENS_LD];
    const int r0 = blockIdx.x * ENS_BLOCK, r = r0 + threadIdx.x;
    if (r < n) {
        double* st = stage + threadIdx.x * ENS_LD;
        const float a = ensemble_block<0, 36>(n, r, members, T, st);
        const float b = ensemble_block<36, 45>(n, r, members, T, st);
        const float c = ensemble_block<45, 54>(n, r, members, T, st);
        spread[r] = (double)fmaxf(a, fmaxf(b, c));
    }
    __syncthreads();
    const int rows = min(ENS_BLOCK, n - r0);
    for (int i = threadIdx.x; i < rows * 36; i += ENS_BLOCK)
        C[(int64_t)r0 * 36 + i] = stage[(i / 36) * ENS_LD + i % 36] * rc;
    for (int i = threadIdx.x; i < rows * 9; i += ENS_BLOCK) {
        K[(int64_t)r0 * 9 + i] = stage[(i / 9) * ENS_LD + 36 + i % 9] * rk;
        D[(int64_t)r0 * 9 + i] = stage[(i / 9) * ENS_LD + 45 + i % 9] * rd;
    }
}

void launch_ensemble(int n, int members, const float* T, double rc, double rk, double rd, double* C, double* K,
                     double* D, double* spread, cudaStream_t s) {
    k_ensemble<<<(n + ENS_BLOCK - 1) / ENS_BLOCK, ENS_BLOCK, 0, s>>>(n, members, T, rc, rk, rd, C, K, D, spread);
}

}  // namespace rve
