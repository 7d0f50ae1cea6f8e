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
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "surrogate.h"

namespace rve {

namespace {

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ float silu_f(float a) { return a / (1.f + __expf(-a)); }
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
__device__ __forceinline__ void cp16_zfill(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
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
//           2 = bias, FP32 out, 3 = accumulate FP32 into Cf (C += A B)
template <int NT>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                 const __nv_bfloat16* __restrict__ Bt,
                                                 const float* __restrict__ bias, int epilogue,
                                                 __nv_bfloat16* __restrict__ Cb, float* __restrict__ Cf) {
    constexpr int A_BYTES = 128 * 128, B_BYTES = NT * 128, STAGE = A_BYTES + B_BYTES;
    extern __shared__ uint8_t gsm_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + 2 * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
    const int t = threadIdx.x, warp = t >> 5;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * NT;
    const int KB = K / 64;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"((uint32_t)NT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // kind::f16, D FP32, A and B BF16, both K-major, N = NT, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) | ((128u >> 4) << 24);
    // one K step (64 values) of A and B into stage s: 16-byte chunks, chunk c of row r
    // at r * 128 + ((c ^ (r mod 8)) << 4)
    auto load_step = [&](int kb, int s) {
        const uint32_t sa = smem_addr(base + s * STAGE), sb = sa + A_BYTES;
        for (int i = t; i < 128 * 8; i += 128) {
            const int r = i >> 3, c = i & 7;
            const bool in = m0 + r < M;
            const __nv_bfloat16* src = A + (int64_t)(in ? m0 + r : 0) * K + kb * 64 + c * 8;
            cp16_zfill(sa + r * 128 + ((c ^ (r & 7)) << 4), src, in ? 16u : 0u);
        }
        for (int i = t; i < NT * 8; i += 128) {
            const int r = i >> 3, c = i & 7;
            cp16_zfill(sb + r * 128 + ((c ^ (r & 7)) << 4), Bt + (int64_t)(n0 + r) * K + kb * 64 + c * 8, 16u);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    bool ok = true;
    load_step(0, 0);
    for (int kb = 0; kb < KB && ok; ++kb) {
        const int s = kb & 1;
        if (kb + 1 < KB) {
            // the stage of step kb + 1 was last read by the MMAs of step kb - 1
            if (kb >= 1) {
                bool w = true;
                if ((t & 31) == 0) w = bar_wait(smem_addr(bar + ((kb + 1) & 1)), ((kb - 1) >> 1) & 1);
                w = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
                if (!w) {
                    atomicOr(&g_gemm_timeout, 1);
                    ok = false;
                }
            }
            load_step(kb + 1, (kb + 1) & 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
        if (!ok) break;
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_addr(base + s * STAGE), sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_f16_tmem(tmem, desc_sw128(sa + kk * 32), desc_sw128(sb + kk * 32), idesc,
                             (kb > 0 || kk > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(bar + s))
                         : "memory");
        }
    }
    // the last step's commit completes after every earlier MMA of the tile
    if (ok) {
        bool w = true;
        if ((t & 31) == 0) w = bar_wait(smem_addr(bar + ((KB - 1) & 1)), ((KB - 1) >> 1) & 1);
        w = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
        if (!w) {
            atomicOr(&g_gemm_timeout, 1);
            ok = false;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + t;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 16) {
        uint32_t v[16];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                     "%12, %13, %14, %15}, [%16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                       "=r"(v[14]), "=r"(v[15])
                     : "r"(tmem + lane + c0)
                     : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!ok || row >= M) continue;
        const int col = n0 + c0;
        const int64_t o = (int64_t)row * N + col;
        float f[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) f[u] = __uint_as_float(v[u]);
        if (epilogue == 3) {
#pragma unroll
            for (int u = 0; u < 16; ++u) Cf[o + u] += f[u];
            continue;
        }
        if (bias && epilogue != 0)
#pragma unroll
            for (int u = 0; u < 16; ++u) f[u] += bias[col + u];
        if (epilogue == 1) {
            if (Cf)
#pragma unroll
                for (int u = 0; u < 16; u += 4)
                    *reinterpret_cast<float4*>(Cf + o + u) = make_float4(f[u], f[u + 1], f[u + 2], f[u + 3]);
            uint32_t pk[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                pk[u] = pack_bf16(__float2bfloat16(silu_f(f[2 * u])), __float2bfloat16(silu_f(f[2 * u + 1])));
            *reinterpret_cast<uint4*>(Cb + o) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(Cb + o + 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        } else {
#pragma unroll
            for (int u = 0; u < 16; u += 4)
                *reinterpret_cast<float4*>(Cf + o + u) = make_float4(f[u], f[u + 1], f[u + 2], f[u + 3]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)NT)
                     : "memory");
    }
}

template <int NT>
static size_t gemm_smem() {
    return 1024 + 2 * (size_t)(128 * 128 + NT * 128) + 64;
}

void gemm_tc_prepare() {
    cudaFuncSetAttribute(k_gemm_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<128>());
    cudaFuncSetAttribute(k_gemm_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<64>());
}

int gemm_tc_timed_out() {
    int v = 0;
    cudaMemcpyFromSymbol(&v, g_gemm_timeout, sizeof(int));
    return v;
}

// M a multiple of 64 (rows past a 128-row tile are zero-filled), N 64 or a
// multiple of 128, K a multiple of 64.  128-column tiles: 128 TMEM columns and
// 64 KB of operand stages per CTA, so three CTAs share an SM and hide each
// other's load latency and epilogue.
void launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Bt, const float* bias,
                      int epilogue, __nv_bfloat16* Cb, float* Cf, cudaStream_t s) {
    if (N == 64) {
        dim3 grid(1, (M + 127) / 128);
        k_gemm_tc<64><<<grid, 128, gemm_smem<64>(), s>>>(M, N, K, A, Bt, bias, epilogue, Cb, Cf);
    } else {
        dim3 grid(N / 128, (M + 127) / 128);
        k_gemm_tc<128><<<grid, 128, gemm_smem<128>(), s>>>(M, N, K, A, Bt, bias, epilogue, Cb, Cf);
    }
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
// into out[OO ..] (compile-time indices keep L in registers).
template <int NN, int OFF, int OO>
__device__ __forceinline__ void head_block(const float (&L)[33], float* out) {
#pragma unroll
    for (int i = 0; i < NN; ++i)
#pragma unroll
        for (int j = 0; j < NN; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q <= (i < j ? i : j); ++q)
                acc = fmaf(L[OFF + i * (i + 1) / 2 + q], L[OFF + j * (j + 1) / 2 + q], acc);
            out[OO + i * NN + j] = acc;
        }
}

// Head: z [M][noutp] of member e -> factor entries (softplus diagonals), member
// tensors L L^T into Te [n][54] (C 36, K 9, D 9).  FP32 arithmetic (the network
// itself is BF16 with FP32 accumulation; FP64 runs at a small fraction of the FP32
// rate on this GPU).
__global__ void k_head_tensors(int n, int noutp, const float* __restrict__ z, const uint8_t* __restrict__ diag,
                               float* __restrict__ Te) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float L[33];
#pragma unroll
    for (int c = 0; c < 33; ++c) {
        const float zz = z[(int64_t)r * noutp + c];
        L[c] = diag[c] ? (zz > 20.f ? zz : log1pf(expf(zz))) : zz;
    }
    float* out = Te + (int64_t)r * 54;
    head_block<6, 0, 0>(L, out);
    head_block<3, 21, 36>(L, out);
    head_block<3, 27, 45>(L, out);
}

void launch_head_tensors(int n, int noutp, const float* z, const uint8_t* diag, float* Te, cudaStream_t s) {
    k_head_tensors<<<(n + 127) / 128, 128, 0, s>>>(n, noutp, z, diag, Te);
}

// Mean over the members of entries [LO, HI) of row r (written to Tm in FP64) and
// the largest relative member deviation max_e ||T_e - mean|| / ||mean|| over them.
template <int LO, int HI>
__device__ __forceinline__ float ensemble_block(int n, int r, int members, const float* __restrict__ T,
                                                double* __restrict__ Tm) {
    float mean[HI - LO];
    const float inv = 1.f / (float)members;
#pragma unroll
    for (int c = 0; c < HI - LO; ++c) {
        float sacc = 0.f;
        for (int e = 0; e < members; ++e) sacc += T[((int64_t)e * n + r) * 54 + LO + c];
        mean[c] = sacc * inv;
        Tm[(int64_t)r * 54 + LO + c] = (double)mean[c];
    }
    float den = 0.f;
#pragma unroll
    for (int c = 0; c < HI - LO; ++c) den = fmaf(mean[c], mean[c], den);
    float worst = 0.f;
    for (int e = 0; e < members; ++e) {
        float num = 0.f;
#pragma unroll
        for (int c = 0; c < HI - LO; ++c) {
            const float d = T[((int64_t)e * n + r) * 54 + LO + c] - mean[c];
            num = fmaf(d, d, num);
        }
        const float q = den > 0.f ? sqrtf(num / den) : 0.f;
        worst = q > worst ? q : worst;
    }
    return worst;
}

// Ensemble mean and spread: Tm [n][54] = mean over members (FP64 storage),
// spread[n] = max over the three tensors of max_e ||T_e - Tm||_F / ||Tm||_F.
__global__ void k_ensemble(int n, int members, const float* __restrict__ T, double* __restrict__ Tm,
                           double* __restrict__ spread) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float a = ensemble_block<0, 36>(n, r, members, T, Tm);
    const float b = ensemble_block<36, 45>(n, r, members, T, Tm);
    const float c = ensemble_block<45, 54>(n, r, members, T, Tm);
    spread[r] = (double)fmaxf(a, fmaxf(b, c));
}

void launch_ensemble(int n, int members, const float* T, double* Tm, double* spread, cudaStream_t s) {
    k_ensemble<<<(n + 127) / 128, 128, 0, s>>>(n, members, T, Tm, spread);
}

// Tm [n][54] (C 36, K 9, D 9 in the network's units) -> C [n][36], K [n][9], D [n][9] in SI units
__global__ void k_split_tensors(int64_t n, const double* __restrict__ Tm, double rc, double rk, double rd,
                                double* __restrict__ C, double* __restrict__ K, double* __restrict__ D) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * 54; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / 54;
        const int c = (int)(i % 54);
        const double v = Tm[i];
        if (c < 36) C[r * 36 + c] = v * rc;
        else if (c < 45) K[r * 9 + c - 36] = v * rk;
        else D[r * 9 + c - 45] = v * rd;
    }
}

void launch_split_tensors(int64_t n, const double* Tm, double rc, double rk, double rd, double* C, double* K,
                          double* D, cudaStream_t s) {
    int64_t b = (n * 54 + 255) / 256;
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    k_split_tensors<<<(unsigned)b, 256, 0, s>>>(n, Tm, rc, rk, rd, C, K, D);
}

}  // namespace rve
