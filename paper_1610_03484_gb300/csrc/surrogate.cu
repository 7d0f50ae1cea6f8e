// Learned surrogate of the RVE homogenisation (no counterpart in the paper).
//
// An ensemble of MLPs maps 8 features of a macro Gauss point to the 33
// Cholesky-factor entries of its normalised C (21), K (6) and D (6):
//   h_{l+1} = silu(h_l W_l + b_l), l = 0..3 (width 256), z = h_4 W_4 + b_4,
//   L = tril(z) with softplus on the diagonal, tensor = L L^T (always SPD).
// Weights and activations are BF16, every product accumulates in FP32 on the
// tensor cores (mma.sync m16n8k16), master weights and Adam moments are FP32.
//
// GEMM convention: C[M][N] = A[M][K] * B, with A row-major and B supplied as
// Bt[N][K] row-major (K contiguous in both), M, N multiples of 64, K of 16.
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

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float silu_f(float a) { return a / (1.f + __expf(-a)); }
__device__ __forceinline__ float dsilu_f(float a) {
    const float s = 1.f / (1.f + __expf(-a));
    return s * (1.f + a * (1.f - s));
}

}  // namespace

// Block tile 64 x 64, 4 warps (each 16 rows x 64 columns), K step 16.
// epilogue: 0 = store FP32 only, 1 = bias + silu -> BF16 (pre-activation to zf if non-null),
//           2 = bias, FP32 out, 3 = accumulate FP32 into Cf (C += A B)
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                   const __nv_bfloat16* __restrict__ Bt,
                                                   const float* __restrict__ bias, int epilogue,
                                                   __nv_bfloat16* __restrict__ Cb, float* __restrict__ Cf) {
    __shared__ __nv_bfloat16 As[64][16 + 8];
    __shared__ __nv_bfloat16 Bs[64][16 + 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[i][r] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        // stage A and B tiles: 64 x 16 each, 128 threads x 8 elements
        for (int i = threadIdx.x; i < 64 * 16; i += 128) {
            const int r = i >> 4, c = i & 15;
            As[r][c] = A[(int64_t)(m0 + r) * K + k0 + c];
            Bs[r][c] = Bt[(int64_t)(n0 + r) * K + k0 + c];
        }
        __syncthreads();
        uint32_t a[4];
        const int ar = warp * 16 + g;
        a[0] = pack_bf16(As[ar][2 * t], As[ar][2 * t + 1]);
        a[1] = pack_bf16(As[ar + 8][2 * t], As[ar + 8][2 * t + 1]);
        a[2] = pack_bf16(As[ar][2 * t + 8], As[ar][2 * t + 9]);
        a[3] = pack_bf16(As[ar + 8][2 * t + 8], As[ar + 8][2 * t + 9]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            uint32_t b[2];
            const int bn = nt * 8 + g;
            b[0] = pack_bf16(Bs[bn][2 * t], Bs[bn][2 * t + 1]);
            b[1] = pack_bf16(Bs[bn][2 * t + 8], Bs[bn][2 * t + 9]);
            mma_bf16_16816(acc[nt], a, b);
        }
        __syncthreads();
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = m0 + warp * 16 + g + (r >= 2 ? 8 : 0);
            const int col = n0 + nt * 8 + 2 * t + (r & 1);
            const int64_t o = (int64_t)row * N + col;
            float v = acc[nt][r];
            if (epilogue == 3) {
                Cf[o] += v;
                continue;
            }
            if (bias && epilogue != 0) v += bias[col];
            if (epilogue == 1) {
                if (Cf) Cf[o] = v;
                Cb[o] = __float2bfloat16(silu_f(v));
            } else {
                Cf[o] = v;
            }
        }
}

void launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Bt, const float* bias,
                      int epilogue, __nv_bfloat16* Cb, float* Cf, cudaStream_t s) {
    dim3 grid(N / 64, M / 64);
    k_gemm_bf16<<<grid, 128, 0, s>>>(M, N, K, A, Bt, bias, epilogue, Cb, Cf);
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

// Head: z [M][noutp] of member e -> factor entries (softplus diagonals), accumulated
// into the ensemble mean tensors; writes member tensors to T_e [n][54] (C 36, K 9, D 9).
__global__ void k_head_tensors(int n, int noutp, const float* __restrict__ z, const uint8_t* __restrict__ diag,
                               double* __restrict__ Te) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double L[33];
    for (int c = 0; c < 33; ++c) {
        const double zz = z[(int64_t)r * noutp + c];
        L[c] = diag[c] ? (zz > 30 ? zz : log1p(exp(zz))) : zz;
    }
    double* out = Te + (int64_t)r * 54;
    const int sizes[3] = {6, 3, 3}, offs[3] = {0, 21, 27}, oofs[3] = {0, 36, 45};
    for (int b = 0; b < 3; ++b) {
        const int nn = sizes[b];
        double Lm[6][6] = {};
        int k = 0;
        for (int i = 0; i < nn; ++i)
            for (int j = 0; j <= i; ++j) Lm[i][j] = L[offs[b] + k++];
        for (int i = 0; i < nn; ++i)
            for (int j = 0; j < nn; ++j) {
                double sacc = 0;
                for (int q = 0; q <= (i < j ? i : j); ++q) sacc += Lm[i][q] * Lm[j][q];
                out[oofs[b] + i * nn + j] = sacc;
            }
    }
}

void launch_head_tensors(int n, int noutp, const float* z, const uint8_t* diag, double* Te, cudaStream_t s) {
    k_head_tensors<<<(n + 127) / 128, 128, 0, s>>>(n, noutp, z, diag, Te);
}

// Ensemble mean and spread: Tm [n][54] = mean over members, spread[n] = max over
// the three tensors of max_e ||T_e - Tm||_F / ||Tm||_F.
__global__ void k_ensemble(int n, int members, const double* __restrict__ T, double* __restrict__ Tm,
                           double* __restrict__ spread) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double mean[54];
    for (int c = 0; c < 54; ++c) {
        double sacc = 0;
        for (int e = 0; e < members; ++e) sacc += T[((int64_t)e * n + r) * 54 + c];
        mean[c] = sacc / members;
        Tm[(int64_t)r * 54 + c] = mean[c];
    }
    const int lo[3] = {0, 36, 45}, hi[3] = {36, 45, 54};
    double worst = 0;
    for (int b = 0; b < 3; ++b) {
        double den = 0;
        for (int c = lo[b]; c < hi[b]; ++c) den += mean[c] * mean[c];
        for (int e = 0; e < members; ++e) {
            double num = 0;
            for (int c = lo[b]; c < hi[b]; ++c) {
                const double d = T[((int64_t)e * n + r) * 54 + c] - mean[c];
                num += d * d;
            }
            const double q = den > 0 ? sqrt(num / den) : 0.0;
            worst = q > worst ? q : worst;
        }
    }
    spread[r] = worst;
}

void launch_ensemble(int n, int members, const double* T, double* Tm, double* spread, cudaStream_t s) {
    k_ensemble<<<(n + 127) / 128, 128, 0, s>>>(n, members, T, Tm, spread);
}

}  // namespace rve
