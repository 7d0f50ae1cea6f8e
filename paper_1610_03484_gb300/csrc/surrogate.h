// Launch wrappers of the surrogate kernels (surrogate.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace rve {

// sets the GEMM kernels' shared-memory limit (once per device, before the first launch)
void gemm_tc_prepare();
// nonzero once a bounded wait inside the GEMM gave up (sticky for the process)
int gemm_tc_timed_out();
// C = A Bt^T on the tensor cores (TMA-fed); an error if a tensor map cannot be encoded
cudaError_t launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, const __nv_bfloat16* Bt,
                             const float* bias, int epilogue, __nv_bfloat16* Cb, float* Cf, cudaStream_t s);
// Fused ensemble inference: all layers of up to mlp_fused_max_members() members per
// 128-row tile with the activations kept on chip; X [M][64] BF16 features, member e's
// W^T of layer l at wt[e] + w_off[l], biases bias[e * 5 + l]; z of member e written
// transposed to zT + e * 64 * ldz ([64][ldz]).  An error if a tensor map cannot be encoded.
int mlp_fused_max_members();
cudaError_t launch_mlp_fused(int M, int members, const __nv_bfloat16* X, const __nv_bfloat16* const* wt,
                             const int64_t* w_off, const float* const* bias, float* zT, int ldz, cudaStream_t s);
void launch_transpose_bf16(int rows, int cols, const __nv_bfloat16* in, __nv_bfloat16* out, cudaStream_t s);
void launch_silu_backward(int64_t n, const float* dY, const float* Z, __nv_bfloat16* g, cudaStream_t s);
void launch_head_loss(int M, int m_valid, int noutp, const float* z, const float* target, const float* sigma,
                      const uint8_t* diag, __nv_bfloat16* dz, float* loss_acc, cudaStream_t s);
void launch_colsum_bf16(int rows, int cols, const __nv_bfloat16* in, float* out, cudaStream_t s);
void launch_adam(int K, int N, float* W, const float* Gt, float* m1, float* m2, float lr, int step,
                 __nv_bfloat16* Wt, __nv_bfloat16* Wn, int n_valid_out, cudaStream_t s);
void launch_adam_bias(int N, float* b, const float* g, float* m1, float* m2, float lr, int step, int n_valid_out,
                      cudaStream_t s);
void launch_features(int n, int M, int kin, const double* feat, const float* mean, const float* inv_std,
                     __nv_bfloat16* X, cudaStream_t s);
// zT [noutp][ldz] (transposed last-layer output) -> member tensors TeT [54][n]
void launch_head_tensors(int n, int ldz, const float* zT, const uint8_t* diag, float* TeT, cudaStream_t s);
// T [members][54][n] -> ensemble means C [n][36], K [n][9], D [n][9] (times the
// reference scales rc, rk, rd; FP64) and spread [n]
void launch_ensemble(int n, int members, const float* T, double rc, double rk, double rd, double* C, double* K,
                     double* D, double* spread, cudaStream_t s);

}  // namespace rve
