// C ABI of the learned surrogate: ensemble MLP training and inference on the
// GPU (surrogate.cu kernels) and the surrogate-plus-fallback batched FE^2 call.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "api_internal.h"
#include "surrogate.h"

namespace rve {
namespace {

constexpr int KIN = 64;      // 8 features padded to one GEMM tile
constexpr int HID = 256;     // hidden width
constexpr int NOUTP = 64;    // 33 outputs padded
constexpr int NOUT = 33;
constexpr int NLAYER = 5;
constexpr int NFEAT = 8;
constexpr int HEADER = 8 + 8 + 33 + 3;   // feature mean, feature std, sigma, reference scales

const int LK[NLAYER] = {KIN, HID, HID, HID, HID};
const int LN[NLAYER] = {HID, HID, HID, HID, NOUTP};

int64_t layer_w_off(int l) {
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += (int64_t)LK[i] * LN[i] + LN[i];
    return o;
}
int64_t n_params() { return layer_w_off(NLAYER); }

std::vector<uint8_t> diag_mask() {
    std::vector<uint8_t> d(NOUT, 0);
    const int sizes[3] = {6, 3, 3}, offs[3] = {0, 21, 27};
    for (int b = 0; b < 3; ++b) {
        int k = 0;
        for (int i = 0; i < sizes[b]; ++i)
            for (int j = 0; j <= i; ++j) d[offs[b] + k++] = (i == j);
    }
    return d;
}

}  // namespace
}  // namespace rve

using namespace rve;

struct rve_surrogate_s {
    rve_ctx ctx = nullptr;
    int members = 0;
    bool trained = false;
    float feat_mean[8] = {0}, feat_std[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    float sigma[33];
    double ref[3] = {1, 1, 1};
    // per member: FP32 master params, Adam moments, BF16 weights in both layouts
    std::vector<DevBuf> P, M1, M2, Wt, Wn;
    DevBuf d_norm, d_diag;
    // workspace
    DevBuf X, H[NLAYER], Z[NLAYER], zout, dz, G, Gt, Ht, dH, gradT, gradb, loss, feat_dev, Tmem, spr;
    // inference: the fused kernel (all members' layers per tile, activations on chip)
    // or one GEMM launch per member and layer
    bool fused = true;
    DevBuf zall;
};

namespace {

int refresh_bf16(rve_surrogate s, int e) {
    // rebuild BF16 copies from the FP32 master parameters via a zero-lr Adam pass
    cudaStream_t st = s->ctx->stream;
    for (int l = 0; l < NLAYER; ++l) {
        const int64_t o = layer_w_off(l);
        float* W = s->P[e].as<float>() + o;
        float* m1 = s->M1[e].as<float>() + o;
        float* m2 = s->M2[e].as<float>() + o;
        __nv_bfloat16* wt = s->Wt[e].as<__nv_bfloat16>() + o;
        __nv_bfloat16* wn = s->Wn[e].as<__nv_bfloat16>() + o;
        // gradient buffer of zeros of the right shape
        RVE_TRY(s->gradT.ensure((size_t)LK[l] * LN[l] * 4));
        RVE_CUDA(cudaMemsetAsync(s->gradT.p, 0, (size_t)LK[l] * LN[l] * 4, st));
        launch_adam(LK[l], LN[l], W, s->gradT.as<float>(), m1, m2, 0.f, 1, wt, wn, LN[l], st);
    }
    return RVE_OK;
}

int alloc_work(rve_surrogate s, int M) {
    RVE_TRY(s->X.ensure((size_t)M * KIN * 2));
    for (int l = 0; l < NLAYER; ++l) {
        RVE_TRY(s->H[l].ensure((size_t)M * LK[l] * 2));
        RVE_TRY(s->Z[l].ensure((size_t)M * LN[l] * 4));
    }
    RVE_TRY(s->zout.ensure((size_t)M * NOUTP * 4));
    RVE_TRY(s->dz.ensure((size_t)M * HID * 2));
    RVE_TRY(s->G.ensure((size_t)M * HID * 2));
    RVE_TRY(s->Gt.ensure((size_t)M * HID * 2));
    RVE_TRY(s->Ht.ensure((size_t)M * HID * 2));
    RVE_TRY(s->dH.ensure((size_t)M * HID * 4));
    RVE_TRY(s->gradT.ensure((size_t)HID * HID * 4));
    RVE_TRY(s->gradb.ensure((size_t)HID * 4));
    RVE_TRY(s->loss.ensure(64));
    return RVE_OK;
}

// forward pass of member e on M rows already in s->H[0] (BF16 [M][KIN]); z -> s->zout,
// [M][NOUTP] (training) or transposed [NOUTP][M] (inference, transposed_out)
int forward(rve_surrogate s, int e, int M, bool keep_pre, bool transposed_out = false) {
    cudaStream_t st = s->ctx->stream;
    for (int l = 0; l < NLAYER; ++l) {
        const int64_t o = layer_w_off(l);
        const __nv_bfloat16* wt = s->Wt[e].as<__nv_bfloat16>() + o;
        const float* b = s->P[e].as<float>() + o + (int64_t)LK[l] * LN[l];
        if (l < NLAYER - 1)
            RVE_CUDA(launch_gemm_bf16(M, LN[l], LK[l], s->H[l].as<__nv_bfloat16>(), wt, b, 1,
                                      s->H[l + 1].as<__nv_bfloat16>(), keep_pre ? s->Z[l].as<float>() : nullptr,
                                      st));
        else
            RVE_CUDA(launch_gemm_bf16(M, LN[l], LK[l], s->H[l].as<__nv_bfloat16>(), wt, b, transposed_out ? 4 : 2,
                                      nullptr, s->zout.as<float>(), st));
    }
    s->ctx->launches += NLAYER;
    return RVE_OK;
}

// Backward pass of member e after forward(keep_pre) and the head loss (dz
// holds d loss / d z).  With grads_host == nullptr the Adam update is applied;
// otherwise every layer's gradient is copied to grads_host in the parameter
// layout ([K][N] weights then [N] bias per layer) and the weights are kept.
int backward_step(rve_surrogate s, int e, int M, int step, float lr, float* grads_host) {
    cudaStream_t st = s->ctx->stream;
    __nv_bfloat16* Gcur = s->dz.as<__nv_bfloat16>();
    std::vector<float> gT, gb;
    for (int l = NLAYER - 1; l >= 0; --l) {
        const int K = LK[l], N = LN[l];
        const int64_t o = layer_w_off(l);
        // dW^T [N][K] = G^T H_l
        launch_transpose_bf16(M, N, Gcur, s->Gt.as<__nv_bfloat16>(), st);
        launch_transpose_bf16(M, K, s->H[l].as<__nv_bfloat16>(), s->Ht.as<__nv_bfloat16>(), st);
        RVE_CUDA(launch_gemm_bf16(N, K, M, s->Gt.as<__nv_bfloat16>(), s->Ht.as<__nv_bfloat16>(), nullptr, 0,
                                  nullptr, s->gradT.as<float>(), st));
        launch_colsum_bf16(M, N, Gcur, s->gradb.as<float>(), st);
        if (l > 0) {
            // dH_l = G W_l^T, then through the silu of layer l-1
            RVE_CUDA(launch_gemm_bf16(M, K, N, Gcur, s->Wn[e].as<__nv_bfloat16>() + o, nullptr, 0, nullptr,
                                      s->dH.as<float>(), st));
            launch_silu_backward((int64_t)M * K, s->dH.as<float>(), s->Z[l - 1].as<float>(),
                                 s->G.as<__nv_bfloat16>(), st);
        }
        const int nvalid = (l == NLAYER - 1) ? NOUT : N;
        if (grads_host) {
            gT.resize((size_t)N * K);
            gb.resize(N);
            RVE_CUDA(cudaMemcpyAsync(gT.data(), s->gradT.p, gT.size() * 4, cudaMemcpyDeviceToHost, st));
            RVE_CUDA(cudaMemcpyAsync(gb.data(), s->gradb.p, gb.size() * 4, cudaMemcpyDeviceToHost, st));
            RVE_CUDA(cudaStreamSynchronize(st));
            for (int k = 0; k < K; ++k)
                for (int n = 0; n < N; ++n) grads_host[o + (int64_t)k * N + n] = n < nvalid ? gT[(size_t)n * K + k] : 0.f;
            for (int n = 0; n < N; ++n) grads_host[o + (int64_t)K * N + n] = n < nvalid ? gb[n] : 0.f;
        } else {
            launch_adam(K, N, s->P[e].as<float>() + o, s->gradT.as<float>(), s->M1[e].as<float>() + o,
                        s->M2[e].as<float>() + o, lr, step, s->Wt[e].as<__nv_bfloat16>() + o,
                        s->Wn[e].as<__nv_bfloat16>() + o, nvalid, st);
            const int64_t ob = o + (int64_t)K * N;
            launch_adam_bias(N, s->P[e].as<float>() + ob, s->gradb.as<float>(), s->M1[e].as<float>() + ob,
                             s->M2[e].as<float>() + ob, lr, step, nvalid, st);
        }
        if (l > 0) {
            RVE_CUDA(cudaMemcpyAsync(s->dz.p, s->G.p, (size_t)M * K * 2, cudaMemcpyDeviceToDevice, st));
            Gcur = s->dz.as<__nv_bfloat16>();
        }
        s->ctx->launches += 7;
    }
    return RVE_OK;
}

}  // namespace

extern "C" {

int rve_surrogate_create(rve_ctx c, int members, uint64_t seed, rve_surrogate* out) {
    RVE_TRY(check_ctx(c));
    if (!out || members < 1 || members > 16) {
        set_error("rve_surrogate_create: members must be 1..16");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    gemm_tc_prepare();
    auto* s = new rve_surrogate_s();
    s->ctx = c;
    s->members = members;
    for (int i = 0; i < NOUT; ++i) s->sigma[i] = 1.f;
    s->P.resize(members);
    s->M1.resize(members);
    s->M2.resize(members);
    s->Wt.resize(members);
    s->Wn.resize(members);
    const int64_t np = n_params();
    cudaStream_t st = c->stream;
    for (int e = 0; e < members; ++e) {
        std::mt19937_64 rng(seed * 1000003ull + (uint64_t)e);
        std::vector<float> h(np, 0.f);
        for (int l = 0; l < NLAYER; ++l) {
            const int64_t o = layer_w_off(l);
            const int kin = l == 0 ? NFEAT : LK[l];   // padded inputs stay zero
            const float lim = std::sqrt(6.f / kin);
            std::uniform_real_distribution<float> U(-lim, lim);
            for (int k = 0; k < LK[l]; ++k)
                for (int n = 0; n < LN[l]; ++n)
                    h[o + (int64_t)k * LN[l] + n] = (k < kin && (l < NLAYER - 1 || n < NOUT)) ? U(rng) : 0.f;
        }
        int rc = upload(s->P[e], h.data(), h.size(), st);
        if (rc == RVE_OK) rc = s->M1[e].ensure(np * 4);
        if (rc == RVE_OK) rc = s->M2[e].ensure(np * 4);
        if (rc == RVE_OK) rc = s->Wt[e].ensure(np * 2);
        if (rc == RVE_OK) rc = s->Wn[e].ensure(np * 2);
        if (rc != RVE_OK) {
            delete s;
            return rc;
        }
        cudaMemsetAsync(s->M1[e].p, 0, np * 4, st);
        cudaMemsetAsync(s->M2[e].p, 0, np * 4, st);
        rc = refresh_bf16(s, e);
        if (rc != RVE_OK) {
            delete s;
            return rc;
        }
    }
    auto dm = diag_mask();
    if (upload(s->d_diag, dm.data(), dm.size(), st) != RVE_OK) {
        delete s;
        return RVE_ERR_OUT_OF_MEMORY;
    }
    *out = s;
    return RVE_OK;
}

int rve_surrogate_free(rve_ctx c, rve_surrogate s) {
    if (!s) return RVE_OK;
    if (c) cudaSetDevice(c->device);
    cudaStreamSynchronize(s->ctx->stream);
    delete s;
    return RVE_OK;
}

int rve_gauss_point_features(rve_ctx c, rve_mesh m, int64_t G, const double* T_C, const double* c_wt,
                             const double* t_h, double* feat) {
    RVE_TRY(check_ctx(c));
    if (!m || G < 0 || (G > 0 && (!T_C || !c_wt || !t_h || !feat))) return RVE_ERR_INVALID_ARGUMENT;
    if (!m->have_materials) return RVE_ERR_STATE;
    if (G == 0) return RVE_OK;
    std::vector<double> w(G);
    RVE_TRY(rve_degradation_factor(c, G, T_C, c_wt, t_h, &m->deg, w.data()));
    const MaterialConsts& mc = m->mc;
    for (int64_t g = 0; g < G; ++g) {
        const double wy = m->deg.apply_to_yarn ? w[g] : 1.0;
        const double f[8] = {T_C[g], c_wt[g], std::log10(std::max(t_h[g], 1e-30)), mc.Em * w[g],
                             mc.E1 * wy, mc.E2 * wy, mc.G12 * wy, mc.km};
        std::memcpy(feat + 8 * g, f, sizeof(f));
    }
    return RVE_OK;
}

int rve_surrogate_train(rve_ctx c, rve_surrogate s, int64_t n, const double* feat, const double* Ct,
                        const double* Kt, const double* Dt, int epochs, int batch, double lr,
                        uint64_t seed, double* loss_history) {
    NvtxRange nvtx_("surrogate training: %lld points, %d members", (long long)n, s ? s->members : 0);
    RVE_TRY(check_ctx(c));
    if (!s || n < 64 || !feat || !Ct || !Kt || !Dt || epochs < 1 || batch < 64 || batch % 64 || !(lr > 0)) {
        set_error("rve_surrogate_train: invalid argument (n >= 64, batch a multiple of 64)");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t st = c->stream;
    // ---- normalisation from the data
    double mean[8] = {0}, var[8] = {0};
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 8; ++k) mean[k] += feat[8 * i + k] / n;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 8; ++k) var[k] += (feat[8 * i + k] - mean[k]) * (feat[8 * i + k] - mean[k]) / n;
    for (int k = 0; k < 8; ++k) {
        s->feat_mean[k] = (float)mean[k];
        s->feat_std[k] = var[k] > 1e-30 * (mean[k] * mean[k] + 1e-30) ? (float)std::sqrt(var[k]) : 1.f;
    }
    double tr[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 6; ++a) tr[0] += Ct[36 * i + 7 * a] / (6.0 * n);
        for (int a = 0; a < 3; ++a) {
            tr[1] += Kt[9 * i + 4 * a] / (3.0 * n);
            tr[2] += Dt[9 * i + 4 * a] / (3.0 * n);
        }
    }
    for (int b = 0; b < 3; ++b) s->ref[b] = tr[b];
    // targets: Cholesky factors of the normalised tensors, row-major lower triangles
    std::vector<float> tgt((size_t)n * NOUT);
    for (int64_t i = 0; i < n; ++i) {
        const double* src[3] = {Ct + 36 * i, Kt + 9 * i, Dt + 9 * i};
        const int sizes[3] = {6, 3, 3}, offs[3] = {0, 21, 27};
        for (int b = 0; b < 3; ++b) {
            const int nn = sizes[b];
            double A[6][6], L[6][6] = {};
            for (int r = 0; r < nn; ++r)
                for (int q = 0; q < nn; ++q) A[r][q] = 0.5 * (src[b][r * nn + q] + src[b][q * nn + r]) / s->ref[b];
            for (int j = 0; j < nn; ++j) {
                double d = A[j][j];
                for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
                if (!(d > 0)) {
                    set_error("rve_surrogate_train: a training tensor is not positive definite");
                    return RVE_ERR_NOT_SPD;
                }
                L[j][j] = std::sqrt(d);
                for (int r = j + 1; r < nn; ++r) {
                    double t = A[r][j];
                    for (int k = 0; k < j; ++k) t -= L[r][k] * L[j][k];
                    L[r][j] = t / L[j][j];
                }
            }
            int k = 0;
            for (int r = 0; r < nn; ++r)
                for (int q = 0; q <= r; ++q) tgt[i * NOUT + offs[b] + k++] = (float)L[r][q];
        }
    }
    // The factors of tensors normalised by their mean trace are O(1); an equal
    // scale for every entry makes the loss the squared error relative to the
    // tensor's own size (what the accuracy target is stated in).
    for (int o = 0; o < NOUT; ++o) s->sigma[o] = 1.f;
    // ---- device data: normalised features (BF16 rows) and targets
    const int M = batch;
    RVE_TRY(alloc_work(s, M));
    DevBuf dfeat, dtgt, dsig, dmean, dstd, bfeat, btgt, didx;
    std::vector<float> fm(s->feat_mean, s->feat_mean + 8), fis(8);
    for (int k = 0; k < 8; ++k) fis[k] = 1.f / s->feat_std[k];
    RVE_TRY(upload(dfeat, feat, (size_t)n * 8, st));
    RVE_TRY(upload(dtgt, tgt.data(), tgt.size(), st));
    RVE_TRY(upload(dsig, s->sigma, NOUT, st));
    RVE_TRY(upload(dmean, fm.data(), 8, st));
    RVE_TRY(upload(dstd, fis.data(), 8, st));
    RVE_TRY(bfeat.ensure((size_t)M * 8 * 8));
    RVE_TRY(btgt.ensure((size_t)M * NOUT * 4));
    std::vector<double> hb((size_t)M * 8);
    std::vector<float> ht((size_t)M * NOUT);
    const int64_t steps_per_epoch = n / M;
    std::vector<double> hist(epochs, 0.0);
    for (int e = 0; e < s->members; ++e) {
        std::mt19937_64 rng(seed * 7919ull + (uint64_t)e);
        std::vector<int64_t> perm(n);
        std::iota(perm.begin(), perm.end(), 0);
        int step = 0;
        for (int ep = 0; ep < epochs; ++ep) {
            std::shuffle(perm.begin(), perm.end(), rng);
            RVE_CUDA(cudaMemsetAsync(s->loss.p, 0, 4, st));
            for (int64_t b = 0; b < steps_per_epoch; ++b) {
                for (int r = 0; r < M; ++r) {
                    const int64_t i = perm[b * M + r];
                    std::memcpy(&hb[(size_t)r * 8], feat + 8 * i, 64);
                    std::memcpy(&ht[(size_t)r * NOUT], &tgt[(size_t)i * NOUT], NOUT * 4);
                }
                RVE_CUDA(cudaMemcpyAsync(bfeat.p, hb.data(), hb.size() * 8, cudaMemcpyHostToDevice, st));
                RVE_CUDA(cudaMemcpyAsync(btgt.p, ht.data(), ht.size() * 4, cudaMemcpyHostToDevice, st));
                launch_features(M, M, KIN, bfeat.as<double>(), dmean.as<float>(), dstd.as<float>(),
                                s->H[0].as<__nv_bfloat16>(), st);
                RVE_TRY(forward(s, e, M, true));
                launch_head_loss(M, M, NOUTP, s->zout.as<float>(), btgt.as<float>(), dsig.as<float>(),
                                 s->d_diag.as<uint8_t>(), s->dz.as<__nv_bfloat16>(), s->loss.as<float>(), st);
                ++step;
                // cosine decay of the learning rate over all steps of this member
                const double total = (double)epochs * steps_per_epoch;
                const double lr_t = lr * (0.02 + 0.98 * 0.5 * (1.0 + std::cos(M_PI * (step - 1) / total)));
                RVE_TRY(backward_step(s, e, M, step, (float)lr_t, nullptr));
            }
            float lsum = 0;
            RVE_CUDA(cudaMemcpyAsync(&lsum, s->loss.p, 4, cudaMemcpyDeviceToHost, st));
            RVE_CUDA(cudaStreamSynchronize(st));
            hist[ep] += lsum / steps_per_epoch / s->members;
        }
    }
    RVE_CUDA(cudaGetLastError());
    if (loss_history) std::memcpy(loss_history, hist.data(), sizeof(double) * epochs);
    s->trained = true;
    if (gemm_tc_timed_out()) {
        set_error("a bounded wait inside the surrogate GEMM gave up");
        return RVE_ERR_TIMEOUT;
    }
    return RVE_OK;
}

int rve_surrogate_gradients(rve_ctx c, rve_surrogate s, int member, int n, const double* feat,
                            const float* target_factors, float* grads, double* loss) {
    RVE_TRY(check_ctx(c));
    if (!s || member < 0 || member >= s->members || n < 1 || n % 64 || !feat || !target_factors || !grads) {
        set_error("rve_surrogate_gradients: invalid argument (n a positive multiple of 64)");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t st = c->stream;
    RVE_TRY(alloc_work(s, n));
    DevBuf df, dt, dsig, dmean, dstd;
    std::vector<float> fis(8);
    for (int k = 0; k < 8; ++k) fis[k] = 1.f / s->feat_std[k];
    RVE_TRY(upload(df, feat, (size_t)n * 8, st));
    RVE_TRY(upload(dt, target_factors, (size_t)n * NOUT, st));
    RVE_TRY(upload(dsig, s->sigma, NOUT, st));
    RVE_TRY(upload(dmean, s->feat_mean, 8, st));
    RVE_TRY(upload(dstd, fis.data(), 8, st));
    RVE_CUDA(cudaMemsetAsync(s->loss.p, 0, 4, st));
    launch_features(n, n, KIN, df.as<double>(), dmean.as<float>(), dstd.as<float>(), s->H[0].as<__nv_bfloat16>(), st);
    RVE_TRY(forward(s, member, n, true));
    launch_head_loss(n, n, NOUTP, s->zout.as<float>(), dt.as<float>(), dsig.as<float>(), s->d_diag.as<uint8_t>(),
                     s->dz.as<__nv_bfloat16>(), s->loss.as<float>(), st);
    RVE_TRY(backward_step(s, member, n, 1, 0.f, grads));
    float l = 0;
    RVE_CUDA(cudaMemcpyAsync(&l, s->loss.p, 4, cudaMemcpyDeviceToHost, st));
    RVE_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = l;
    if (gemm_tc_timed_out()) {
        set_error("a bounded wait inside the surrogate GEMM gave up");
        return RVE_ERR_TIMEOUT;
    }
    return RVE_OK;
}

// Ensemble prediction on device features: member tensors, mean and spread.
static int predict_dev(rve_surrogate s, int64_t n, const double* feat_dev, double* C_dev, double* K_dev,
                       double* D_dev, double* spread_dev) {
    NvtxRange nvtx_("surrogate inference: %lld points, %d members", (long long)n, s->members);
    cudaStream_t st = s->ctx->stream;
    const int64_t chunk = 65536;
    RVE_TRY(alloc_work(s, (int)chunk));
    RVE_TRY(s->Tmem.ensure((size_t)s->members * chunk * 54 * 4));
    const bool use_fused = s->fused && s->members <= mlp_fused_max_members();
    std::vector<const __nv_bfloat16*> wt;
    std::vector<const float*> bias;
    int64_t w_off[NLAYER];
    if (use_fused) {
        RVE_TRY(s->zall.ensure((size_t)s->members * 64 * chunk * 4));
        for (int l = 0; l < NLAYER; ++l) w_off[l] = layer_w_off(l);
        for (int e = 0; e < s->members; ++e) {
            wt.push_back(s->Wt[e].as<__nv_bfloat16>());
            for (int l = 0; l < NLAYER; ++l)
                bias.push_back(s->P[e].as<float>() + layer_w_off(l) + (int64_t)LK[l] * LN[l]);
        }
    }
    DevBuf dmean, dstd;
    std::vector<float> fis(8);
    for (int k = 0; k < 8; ++k) fis[k] = 1.f / s->feat_std[k];
    RVE_TRY(upload(dmean, s->feat_mean, 8, st));
    RVE_TRY(upload(dstd, fis.data(), 8, st));
    for (int64_t off = 0; off < n; off += chunk) {
        const int nn = (int)std::min<int64_t>(chunk, n - off);
        const int M = ((nn + 63) / 64) * 64;
        launch_features(nn, M, KIN, feat_dev + off * 8, dmean.as<float>(), dstd.as<float>(),
                        s->H[0].as<__nv_bfloat16>(), st);
        if (use_fused) {
            RVE_CUDA(launch_mlp_fused(M, s->members, s->H[0].as<__nv_bfloat16>(), wt.data(), w_off,
                                      bias.data(), s->zall.as<float>(), M, st));
            s->ctx->launches += 1;
        }
        for (int e = 0; e < s->members; ++e) {
            const float* zT = s->zout.as<float>();
            if (use_fused)
                zT = s->zall.as<float>() + (size_t)e * 64 * M;
            else
                RVE_TRY(forward(s, e, M, false, true));
            launch_head_tensors(nn, M, zT, s->d_diag.as<uint8_t>(), s->Tmem.as<float>() + (size_t)e * nn * 54, st);
        }
        launch_ensemble(nn, s->members, s->Tmem.as<float>(), s->ref[0], s->ref[1], s->ref[2], C_dev + off * 36,
                        K_dev + off * 9, D_dev + off * 9, spread_dev + off, st);
        s->ctx->launches += 2 + s->members;
    }
    RVE_CUDA(cudaGetLastError());
    return RVE_OK;
}

int rve_surrogate_predict(rve_ctx c, rve_surrogate s, int64_t n, const double* feat, double* C, double* K,
                          double* D, double* spread) {
    RVE_TRY(check_ctx(c));
    if (!s || n < 0 || (n > 0 && (!feat || !C || !K || !D || !spread))) return RVE_ERR_INVALID_ARGUMENT;
    if (!s->trained) {
        set_error("surrogate has not been trained or loaded");
        return RVE_ERR_STATE;
    }
    if (n == 0) return RVE_OK;
    cudaStream_t st = c->stream;
    DevBuf df, dC, dK, dD, dsp;
    RVE_TRY(upload(df, feat, (size_t)n * 8, st));
    RVE_TRY(dC.ensure((size_t)n * 36 * 8));
    RVE_TRY(dK.ensure((size_t)n * 9 * 8));
    RVE_TRY(dD.ensure((size_t)n * 9 * 8));
    RVE_TRY(dsp.ensure((size_t)n * 8));
    RVE_TRY(predict_dev(s, n, df.as<double>(), dC.as<double>(), dK.as<double>(), dD.as<double>(),
                        dsp.as<double>()));
    RVE_CUDA(cudaMemcpyAsync(C, dC.p, (size_t)n * 36 * 8, cudaMemcpyDeviceToHost, st));
    RVE_CUDA(cudaMemcpyAsync(K, dK.p, (size_t)n * 9 * 8, cudaMemcpyDeviceToHost, st));
    RVE_CUDA(cudaMemcpyAsync(D, dD.p, (size_t)n * 9 * 8, cudaMemcpyDeviceToHost, st));
    RVE_CUDA(cudaMemcpyAsync(spread, dsp.p, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    RVE_CUDA(cudaStreamSynchronize(st));
    if (gemm_tc_timed_out()) {
        set_error("a bounded wait inside the surrogate GEMM gave up");
        return RVE_ERR_TIMEOUT;
    }
    return RVE_OK;
}

int rve_surrogate_set_fused(rve_ctx c, rve_surrogate s, int fused) {
    RVE_TRY(check_ctx(c));
    if (!s) return RVE_ERR_INVALID_ARGUMENT;
    s->fused = fused != 0;
    return RVE_OK;
}

int rve_surrogate_predict_dev(rve_ctx c, rve_surrogate s, int64_t n, const double* feat_dev, double* C_dev,
                              double* K_dev, double* D_dev, double* spread_dev) {
    RVE_TRY(check_ctx(c));
    if (!s || n < 0 || (n > 0 && (!feat_dev || !C_dev || !K_dev || !D_dev || !spread_dev)))
        return RVE_ERR_INVALID_ARGUMENT;
    if (!s->trained) {
        set_error("surrogate has not been trained or loaded");
        return RVE_ERR_STATE;
    }
    if (n == 0) return RVE_OK;
    RVE_TRY(predict_dev(s, n, feat_dev, C_dev, K_dev, D_dev, spread_dev));
    RVE_CUDA(cudaGetLastError());
    return RVE_OK;
}

int rve_surrogate_get_params(rve_ctx c, rve_surrogate s, float* buf, int64_t* len) {
    RVE_TRY(check_ctx(c));
    if (!s || !len) return RVE_ERR_INVALID_ARGUMENT;
    const int64_t np = n_params();
    const int64_t need = HEADER + (int64_t)s->members * np;
    if (!buf) {
        *len = need;
        return RVE_OK;
    }
    if (*len < need) return RVE_ERR_INVALID_ARGUMENT;
    std::memcpy(buf, s->feat_mean, 32);
    std::memcpy(buf + 8, s->feat_std, 32);
    std::memcpy(buf + 16, s->sigma, 33 * 4);
    for (int b = 0; b < 3; ++b) buf[49 + b] = (float)s->ref[b];
    for (int e = 0; e < s->members; ++e)
        RVE_CUDA(cudaMemcpyAsync(buf + HEADER + e * np, s->P[e].p, np * 4, cudaMemcpyDeviceToHost, c->stream));
    RVE_CUDA(cudaStreamSynchronize(c->stream));
    *len = need;
    return RVE_OK;
}

int rve_surrogate_set_params(rve_ctx c, rve_surrogate s, const float* buf, int64_t len) {
    RVE_TRY(check_ctx(c));
    const int64_t np = n_params();
    if (!s || !buf || len != HEADER + (int64_t)s->members * np) {
        set_error("rve_surrogate_set_params: length does not match the ensemble size");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    std::memcpy(s->feat_mean, buf, 32);
    std::memcpy(s->feat_std, buf + 8, 32);
    std::memcpy(s->sigma, buf + 16, 33 * 4);
    for (int b = 0; b < 3; ++b) s->ref[b] = buf[49 + b];
    for (int e = 0; e < s->members; ++e) {
        RVE_CUDA(cudaMemcpyAsync(s->P[e].p, buf + HEADER + e * np, np * 4, cudaMemcpyHostToDevice, c->stream));
        RVE_TRY(refresh_bf16(s, e));
    }
    RVE_CUDA(cudaStreamSynchronize(c->stream));
    s->trained = true;
    return RVE_OK;
}

int macro_update_gauss_points_surrogate(rve_ctx c, const rve_mesh* meshes, const rve_surrogate* surrogates,
                                        int n_meshes, double tau, int64_t G, const double* T_C,
                                        const double* c_wt, const double* t_h, const int32_t* mesh_id,
                                        double* C, double* K, double* D, int32_t* status, uint8_t* fallback,
                                        rve_stats* st) {
    RVE_TRY(check_ctx(c));
    if (!meshes || !surrogates || n_meshes <= 0 || G < 0 || !(tau >= 0) ||
        (G > 0 && (!T_C || !c_wt || !t_h || !mesh_id || !C || !K || !D || !status || !fallback))) {
        set_error("macro_update_gauss_points_surrogate: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    auto t0 = std::chrono::steady_clock::now();
    const int64_t l0 = c->launches;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->converged = 1;
    }
    cudaStream_t s = c->stream;
    std::vector<std::vector<int64_t>> groups(n_meshes);
    for (int64_t g = 0; g < G; ++g) {
        if (mesh_id[g] < 0 || mesh_id[g] >= n_meshes) return RVE_ERR_INVALID_ARGUMENT;
        groups[mesh_id[g]].push_back(g);
    }
    std::vector<int64_t> fb_idx;
    std::vector<int32_t> fb_mesh;
    for (int mi = 0; mi < n_meshes; ++mi) {
        auto& grp = groups[mi];
        if (grp.empty()) continue;
        rve_surrogate sg = surrogates[mi];
        if (!sg || !sg->trained) {
            for (auto g : grp) {
                fb_idx.push_back(g);
                fb_mesh.push_back(mi);
            }
            continue;
        }
        const int64_t n = (int64_t)grp.size();
        std::vector<double> T(n), cc(n), tt(n), feat((size_t)n * 8);
        for (int64_t i = 0; i < n; ++i) {
            T[i] = T_C[grp[i]];
            cc[i] = c_wt[grp[i]];
            tt[i] = t_h[grp[i]];
        }
        RVE_TRY(rve_gauss_point_features(c, meshes[mi], n, T.data(), cc.data(), tt.data(), feat.data()));
        std::vector<double> Cp((size_t)n * 36), Kp((size_t)n * 9), Dp((size_t)n * 9), spr(n);
        RVE_TRY(rve_surrogate_predict(c, sg, n, feat.data(), Cp.data(), Kp.data(), Dp.data(), spr.data()));
        for (int64_t i = 0; i < n; ++i) {
            const int64_t g = grp[i];
            if (!(spr[i] <= tau)) {
                fb_idx.push_back(g);
                fb_mesh.push_back(mi);
                continue;
            }
            std::memcpy(C + 36 * g, &Cp[36 * i], 36 * 8);
            std::memcpy(K + 9 * g, &Kp[9 * i], 9 * 8);
            std::memcpy(D + 9 * g, &Dp[9 * i], 9 * 8);
            status[g] = RVE_OK;
            fallback[g] = 0;
        }
    }
    int rc = RVE_OK;
    if (!fb_idx.empty()) {
        const int64_t nf = (int64_t)fb_idx.size();
        std::vector<double> T(nf), cc(nf), tt(nf), Cf((size_t)nf * 36), Kf((size_t)nf * 9), Df((size_t)nf * 9);
        std::vector<int32_t> sf(nf);
        for (int64_t i = 0; i < nf; ++i) {
            T[i] = T_C[fb_idx[i]];
            cc[i] = c_wt[fb_idx[i]];
            tt[i] = t_h[fb_idx[i]];
        }
        rve_stats fs;
        rc = macro_update_gauss_points(c, meshes, n_meshes, nf, T.data(), cc.data(), tt.data(), fb_mesh.data(),
                                       Cf.data(), Kf.data(), Df.data(), sf.data(), RVE_MODE_PCG, &fs);
        if (rc != RVE_OK && rc != RVE_ERR_NOT_CONVERGED && rc != RVE_ERR_NUMERIC) return rc;
        for (int64_t i = 0; i < nf; ++i) {
            const int64_t g = fb_idx[i];
            std::memcpy(C + 36 * g, &Cf[36 * i], 36 * 8);
            std::memcpy(K + 9 * g, &Kf[9 * i], 9 * 8);
            std::memcpy(D + 9 * g, &Df[9 * i], 9 * 8);
            status[g] = sf[i];
            fallback[g] = 1;
        }
        if (st) {
            *st = fs;
        }
    }
    if (st) {
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        st->kernel_launches = c->launches - l0;
    }
    if (gemm_tc_timed_out()) {
        set_error("a bounded wait inside the surrogate GEMM gave up");
        return RVE_ERR_TIMEOUT;
    }
    return rc;
}

}  // extern "C"
