// Internal definitions shared by the host files of the C ABI (api.cu,
// surrogate_api.cu): device buffers, handles and error macros.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "rve_internal.h"

#define RVE_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::rve::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
            return e_ == cudaErrorMemoryAllocation ? RVE_ERR_OUT_OF_MEMORY : RVE_ERR_CUDA; \
        }                                                                                \
    } while (0)

#define RVE_TRY(call)                  \
    do {                               \
        int rc_ = (call);              \
        if (rc_ != RVE_OK) return rc_; \
    } while (0)

namespace rve {

const std::string& last_error();

// NVTX range over a host scope (header-only NVTX v3: a no-op unless a profiler is
// attached); the name is printf-formatted.
struct NvtxRange {
    explicit NvtxRange(const char* fmt, ...) {
        char buf[128];
        va_list ap;
        va_start(ap, fmt);
        std::vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------ device buffer
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) {
        o.p = nullptr;
        o.bytes = 0;
    }
    void swap(DevBuf& o) noexcept {
        void* tp = p;
        p = o.p;
        o.p = tp;
        const size_t tb = bytes;
        bytes = o.bytes;
        o.bytes = tb;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int ensure(size_t b) {
        if (b <= bytes && p) return RVE_OK;
        release();
        if (b == 0) b = 16;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
            return RVE_ERR_OUT_OF_MEMORY;
        }
        bytes = b;
        return RVE_OK;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

template <typename T>
inline int upload(DevBuf& d, const T* h, size_t n, cudaStream_t s) {
    RVE_TRY(d.ensure(n * sizeof(T)));
    if (n) RVE_CUDA(cudaMemcpyAsync(d.p, h, n * sizeof(T), cudaMemcpyHostToDevice, s));
    return RVE_OK;
}

// Constraint rows and preconditioner data of one field on the current BC.
struct FieldDev {
    int nc = 3;
    int nfield = 1;
    int64_t n_rows = 0;
    DevBuf diag64, diag32, mask;
    int m = 0;
    int64_t n_sup = 0;
    DevBuf sup_row, sup_coef, sup_of_row;
    std::vector<int64_t> h_sup_row;   // host copies of the rows (the multiplier route's D = C X)
    std::vector<double> h_sup_coef;
};

}  // namespace rve

namespace rve {
// Profile-mode counters of a context (summed device times from CUDA events and the
// algorithmic bytes / flops of the timed launches).  Operator classes are indexed
// by 2 (p - 1) + (scalar field ? 1 : 0).
// Result of one field's solve over a batch of B RVEs.
struct SolveOut {
    std::vector<double> tensor;    // [B][6][6] energy form (internal units)
    std::vector<double> sig;       // [B][6][6] sigma form (diagnostic)
    int iterations = 0;
    int sweeps = 0;
    bool converged = true;
    double rel_res = 0;
    bool numeric = false;
    bool timeout = false;   // a bounded device wait gave up
};

struct ProfCounters {
    double op_ms = 0, op_bytes = 0, op_flops = 0, op_cols = 0, op_cols_all = 0;
    int64_t op_launches = 0;
    double upd_ms = 0, upd_bytes = 0, pup_ms = 0, pup_bytes = 0, fin_ms = 0;
    double res_ms = 0;
    int64_t res_launches = 0;
    double graph_host_ms = 0;   // host time capturing and instantiating PCG graphs (always counted)
    int64_t graphs = 0;
    double cls_ms[6] = {}, cls_bytes[6] = {}, cls_flops[6] = {}, cls_cols[6] = {}, cls_cols_all[6] = {};
    int64_t cls_launches[6] = {};
};
}  // namespace rve

struct rve_ctx_s {
    rve_options opt;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;   // private stream used only to capture graphs
    bool own_stream = false;
    int device = 0;
    std::atomic<int64_t> launches{0};
    // profile mode: event pairs around every operator launch of a captured body
    std::vector<cudaEvent_t> ev;
    rve::ProfCounters prof;
    std::mutex prof_mu;   // guards prof against the batched call's per-mesh threads
    ~rve_ctx_s() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

struct rve_mesh_s {
    rve_ctx ctx = nullptr;
    // the mesh's own streams, used (on_own_streams) only while the batched call
    // solves several meshes concurrently, one host thread per mesh; every other
    // call runs on the context's streams
    cudaStream_t stream = nullptr, capture = nullptr;
    bool on_own_streams = false;
    // instantiated PCG iteration graphs per field and precision, reused while the
    // captured launch parameters (kept as raw bytes in key) stay the same
    struct GraphCache {
        cudaGraphExec_t exec = nullptr;
        std::vector<unsigned char> key;
    } graph_cache[2][2];
    ~rve_mesh_s() {
        for (auto& row : graph_cache)
            for (auto& g : row)
                if (g.exec) cudaGraphExecDestroy(g.exec);
        if (stream) cudaStreamDestroy(stream);
        if (capture) cudaStreamDestroy(capture);
    }
    int p = 1;
    int bc = RVE_BC_DIRICHLET;
    int64_t nv = 0, nt = 0;
    std::vector<double> xyz;
    std::vector<int32_t> tets;
    std::vector<uint8_t> phase;
    std::vector<double> tangent;
    rve::DofMap map;
    double volume = 0;
    // device mesh
    rve::DevBuf d_xyz, d_edofs, d_lverts, d_geo64, d_geo32, d_phase, d_tangent, d_flag;
    rve::DevBuf d_matm64, d_matm32, d_mats64, d_mats32;
    // tensor-core operator: packed FP32 element matrices of the mechanics (formed lazily,
    // invalidated whenever the DOF map or the materials change) and their index tables
    rve::DevBuf d_ke32, d_kepairs, d_keptab;
    bool ke_valid = false;
    // element colouring of the current DOF map (no two elements of a colour share a
    // DOF): elements sorted by colour on the device, colour offsets on the host
    rve::DevBuf d_colour_elems;
    std::vector<int64_t> colour_off;
    int ncolour = 0;
    // checking build: DOF-index bound the kernels test against (0: the map's own count)
    int64_t debug_node_bound = 0;
    rve::FieldDev mech, scal;
    bool have_materials = false;
    int tuned_batch = 0;   // batch size chosen by rve_autotune_batch (0: the built-in rule)
    int tuned_kernel = 0;  // operator kernel chosen by rve_autotune_schedule (0: not tuned)
    // batched call: the scalar-field solution of this mesh (independent of the
    // degradation state), formed by the call's first batch of the mesh
    bool scal_cached = false;
    rve::SolveOut scal_out;
    // per phase: sum over its tets of |T| times the diagonal of D (6, mechanics) and of
    // k (3) and d (3), internal units; the energy scale of each unit load case
    double phase_voigt[2][12] = {};
    rve::MaterialConsts mc{};
    rve_degradation deg{};
    double T_C = 20, c_wt = 0, t_h = 0;
    // solve workspace
    // FP64 solution and residual per field (mechanics, scalar); swapped with the
    // warm-start buffers after a batch instead of copied
    rve::DevBuf x64f[2], r64f[2];
    rve::DevBuf b64, p64, q64, x32, r32, p32, q32;
    rve::DevBuf epart, rzp, cpart, gpart, mpart, gsum, msum;
    rve::DevBuf colstate, scale64, scale32, wdev, coltol;
    // warm start: the previous batch's FP64 solutions per field and their factors
    rve::DevBuf warm[2], warm_r[2], warm_map, warm_coef, warm_dcoef;
    // energy-optimal warm start: source list, one-hot map of the compact source copy,
    // the phase scales of the product pass (FP32 and negated FP64), the sources (FP64 and
    // split into FP32 high and low words), minus the degraded and the other phases'
    // products of them (FP64 plus FP32 low words), their inner products, and the column
    // map of r0 into the products
    rve::DevBuf warm_src, warm_omap, warm_ocoef, warm_ksc, warm_phs, warm_xs64, warm_xs, warm_kx, warm_klo, warm_gram,
        warm_kxmap;
    rve::DevBuf dscale32, dscale64;   // per-column phase scales of the warm-start residual
    // per field: K_ph u_macro for each phase at unit modulus, [2][n_rows][6] (FP64),
    // so that a batch's right-hand side is a per-column combination of them
    rve::DevBuf bph[2];
    bool bph_valid[2] = {false, false};
    int bph_prec[2] = {0, 0};         // precision the cached loads were formed in
    int warm_cols[2] = {0, 0};
    std::vector<double> warm_w[2];
};

namespace rve {
// Batched PCG homogenisation of B RVEs of one mesh (degradation factors d_w on
// the device); host outputs C [B][36], K [B][9], D [B][9] (any may be null).
// w_host (optional, [B]) enables the warm start from the mesh's previous batch
// (see macro_update_gauss_points); the batch's solutions become the next start.
int homogenise_batch(rve_mesh m, int B, const double* d_w, double* C, double* K, double* D, rve_stats* st,
                     const double* w_host = nullptr);
int check_ctx(rve_ctx c);
}  // namespace rve
