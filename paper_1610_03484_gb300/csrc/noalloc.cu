// Scratch memory for the allocation-free operator entry point.
//
// The array below is the only scratch that rve_operator_energy_noalloc uses.
// It is a file-scope __device__ array, so every GPU that loads librve holds it
// (about 0.9 MB) until the process exits.  In host code its name is only a
// host-side stand-in; the device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"

namespace rve {

// per-block partial energies [nby][ncols] followed by the column scales [ncols][2]
constexpr int kNoAllocMaxCols = 96;
constexpr int kNoAllocMaxBlocksY = 1216;
constexpr size_t kNoAllocDoubles =
    (size_t)kNoAllocMaxBlocksY * kNoAllocMaxCols + (size_t)kNoAllocMaxCols * 2;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

int noalloc_max_cols() { return kNoAllocMaxCols; }
int noalloc_max_blocks_y() { return kNoAllocMaxBlocksY; }

// Device address of the scratch array on the current device (looked up once
// per device).  Returns nullptr and the CUDA error on failure.
double* noalloc_scratch(int device, cudaError_t* err) {
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    *err = cudaSuccess;
    if (device < 0 || device >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        addr[device] = static_cast<double*>(p);
    }
    return addr[device];
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}
__global__ void k_scale(int64_t n, double v, double* __restrict__ a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] *= v;
}

// y[row][col] *= (col % 6 < 3 ? f_lo : f_hi)
__global__ void k_scale_cols(int64_t n_rows, int ncols, double f_lo, double f_hi, double* __restrict__ y) {
    const int64_t n = n_rows * ncols;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] *= ((i % ncols) % 6) < 3 ? f_lo : f_hi;
}

void launch_scale_cols(int64_t n_rows, int ncols, double f_lo, double f_hi, double* y, cudaStream_t s) {
    int64_t b = (n_rows * ncols + 255) / 256;
    if (b > 2432) b = 2432;
    if (b < 1) b = 1;
    k_scale_cols<<<(unsigned)b, 256, 0, s>>>(n_rows, ncols, f_lo, f_hi, y);
}

void launch_fill(int64_t n, double v, double* a, cudaStream_t s) {
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, v, a);
}
void launch_scale(int64_t n, double v, double* a, cudaStream_t s) {
    int64_t b = (n + 255) / 256;
    if (b > 2432) b = 2432;
    if (b < 1) b = 1;
    k_scale<<<(unsigned)b, 256, 0, s>>>(n, v, a);
}

}  // namespace rve
