// Low-rank block times a panel, y = U (V^T x), without any device allocation.
//
// For callers that must not allocate device memory at the time of the call:
// code running where cudaMalloc is not allowed or not wanted (a fixed memory
// budget handed out in advance, a real-time loop that must not stall in the
// allocator, a plug-in that does not own the device's memory).  The k x nrhs
// intermediate V^T x, which the library's matrix-vector product keeps in the
// arena that hlu_create allocated, lives here in one fixed array in device
// memory that belongs to the library and exists on every GPU that loads it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hlu.h"

namespace {

// Largest k * nrhs the entry point accepts: 65536 doubles = 512 KiB.
constexpr int64_t kStaticScratchDoubles = int64_t(1) << 16;

// The scratch array.  Its name is only a host-side handle: device code may use
// it directly, host code must pass the address obtained from
// cudaGetSymbolAddress on the device in question.
static __device__ __align__(256) double g_lowrank_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).  Returns nullptr on failure.
double *scratch_on_current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lowrank_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    return g_scratch_addr[dev];
}

// T (k x nrhs, zeroed by the caller) += V[rows]^T x[rows] over this CTA's row range.
__global__ void k_project_rows(const double *V, int64_t ldv, const double *x, int64_t ldx, int n, int k, int nrhs,
                               int rows_per_cta, double *T) {
    const int r0 = blockIdx.x * rows_per_cta;
    const int r1 = min(n, r0 + rows_per_cta);
    for (int p = threadIdx.x; p < k * nrhs; p += blockDim.x) {
        const int a = p % k, j = p / k;
        double s = 0.0;
        for (int r = r0; r < r1; ++r) s += V[r + a * ldv] * x[r + j * ldx];
        atomicAdd(T + p, s);
    }
}

// y (m x nrhs) = U (m x k) T (k x nrhs)
__global__ void k_apply_rows(const double *U, int64_t ldu, const double *T, int m, int k, int nrhs, double *y,
                             int64_t ldy) {
    const int64_t tot = (int64_t)m * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = int(e % m), j = int(e / m);
        double s = 0.0;
        for (int a = 0; a < k; ++a) s += U[i + a * ldu] * T[a + (int64_t)j * k];
        y[i + j * ldy] = s;
    }
}

}  // namespace

extern "C" int hlu_lowrank_apply_noalloc(int32_t m, int32_t n, int32_t k, int32_t nrhs, const double *U, int64_t ldu,
                                         const double *V, int64_t ldv, const double *x, int64_t ldx, double *y,
                                         int64_t ldy, void *cuda_stream) {
    if (m < 0 || n < 0 || k < 0 || nrhs < 0) return HLU_EINVAL;
    if ((int64_t)k * nrhs > kStaticScratchDoubles) return HLU_EINVAL;  // beyond the fixed scratch array
    if (m == 0 || nrhs == 0) return HLU_OK;
    if (!y || ldy < m) return HLU_EINVAL;
    if (k > 0 && (!U || !V || !x || ldu < m || ldv < n || ldx < n)) return HLU_EINVAL;
    double *T = scratch_on_current_device();
    if (!T) return HLU_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    // the array keeps the previous call's values: the accumulator starts from zero
    if (k > 0 && cudaMemsetAsync(T, 0, sizeof(double) * (size_t)k * nrhs, s) != cudaSuccess) return HLU_ECUDA;
    if (k > 0 && n > 0) {
        const int rows_per_cta = 256;
        const int grid = (n + rows_per_cta - 1) / rows_per_cta;
        k_project_rows<<<grid, 256, 0, s>>>(V, ldv, x, ldx, n, k, nrhs, rows_per_cta, T);
    }
    const int64_t tot = (int64_t)m * nrhs;
    const int grid = (int)((tot + 255) / 256 < 1024 ? (tot + 255) / 256 : 1024);
    k_apply_rows<<<grid, 256, 0, s>>>(U, ldu, T, m, k, nrhs, y, ldy);
    return cudaGetLastError() == cudaSuccess ? HLU_OK : HLU_ECUDA;
}
