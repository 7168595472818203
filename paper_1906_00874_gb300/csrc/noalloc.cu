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

#include "../../include/hlu.h"

namespace {

// Largest k * nrhs the entry point accepts: 65536 doubles = 512 KiB.
constexpr int64_t kStaticScratchDoubles = int64_t(1) << 16;

// The scratch array.  Its name is only a host-side handle: device code may use
// it directly, host code must pass the address obtained from
// cudaGetSymbolAddress on the device in question.
static __device__ __align__(256) double g_lowrank_scratch[kStaticScratchDoubles];

// Device address of the scratch array in the current device's context, looked
// up on every call (a cheap query once the module is loaded), so that an
// address never outlives the context it belongs to (cudaDeviceReset, a new
// primary context).  The first lookup on a device loads the library's module
// there, which is why the first call on a device must come before any stream
// capture.  Returns nullptr on failure.
double *scratch_on_current_device() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lowrank_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<double *>(p);
}

// T (k x nrhs, zeroed before the launch) += V[rows]^T x[rows].  CTA (bx, by,
// bz) takes rows [128 bx, 128 bx + 128), the 16 columns a0 = 16 by of V and the
// 16 columns j0 = 16 bz of x: both 128 x 16 slices are staged in shared memory
// by coalesced loads (consecutive threads read consecutive rows of a column),
// then thread t forms output (a0 + t % 16, j0 + t / 16) over the staged rows
// and adds it to T with one atomicAdd per CTA and output.
constexpr int kRowsPerCta = 128, kTile = 16;

__global__ void __launch_bounds__(256) k_project_rows(const double *V, int64_t ldv, const double *x, int64_t ldx,
                                                      int n, int k, int nrhs, double *T) {
    __shared__ double sV[kTile][kRowsPerCta + 1], sX[kTile][kRowsPerCta + 1];
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerCta;
    const int a0 = blockIdx.y * kTile, j0 = blockIdx.z * kTile;
    const int64_t left = (int64_t)n - r0;
    const int rows = left < kRowsPerCta ? (int)left : kRowsPerCta;
    const int ta = min(kTile, k - a0), tj = min(kTile, nrhs - j0);
    for (int e = threadIdx.x; e < kTile * kRowsPerCta; e += blockDim.x) {
        const int c = e / kRowsPerCta, i = e - c * kRowsPerCta;
        sV[c][i] = (c < ta && i < rows) ? V[r0 + i + (int64_t)(a0 + c) * ldv] : 0.0;
        sX[c][i] = (c < tj && i < rows) ? x[r0 + i + (int64_t)(j0 + c) * ldx] : 0.0;
    }
    __syncthreads();
    const int ca = threadIdx.x % kTile, cj = threadIdx.x / kTile;
    if (ca < ta && cj < tj) {
        double s = 0.0;
        for (int i = 0; i < rows; ++i) s = fma(sV[ca][i], sX[cj][i], s);
        atomicAdd(T + (a0 + ca) + (int64_t)(j0 + cj) * k, s);
    }
}

// y (m x nrhs) = U (m x k) T (k x nrhs); consecutive threads take consecutive rows (coalesced U and y).
__global__ void k_apply_rows(const double *U, int64_t ldu, const double *T, int m, int k, int nrhs, double *y,
                             int64_t ldy) {
    const int64_t tot = (int64_t)m * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % m, j = e / m;
        double s = 0.0;
        for (int a = 0; a < k; ++a) s = fma(U[i + a * ldu], T[a + j * k], s);
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
    // the array keeps the previous call's values: the accumulator starts from zero (k = 0: y = 0 below)
    if (k > 0 && cudaMemsetAsync(T, 0, sizeof(double) * (size_t)k * nrhs, s) != cudaSuccess) return HLU_ECUDA;
    if (k > 0 && n > 0) {
        const int64_t gx = ((int64_t)n + kRowsPerCta - 1) / kRowsPerCta;  // <= 2^24 for int32 n
        const dim3 grid((unsigned)gx, (unsigned)((k + kTile - 1) / kTile), (unsigned)((nrhs + kTile - 1) / kTile));
        k_project_rows<<<grid, 256, 0, s>>>(V, ldv, x, ldx, n, k, nrhs, T);
    }
    const int64_t tot = (int64_t)m * nrhs;
    const int grid = (int)((tot + 255) / 256 < 1216 ? (tot + 255) / 256 : 1216);
    k_apply_rows<<<grid, 256, 0, s>>>(U, ldu, T, m, k, nrhs, y, ldy);
    return cudaGetLastError() == cudaSuccess ? HLU_OK : HLU_ECUDA;
}
