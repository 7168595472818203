// Device kernels of the restarted GMRES(m) solver (Saad and Schultz 1986), in FP64, right-preconditioned
// by the H-LU solve.  All right-hand sides advance in lockstep; every column c of a panel (n rows,
// leading dimension n) is an independent system.  Basis vectors i of a family are panels at
// base + i * stride.  Every reduction has a fixed order (one block per output), so the iteration is
// deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include "gmres.cuh"

namespace hlu {

namespace {

constexpr int kGmThreads = 256;

__device__ __forceinline__ double gm_warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out[c * ld + i] = (X_i[:, c], Y[:, c]) for i < k (blockIdx.x), c < ncol (blockIdx.y).
__global__ void __launch_bounds__(kGmThreads) k_gm_dots(const double *X, int64_t xs, const double *Y, int64_t n,
                                                         double *out, int ld) {
    __shared__ double red[kGmThreads / 32];
    const int i = blockIdx.x, c = blockIdx.y;
    const double *x = X + i * xs + c * n, *y = Y + c * n;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += kGmThreads) s = fma(x[r], y[r], s);
    s = gm_warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kGmThreads / 32 ? red[threadIdx.x] : 0.0;
        s = gm_warp_sum(s);
        if (threadIdx.x == 0) out[c * ld + i] = s;
    }
}

// Y[:, c] += alpha * sum_{i < k} h[c * ld + i] X_i[:, c].
__global__ void k_gm_axpy(const double *X, int64_t xs, int k, const double *h, int ld, double alpha, double *Y,
                          int64_t n, int ncol) {
    const int64_t tot = n * ncol;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const int64_t r = e - (int64_t)c * n;
        const double *hc = h + c * ld;
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(hc[i], X[i * xs + c * n + r], s);
        Y[e] = fma(alpha, s, Y[e]);
    }
}

// Y[:, c] = X[:, c] * f[c].
__global__ void k_gm_scale(const double *X, const double *f, double *Y, int64_t n, int ncol) {
    const int64_t tot = n * ncol;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
        Y[e] = X[e] * f[e / n];
}

// Start of a cycle, one thread per column: beta = sqrt(nrm2), g = beta e_1, inv = 1 / beta (0 for beta = 0).
__global__ void k_gm_start(const double *nrm2, GmState s, int ncol) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const int m = s.m;
    const double beta = sqrt(nrm2[c]);
    double *g = s.g + c * (m + 1);
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    s.inv[c] = beta > 0.0 ? 1.0 / beta : 0.0;
    s.est[c] = beta;
}

// Step j of the Arnoldi process, one thread per column: H[0..j, j] = t1 + t2 (the two classical
// Gram-Schmidt passes), H[j+1, j] = |w|; the previous Givens rotations are applied to the new column,
// a new rotation zeroes H[j+1, j]; g is rotated and |g[j+1]| is the residual norm of the current
// iterate (Saad's estimate).  inv = 1 / H[j+1, j], or 0 on breakdown (w = 0: the Krylov space is
// invariant and the estimate is exact).
__global__ void k_gm_arnoldi(const double *t1, const double *t2, const double *nrm2, GmState s, int j, int ncol) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const int m = s.m, ld = m + 1;
    double *col = s.H + (int64_t)c * ld * m + (int64_t)j * ld;
    double *cs = s.cs + c * m, *sn = s.sn + c * m, *g = s.g + c * ld;
    for (int i = 0; i <= j; ++i) col[i] = t1[c * ld + i] + t2[c * ld + i];
    const double hn = sqrt(nrm2[c]);
    col[j + 1] = hn;
    s.inv[c] = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    const double a = col[j], b = col[j + 1];
    const double rr = hypot(a, b);
    const double cj = rr > 0.0 ? a / rr : 1.0, sj = rr > 0.0 ? b / rr : 0.0;
    cs[j] = cj;
    sn[j] = sj;
    col[j] = rr;
    col[j + 1] = 0.0;
    g[j + 1] = -sj * g[j];
    g[j] = cj * g[j];
    s.est[c] = fabs(g[j + 1]);
}

// y = R^{-1} g[0..k) by back substitution (R: the rotated k x k Hessenberg, upper triangular), one
// thread per column; y goes to y[c * (m + 1) + i].  A zero pivot (exact breakdown before step k)
// gives y_i = 0 for that and the later directions, which do not exist.
__global__ void k_gm_hsolve(GmState s, int k, double *y, int ncol) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const int m = s.m, ld = m + 1;
    const double *Hc = s.H + (int64_t)c * ld * m, *g = s.g + c * ld;
    double *yc = y + c * ld;
    for (int i = k - 1; i >= 0; --i) {
        double v = g[i];
        for (int l = i + 1; l < k; ++l) v -= Hc[i + (int64_t)l * ld] * yc[l];
        const double d = Hc[i + (int64_t)i * ld];
        yc[i] = d != 0.0 ? v / d : 0.0;
    }
}

int grid_for(int64_t tot) {
    int64_t b = (tot + kGmThreads - 1) / kGmThreads;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

}  // namespace

void gm_dots(const double *X, int64_t xs, int k, const double *Y, int64_t n, int ncol, double *out, int ld,
             cudaStream_t st) {
    if (k > 0 && ncol > 0) k_gm_dots<<<dim3(k, ncol), kGmThreads, 0, st>>>(X, xs, Y, n, out, ld);
}

void gm_axpy(const double *X, int64_t xs, int k, const double *h, int ld, double alpha, double *Y, int64_t n,
             int ncol, cudaStream_t st) {
    if (k > 0 && ncol > 0) k_gm_axpy<<<grid_for(n * ncol), kGmThreads, 0, st>>>(X, xs, k, h, ld, alpha, Y, n, ncol);
}

void gm_scale(const double *X, const double *f, double *Y, int64_t n, int ncol, cudaStream_t st) {
    if (ncol > 0) k_gm_scale<<<grid_for(n * ncol), kGmThreads, 0, st>>>(X, f, Y, n, ncol);
}

void gm_start(const double *nrm2, const GmState &s, int ncol, cudaStream_t st) {
    k_gm_start<<<(ncol + 63) / 64, 64, 0, st>>>(nrm2, s, ncol);
}

void gm_arnoldi(const double *t1, const double *t2, const double *nrm2, const GmState &s, int j, int ncol,
                cudaStream_t st) {
    k_gm_arnoldi<<<(ncol + 63) / 64, 64, 0, st>>>(t1, t2, nrm2, s, j, ncol);
}

void gm_hsolve(const GmState &s, int k, double *y, int ncol, cudaStream_t st) {
    k_gm_hsolve<<<(ncol + 63) / 64, 64, 0, st>>>(s, k, y, ncol);
}

}  // namespace hlu
