// Factorisation error E_fac = ||A_H - L U||_2 / ||A_H||_2 of a factorised handle, estimated on the
// device by power iteration on M^T M (M = A_H - L U, and A_H alone for the denominator), with M
// applied through the leaves of the block structure and never formed.
//
// The factors overwrite the working copy of A_H leaf by leaf (Sec. 3.1): a leaf (t, s) with
// begin(t) < begin(s) belongs to U, one with begin(t) > begin(s) to L, and a diagonal leaf holds
// L strictly below and U on and above its diagonal; L has a unit diagonal that is not stored.
// All sums are in FP64 (single-precision factors are promoted exactly).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/hlu.h"
#include "errest.cuh"

namespace hlu {

namespace {

constexpr int kApplyThreads = 128;
constexpr int kRankChunk = 128;  // low-rank products go through shared memory in chunks of this rank

enum Which : int { W_AH = 0, W_UPPER = 1, W_LOWER = 2 };

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Entry (i, j) of a dense leaf of side `side` takes part in operator `which`.
__device__ __forceinline__ bool dense_takes(int which, int side, int i, int j) {
    if (which == W_AH || side != 0) return true;
    return which == W_UPPER ? j >= i : j < i;
}

// y += Op x (trans = 0) or y += Op^T x (trans = 1) over the leaves of operator `which`; one CTA per
// leaf (grid-stride), accumulation by atomicAdd (the order of the sums is not fixed).
template <class T>
__global__ void __launch_bounds__(kApplyThreads) k_leaf_apply(const ErrLeaf *leaves, int64_t nl, const double *Aa,
                                                              const T *F, const int32_t *kd, int which, int trans,
                                                              const double *x, double *y) {
    __shared__ double t[kRankChunk];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t l = blockIdx.x; l < nl; l += gridDim.x) {
        const ErrLeaf L = leaves[l];
        if ((which == W_UPPER && L.side == 2) || (which == W_LOWER && L.side == 1)) continue;
        const bool fac = which != W_AH;
        // rows / columns of the operator application: out = rows of the result, in = rows of x
        const int m = L.m, n = L.n;
        const int64_t ro = trans ? L.c0 : L.r0, ci = trans ? L.r0 : L.c0;
        if (L.kind == 0) {
            const int64_t off = fac ? L.f_off : L.a_off;
            if (!trans) {
                for (int i = threadIdx.x; i < m; i += blockDim.x) {
                    double s = 0.0;
                    for (int j = 0; j < n; ++j)
                        if (dense_takes(which, L.side, i, j)) {
                            const double d = fac ? (double)F[off + i + (int64_t)j * m] : Aa[off + i + (int64_t)j * m];
                            s = fma(d, x[ci + j], s);
                        }
                    atomicAdd(y + ro + i, s);
                }
            } else {
                for (int j = warp; j < n; j += nw) {
                    double s = 0.0;
                    for (int i = lane; i < m; i += 32)
                        if (dense_takes(which, L.side, i, j)) {
                            const double d = fac ? (double)F[off + i + (int64_t)j * m] : Aa[off + i + (int64_t)j * m];
                            s = fma(d, x[ci + i], s);
                        }
                    s = warp_sum_d(s);
                    if (lane == 0) atomicAdd(y + ro + j, s);
                }
            }
        } else {
            const int k = fac ? kd[L.kslot] : L.ak;
            // y_out += P (Q^T x_in): (P, Q) = (U, V) for A, (V, U) for A^T
            const int64_t po = fac ? (trans ? L.f_voff : L.f_off) : (trans ? L.a_voff : L.a_off);
            const int64_t qo = fac ? (trans ? L.f_off : L.f_voff) : (trans ? L.a_off : L.a_voff);
            const int mp = trans ? n : m, mq = trans ? m : n;
            for (int a0 = 0; a0 < k; a0 += kRankChunk) {
                const int kc = min(kRankChunk, k - a0);
                for (int a = warp; a < kc; a += nw) {
                    double s = 0.0;
                    for (int j = lane; j < mq; j += 32) {
                        const int64_t e = qo + j + (int64_t)(a0 + a) * mq;
                        s = fma(fac ? (double)F[e] : Aa[e], x[ci + j], s);
                    }
                    s = warp_sum_d(s);
                    if (lane == 0) t[a] = s;
                }
                __syncthreads();
                for (int i = threadIdx.x; i < mp; i += blockDim.x) {
                    double s = 0.0;
                    for (int a = 0; a < kc; ++a) {
                        const int64_t e = po + i + (int64_t)(a0 + a) * mp;
                        s = fma(fac ? (double)F[e] : Aa[e], t[a], s);
                    }
                    atomicAdd(y + ro + i, s);
                }
                __syncthreads();
            }
        }
    }
}

// out = a x + b z (n values)
__global__ void k_axpby(int64_t n, double a, const double *x, double b, const double *z, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (z ? b * z[i] : 0.0);
}

// *acc += sum x_i^2
__global__ void k_sumsq(int64_t n, const double *x, double *acc) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(x[i], x[i], s);
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s = warp_sum_d(s);
        if (threadIdx.x == 0) atomicAdd(acc, s);
    }
}

// x_cluster[p] = x_orig[perm[p]]
__global__ void k_gather(int64_t n, const int32_t *perm, const double *x, double *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[perm[i]];
}

int grid_of(int64_t n) {
    const int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : g > 1216 ? 1216 : g);
}

}  // namespace

int ErrEstimator::apply(int which, int trans, const double *x, double *y) {
    cudaMemsetAsync(y, 0, sizeof(double) * n, stream);
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(n_leaves, 1), 152 * 16);
    if (fp64)
        k_leaf_apply<double><<<grid, kApplyThreads, 0, stream>>>(leaves, n_leaves, aarena,
                                                                  static_cast<const double *>(farena), kdyn, which,
                                                                  trans, x, y);
    else
        k_leaf_apply<float><<<grid, kApplyThreads, 0, stream>>>(leaves, n_leaves, aarena,
                                                                 static_cast<const float *>(farena), kdyn, which,
                                                                 trans, x, y);
    launched += 2;
    return cudaGetLastError() == cudaSuccess ? HLU_OK : HLU_ECUDA;
}

// z = M^T M x (with_factors) or A^T A x, work vectors w1 .. w3 of n values
int ErrEstimator::normal_apply(bool with_factors, const double *x, double *z) {
    int st;
    if ((st = apply(W_AH, 0, x, w1))) return st;  // w1 = A x
    if (with_factors) {
        if ((st = apply(W_UPPER, 0, x, w2))) return st;   // w2 = U x
        if ((st = apply(W_LOWER, 0, w2, w3))) return st;  // w3 = Ls U x
        k_axpby<<<grid_of(n), 256, 0, stream>>>(n, 1.0, w2, 1.0, w3, w3);  // w3 = L U x
        k_axpby<<<grid_of(n), 256, 0, stream>>>(n, 1.0, w1, -1.0, w3, w1); // w1 = M x
        launched += 2;
    }
    if ((st = apply(W_AH, 1, w1, z))) return st;  // z = A^T w1
    if (with_factors) {
        if ((st = apply(W_LOWER, 1, w1, w2))) return st;  // w2 = Ls^T w1
        k_axpby<<<grid_of(n), 256, 0, stream>>>(n, 1.0, w1, 1.0, w2, w2);  // w2 = L^T w1
        if ((st = apply(W_UPPER, 1, w2, w3))) return st;  // w3 = U^T L^T w1
        k_axpby<<<grid_of(n), 256, 0, stream>>>(n, 1.0, z, -1.0, w3, z);   // z = M^T M x
        launched += 2;
    }
    return cudaGetLastError() == cudaSuccess ? HLU_OK : HLU_ECUDA;
}

// ||Op||_2 by power iteration on Op^T Op from the cluster-order start vector x0 (unnormalised):
// x = x0 / |x0|; repeat z = Op^T Op x, lam = |z|, x = z / lam until |lam - lam_old| <= rtol lam or
// `iters` products; returns sqrt(lam).
int ErrEstimator::power(bool with_factors, const double *x0, int iters, double rtol, double *out) {
    double *acc = host_acc;
    cudaMemsetAsync(dacc, 0, sizeof(double), stream);
    k_sumsq<<<grid_of(n), 256, 0, stream>>>(n, x0, dacc);
    cudaMemcpyAsync(acc, dacc, sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess) return HLU_ECUDA;
    const double nx = std::sqrt(*acc);
    if (!(nx > 0.0)) return HLU_EINVAL;
    k_axpby<<<grid_of(n), 256, 0, stream>>>(n, 1.0 / nx, x0, 0.0, nullptr, x);
    launched += 2;
    double lam = 0.0, lam_old = 0.0;
    for (int it = 0; it < iters; ++it) {
        int st = normal_apply(with_factors, x, z);
        if (st) return st;
        cudaMemsetAsync(dacc, 0, sizeof(double), stream);
        k_sumsq<<<grid_of(n), 256, 0, stream>>>(n, z, dacc);
        cudaMemcpyAsync(acc, dacc, sizeof(double), cudaMemcpyDeviceToHost, stream);
        launched += 1;
        if (cudaStreamSynchronize(stream) != cudaSuccess) return HLU_ECUDA;
        lam = std::sqrt(*acc);
        if (!std::isfinite(lam)) return HLU_ENUMERIC;
        if (lam == 0.0) {
            *out = 0.0;
            return HLU_OK;
        }
        k_axpby<<<grid_of(n), 256, 0, stream>>>(n, 1.0 / lam, z, 0.0, nullptr, x);
        launched += 1;
        if (lam_old != 0.0 && std::fabs(lam - lam_old) <= rtol * lam) break;
        lam_old = lam;
    }
    *out = std::sqrt(lam);
    return HLU_OK;
}

int ErrEstimator::run(const double *x0_orig, const int32_t *perm, int iters, double rtol, double *efac,
                      double *norm_a) {
    k_gather<<<grid_of(n), 256, 0, stream>>>(n, perm, x0_orig, x0c);
    launched += 1;
    double num = 0.0, den = 0.0;
    int st = power(true, x0c, iters, rtol, &num);
    if (st) return st;
    if ((st = power(false, x0c, iters, rtol, &den))) return st;
    if (norm_a) *norm_a = den;
    *efac = den > 0.0 ? num / den : 0.0;
    return HLU_OK;
}

}  // namespace hlu
