// Device kernels of the H-LU task graph (sm_103a).  One CTA (256 threads)
// executes one task; the launch of a wave passes the slice of the task array
// that belongs to it.  T is the storage type of the factors (double or
// float); the core of every rounded addition is always computed in double.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <algorithm>

#include "kernels.cuh"

namespace hlu {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxLeaf = 128;        // largest dense diagonal leaf (4 rows per lane)
constexpr int kRowsPerLane = kMaxLeaf / 32;

__device__ __forceinline__ int dim_r(const Panel &p, const int32_t *kd) { return p.rslot >= 0 ? kd[p.rslot] : p.rows; }
__device__ __forceinline__ int dim_c(const Panel &p, const int32_t *kd) { return p.cslot >= 0 ? kd[p.cslot] : p.cols; }

template <class T>
__device__ __forceinline__ T &at(T *A, const Panel &p, int i, int j) {
    return A[p.off + (int64_t)i * p.rs + (int64_t)j * p.cs];
}

__device__ void set_error(long long *err, int code, long long index, double value) {
    if (atomicCAS((unsigned long long *)err, 0ull, (unsigned long long)code) == 0ull) {
        err[1] = index;
        err[2] = __double_as_longlong(value);
    }
    atomicAdd((unsigned long long *)(err + 3), 1ull);
}

// Profiling of rounded-addition phases (only when a.phase is set): thread 0
// adds the time since `t` to slot `s` and returns the new time stamp.
__device__ __forceinline__ unsigned long long phase_mark(const LaunchArgs &a, int s, unsigned long long t) {
    if (!a.phase || threadIdx.x != 0) return 0ull;
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (t) atomicAdd(a.phase + s, now - t);
    return now;
}

// Model flop counts (standard operation counts, Golub and Van Loan).
__device__ __forceinline__ void add_flops(const LaunchArgs &a, int kind, double f) {
    if (a.flops && f > 0.0) atomicAdd(a.flops + kind, f);
}

__device__ __forceinline__ double qr_model_flops(double m, double K) {
    const double hi = m > K ? m : K, lo = m > K ? K : m;
    return 2.0 * hi * lo * lo - 2.0 * lo * lo * lo / 3.0;
}

// Model flops of one rounded addition (the oracle's count, whichever route the
// kernel takes): QR of both stacks, Jacobi SVD of the K x K core, Q times the
// kept vectors.
__device__ __forceinline__ double radd_model_flops(int m, int n, int K, int knew) {
    const double ku = m < K ? m : K, kv = n < K ? n : K, kb = ku > kv ? ku : kv;
    return qr_model_flops(m, K) + qr_model_flops(n, K) + 21.0 * kb * kb * kb + 2.0 * (m * ku + n * kv) * knew;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sum over the CTA; `red` holds >= 33 doubles of shared memory.
__device__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double s = l < nw ? red[l] : 0.0;
        s = warp_sum(s);
        if (l == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// ------------------------------------------------------------------ GETRF
// Unpivoted LU of an m x m dense diagonal leaf in shared memory (Sec. 3.1,
// "Dense blocks": L unit lower and U overwrite A).
template <class T>
__device__ void dev_getrf(const TGetrf &t, const LaunchArgs &a, unsigned char *smem_raw) {
    T *s = reinterpret_cast<T *>(smem_raw);
    const int m = t.m;
    T *g = reinterpret_cast<T *>(a.arena) + t.off;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) s[e] = g[e];
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        const T piv = s[k + k * m];
        if (threadIdx.x == 0 && (!(piv != T(0)) || !isfinite((double)piv)))
            set_error(a.err, DE_PIVOT, t.leaf, (double)piv);
        for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) s[i + k * m] /= piv;
        __syncthreads();
        const int rem = m - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e % rem, j = k + 1 + e / rem;
            s[i + j * m] -= s[i + k * m] * s[k + j * m];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) g[e] = s[e];
    if (threadIdx.x == 0) add_flops(a, K_GETRF, 2.0 * m * m * m / 3.0);
}

// ------------------------------------------------------------------- TRSM
// Triangular solve of a panel with a dense diagonal leaf; one warp per panel
// column, the column held in registers (rows lane + 32 r), the triangle in
// shared memory laid out so that lane accesses are contiguous.
template <class T>
__device__ void dev_trsm(const TTrsm &t, const LaunchArgs &a, unsigned char *smem_raw) {
    T *L = reinterpret_cast<T *>(smem_raw);
    const int m = t.m;
    const T *g = reinterpret_cast<const T *>(a.arena) + t.L_off;
    if (t.mode == TR_UPPER_TRANS) {
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = e % m, j = e / m;
            L[j + i * m] = g[e];  // L = U^T
        }
    } else {
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) L[e] = g[e];
    }
    __syncthreads();
    T *A = reinterpret_cast<T *>(a.arena);
    const int p = dim_c(t.P, a.kdyn);
    if (threadIdx.x == 0) add_flops(a, K_TRSM, (double)m * m * p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < p; c += nw) {
        T x[kRowsPerLane];
#pragma unroll
        for (int r = 0; r < kRowsPerLane; ++r) {
            const int row = lane + 32 * r;
            x[r] = row < m ? at(A, t.P, row, c) : T(0);
        }
        if (t.mode == TR_LOWER_UNIT || t.mode == TR_UPPER_TRANS) {
            const bool unit = t.mode == TR_LOWER_UNIT;
            for (int i = 0; i < m; ++i) {
                const int ri = i >> 5, li = i & 31;
                if (!unit && lane == li) {
#pragma unroll
                    for (int r = 0; r < kRowsPerLane; ++r)
                        if (r == ri) x[r] /= L[i + i * m];
                }
                T xv = 0;
#pragma unroll
                for (int r = 0; r < kRowsPerLane; ++r)
                    if (r == ri) xv = x[r];
                const T xi = __shfl_sync(kFull, xv, li);
#pragma unroll
                for (int r = 0; r < kRowsPerLane; ++r) {
                    const int row = lane + 32 * r;
                    if (row > i && row < m) x[r] -= L[row + i * m] * xi;
                }
            }
        } else {  // TR_UPPER: backward substitution
            for (int i = m - 1; i >= 0; --i) {
                const int ri = i >> 5, li = i & 31;
                if (lane == li) {
#pragma unroll
                    for (int r = 0; r < kRowsPerLane; ++r)
                        if (r == ri) x[r] /= L[i + i * m];
                }
                T xv = 0;
#pragma unroll
                for (int r = 0; r < kRowsPerLane; ++r)
                    if (r == ri) xv = x[r];
                const T xi = __shfl_sync(kFull, xv, li);
#pragma unroll
                for (int r = 0; r < kRowsPerLane; ++r) {
                    const int row = lane + 32 * r;
                    if (row < i) x[r] -= L[row + i * m] * xi;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kRowsPerLane; ++r) {
            const int row = lane + 32 * r;
            if (row < m) at(A, t.P, row, c) = x[r];
        }
    }
}

// ---------------------------------------------------------------- PROJECT
// T (k x p) = F^T X (F: len x k, X: len x p): the V^T z (or U^T z) half of a
// low-rank product (Sec. 3.1).  Rows are streamed through shared memory in
// chunks of 32; each thread owns up to 16 outputs of a 64 x 64 output tile.
template <class T>
__device__ void dev_project(const TProject &t, const LaunchArgs &a, unsigned char *smem_raw) {
    T(*sF)[65] = reinterpret_cast<T(*)[65]>(smem_raw);
    T(*sX)[65] = sF + 32;
    T *A = reinterpret_cast<T *>(a.arena);
    const int len = dim_r(t.F, a.kdyn), k = dim_c(t.F, a.kdyn), p = dim_c(t.X, a.kdyn);
    if (threadIdx.x == 0) add_flops(a, K_PROJECT, 2.0 * len * k * p);
    for (int a0 = 0; a0 < k; a0 += 64)
        for (int b0 = 0; b0 < p; b0 += 64) {
            const int ka = min(64, k - a0), pb = min(64, p - b0);
            T acc[16];
#pragma unroll
            for (int s = 0; s < 16; ++s) acc[s] = T(0);
            for (int r0 = 0; r0 < len; r0 += 32) {
                const int rr = min(32, len - r0);
                for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
                    const int r = e & 31, c = e >> 5;
                    sF[r][c] = (r < rr && c < ka) ? at(A, t.F, r0 + r, a0 + c) : T(0);
                    sX[r][c] = (r < rr && c < pb) ? at(A, t.X, r0 + r, b0 + c) : T(0);
                }
                __syncthreads();
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const int idx = threadIdx.x + kThreads * s;
                    const int ia = idx & 63, ib = idx >> 6;
                    T v = acc[s];
                    for (int r = 0; r < rr; ++r) v += sF[r][ia] * sX[r][ib];
                    acc[s] = v;
                }
                __syncthreads();
            }
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const int idx = threadIdx.x + kThreads * s;
                const int ia = idx & 63, ib = idx >> 6;
                if (ia < ka && ib < pb) at(A, t.T, a0 + ia, b0 + ib) = acc[s];
            }
        }
}

// ------------------------------------------------------------------ ACCUM
// out (m x p) = beta out + alpha sum_t A_t X_t over the leaves that cover one
// leaf cluster of the output rows (dense leaves: A = D, X = panel slice;
// low-rank leaves: A = U slice, X = projected V^T z).
template <class T>
__device__ void dev_accum(const TAccum &t, const Term *terms, const LaunchArgs &a) {
    T *A = reinterpret_cast<T *>(a.arena);
    const int m = dim_r(t.out, a.kdyn);
    const int p = t.dst >= 0 ? a.kdyn[t.src] : dim_c(t.out, a.kdyn);
    if (t.dst >= 0 && threadIdx.x == 0) a.kdyn[t.dst] = p;
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int q = 0; q < t.nterms; ++q) f += 2.0 * m * (double)dim_c(terms[t.term0 + q].A, a.kdyn) * p;
        add_flops(a, K_ACCUM, f);
    }
    const T alpha = T(t.alpha);
    for (int e0 = 0; e0 < m * p; e0 += blockDim.x) {
        const int e = e0 + threadIdx.x;
        if (e >= m * p) break;
        const int i = e % m, j = e / m;
        T acc = T(0);
        for (int q = 0; q < t.nterms; ++q) {
            const Term tm = terms[t.term0 + q];
            const int inner = dim_c(tm.A, a.kdyn);
            const T *pa = A + tm.A.off + (int64_t)i * tm.A.rs;
            const T *px = A + tm.X.off + (int64_t)j * tm.X.cs;
            for (int l = 0; l < inner; ++l) acc += pa[(int64_t)l * tm.A.cs] * px[(int64_t)l * tm.X.rs];
        }
        T &o = at(A, t.out, i, j);
        o = (t.overwrite ? T(0) : o) + alpha * acc;
    }
}

// ------------------------------------------------------------------ SPLIT
template <class T>
__device__ void dev_split(const TSplit &t, const LaunchArgs &a) {
    T *A = reinterpret_cast<T *>(a.arena);
    const int k = a.kdyn[t.src_kslot];
    if (threadIdx.x == 0) a.kdyn[t.dst_kslot] = k;
    for (int e = threadIdx.x; e < t.mu * k; e += blockDim.x) {
        const int i = e % t.mu, j = e / t.mu;
        A[t.dstU + e] = at(A, t.srcU, i, j);
    }
    for (int e = threadIdx.x; e < t.nv * k; e += blockDim.x) {
        const int i = e % t.nv, j = e / t.nv;
        A[t.dstV + e] = at(A, t.srcV, i, j);
    }
}

// ------------------------------------------------------------------- RADD
template <class R>
__device__ __forceinline__ R warp_sum_t(R v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Householder QR of the m x K panel W in place, in the panel's own precision T
// (reflector j: v_j = 1 implied, v_j[i] stored below the diagonal, tau[j]);
// R in the upper triangle.
template <class T>
__device__ void block_householder_qr(T *W, int m, int K, double *tau, double *red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int kk = min(m, K);
    for (int j = 0; j < kk; ++j) {
        T *x = W + (int64_t)j * m;
        T s = T(0);
        for (int i = j + threadIdx.x; i < m; i += blockDim.x) s += x[i] * x[i];
        s = warp_sum_t(s);
        __syncthreads();
        if (lane == 0) red[warp] = (double)s;
        __syncthreads();
        if (warp == 0) {
            double q = lane < nw ? red[lane] : 0.0;
            q = warp_sum(q);
            if (lane == 0) red[32] = q;
        }
        __syncthreads();
        const T x0 = x[j];
        const T nrm = T(sqrt(red[32]));
        if (nrm == T(0)) {
            if (threadIdx.x == 0) tau[j] = 0.0;
            __syncthreads();
            continue;
        }
        const T alpha = x0 >= T(0) ? -nrm : nrm;
        const T v0 = x0 - alpha;
        const T tj = (alpha - x0) / alpha;
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) x[i] = x[i] / v0;
        if (threadIdx.x == 0) {
            x[j] = alpha;
            tau[j] = (double)tj;
        }
        __syncthreads();
        for (int c = j + 1 + warp; c < K; c += nw) {
            T *y = W + (int64_t)c * m;
            T d = T(0);
            for (int i = j + 1 + lane; i < m; i += 32) d += x[i] * y[i];
            d = warp_sum_t(d);
            d = (d + y[j]) * tj;
            __syncwarp();
            if (lane == 0) y[j] -= d;
            for (int i = j + 1 + lane; i < m; i += 32) y[i] -= d * x[i];
        }
        __syncthreads();
    }
}

// Z (m x nc, ld m) := Q Z with Q = H_0 ... H_{kk-1} from block_householder_qr,
// in precision T; each warp owns whole columns, so no CTA barrier is needed
// between reflectors.
template <class T>
__device__ void block_apply_q(const T *W, int m, int kk, const double *tau, T *Z, int nc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < nc; c += nw) {
        T *y = Z + (int64_t)c * m;
        for (int j = kk - 1; j >= 0; --j) {
            const T *x = W + (int64_t)j * m;
            T d = T(0);
            for (int i = j + 1 + lane; i < m; i += 32) d += x[i] * y[i];
            d = warp_sum_t(d);
            d = (d + y[j]) * T(tau[j]);
            __syncwarp();
            if (lane == 0) y[j] -= d;
            for (int i = j + 1 + lane; i < m; i += 32) y[i] -= d * x[i];
            __syncwarp();
        }
    }
}

// One-sided (Hestenes) Jacobi on the columns of M (ku x kv, double, shared):
// M J = B with orthogonal columns; the singular values are the column norms of
// B, the right singular vectors the columns of J.  Round-robin ordering, one
// warp per column pair.  A pair is rotated while |x.y| > tol |x||y| with
// tol = 4 ku eps_double, the rounding level of the dot product itself (a
// smaller tolerance is never met reliably and only burns sweeps); at most 30
// sweeps.
__device__ void block_jacobi(double *M, int ku, int kv, double *J, int *flag) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int np = (kv + 1) & ~1;
    const double tol = 4.0 * ku * DBL_EPSILON;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (threadIdx.x == 0) *flag = 0;
        __syncthreads();
        for (int r = 0; r < np - 1; ++r) {
            for (int pi = warp; pi < np / 2; pi += nw) {
                int p, q;
                if (pi == 0) {
                    p = r;
                    q = np - 1;
                } else {
                    p = (r + pi) % (np - 1);
                    q = (r - pi + np - 1) % (np - 1);
                }
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                if (q >= kv) continue;
                double *cp = M + (int64_t)p * ku, *cq = M + (int64_t)q * ku;
                double aa = 0.0, bb = 0.0, gg = 0.0;
                for (int i = lane; i < ku; i += 32) {
                    const double x = cp[i], y = cq[i];
                    aa += x * x;
                    bb += y * y;
                    gg += x * y;
                }
                aa = warp_sum(aa);
                bb = warp_sum(bb);
                gg = warp_sum(gg);
                if (gg == 0.0 || !(fabs(gg) > tol * sqrt(aa * bb))) continue;
                if (lane == 0) *flag = 1;
                const double zeta = (bb - aa) / (2.0 * gg);
                const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
                __syncwarp();
                for (int i = lane; i < ku; i += 32) {
                    const double x = cp[i], y = cq[i];
                    cp[i] = cs * x - sn * y;
                    cq[i] = sn * x + cs * y;
                }
                double *jp = J + (int64_t)p * kv, *jq = J + (int64_t)q * kv;
                for (int i = lane; i < kv; i += 32) {
                    const double x = jp[i], y = jq[i];
                    jp[i] = cs * x - sn * y;
                    jq[i] = sn * x + cs * y;
                }
            }
            __syncthreads();
        }
        const int f = *flag;
        __syncthreads();
        if (!f) break;
    }
}

// FP64 core buffers of a rounded addition with stacked rank K (see dev_radd).
__host__ __device__ size_t radd_core_bytes(int K) {
    return sizeof(double) * (3 * (size_t)K * K + 5 * (size_t)K + 40) + sizeof(int) * (2 * (size_t)K + 8);
}

size_t radd_smem_bytes(int kc) { return radd_core_bytes(kc); }

// QR with column pivoting of the ku x kv core M (double, shared memory, column
// major), stopped at the first step whose largest remaining column norm is at
// most delta times the first pivot's (the neglected block is at the level of
// double rounding): M P = Q [R'; ~0] with R' of r rows.  Reflectors are kept
// below the diagonal of M (v_j = 1 implied), tau[j]; perm holds P.  The pivot
// is the largest column norm, lowest index on ties.
__device__ int block_qrcp(double *M, int ku, int kv, double *tau, double *cn, int *perm, double delta,
                          double *red, int *iflag) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = threadIdx.x; j < kv; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < ku; ++i) s += M[i + (size_t)j * ku] * M[i + (size_t)j * ku];
        cn[j] = s;
        perm[j] = j;
    }
    __syncthreads();
    double n0 = 0.0;  // first pivot norm (kept by warp 0)
    int r = 0;
    const int kk = min(ku, kv);
    for (int j = 0; j < kk; ++j) {
        double *x = M + (size_t)j * ku;
        // warp 0: pivot, stopping test, column swap and reflector; one barrier
        if (warp == 0) {
            double bv = -1.0;
            int bi = j;
            for (int c = j + lane; c < kv; c += 32)
                if (cn[c] > bv) {
                    bv = cn[c];
                    bi = c;
                }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(kFull, bv, o);
                const int oi = __shfl_xor_sync(kFull, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (j == 0) n0 = bv;
            const bool stop = !(bv > delta * delta * n0);
            if (lane == 0) iflag[1] = stop ? -1 : bi;
            if (!stop) {
                const int p = bi;
                if (p != j) {
                    for (int i = lane; i < ku; i += 32) {
                        const double tmp = x[i];
                        x[i] = M[i + (size_t)p * ku];
                        M[i + (size_t)p * ku] = tmp;
                    }
                    if (lane == 0) {
                        const double tc = cn[j];
                        cn[j] = cn[p];
                        cn[p] = tc;
                        const int tp = perm[j];
                        perm[j] = perm[p];
                        perm[p] = tp;
                    }
                    __syncwarp();
                }
                double s = 0.0;
                for (int i = j + lane; i < ku; i += 32) s += x[i] * x[i];
                s = warp_sum(s);
                const double x0 = x[j];
                const double nrm = sqrt(s);
                double tj = 0.0;
                __syncwarp();
                if (nrm > 0.0) {
                    const double alpha = x0 >= 0.0 ? -nrm : nrm;
                    const double v0 = x0 - alpha;
                    for (int i = j + 1 + lane; i < ku; i += 32) x[i] /= v0;
                    tj = (alpha - x0) / alpha;
                    __syncwarp();
                    if (lane == 0) x[j] = alpha;
                }
                if (lane == 0) tau[j] = tj;
            }
        }
        __syncthreads();
        if (iflag[1] < 0) break;  // uniform: every thread reads the same flag
        const double tj = tau[j];
        for (int c = j + 1 + warp; c < kv; c += nw) {
            double *y = M + (size_t)c * ku;
            double d = 0.0;
            for (int i = j + 1 + lane; i < ku; i += 32) d += x[i] * y[i];
            d = warp_sum(d);
            d = (d + y[j]) * tj;
            __syncwarp();
            if (lane == 0) y[j] -= d;
            double t2 = 0.0;
            for (int i = j + 1 + lane; i < ku; i += 32) {
                y[i] -= d * x[i];
                t2 += y[i] * y[i];
            }
            t2 = warp_sum(t2);
            if (lane == 0) cn[c] = t2;
        }
        __syncthreads();
        r = j + 1;
    }
    return r;
}

// Z (ku x nc in shared memory, leading dimension ku) := Q Z with the r
// reflectors of block_qrcp; one warp per column.
__device__ void block_apply_qcp(const double *M, int ku, int r, const double *tau, double *Z, int nc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < nc; c += nw) {
        double *y = Z + (size_t)c * ku;
        for (int j = r - 1; j >= 0; --j) {
            const double *x = M + (size_t)j * ku;
            double d = 0.0;
            for (int i = j + 1 + lane; i < ku; i += 32) d += x[i] * y[i];
            d = warp_sum(d);
            d = (d + y[j]) * tau[j];
            __syncwarp();
            if (lane == 0) y[j] -= d;
            for (int i = j + 1 + lane; i < ku; i += 32) y[i] -= d * x[i];
            __syncwarp();
        }
    }
}

// Rounded addition (Sec. 3.1): the target's factors and every contribution are
// stacked, U_s = [U_c, c_1 U_1, ...], V_s = [V_c, V_1, ...] (pieces
// zero-padded to the target's index ranges); both stacks are reduced by
// Householder QR, and the core M = R_u R_v^T (double) is decomposed: a QR with
// column pivoting M P = Q_M [R'; ~0] (stopped at double-rounding level)
// followed by one-sided Jacobi on R'^T gives M = X Sigma Y^T with X = Q_M [J; 0]
// and Y = P W Sigma^{-1}; singular values sigma_i <= eps sigma_1 are dropped and
// the new factors are U = Q_u [X Sigma; 0], V = Q_v [Y; 0].
//
// Shared memory is carved by the task's own stacked rank K: the FP64 core
// buffers first (radd_smem_bytes(K)), then, when they fit in the rest of the
// CTA's `smem_bytes`, the stacked panels themselves; larger panels stay in
// the global `scratch`.  The pivoted QR of the core stops at delta times the
// first pivot: 1e-13 for FP64 factors (double rounding level) and 1e-6 for
// FP32 factors (an order above the FP32 rounding of the stacked panels, two
// below the relative tolerances eps the method uses).
// Small targets (m n <= kSmallTarget, m, n <= 128): the sum X = U_c V_c^T + sum_i c_i U_i V_i^T
// is formed densely (in the factor precision) and its truncated SVD is taken
// directly - pivoted QR of X (double) and one-sided Jacobi on the reduced
// factor - which is the same T_eps of the same sum without the two stacked
// QRs.  Returns false (before touching anything) when X and its buffers do
// not fit in `smem_bytes`.
constexpr int kSmallTarget = 4096;

template <class T>
__device__ bool radd_small(const TRadd &t, const Piece *pieces, const LaunchArgs &a, int kself,
                           unsigned char *smem_raw, size_t smem_bytes, double delta) {
    const int m = t.m, n = t.n, mn = min(m, n), mx = max(m, n);
    const size_t need = sizeof(double) * ((size_t)m * n + (size_t)mx * mn + (size_t)mn * mn + 2 * mn + n + 40) +
                        sizeof(int) * ((size_t)mn + n + 8);
    // every launch provides radd_smem_bytes(64) >= the largest `need` of a target
    // with m n <= kSmallTarget and m, n <= 128 (100704 bytes at m = n = 64), so
    // the choice depends on the task alone
    if ((int64_t)m * n > kSmallTarget || mx > 128 || need > smem_bytes) return false;
    T *A = reinterpret_cast<T *>(a.arena);
    int32_t *kd = a.kdyn;
    double *X = reinterpret_cast<double *>(smem_raw);
    double *C = X + (size_t)m * n;  // n x r, later m x knew
    double *J = C + (size_t)mx * mn;
    double *tau = J + (size_t)mn * mn;
    double *sig = tau + mn;
    double *cn = sig + mn;
    double *red = cn + n;
    int *order = reinterpret_cast<int *>(red + 40);
    int *perm = order + mn;
    int *iflag = perm + n;
    unsigned long long ph = phase_mark(a, 0, 0ull);
    // ---- X = U_c V_c^T + sum of the zero-padded contributions
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        const int i = e % m, j = e / m;
        T acc = T(0);
        for (int c = 0; c < kself; ++c) acc += A[t.U_off + i + (int64_t)c * m] * A[t.V_off + j + (int64_t)c * n];
        for (int q = 0; q < t.npieces; ++q) {
            const Piece &pc = pieces[t.piece0 + q];
            const int ii = i - pc.roff, jj = j - pc.coff;
            if (ii < 0 || ii >= pc.U.rows || jj < 0 || jj >= pc.V.rows) continue;
            const int k = dim_c(pc.U, kd);
            T s = T(0);
            for (int l = 0; l < k; ++l) s += at(A, pc.U, ii, l) * at(A, pc.V, jj, l);
            acc += T(pc.coef) * s;
        }
        X[e] = (double)acc;
    }
    __syncthreads();
    ph = phase_mark(a, 0, ph);
    // ---- X P = Q [R'; ~0], one-sided Jacobi on C = R'^T (n x r)
    const int r = block_qrcp(X, m, n, tau, cn, perm, delta, red, iflag);
    ph = phase_mark(a, 1, ph);
    for (int e = threadIdx.x; e < n * r; e += blockDim.x) {
        const int c = e % n, i = e / n;
        C[e] = c >= i ? X[i + (size_t)c * m] : 0.0;
    }
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) J[e] = (e % r == e / r) ? 1.0 : 0.0;
    __syncthreads();
    block_jacobi(C, n, r, J, iflag);
    ph = phase_mark(a, 2, ph);
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += C[i + (size_t)j * n] * C[i + (size_t)j * n];
        sig[j] = sqrt(s);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        int rk = 0;
        for (int l = 0; l < r; ++l) rk += (sig[l] > sig[j]) || (sig[l] == sig[j] && l < j);
        order[rk] = j;
    }
    __syncthreads();
    const double s1 = r > 0 ? sig[order[0]] : 0.0;
    int knew = 0;
    if (!isfinite(s1)) {
        if (threadIdx.x == 0) set_error(a.err, DE_NONFINITE, t.target, s1);
    } else if (s1 > 0.0) {
        for (int l = 0; l < r; ++l) knew += sig[order[l]] > a.eps * s1;
    }
    if (knew > t.cap) {
        if (threadIdx.x == 0) set_error(a.err, DE_RANKCAP, t.target, (double)knew);
        knew = t.cap;
    }
    ph = phase_mark(a, 3, ph);
    if (a.phase && threadIdx.x == 0) {  // Jacobi problem size: columns, rows
        atomicAdd(a.phase + 6, (unsigned long long)r);
        atomicAdd(a.phase + 7, 1ull);
    }
    // ---- V = P W_sel Sigma^{-1} (every row of V is covered by the permutation)
    T *Uc = A + t.U_off;
    T *Vc = A + t.V_off;
    for (int e = threadIdx.x; e < n * knew; e += blockDim.x) {
        const int i = e % n, c = e / n;
        const int j = order[c];
        Vc[perm[i] + (int64_t)c * n] = T(C[i + (size_t)j * n] / sig[j]);
    }
    __syncthreads();
    // ---- U = Q [J_sel Sigma; 0] (C reused for the m x knew product)
    for (int e = threadIdx.x; e < m * knew; e += blockDim.x) {
        const int i = e % m, c = e / m;
        const int j = order[c];
        C[e] = i < r ? J[i + (size_t)j * r] * sig[j] : 0.0;
    }
    __syncthreads();
    block_apply_qcp(X, m, r, tau, C, knew);
    __syncthreads();
    for (int e = threadIdx.x; e < m * knew; e += blockDim.x) Uc[e] = T(C[e]);
    if (threadIdx.x == 0) kd[t.kslot] = knew;
    phase_mark(a, 4, ph);
    return true;
}

// When even the core does not fit (K above the CTA's shared-memory capacity),
// it is placed in `core_scratch` (global, radd_core_bytes(K) bytes).
template <class T>
__device__ void dev_radd(const TRadd &t, const Piece *pieces, const LaunchArgs &a, int kc, unsigned char *smem_raw,
                         T *scratch, size_t smem_bytes, unsigned char *core_scratch) {
    T *A = reinterpret_cast<T *>(a.arena);
    int32_t *kd = a.kdyn;
    const int m = t.m, n = t.n;
    const int kself = t.include_self ? kd[t.kslot] : 0;
    int K = kself;
    for (int q = 0; q < t.npieces; ++q) K += dim_c(pieces[t.piece0 + q].U, kd);
    __syncthreads();  // every thread has read the target's rank before it is rewritten
    if (K > t.Kcap) {
        if (threadIdx.x == 0) set_error(a.err, DE_RANKCAP, t.target, (double)K);
        return;
    }
    if (K == 0) {
        if (threadIdx.x == 0) kd[t.kslot] = 0;
        return;
    }
    const double delta = sizeof(T) == 8 ? 1e-13 : 1e-6;
    if (radd_small<T>(t, pieces, a, kself, smem_raw, smem_bytes, delta)) {
        if (threadIdx.x == 0) add_flops(a, K_RADD, radd_model_flops(m, n, K, kd[t.kslot]));
        return;
    }
    if (K > kc) {
        if (threadIdx.x == 0) set_error(a.err, DE_RANKCAP, t.target, (double)K);
        return;
    }
    const size_t core_bytes = (radd_core_bytes(K) + 15) & ~size_t(15);
    const bool core_in_smem = core_bytes <= smem_bytes;
    unsigned char *core = core_in_smem ? smem_raw : core_scratch;
    double *M = reinterpret_cast<double *>(core);  // core, then QRCP reflectors
    double *C = M + (size_t)K * K;                        // R'^T (kv x r), later Q_M [J Sigma; 0]
    double *J = C + (size_t)K * K;                        // Jacobi rotations (r x r)
    double *tauU = J + (size_t)K * K;
    double *tauV = tauU + K;
    double *tauM = tauV + K;
    double *sig = tauM + K;
    double *cn = sig + K;
    double *red = cn + K;  // 40 doubles
    int *order = reinterpret_cast<int *>(red + 40);
    int *perm = order + K;
    int *iflag = perm + K;  // 8 ints
    const size_t panel_bytes = (size_t)(m + n) * K * sizeof(T);
    T *WU = core_in_smem && core_bytes + panel_bytes <= smem_bytes ? reinterpret_cast<T *>(smem_raw + core_bytes)
                                                                    : scratch;
    T *WV = WU + (int64_t)m * K;
    // ---- stack the factors
    for (int64_t e = threadIdx.x; e < (int64_t)(m + n) * K; e += blockDim.x) WU[e] = T(0);
    __syncthreads();
    for (int e = threadIdx.x; e < m * kself; e += blockDim.x) WU[e] = A[t.U_off + e];
    for (int e = threadIdx.x; e < n * kself; e += blockDim.x) WV[e] = A[t.V_off + e];
    int col = kself;
    for (int q = 0; q < t.npieces; ++q) {
        const Piece pc = pieces[t.piece0 + q];
        const int k = dim_c(pc.U, kd), mu = pc.U.rows, nv = pc.V.rows;
        const T coef = T(pc.coef);
        for (int e = threadIdx.x; e < mu * k; e += blockDim.x) {
            const int i = e % mu, j = e / mu;
            WU[pc.roff + i + (int64_t)(col + j) * m] = coef * at(A, pc.U, i, j);
        }
        for (int e = threadIdx.x; e < nv * k; e += blockDim.x) {
            const int i = e % nv, j = e / nv;
            WV[pc.coff + i + (int64_t)(col + j) * n] = at(A, pc.V, i, j);
        }
        col += k;
    }
    __syncthreads();
    // ---- QR of both stacks
    block_householder_qr(WU, m, K, tauU, red);
    block_householder_qr(WV, n, K, tauV, red);
    const int ku = min(m, K), kv = min(n, K);
    // ---- core M = R_u R_v^T (double)
    for (int e = threadIdx.x; e < ku * kv; e += blockDim.x) {
        const int i = e % ku, j = e / ku;
        double s = 0.0;
        for (int l = max(i, j); l < K; ++l) s += (double)WU[i + (int64_t)l * m] * (double)WV[j + (int64_t)l * n];
        M[e] = s;
    }
    __syncthreads();
    // ---- M P = Q_M [R'; ~0], then one-sided Jacobi on C = R'^T (kv x r)
    const int r = block_qrcp(M, ku, kv, tauM, cn, perm, delta, red, iflag);
    for (int e = threadIdx.x; e < kv * r; e += blockDim.x) {
        const int c = e % kv, i = e / kv;
        C[e] = c >= i ? M[i + (size_t)c * ku] : 0.0;
    }
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) J[e] = (e % r == e / r) ? 1.0 : 0.0;
    __syncthreads();
    block_jacobi(C, kv, r, J, iflag);
    // ---- singular values, ordering, truncation rank
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < kv; ++i) s += C[i + (size_t)j * kv] * C[i + (size_t)j * kv];
        sig[j] = sqrt(s);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        int rk = 0;
        for (int l = 0; l < r; ++l) rk += (sig[l] > sig[j]) || (sig[l] == sig[j] && l < j);
        order[rk] = j;
    }
    __syncthreads();
    const double s1 = r > 0 ? sig[order[0]] : 0.0;
    int knew = 0;
    if (!isfinite(s1)) {
        if (threadIdx.x == 0) set_error(a.err, DE_NONFINITE, t.target, s1);
    } else if (s1 > 0.0) {
        for (int l = 0; l < r; ++l) knew += sig[order[l]] > a.eps * s1;
    }
    if (knew > t.cap) {
        if (threadIdx.x == 0) set_error(a.err, DE_RANKCAP, t.target, (double)knew);
        knew = t.cap;
    }
    T *Uc = A + t.U_off;
    T *Vc = A + t.V_off;
    // ---- V = Q_v [P W_sel Sigma^{-1}; 0]
    for (int e = threadIdx.x; e < n * knew; e += blockDim.x) Vc[e] = T(0);
    __syncthreads();
    for (int e = threadIdx.x; e < kv * knew; e += blockDim.x) {
        const int i = e % kv, c = e / kv;
        const int j = order[c];
        Vc[perm[i] + (int64_t)c * n] = T(C[i + (size_t)j * kv] / sig[j]);
    }
    __syncthreads();
    // ---- U = Q_u [Q_M [J_sel Sigma; 0]; 0] (C now holds the ku x knew product)
    for (int e = threadIdx.x; e < ku * knew; e += blockDim.x) {
        const int i = e % ku, c = e / ku;
        const int j = order[c];
        C[e] = i < r ? J[i + (size_t)j * r] * sig[j] : 0.0;
    }
    __syncthreads();
    block_apply_qcp(M, ku, r, tauM, C, knew);
    __syncthreads();
    for (int e = threadIdx.x; e < m * knew; e += blockDim.x) {
        const int i = e % m, c = e / m;
        Uc[e] = i < ku ? T(C[i + (size_t)c * ku]) : T(0);
    }
    __syncthreads();
    block_apply_q(WU, m, ku, tauU, Uc, knew);
    block_apply_q(WV, n, kv, tauV, Vc, knew);
    if (threadIdx.x == 0) {
        kd[t.kslot] = knew;
        add_flops(a, K_RADD, radd_model_flops(m, n, K, knew));
    }
}

// ------------------------------------------------------------ wave kernels
// One launch per (wave, kind): CTA b executes task b of the launch's slice.
template <class T>
__global__ void __launch_bounds__(kThreads) k_getrf(const TGetrf *tasks, LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TGetrf t = tasks[blockIdx.x];
    dev_getrf<T>(t, a, smem_raw);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_trsm(const TTrsm *tasks, LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TTrsm t = tasks[blockIdx.x];
    dev_trsm<T>(t, a, smem_raw);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_project(const TProject *tasks, LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TProject t = tasks[blockIdx.x];
    dev_project<T>(t, a, smem_raw);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_accum(const TAccum *tasks, const Term *terms, LaunchArgs a) {
    const TAccum t = tasks[blockIdx.x];
    dev_accum<T>(t, terms, a);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_split(const TSplit *tasks, LaunchArgs a) {
    const TSplit t = tasks[blockIdx.x];
    dev_split<T>(t, a);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_radd(const TRadd *tasks, const Piece *pieces, LaunchArgs a, int kc,
                                                   size_t smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TRadd t = tasks[blockIdx.x];
    dev_radd<T>(t, pieces, a, kc, smem_raw, reinterpret_cast<T *>(a.arena) + t.scratch_off, smem_bytes, nullptr);
}

// -------------------------------------------------------- data-flow kernel
// One persistent launch executes the whole task graph.  Worker CTAs claim
// queue slots in order (atomic head); a slot holds the id of a ready task once
// the last predecessor of that task has finished and pushed it (atomic tail).
// A finished task releases its successors: the last one to decrement a
// successor's in-degree pushes it.  Writes of a task are published with a
// device-scope fence before the release; the consumer reads the slot with an
// acquire load.  Every wait has a deadline (%globaltimer): on expiry, or when
// another worker has recorded an error, the worker records DE_TIMEOUT (first
// error wins) and leaves, so the launch always ends.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_dataflow(FlowArgs f, LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task;
    T *scratch = reinterpret_cast<T *>(f.scratch) + (int64_t)blockIdx.x * f.scratch_stride;
    for (;;) {
        if (threadIdx.x == 0) {
            const int slot = atomicAdd(f.counters, 1);
            int g = -1;
            if (slot < f.n_tasks) {
                const unsigned long long deadline = global_ns() + f.timeout_ns;
                for (;;) {
                    g = ld_acquire(f.queue + slot);
                    if (g >= 0) break;
                    if (*(volatile long long *)a.err != 0) {
                        g = -2;
                        break;
                    }
                    if (global_ns() > deadline) {
                        set_error(a.err, DE_TIMEOUT, slot, 0.0);
                        g = -2;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            s_task = g;
        }
        __syncthreads();
        const int g = s_task;
        if (g < 0) break;
        const int code = f.code[g];
        const int kind = code >> kCodeShift, idx = code & kCodeMask;
        const unsigned long long t_start = (f.busy && threadIdx.x == 0) ? global_ns() : 0ull;
        switch (kind) {
            case K_GETRF: {
                const TGetrf t = f.getrf[idx];
                dev_getrf<T>(t, a, smem_raw);
                break;
            }
            case K_TRSM: {
                const TTrsm t = f.trsm[idx];
                dev_trsm<T>(t, a, smem_raw);
                break;
            }
            case K_PROJECT: {
                const TProject t = f.project[idx];
                dev_project<T>(t, a, smem_raw);
                break;
            }
            case K_ACCUM: {
                const TAccum t = f.accum[idx];
                dev_accum<T>(t, f.terms, a);
                break;
            }
            case K_RADD: {
                const TRadd t = f.radd[idx];
                dev_radd<T>(t, f.pieces, a, f.kc, smem_raw, scratch, f.smem_bytes,
                            reinterpret_cast<unsigned char *>(f.core_scratch) +
                                (int64_t)blockIdx.x * f.core_stride);
                break;
            }
            case K_SPLIT: {
                const TSplit t = f.split[idx];
                dev_split<T>(t, a);
                break;
            }
            default:
                break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (f.busy) {
                const unsigned long long dt = global_ns() - t_start;
                atomicAdd(f.busy + kind, dt);
                atomicAdd(f.busy + 8 + kind, 1ull);
                if (kind == K_RADD) {  // rounded additions by size m + n: < 128, < 256, ..., >= 8192
                    const TRadd &t = f.radd[idx];
                    int b = 0;
                    for (int s = t.m + t.n; s >= 128 && b < 7; s >>= 1) ++b;
                    atomicAdd(f.busy + 16 + b, dt);
                    atomicAdd(f.busy + 24 + b, 1ull);
                }
            }
            __threadfence();
            for (int e = f.succ_ptr[g]; e < f.succ_ptr[g + 1]; ++e) {
                const int s = f.succ_idx[e];
                if (atomicSub(f.indeg + s, 1) == 1) {
                    __threadfence();
                    const int pos = atomicAdd(f.counters + 1, 1);
                    st_release(f.queue + pos, s);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ RESET
// leaf_desc per leaf (int64 x kLeafDesc): kind, m, n, k, a_off (D or U), a_voff, f_off (D or U), f_voff, kslot
template <class T>
__global__ void k_reset(const int64_t *desc, const double *Aa, T *F, int32_t *kd) {
    const int64_t *d = desc + kLeafDesc * (int64_t)blockIdx.x;
    const int64_t kind = d[0], m = d[1], n = d[2], k = d[3], ao = d[4], av = d[5], fo = d[6], fv = d[7];
    if (kind == 0) {
        for (int64_t e = threadIdx.x; e < m * n; e += blockDim.x) F[fo + e] = T(Aa[ao + e]);
    } else {
        for (int64_t e = threadIdx.x; e < m * k; e += blockDim.x) F[fo + e] = T(Aa[ao + e]);
        for (int64_t e = threadIdx.x; e < n * k; e += blockDim.x) F[fv + e] = T(Aa[av + e]);
        if (threadIdx.x == 0) kd[d[8]] = int32_t(k);
    }
}

template <class Tin, class Tout>
__global__ void k_permute(const int32_t *perm, int32_t n, int32_t nrhs, const Tin *x, int64_t ldx, Tout *y,
                          int64_t ldy, int to_cluster) {
    const int64_t tot = (int64_t)n * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e % n, j = e / n;
        if (to_cluster)
            y[p + j * ldy] = Tout(x[perm[p] + j * ldx]);
        else
            y[perm[p] + j * ldy] = Tout(x[p + j * ldx]);
    }
}

__global__ void k_set_slot(int32_t *kd, int32_t slot, int32_t v) { kd[slot] = v; }

template <class T>
__global__ void k_to_work(const double *x, T *y, int64_t tot) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = T(x[e]);
}

template <class T>
__global__ void k_add_from_work(double *x, const T *y, int64_t tot) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
        x[e] += (double)y[e];
}

// r = b - ax per column j (one block row of columns per blockIdx.y), squared norms accumulated
__global__ void k_residual(const double *b, const double *ax, double *r, int64_t n, double *nrm2, double *bn2) {
    __shared__ double red[2][32];
    const int64_t j = blockIdx.y;
    double sr = 0.0, sb = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i + j * n], ri = bi - ax[i + j * n];
        r[i + j * n] = ri;
        sr += ri * ri;
        sb += bi * bi;
    }
    sr = warp_sum(sr);
    sb = warp_sum(sb);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = sr;
        red[1][w] = sb;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        sr = l < nw ? red[0][l] : 0.0;
        sb = l < nw ? red[1][l] : 0.0;
        sr = warp_sum(sr);
        sb = warp_sum(sb);
        if (l == 0) {
            atomicAdd(nrm2 + j, sr);
            atomicAdd(bn2 + j, sb);
        }
    }
}

// -------------------------------------------------------------- dispatch
size_t getrf_smem_bytes(int max_leaf, int elem) { return (size_t)max_leaf * max_leaf * elem; }

template <class T>
void launch_kind(int kind, const void *tasks, const Term *terms, const Piece *pieces, int start, int count,
                 int aux, const LaunchArgs &a, cudaStream_t s) {
    switch (kind) {
        case K_GETRF:
            k_getrf<T><<<count, kThreads, getrf_smem_bytes(aux, sizeof(T)), s>>>(
                reinterpret_cast<const TGetrf *>(tasks) + start, a);
            break;
        case K_TRSM:
            k_trsm<T><<<count, kThreads, getrf_smem_bytes(aux, sizeof(T)), s>>>(
                reinterpret_cast<const TTrsm *>(tasks) + start, a);
            break;
        case K_PROJECT:
            k_project<T><<<count, kThreads, 2 * 32 * 65 * sizeof(T), s>>>(
                reinterpret_cast<const TProject *>(tasks) + start, a);
            break;
        case K_ACCUM:
            k_accum<T><<<count, kThreads, 0, s>>>(reinterpret_cast<const TAccum *>(tasks) + start, terms, a);
            break;
        case K_RADD: {
            // at least the dense route's worst case (m n <= kSmallTarget) so that the
            // route a task takes does not depend on the schedule
            const size_t smem = std::max(radd_smem_bytes(aux), radd_smem_bytes(64));
            k_radd<T><<<count, kThreads, smem, s>>>(reinterpret_cast<const TRadd *>(tasks) + start, pieces, a, aux,
                                                    smem);
            break;
        }
        case K_SPLIT:
            k_split<T><<<count, kThreads, 0, s>>>(reinterpret_cast<const TSplit *>(tasks) + start, a);
            break;
        default:
            break;
    }
}

// Lets a kernel use all of the opt-in shared memory beside its static share.
template <class K>
static bool allow_dynamic_smem(K kernel, int optin) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return false;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes) == cudaSuccess;
}

template <class T>
bool set_kernel_attributes() {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    bool ok = allow_dynamic_smem(k_radd<T>, optin);
    ok = allow_dynamic_smem(k_getrf<T>, optin) && ok;
    ok = allow_dynamic_smem(k_trsm<T>, optin) && ok;
    ok = allow_dynamic_smem(k_project<T>, optin) && ok;
    ok = allow_dynamic_smem(k_dataflow<T>, optin) && ok;
    cudaGetLastError();  // a failure is reported through the return value, not left pending
    return ok;
}

size_t dataflow_smem_bytes(int max_leaf, int elem, int kc) {
    size_t s = getrf_smem_bytes(max_leaf, elem);
    s = std::max(s, (size_t)2 * 32 * 65 * elem);
    s = std::max(s, radd_smem_bytes(kc));
    return s;
}

template <class T>
int dataflow_workers(size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dataflow<T>, kThreads, smem) != cudaSuccess || per < 1)
        per = 1;
    return sms * per;
}

template <class T>
void launch_dataflow(const FlowArgs &f, const LaunchArgs &a, int grid, size_t smem, cudaStream_t s) {
    k_dataflow<T><<<grid, kThreads, smem, s>>>(f, a);
}

template int dataflow_workers<double>(size_t);
template int dataflow_workers<float>(size_t);
template void launch_dataflow<double>(const FlowArgs &, const LaunchArgs &, int, size_t, cudaStream_t);
template void launch_dataflow<float>(const FlowArgs &, const LaunchArgs &, int, size_t, cudaStream_t);

template <class T>
void launch_reset(const int64_t *leaf_desc, int64_t n_leaves, const double *aarena, T *farena, int32_t *kdyn,
                  cudaStream_t s) {
    if (n_leaves > 0) k_reset<T><<<(unsigned)n_leaves, kThreads, 0, s>>>(leaf_desc, aarena, farena, kdyn);
}

template <class Tin, class Tout>
void launch_permute(const int32_t *perm, int32_t n, int32_t nrhs, const Tin *x, int64_t ldx, Tout *y, int64_t ldy,
                    int to_cluster, cudaStream_t s) {
    const int64_t tot = (int64_t)n * nrhs;
    const int blocks = (int)std::min<int64_t>((tot + kThreads - 1) / kThreads, 152 * 8);
    if (tot > 0) k_permute<Tin, Tout><<<blocks, kThreads, 0, s>>>(perm, n, nrhs, x, ldx, y, ldy, to_cluster);
}

void launch_set_slot(int32_t *kdyn, int32_t slot, int32_t value, cudaStream_t s) {
    k_set_slot<<<1, 1, 0, s>>>(kdyn, slot, value);
}

static int grid_for(int64_t tot) { return (int)std::max<int64_t>(1, std::min<int64_t>((tot + kThreads - 1) / kThreads, 152 * 8)); }

template <class T>
void launch_to_work(const double *x, T *y, int64_t n, int32_t nc, cudaStream_t s) {
    const int64_t tot = n * nc;
    if (tot > 0) k_to_work<T><<<grid_for(tot), kThreads, 0, s>>>(x, y, tot);
}

template <class T>
void launch_add_from_work(double *x, const T *y, int64_t n, int32_t nc, cudaStream_t s) {
    const int64_t tot = n * nc;
    if (tot > 0) k_add_from_work<T><<<grid_for(tot), kThreads, 0, s>>>(x, y, tot);
}

void launch_residual(const double *b, const double *ax, double *r, int64_t n, int32_t nc, double *nrm2,
                     double *bn2, cudaStream_t s) {
    if (n * nc == 0) return;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 64));
    k_residual<<<dim3(gx, nc), kThreads, 0, s>>>(b, ax, r, n, nrm2, bn2);
}

template void launch_to_work<double>(const double *, double *, int64_t, int32_t, cudaStream_t);
template void launch_to_work<float>(const double *, float *, int64_t, int32_t, cudaStream_t);
template void launch_add_from_work<double>(double *, const double *, int64_t, int32_t, cudaStream_t);
template void launch_add_from_work<float>(double *, const float *, int64_t, int32_t, cudaStream_t);

template void launch_kind<double>(int, const void *, const Term *, const Piece *, int, int, int, const LaunchArgs &,
                                  cudaStream_t);
template void launch_kind<float>(int, const void *, const Term *, const Piece *, int, int, int, const LaunchArgs &,
                                 cudaStream_t);
template bool set_kernel_attributes<double>();
template bool set_kernel_attributes<float>();
template void launch_reset<double>(const int64_t *, int64_t, const double *, double *, int32_t *, cudaStream_t);
template void launch_reset<float>(const int64_t *, int64_t, const double *, float *, int32_t *, cudaStream_t);
template void launch_permute<double, double>(const int32_t *, int32_t, int32_t, const double *, int64_t, double *,
                                             int64_t, int, cudaStream_t);
template void launch_permute<double, float>(const int32_t *, int32_t, int32_t, const double *, int64_t, float *,
                                            int64_t, int, cudaStream_t);
template void launch_permute<float, double>(const int32_t *, int32_t, int32_t, const float *, int64_t, double *,
                                            int64_t, int, cudaStream_t);

}  // namespace hlu
