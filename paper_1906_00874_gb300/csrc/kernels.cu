// Device kernels of the H-LU task graph (sm_103a).  One CTA (256 threads)
// executes one task; the launch of a wave passes the slice of the task array
// that belongs to it.  T is the storage type of the factors (double or
// float).  With double factors every step is double.  With float factors the
// stacked QRs, the pivoted QR and the QR of R'^T of each truncation core are
// single precision, and the one-sided Jacobi SVD of the core is double
// (LaunchArgs::core64, the default) or single precision (the HLU_FP32_CORE32
// variant).
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>

#include <algorithm>

#include "kernels.cuh"

namespace hlu {

constexpr unsigned kFull = 0xffffffffu;

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

template <class R>
__device__ __forceinline__ R warp_sum_t(R v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ float warp_max_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Largest column count of a truncation core: the dense route takes n <= 128,
// the stacked route kv <= the stacked-rank limit (96).
constexpr int kVRows = 128;

// Cooperative copy of n elements: element e is read by src(e) and written by
// dst(e, v), one element per thread and step.
template <class T, class Src, class Dst>
__device__ __forceinline__ void block_copy(int n, Src src, Dst dst) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) dst(e, src(e));
}

// ------------------------------------------------------------------ GETRF
// Unpivoted LU of an m x m dense diagonal leaf in shared memory (Sec. 3.1,
// "Dense blocks": L unit lower and U overwrite A).
template <class T>
__device__ void dev_getrf(const TGetrf &t, const LaunchArgs &a, unsigned char *smem_raw) {
    T *s = reinterpret_cast<T *>(smem_raw);
    const int m = t.m;
    T *g = reinterpret_cast<T *>(a.arena) + t.off;
    block_copy<T>(m * m, [&](int e) { return g[e]; }, [&](int e, T v) { s[e] = v; });
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
// Triangular solve of an m x p panel with a dense diagonal leaf (m <= 128).
// The triangle is staged in shared memory (transposed for TR_UPPER_TRANS, so
// that every mode reads a column of L per step) with the reciprocals of its
// diagonal (ones for the unit lower factor).  Every panel column is solved by
// a group of 16 lanes, each holding R rows (lane + 16 r) in registers, 16
// columns at a time; the steps i are fully unrolled, so that the lane that
// owns x_i and the rows a step updates are known at compile time: step i
// scales x_i by the reciprocal pivot, broadcasts it within the group and
// subtracts its multiple of column i from the rows below (forward) or above
// (backward) it.
constexpr int kTrsmSlack = 128;  // zeroed elements after the triangle (reads past the last column)

size_t trsm_smem_bytes(int max_leaf, int elem) {
    return (size_t)(max_leaf * max_leaf + kTrsmSlack + max_leaf) * elem;
}

template <class T, int R>
__device__ __forceinline__ void trsm_group16(const T *L, const T *dinv, T *A, const Panel &P, int m, int p,
                                             bool forward) {
    constexpr int GS = 16;
    const int lane = threadIdx.x & (GS - 1), grp = threadIdx.x / GS, per_pass = blockDim.x / GS;
    for (int c0 = 0; c0 < p; c0 += per_pass) {
        const int c = c0 + grp;
        const bool live = c < p;  // dead groups still take part in the shuffles
        T *col_p = A + P.off + (int64_t)(live ? c : 0) * P.cs;
        T x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int row = lane + GS * r;
            x[r] = (live && row < m) ? col_p[(int64_t)row * P.rs] : T(0);
        }
        if (forward) {
#pragma unroll
            for (int ri = 0; ri < R; ++ri)
#pragma unroll
                for (int li = 0; li < GS; ++li) {
                    const int i = ri * GS + li;
                    if (i < m) {
                        if (lane == li) x[ri] *= dinv[i];
                        const T xi = __shfl_sync(kFull, x[ri], li, GS);
                        const T *col = L + i * m + lane;
                        if (lane > li) x[ri] -= col[GS * ri] * xi;
#pragma unroll
                        for (int r = ri + 1; r < R; ++r) x[r] -= col[GS * r] * xi;
                    }
                }
        } else {
#pragma unroll
            for (int ri = R - 1; ri >= 0; --ri)
#pragma unroll
                for (int li = GS - 1; li >= 0; --li) {
                    const int i = ri * GS + li;
                    if (i < m) {
                        if (lane == li) x[ri] *= dinv[i];
                        const T xi = __shfl_sync(kFull, x[ri], li, GS);
                        const T *col = L + i * m + lane;
                        if (lane < li) x[ri] -= col[GS * ri] * xi;
#pragma unroll
                        for (int r = 0; r < ri; ++r) x[r] -= col[GS * r] * xi;
                    }
                }
        }
        if (live) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = lane + GS * r;
                if (row < m) col_p[(int64_t)row * P.rs] = x[r];
            }
        }
    }
}

template <class T>
__device__ void dev_trsm(const TTrsm &t, const LaunchArgs &a, unsigned char *smem_raw) {
    const int mode = t.mode & 0xff;
    const int m = t.m, mm = m * m;
    T *L = reinterpret_cast<T *>(smem_raw);
    T *dinv = L + mm + kTrsmSlack;
    const T *g = reinterpret_cast<const T *>(a.arena) + t.L_off;
    if (mode == TR_UPPER_TRANS)  // L = U^T
        block_copy<T>(mm, [&](int e) { return g[e]; }, [&](int e, T v) {
            const int j = e / m;
            L[j + (e - j * m) * m] = v;
        });
    else
        block_copy<T>(mm, [&](int e) { return g[e]; }, [&](int e, T v) { L[e] = v; });
    for (int e = mm + threadIdx.x; e < mm + kTrsmSlack; e += blockDim.x) L[e] = T(0);
    __syncthreads();
    const bool unit = mode == TR_LOWER_UNIT;
    for (int i = threadIdx.x; i < m; i += blockDim.x) dinv[i] = unit ? T(1) : T(1) / L[i + i * m];
    T *A = reinterpret_cast<T *>(a.arena);
    const int p = dim_c(t.P, a.kdyn);
    if (threadIdx.x == 0 && !(t.mode & kTrsmNoFlops)) add_flops(a, K_TRSM, (double)m * m * p);
    const bool forward = mode != TR_UPPER;
    __syncthreads();
    if (m <= 32)
        trsm_group16<T, 2>(L, dinv, A, t.P, m, p, forward);
    else if (m <= 64)
        trsm_group16<T, 4>(L, dinv, A, t.P, m, p, forward);
    else
        trsm_group16<T, 8>(L, dinv, A, t.P, m, p, forward);
}

// ---------------------------------------------------------------- PROJECT
// T (k x p) = F^T X (F: len x k, X: len x p): the V^T z (or U^T z) half of a
// low-rank product (Sec. 3.1).  The output is cut into 4 x 4 tiles held in
// registers; the lanes of a warp take consecutive rows (coalesced loads of
// the 4 + 4 columns of the tile), kU rows per lane in flight at a time, and
// the 32 lane partials are added by shuffles.  With fewer tiles than warps,
// G warps share a tile (row groups) and their partials meet in shared memory.
size_t project_smem_bytes(int elem) { return (size_t)(kThreads / 32) * 16 * elem; }

template <class T>
__device__ void dev_project(const TProject &t, const LaunchArgs &a, unsigned char *smem_raw) {
    constexpr int kU = sizeof(T) == 8 ? 2 : 4;
    T *A = reinterpret_cast<T *>(a.arena);
    T *red = reinterpret_cast<T *>(smem_raw);
    const int len = dim_r(t.F, a.kdyn), k = dim_c(t.F, a.kdyn), p = dim_c(t.X, a.kdyn);
    if (threadIdx.x == 0 && !t.no_flops) add_flops(a, K_PROJECT, 2.0 * len * k * p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int ta = (k + 3) >> 2, tb = (p + 3) >> 2, ntile = ta * tb;
    if (ntile == 0) return;
    const int G = ntile >= nw ? 1 : nw / ntile, per = nw / G;
    const int64_t frs = t.F.rs, xrs = t.X.rs;
    for (int tile0 = 0; tile0 < ntile; tile0 += per) {
        const int tile = tile0 + warp / G, g = warp % G;
        const bool live = warp / G < per && tile < ntile;
        const int ia = (tile % ta) * 4, ib = (tile / ta) * 4;
        T acc[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) acc[s] = T(0);
        int na = 0, nb = 0;
        if (live) {
            na = min(4, k - ia);
            nb = min(4, p - ib);
            const T *pf[4], *px[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                pf[u] = A + t.F.off + (int64_t)(ia + min(u, na - 1)) * t.F.cs;
                px[u] = A + t.X.off + (int64_t)(ib + min(u, nb - 1)) * t.X.cs;
            }
            const int step = G * 32;
            int r = g * 32 + lane;
            for (; r + (kU - 1) * step < len; r += kU * step) {
                T f[kU][4], x[kU][4];
#pragma unroll
                for (int q = 0; q < kU; ++q)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        f[q][u] = pf[u][(int64_t)(r + q * step) * frs];
                        x[q][u] = px[u][(int64_t)(r + q * step) * xrs];
                    }
#pragma unroll
                for (int q = 0; q < kU; ++q)
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u * 4 + v] += f[q][u] * x[q][v];
            }
            for (; r < len; r += step) {
                T f[4], x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    f[u] = pf[u][(int64_t)r * frs];
                    x[u] = px[u][(int64_t)r * xrs];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u * 4 + v] += f[u] * x[v];
            }
        }
#pragma unroll
        for (int s = 0; s < 16; ++s) acc[s] = warp_sum_t(acc[s]);
        if (G > 1) {
            __syncthreads();
            if (lane == 0)
#pragma unroll
                for (int s = 0; s < 16; ++s) red[warp * 16 + s] = acc[s];
            __syncthreads();
            if (live && g == 0 && lane < 16) {
                T v = T(0);
                for (int q = 0; q < G; ++q) v += red[(warp + q) * 16 + lane];
                const int u = lane >> 2, w = lane & 3;
                if (u < na && w < nb) at(A, t.T, ia + u, ib + w) = v;
            }
        } else if (live && lane == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (u < na && w < nb) at(A, t.T, ia + u, ib + w) = acc[u * 4 + w];
        }
    }
}

// ------------------------------------------------------------------ ACCUM
// out (m x p) = beta out + alpha sum_t A_t X_t over the leaves that cover one
// leaf cluster of the output rows (dense leaves: A = D, X = panel slice;
// low-rank leaves: A = U slice, X = projected V^T z).  The term descriptors
// and their inner sizes are read in parallel into a shared table (at most
// kAccTerms at a time) with the exclusive prefix of the inner sizes.  The
// inner columns of all terms are then packed, as many as the CTA's shared
// memory holds, into an m x L matrix sA and an L x p matrix sX: a warp takes
// one packed column at a time and its lanes issue asynchronous global-to-
// shared copies (cp.async) of that column's rows, so that all copies of a
// batch are in flight together; one wait, then the batch is consumed as a
// small GEMM from shared memory, every thread owning up to 4 outputs of a row.
constexpr int kAccTerms = 64, kAccCols = 1024;

__host__ __device__ constexpr size_t accum_header_bytes() {
    return (kAccTerms * sizeof(Term) + sizeof(int) * (kAccTerms + 1 + kAccCols) + 15) & ~size_t(15);
}

size_t accum_smem_bytes(int elem) { return accum_header_bytes() + (size_t)12288 * elem; }

template <class T>
__device__ __forceinline__ void cp_async_el(T *dst_smem, const T *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst_smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ int accum_load_terms(const TAccum &t, const Term *terms, const LaunchArgs &a, Term *sT,
                                                int *sP, int q0, int nq);
struct TcState;
__device__ bool dev_accum_tc(const TAccum &t, const Term *terms, const LaunchArgs &a, unsigned char *smem_raw,
                             size_t smem_bytes, TcState &tc, int m, int p);
__device__ __forceinline__ bool tc_on(const TcState *tc);

// TC: the kernel that calls this holds the tensor-core form (only the data-flow kernel does; a
// kernel with tcgen05 code in it needs the TMEM permit handling of k_dataflow).
template <class T, bool TC = false>
__device__ void dev_accum(const TAccum &t, const Term *terms, const LaunchArgs &a, unsigned char *smem_raw,
                          size_t smem_bytes, TcState *tc = nullptr) {
    T *A = reinterpret_cast<T *>(a.arena);
    Term *sT = reinterpret_cast<Term *>(smem_raw);
    int *sP = reinterpret_cast<int *>(sT + kAccTerms);  // exclusive prefix of the inner sizes
    int *sC = sP + kAccTerms + 1;                      // packed column -> (term << 16) | column
    T *sm = reinterpret_cast<T *>(smem_raw + accum_header_bytes());
    const int data = (int)((smem_bytes - accum_header_bytes()) / sizeof(T));
    const int m = dim_r(t.out, a.kdyn);
    const int p = t.dst >= 0 ? a.kdyn[t.src] : dim_c(t.out, a.kdyn);
    if (t.dst >= 0 && threadIdx.x == 0) a.kdyn[t.dst] = p;
    if (m == 0 || p == 0) return;
    bool loaded = false;  // the table of term batch 0 is in shared memory
    if constexpr (TC && sizeof(T) == 4) {
        // dense products with at least 32 rows and 16 columns go to the tensor cores
        if (tc_on(tc) && m >= 32 && m <= kMaxLeafRows && p >= 16) {
            if (dev_accum_tc(t, terms, a, smem_raw, smem_bytes, *tc, m, p)) return;
            loaded = true;
        }
    }
    const T alpha = T(t.alpha);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int kSlots = 4;  // (row, 4-column block) outputs per thread
    // output column tiles of pb columns: m * ceil(pb / 4) <= kSlots * blockDim
    const int pbmax = max(4, min((p + 3) & ~3, 4 * (kSlots * (int)blockDim.x / m)));
    for (int b0 = 0; b0 < p; b0 += pbmax) {
        const int pb = min(pbmax, p - b0);
        const int Lcap = min(kAccCols, data / (m + pb));  // >= 1
        T *sA = sm, *sX = sm + m * Lcap;                 // sA: m x Lcap (ld m); sX: Lcap x pb (ld Lcap)
        const int work = m * ((pb + 3) >> 2);
        T acc[kSlots][4];
#pragma unroll
        for (int s = 0; s < kSlots; ++s)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[s][u] = T(0);
        for (int q0 = 0; q0 < t.nterms; q0 += kAccTerms) {
            const int nq = min(kAccTerms, t.nterms - q0);
            const int Ltot = (loaded && b0 == 0 && q0 == 0) ? sP[nq] : accum_load_terms(t, terms, a, sT, sP, q0, nq);
            if (b0 == 0 && q0 == 0 && threadIdx.x == 0 && t.credit > 0.0f) add_flops(a, K_ACCUM, (double)t.credit * p);
            if (b0 == 0 && threadIdx.x == 0 && t.credit == 0.0f) add_flops(a, K_ACCUM, 2.0 * m * (double)Ltot * p);
            for (int c0 = 0; c0 < Ltot; c0 += Lcap) {
                const int L = min(Lcap, Ltot - c0);
                if (c0 > 0) __syncthreads();  // the previous batch is consumed
                for (int lb = threadIdx.x; lb < L; lb += blockDim.x) {
                    const int gc = c0 + lb;
                    int lo = 0, hi = nq - 1;  // largest q with sP[q] <= gc (a non-empty term)
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sP[mid] <= gc)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    sC[lb] = (lo << 16) | (gc - sP[lo]);
                }
                __syncthreads();
                for (int lb = warp; lb < L; lb += nw) {
                    const int c = sC[lb], q = c >> 16, l = c & 0xffff;
                    const Panel &PA = sT[q].A;
                    const T *ca = A + PA.off + (int64_t)l * PA.cs;
                    for (int i = lane; i < m; i += 32) cp_async_el(sA + lb * m + i, ca + (int64_t)i * PA.rs);
                    const Panel &PX = sT[q].X;
                    const T *cx = A + PX.off + (int64_t)l * PX.rs + (int64_t)b0 * PX.cs;
                    for (int j = lane; j < pb; j += 32) cp_async_el(sX + lb + j * Lcap, cx + (int64_t)j * PX.cs);
                }
                cp_async_wait_all();
                __syncthreads();
#pragma unroll
                for (int s = 0; s < kSlots; ++s) {
                    const int w = threadIdx.x + s * blockDim.x;
                    if (w < work) {
                        const int jb = w / m, i = w - jb * m, j0 = jb * 4;
                        const T *pa = sA + i;
                        const T *px = sX + j0 * Lcap;
                        const int x1 = min(1, pb - 1 - j0) * Lcap, x2 = min(2, pb - 1 - j0) * Lcap,
                                  x3 = min(3, pb - 1 - j0) * Lcap;
                        T a0 = acc[s][0], a1 = acc[s][1], a2 = acc[s][2], a3 = acc[s][3];
                        for (int lb = 0; lb < L; ++lb) {
                            const T av = pa[lb * m];
                            a0 += av * px[lb];
                            a1 += av * px[lb + x1];
                            a2 += av * px[lb + x2];
                            a3 += av * px[lb + x3];
                        }
                        acc[s][0] = a0;
                        acc[s][1] = a1;
                        acc[s][2] = a2;
                        acc[s][3] = a3;
                    }
                }
            }
        }
        // outputs of the tile (also without terms: an overwrite clears them)
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const int w = threadIdx.x + s * blockDim.x;
            if (w < work) {
                const int jb = w / m, i = w - jb * m, j0 = jb * 4;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (j0 + u < pb) {
                        T &o = at(A, t.out, i, b0 + j0 + u);
                        o = (t.overwrite ? T(0) : o) + alpha * acc[s][u];
                    }
            }
        }
    }
}

// ------------------------------------------------------ ACCUM on tensor cores
// Dense products of the factorisation on the 5th-generation tensor cores (tcgen05), for
// single-precision factors: one output tile of 128 rows (the leaf cluster, zero rows beyond m)
// by Np <= 128 columns accumulates in tensor memory (TMEM, FP32) over the packed inner columns of
// all terms.  Each operand value v is split into two TF32 parts, hi = tf32(v), lo = tf32(v - hi),
// and the tile takes A_hi X_hi + A_hi X_lo + A_lo X_hi (three MMAs of kind::tf32 per K step of 8),
// which keeps the products at FP32 accuracy (the dropped A_lo X_lo term is below 2^-21 of the
// product).  Operands are staged in shared memory in the K-major, unswizzled layout of the MMA
// descriptors: 8-row core matrices of 16 bytes per row, adjacent in K at 128 bytes (leading byte
// offset) and in M / N at 256 bytes (stride byte offset), one block of rows x 8 per K step.  One
// thread issues the MMAs and commits them to an mbarrier that every thread waits on (with a
// deadline) before the staged operands are overwritten or the accumulator is read back with
// tcgen05.ld (warp w reads TMEM lanes 32 (w % 4) ... and half (w / 4) of the columns).
struct TcState {
    uint32_t tmem;   // TMEM address of the accumulators (128 lanes x kTcTmemCols columns)
    uint32_t mbar;   // shared address of the MMA-completion mbarrier
    uint32_t phase;  // parity of the mbarrier phase to wait for next
    bool on;
    unsigned long long timeout_ns;
    int min_inner;
};

// Tiles of at most 128 output columns, one accumulator per tile (128 TMEM columns per worker).  The
// MMAs of a tile may also rotate over kTcAccs accumulators (added in a fixed order by the epilogue)
// so that consecutive MMAs do not wait on each other's results; with four (4 x 64 columns) the
// products of the factorisations here were no faster, so one is used.
constexpr int kTcRows = 128, kTcMaxCols = 128, kTcAccs = 1, kTcTmemCols = kTcAccs * kTcMaxCols;

__device__ __forceinline__ bool tc_on(const TcState *tc) { return tc && tc->on; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, LBO 128 B (K direction), SBO 256 B (M / N).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, k) in a K-major tile of `rows` rows: [k / 8][row / 8][(k / 4) % 2][row % 8][k % 4].
__device__ __forceinline__ uint32_t tc_off(int row, int k, int rows) {
    return (uint32_t)((k >> 3) * rows * 32 + (row >> 3) * 256 + ((k >> 2) & 1) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ unsigned long long tc_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (every thread) for the MMAs committed last; false on timeout (error recorded).
__device__ __forceinline__ bool tc_wait(TcState &tc, const LaunchArgs &a) {
    const unsigned long long deadline = tc_now() + tc.timeout_ns;
    uint32_t ok = 0;
    for (;;) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(tc.mbar), "r"(tc.phase)
            : "memory");
        if (ok) break;
        if (tc_now() > deadline) {
            if (threadIdx.x == 0) set_error(a.err, DE_TIMEOUT, -1, 0.0);
            return false;
        }
    }
    tc.phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return true;
}

// Inclusive scan of the inner sizes of a term batch into sP (exclusive prefix, sP[0] = 0), the
// batch's descriptors into sT; returns the batch's packed inner size.  Ends with a barrier.
__device__ __forceinline__ int accum_load_terms(const TAccum &t, const Term *terms, const LaunchArgs &a, Term *sT,
                                                int *sP, int q0, int nq) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();  // the previous table and batch are no longer read
    if ((int)threadIdx.x < nq) {
        const Term tm = terms[t.term0 + q0 + threadIdx.x];
        sT[threadIdx.x] = tm;
        sP[threadIdx.x + 1] = dim_c(tm.A, a.kdyn);
    }
    __syncthreads();
    if (warp == 0) {
        int carry = 0;
        for (int base = 0; base < nq; base += 32) {
            const int q = base + lane;
            int v = q < nq ? sP[q + 1] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, v, o);
                if (lane >= o) v += y;
            }
            if (q < nq) sP[q + 1] = v + carry;
            carry += __shfl_sync(kFull, v, 31);
        }
        if (lane == 0) sP[0] = 0;
    }
    __syncthreads();
    return sP[nq];
}

// The tensor-core form of dev_accum (single precision, m <= 128).  Returns false, before writing
// anything, when the task is too small to gain (one term batch with fewer than tc.min_inner inner
// columns): the caller then takes the CUDA-core form with the term table of that batch already in
// shared memory.
__device__ bool dev_accum_tc(const TAccum &t, const Term *terms, const LaunchArgs &a, unsigned char *smem_raw,
                             size_t smem_bytes, TcState &tc, int m, int p) {
    float *A = reinterpret_cast<float *>(a.arena);
    Term *sT = reinterpret_cast<Term *>(smem_raw);
    int *sP = reinterpret_cast<int *>(sT + kAccTerms);
    int *sC = sP + kAccTerms + 1;
    unsigned char *data = smem_raw + accum_header_bytes();
    const size_t dbytes = smem_bytes - accum_header_bytes();
    const float alpha = float(t.alpha);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m8 = (m + 7) & ~7;
    // tile rows: M = 64 when the leaf cluster fits (its accumulator row r sits in TMEM lane
    // 32 (r / 16) + r % 16), else M = 128 (row r in lane r)
    const int MT = m <= 64 ? 64 : kTcRows;
    const int nw = blockDim.x >> 5;
    for (int b0 = 0; b0 < p; b0 += kTcMaxCols) {
        const int pb = min(kTcMaxCols, p - b0), Np = (pb + 15) & ~15;
        // tiles hi / lo of A (MT x Lc) and X^T (Np x Lc), then the raw operands as copied: A (m x Lc,
        // ld m) and X (Lc x pb, ld Lc)
        const int Lc = min(128, (int)(dbytes / (4 * (size_t)(3 * MT + 3 * Np))) & ~7);
        if (Lc < 8) return b0 > 0;  // (not reached: every worker has room for 8 inner columns)
        unsigned char *Ahi = data, *Alo = Ahi + (size_t)MT * Lc * 4;
        unsigned char *Xhi = Alo + (size_t)MT * Lc * 4, *Xlo = Xhi + (size_t)Np * Lc * 4;
        float *rawA = reinterpret_cast<float *>(Xlo + (size_t)Np * Lc * 4);
        float *rawX = rawA + (size_t)MT * Lc;
        bool pending = false;
        int nmma = 0;  // MMAs issued for this tile (uniform); accumulator j holds data once nmma > j
        // rows m8 .. MT - 1 of the A tiles stay zero for the whole tile
        for (int l = warp; l < Lc; l += nw)
            for (int i = m8 + lane; i < MT; i += 32) {
                const uint32_t o = tc_off(i, l, MT);
                *reinterpret_cast<float *>(Ahi + o) = 0.0f;
                *reinterpret_cast<float *>(Alo + o) = 0.0f;
            }
        for (int q0 = 0; q0 < t.nterms; q0 += kAccTerms) {
            const int nq = min(kAccTerms, t.nterms - q0);
            const int Ltot = accum_load_terms(t, terms, a, sT, sP, q0, nq);  // (the MMAs read only the tiles)
            if (b0 == 0 && q0 == 0 && Ltot < tc.min_inner && t.nterms <= kAccTerms) return false;  // uniform;
            // the caller reuses the loaded table of batch 0
            if (b0 == 0 && q0 == 0 && threadIdx.x == 0 && t.credit > 0.0f) add_flops(a, K_ACCUM, (double)t.credit * p);
            if (b0 == 0 && threadIdx.x == 0 && t.credit == 0.0f) add_flops(a, K_ACCUM, 2.0 * m * (double)Ltot * p);
            for (int c0 = 0; c0 < Ltot; c0 += Lc) {
                const int L = min(Lc, Ltot - c0), Lp = (L + 7) & ~7;
                for (int lb = threadIdx.x; lb < L; lb += blockDim.x) {
                    const int gc = c0 + lb;
                    int lo = 0, hi = nq - 1;  // largest q with sP[q] <= gc (a non-empty term)
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sP[mid] <= gc)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    sC[lb] = (lo << 16) | (gc - sP[lo]);
                }
                __syncthreads();
                // raw operands by asynchronous copies (one packed column per warp and step, all copies
                // of the chunk in flight), while the tensor cores may still read the previous tiles
                for (int lb = warp; lb < L; lb += nw) {
                    const int c = sC[lb], q = c >> 16, l = c & 0xffff;
                    const Panel &PA = sT[q].A;
                    const float *ca = A + PA.off + (int64_t)l * PA.cs;
                    for (int i = lane; i < m; i += 32) cp_async_el(rawA + lb * m + i, ca + (int64_t)i * PA.rs);
                    const Panel &PX = sT[q].X;
                    const float *cx = A + PX.off + (int64_t)l * PX.rs + (int64_t)b0 * PX.cs;
                    for (int j = lane; j < pb; j += 32) cp_async_el(rawX + lb + j * Lc, cx + (int64_t)j * PX.cs);
                }
                cp_async_wait_all();
                if (pending) {
                    if (!tc_wait(tc, a)) return true;
                    pending = false;
                }
                __syncthreads();
                // split into the TF32 tiles: A rows < m8, X^T rows < Np, inner columns < Lp (zero beyond)
                for (int l = warp; l < Lp; l += nw)
                    for (int i = lane; i < m8; i += 32) {
                        const float v = (i < m && l < L) ? rawA[i + l * m] : 0.0f;
                        const float h = tf32_rna(v);
                        const uint32_t o = tc_off(i, l, MT);
                        *reinterpret_cast<float *>(Ahi + o) = h;
                        *reinterpret_cast<float *>(Alo + o) = tf32_rna(v - h);
                    }
                for (int n = warp; n < Np; n += nw)
                    for (int l = lane; l < Lp; l += 32) {
                        const float v = (n < pb && l < L) ? rawX[l + n * Lc] : 0.0f;
                        const float h = tf32_rna(v);
                        const uint32_t o = tc_off(n, l, Np);
                        *reinterpret_cast<float *>(Xhi + o) = h;
                        *reinterpret_cast<float *>(Xlo + o) = tf32_rna(v - h);
                    }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (threadIdx.x == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t idesc = tc_idesc(MT, Np);
                    const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), xh = smem_u32(Xhi), xl = smem_u32(Xlo);
                    int k = nmma;
                    for (int ks = 0; ks < Lp / 8; ++ks) {
                        const uint32_t ao = ks * MT * 32, xo = ks * Np * 32;
                        const uint32_t pa[3] = {ah + ao, ah + ao, al + ao}, px[3] = {xh + xo, xl + xo, xh + xo};
#pragma unroll
                        for (int u = 0; u < 3; ++u, ++k) {
                            const uint32_t d = tc.tmem + (uint32_t)((k % kTcAccs) * kTcMaxCols);
                            tc_mma(d, tc_desc(pa[u]), tc_desc(px[u]), idesc, k >= kTcAccs ? 1u : 0u);
                        }
                    }
                    tc_commit(tc.mbar);
                }
                nmma += 3 * (Lp / 8);
                pending = true;
            }
        }
        if (pending && !tc_wait(tc, a)) return true;
        // epilogue: out = beta out + alpha acc over rows < m and columns < pb of the tile; warp w reads
        // TMEM lanes 32 (w % 4) .. + 31 and half w / 4 of the columns
        const int row = MT == 64 ? (lane < 16 ? 16 * (warp & 3) + lane : kTcRows) : 32 * (warp & 3) + lane;
        const int half = Np >> 1, cbeg = (warp >> 2) * half;
        for (int c8 = cbeg; c8 < cbeg + half; c8 += 8) {
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int q = 0; q < kTcAccs && q < nmma; ++q) {  // uniform: every lane loads
                uint32_t v[8];
                const uint32_t ta = tc.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(q * kTcMaxCols + c8);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7])
                             : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] += __uint_as_float(v[j]);
            }
            if (row < m)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (c8 + j < pb) {
                        float &o = at(A, t.out, row, b0 + c8 + j);
                        o = (t.overwrite ? 0.0f : o) + alpha * acc[j];
                    }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // the accumulator is read before the next tile's MMAs overwrite it
    }
    return true;
}

// ------------------------------------------------------------------ SPLIT
template <class T>
__device__ void dev_split(const TSplit &t, const LaunchArgs &a) {
    T *A = reinterpret_cast<T *>(a.arena);
    const int k = a.kdyn[t.src_kslot];
    if (threadIdx.x == 0) a.kdyn[t.dst_kslot] = k;
    block_copy<T>(
        t.mu * k, [&](int e) { return at(A, t.srcU, e % t.mu, e / t.mu); },
        [&](int e, T v) { A[t.dstU + e] = v; });
    block_copy<T>(
        t.nv * k, [&](int e) { return at(A, t.srcV, e % t.nv, e / t.nv); },
        [&](int e, T v) { A[t.dstV + e] = v; });
}

// ------------------------------------------------------------------- RADD

// Named barrier over `count` threads (a multiple of 32); id 0 with the whole
// CTA is __syncthreads.
__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Householder QR of the m x K panel W (column major, leading dimension m) in
// place, in precision T, by the nw warps [w0, w0 + nw) of the CTA, which
// synchronise on named barrier `bar`.  Reflector j is H_j = I - tau_j v_j
// v_j^T with v_j[j] = 1 implied and v_j[i > j] stored below the diagonal; R
// is left in the upper triangle.  One barrier per column: in step j every
// warp forms the scalars of reflector j itself from the squared norm of
// column j below row j - 1 (left in nrm[j] by the warp that updated that
// column in step j - 1) and applies it to its own columns with v_j[i] =
// x[i] / v0 taken on the fly; after the barrier the warp j mod nw writes v_j
// back.  nrm holds min(m, K) entries.
template <class T>
__device__ void group_householder_qr(T *W, int m, int K, T *tau, T *nrm, int w0, int nw, int bar) {
    const int warp = (int)(threadIdx.x >> 5) - w0, lane = threadIdx.x & 31, nthr = nw * 32;
    const int kk = min(m, K);
    if (kk == 0) return;  // uniform over the group
    if (warp == 0) {
        T s = T(0);
        for (int i = lane; i < m; i += 32) s += W[i] * W[i];
        s = warp_sum_t(s);
        if (lane == 0) nrm[0] = s;
    }
    bar_sync(bar, nthr);
    for (int j = 0; j < kk; ++j) {
        T *x = W + (int64_t)j * m;
        const T nr = sqrt(nrm[j]);
        const T x0 = x[j];
        T alpha = T(0), inv = T(0), tj = T(0);
        if (nr > T(0)) {
            alpha = x0 >= T(0) ? -nr : nr;
            inv = T(1) / (x0 - alpha);
            tj = (alpha - x0) / alpha;
        }
        // each warp updates its columns c = j + 1 + warp + nw t four at a time (overlapping the
        // shuffle reductions); the warp that holds column j + 1 also leaves its norm below row j
        for (int c0 = j + 1 + warp; c0 < K; c0 += 4 * nw) {
            T *y[4];
            T d[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c0 + q * nw;
                y[q] = W + (int64_t)(c < K ? c : j) * m;  // column j stands in (read only)
                d[q] = T(0);
            }
            for (int i = j + 1 + lane; i < m; i += 32) {
                const T xi = x[i] * inv;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c0 + q * nw < K) d[q] += xi * y[q][i];
            }
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (sizeof(T) != 8 || c0 + q * nw < K) d[q] += __shfl_xor_sync(kFull, d[q], o);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (sizeof(T) != 8 || c0 + q * nw < K) d[q] = (d[q] + y[q][j]) * tj;
            __syncwarp();
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c0 + q * nw < K) y[q][j] -= d[q];
            const bool pivot = c0 == j + 1 && c0 < kk;  // q = 0 is the next pivot column
            T t2 = T(0);
            for (int i = j + 1 + lane; i < m; i += 32) {
                const T xi = x[i] * inv;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c0 + q * nw < K) {
                        const T yi = y[q][i] - d[q] * xi;
                        y[q][i] = yi;
                        if (q == 0) t2 += yi * yi;
                    }
            }
            if (pivot) {
                t2 = warp_sum_t(t2);
                if (lane == 0) nrm[c0] = t2;
            }
        }
        bar_sync(bar, nthr);
        if (warp == j % nw) {
            for (int i = j + 1 + lane; i < m; i += 32) x[i] = x[i] * inv;
            if (lane == 0) {
                x[j] = alpha;
                tau[j] = tj;
            }
        }
    }
    bar_sync(bar, nthr);
}

// y := Q y for one column y (length m) with Q = H_0 ... H_{kk-1} from
// group_householder_qr; executed by one warp.
template <class T>
__device__ void warp_apply_q(const T *W, int m, int kk, const T *tau, T *y) {
    const int lane = threadIdx.x & 31;
    for (int j = kk - 1; j >= 0; --j) {
        const T *x = W + (int64_t)j * m;
        T d = T(0);
        for (int i = j + 1 + lane; i < m; i += 32) d += x[i] * y[i];
        d = warp_sum_t(d);
        d = (d + y[j]) * tau[j];
        __syncwarp();
        if (lane == 0) y[j] -= d;
        for (int i = j + 1 + lane; i < m; i += 32) y[i] -= d * x[i];
        __syncwarp();
    }
}

// y := Q y with Q = H_0 ... H_{kk-1} from group_householder_qr (reflector j in column j of W,
// leading dimension ld, entries below row j for rows < len, v_j[j] = 1), for one column held in
// the registers of a warp: row i = lane + 32 k in y[k] (len <= kVRows).
template <class T, int NK>
__device__ __forceinline__ void reg_apply_q_n(const T *W, int ld, int len, int kk, const T *tau, T (&y)[kVRows / 32]) {
    const int lane = threadIdx.x & 31;
    for (int j = kk - 1; j >= 0; --j) {
        const T *x = W + (int64_t)j * ld;
        T xv[NK];
        T d = T(0);
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const int i = lane + 32 * k;
            xv[k] = i == j ? T(1) : (i > j && i < len ? x[i] : T(0));
            d += xv[k] * y[k];
        }
        d = warp_sum_t(d) * tau[j];
#pragma unroll
        for (int k = 0; k < NK; ++k) y[k] -= d * xv[k];
    }
}

// In double precision only the register rows that hold rows < len take part (no arithmetic on the
// zero rows: on the FP64 pipe of this part every operation counts).
template <class T>
__device__ __forceinline__ void reg_apply_q(const T *W, int ld, int len, int kk, const T *tau, T (&y)[kVRows / 32]) {
    if constexpr (sizeof(T) != 8) {  // single precision: one code path (smaller kernel) is faster
        reg_apply_q_n<T, 4>(W, ld, len, kk, tau, y);
        return;
    }
    switch ((len + 31) >> 5) {
        case 0:
            break;
        case 1:
            reg_apply_q_n<T, 1>(W, ld, len, kk, tau, y);
            break;
        case 2:
            reg_apply_q_n<T, 2>(W, ld, len, kk, tau, y);
            break;
        case 3:
            reg_apply_q_n<T, 3>(W, ld, len, kk, tau, y);
            break;
        default:
            reg_apply_q_n<T, 4>(W, ld, len, kk, tau, y);
    }
}

// x 2^-k rounded toward zero to single precision, by integer operations on the bit pattern (they
// run on the integer pipe; on this part a double-precision conversion instruction takes a slot of
// the narrow FP64 pipe).  Zero, subnormal and underflowing values give a signed zero, values
// above the single-precision range (and infinities) a signed infinity.
__device__ __forceinline__ float dbl_to_flt_scaled(double x, int k) {
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sign = (unsigned)hi & 0x80000000u;
    const int ex = (hi >> 20) & 0x7ff;
    const int fe = ex - 1023 - k + 127;
    if (ex == 0 || fe <= 0) return __uint_as_float(sign);
    if (fe >= 255 || ex == 0x7ff) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)fe << 23) | (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29));
}

// A normal single-precision value in double precision (exact), by integer operations; zero and
// subnormal values give a signed zero.
__device__ __forceinline__ double flt_to_dbl(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const int fe = (u >> 23) & 0xff;
    if (fe == 0) return __hiloint2double((int)sign, 0);
    const unsigned m = u & 0x7fffffu;
    return __hiloint2double((int)(sign | ((unsigned)(fe - 127 + 1023) << 20) | (m >> 3)), (int)(m << 29));
}

// Jacobi rotation (c, s) that makes columns x, y with x.x = aa, y.y = bb,
// x.y = gg orthogonal: t = tan(theta) is the smaller root of
// t^2 + 2 zeta t - 1 = 0, zeta = (bb - aa) / (2 gg) (Rutishauser's form), and
// c = 1 / sqrt(1 + t^2), s = c t.  The angle is evaluated in single precision
// (zeta from a power-of-two scaling of both operands, so that it neither
// overflows nor underflows), then (c, s) is renormalised in double by the
// series 1 / sqrt(1 + d) = 1 - d / 2 + 3 d^2 / 8 + O(d^3), d = c^2 + s^2 - 1
// (|d| ~ 1e-7, so the neglected term is below double rounding): the rotation
// is orthogonal to double precision, and only its angle is single-precision
// accurate, which the convergence test on the double dot products absorbs.
__device__ __forceinline__ void jacobi_rotation(double aa, double bb, double gg, double &c, double &s,
                                                double &tan_theta) {
    const double q = bb - aa;
    // 2 gg and q scaled by 2^-e, e the binary exponent of 2 gg, as single-precision values
    int e = (int)((__double2hiint(gg) >> 20) & 0x7ff) - 1023 + 1;
    e = max(-1000, min(1000, e));
    const float pf = dbl_to_flt_scaled(gg, e - 1), qf = dbl_to_flt_scaled(q, e);
    const float z = qf / pf, az = fabsf(z);
    float t;
    if (!(az < 1e15f))
        t = isinf(z) ? 0.0f : 0.5f / z;  // t ~ 1 / (2 zeta); z = +-inf: a negligible angle
    else
        t = copysignf(1.0f, z) / (az + sqrtf(fmaf(z, z, 1.0f)));
    const float cf = rsqrtf(fmaf(t, t, 1.0f));
    const double cd = flt_to_dbl(cf), sd = flt_to_dbl(cf * t);
    const double d = fma(cd, cd, fma(sd, sd, -1.0));
    const double f = fma(d, fma(0.375, d, -0.5), 1.0);
    c = cd * f;
    s = sd * f;
    tan_theta = flt_to_dbl(t);
}

// One-sided (Hestenes) Jacobi on the columns of D (r x r, double, shared
// memory, leading dimension ld), in place: D W = B with orthogonal columns
// (W is not formed); the singular values of D are the column norms of B and
// B = U_D Sigma holds its left singular vectors.  Round-robin ordering; the r/2 pairs of a round are
// taken by groups of g lanes (g a power of two: the largest that is useful
// for r rows and fits the CTA), each lane holding rows i = lane, lane + g, ...
// of both columns; when all groups fit in one warp, the rounds run in that
// warp alone with warp barriers.  A pair is rotated while
// |x.y|^2 > tol^2 |x|^2 |y|^2 with tol = 4 r eps_double, the rounding level of
// the dot product itself; at most 30 sweeps.  The squared column norms are
// computed exactly at the start of every sweep (nrm, r values of shared
// memory) and carried through its rounds by the rotation's own update
// (x.x - t x.y, y.y + t x.y, t = tan theta), so a round forms only the dot
// product x.y: one reduction instead of three on the FP64 pipe.  The norms only
// steer the rotations and the test; the singular values are formed from the
// final columns by the caller.  Returns the number of sweeps.
__device__ int block_jacobi(double *D, int r, int ld, int *flag, double *nrm) {
    if (r < 2) return 0;
    const int np = (r + 1) & ~1, P = np / 2;
    int g = 32;
    while (g > 1 && g * P > (int)blockDim.x) g >>= 1;
    while (g > 1 && (g >> 1) >= r) g >>= 1;
    const bool one_warp = g * P <= 32;
    const int gid = threadIdx.x / g, gl = threadIdx.x % g;
    const double tol = 4.0 * r * DBL_EPSILON, tol2 = tol * tol;
    int sweep = 0;
    while (sweep < 30) {
        ++sweep;
        if (threadIdx.x == 0) *flag = 0;
        for (int j = threadIdx.x; j < r; j += blockDim.x) {
            const double *cj = D + (int64_t)j * ld;
            double v = 0.0;
            for (int i = 0; i < r; ++i) v = fma(cj[i], cj[i], v);
            nrm[j] = v;
        }
        __syncthreads();
        if (!one_warp || threadIdx.x < 32) {  // uniform per warp
            for (int rd = 0; rd < np - 1; ++rd) {
                int p, q;
                if (gid == 0) {
                    p = rd;
                    q = np - 1;
                } else {
                    p = (rd + gid) % (np - 1);
                    q = (rd - gid + np - 1) % (np - 1);
                }
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                const bool active = gid < P && q < r;
                double *cp = D + (int64_t)p * ld, *cq = D + (int64_t)q * ld;
                double gg = 0.0;
                if (active)
                    for (int i = gl; i < r; i += g) gg = fma(cp[i], cq[i], gg);
                for (int o = g >> 1; o > 0; o >>= 1)  // every lane of the warp takes part
                    gg += __shfl_xor_sync(kFull, gg, o);
                // the butterfly leaves identical sums in every lane of a group
                const double aa = active ? nrm[p] : 0.0, bb = active ? nrm[q] : 0.0;
                if (active && gg * gg > tol2 * aa * bb) {
                    if (gl == 0) *flag = 1;
                    double cs, sn, tn;
                    jacobi_rotation(aa, bb, gg, cs, sn, tn);
                    for (int i = gl; i < r; i += g) {
                        const double x = cp[i], y = cq[i];
                        cp[i] = cs * x - sn * y;
                        cq[i] = sn * x + cs * y;
                    }
                    if (gl == 0) {
                        nrm[p] = fma(-tn, gg, aa);
                        nrm[q] = fma(tn, gg, bb);
                    }
                }
                if (one_warp)
                    __syncwarp();
                else
                    __syncthreads();
            }
        }
        __syncthreads();
        const int f = *flag;
        __syncthreads();
        if (!f) break;
    }
    return sweep;
}

// The same rotation entirely in single precision, for cores whose data are
// single precision (their singular values are only known to that level).
__device__ __forceinline__ void jacobi_rotation_f(float aa, float bb, float gg, float &c, float &s) {
    const float z = (bb - aa) / (2.0f * gg), az = fabsf(z);
    float t;
    if (!(az < 1e15f))
        t = isinf(z) ? 0.0f : 0.5f / z;
    else
        t = copysignf(1.0f, z) / (az + sqrtf(fmaf(z, z, 1.0f)));
    c = rsqrtf(fmaf(t, t, 1.0f));
    s = c * t;
}

// One-sided Jacobi in single precision on the columns of X (r x r, shared
// memory, leading dimension r), in place, with the rotations accumulated in W
// (r x r, W = I on entry): X_in W = X_out = B with orthogonal columns, W
// orthogonal.  Same round-robin ordering and lane groups as block_jacobi; a
// pair is rotated while |x.y| > tol |x| |y|, tol = 4 r eps_single.  X should
// be scaled so that its largest entry is near 1 (no overflow of the squared
// norms).  Returns the number of sweeps (at most 30).
__device__ int block_jacobi_f(float *X, float *W, int r, int *flag) {
    if (r < 2) return 0;
    const int np = (r + 1) & ~1, P = np / 2;
    int g = 32;
    while (g > 1 && g * P > (int)blockDim.x) g >>= 1;
    while (g > 1 && (g >> 1) >= r) g >>= 1;
    const bool one_warp = g * P <= 32;
    const int gid = threadIdx.x / g, gl = threadIdx.x % g;
    const float tol = 4.0f * r * FLT_EPSILON;
    int sweep = 0;
    while (sweep < 30) {
        ++sweep;
        if (threadIdx.x == 0) *flag = 0;
        __syncthreads();
        if (!one_warp || threadIdx.x < 32) {  // uniform per warp
            for (int rd = 0; rd < np - 1; ++rd) {
                int p, q;
                if (gid == 0) {
                    p = rd;
                    q = np - 1;
                } else {
                    p = (rd + gid) % (np - 1);
                    q = (rd - gid + np - 1) % (np - 1);
                }
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                const bool active = gid < P && q < r;
                float *cp = X + p * r, *cq = X + q * r, *wp = W + p * r, *wq = W + q * r;
                float aa = 0.0f, bb = 0.0f, gg = 0.0f;
                if (active)
                    for (int i = gl; i < r; i += g) {
                        const float x = cp[i], y = cq[i];
                        aa = fmaf(x, x, aa);
                        bb = fmaf(y, y, bb);
                        gg = fmaf(x, y, gg);
                    }
                for (int o = g >> 1; o > 0; o >>= 1) {
                    aa += __shfl_xor_sync(kFull, aa, o);
                    bb += __shfl_xor_sync(kFull, bb, o);
                    gg += __shfl_xor_sync(kFull, gg, o);
                }
                if (active && fabsf(gg) > tol * sqrtf(aa) * sqrtf(bb)) {
                    if (gl == 0) *flag = 1;
                    float cs, sn;
                    jacobi_rotation_f(aa, bb, gg, cs, sn);
                    for (int i = gl; i < r; i += g) {
                        const float x = cp[i], y = cq[i], u = wp[i], v = wq[i];
                        cp[i] = cs * x - sn * y;
                        cq[i] = sn * x + cs * y;
                        wp[i] = cs * u - sn * v;
                        wq[i] = sn * u + cs * v;
                    }
                }
                if (one_warp)
                    __syncwarp();
                else
                    __syncthreads();
            }
        }
        __syncthreads();
        const int f = *flag;
        __syncthreads();
        if (!f) break;
    }
    return sweep;
}

// QR with column pivoting of the mr x nc core M (precision R, shared memory,
// column major), stopped at the first step whose largest remaining column
// norm is at most delta times the first pivot's: M P = Q [R'; ~0] with R' of
// r rows.  Reflectors are kept below the diagonal of M (v_j = 1 implied),
// tau[j]; R' stays in rows < r; perm holds P.  The pivot is the largest
// column norm, lowest index on ties; the norms of the remaining columns are
// recomputed (not downdated) after every step.
template <class R>
__device__ int block_qrcp(R *M, int mr, int nc, R *tau, R *cn, int *perm, double delta, int *iflag) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        R s = R(0);
        for (int i = 0; i < mr; ++i) s += M[i + (size_t)j * mr] * M[i + (size_t)j * mr];
        cn[j] = s;
        perm[j] = j;
    }
    __syncthreads();
    const R d2 = R(delta * delta);
    R n0 = R(0);  // first pivot norm (kept by warp 0)
    int r = 0;
    const int kk = min(mr, nc);
    for (int j = 0; j < kk; ++j) {
        R *x = M + (size_t)j * mr;
        // warp 0: pivot, stopping test, column swap and reflector; one barrier
        if (warp == 0) {
            R bv = R(-1);
            int bi = j;
            for (int c = j + lane; c < nc; c += 32)
                if (cn[c] > bv) {
                    bv = cn[c];
                    bi = c;
                }
            for (int o = 16; o > 0; o >>= 1) {
                const R ov = __shfl_xor_sync(kFull, bv, o);
                const int oi = __shfl_xor_sync(kFull, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (j == 0) n0 = bv;
            const bool stop = !(bv > d2 * n0);
            if (lane == 0) iflag[1] = stop ? -1 : bi;
            if (!stop) {
                const int p = bi;
                if (p != j) {
                    for (int i = lane; i < mr; i += 32) {
                        const R tmp = x[i];
                        x[i] = M[i + (size_t)p * mr];
                        M[i + (size_t)p * mr] = tmp;
                    }
                    if (lane == 0) {
                        const R tc = cn[j];
                        cn[j] = cn[p];
                        cn[p] = tc;
                        const int tp = perm[j];
                        perm[j] = perm[p];
                        perm[p] = tp;
                    }
                    __syncwarp();
                }
                R s = R(0);
                for (int i = j + lane; i < mr; i += 32) s += x[i] * x[i];
                s = warp_sum_t(s);
                const R x0 = x[j];
                const R nrm = sqrt(s);
                R tj = R(0);
                __syncwarp();
                if (nrm > R(0)) {
                    const R alpha = x0 >= R(0) ? -nrm : nrm;
                    const R v0 = x0 - alpha;
                    for (int i = j + 1 + lane; i < mr; i += 32) x[i] /= v0;
                    tj = (alpha - x0) / alpha;
                    __syncwarp();
                    if (lane == 0) x[j] = alpha;
                }
                if (lane == 0) tau[j] = tj;
            }
        }
        __syncthreads();
        if (iflag[1] < 0) break;  // uniform: every thread reads the same flag
        const R tj = tau[j];
        // each warp updates its columns c = j + 1 + warp + nw t four at a time, so that the four
        // shuffle reductions overlap
        for (int c0 = j + 1 + warp; c0 < nc; c0 += 4 * nw) {
            R *y[4];
            R d[4], t2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c0 + q * nw;
                y[q] = M + (size_t)(c < nc ? c : j) * mr;  // column j stands in (read only)
                d[q] = R(0);
                t2[q] = R(0);
            }
            for (int i = j + 1 + lane; i < mr; i += 32) {
                const R xi = x[i];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c0 + q * nw < nc) d[q] += xi * y[q][i];
            }
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (sizeof(R) != 8 || c0 + q * nw < nc) d[q] += __shfl_xor_sync(kFull, d[q], o);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (sizeof(R) != 8 || c0 + q * nw < nc) d[q] = (d[q] + y[q][j]) * tj;
            __syncwarp();
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c0 + q * nw < nc) y[q][j] -= d[q];
            for (int i = j + 1 + lane; i < mr; i += 32) {
                const R xi = x[i];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c0 + q * nw < nc) {
                        const R yi = y[q][i] - d[q] * xi;
                        y[q][i] = yi;
                        t2[q] += yi * yi;
                    }
            }
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (sizeof(R) != 8 || c0 + q * nw < nc) t2[q] += __shfl_xor_sync(kFull, t2[q], o);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (c0 + q * nw < nc) cn[c0 + q * nw] = t2[q];
        }
        __syncthreads();
        r = j + 1;
    }
    return r;
}

// Shared buffers of the truncated SVD of an mr x nc core (core_truncate),
// carved from one byte range: double arrays first, then arrays of the core
// precision R, then ints.  With `stacked`, the reflector scalars and column
// norms of the two stacked QRs (mr and nc of each) come along.
template <class R>
struct CoreBufs {
    double *D, *sig;                       // Jacobi factor (rc x rc), singular values
    R *M, *C, *cn, *tauM, *tauC, *B, *isg;  // B: D in precision R (aliases D when R is double)
    R *W;                                   // single precision: accumulated rotations (in D's space)
    R *tauU, *tauV, *nrmU, *nrmV;
    int *order, *perm, *iflag;
    // single-precision cores with the Jacobi SVD in double (core64): 1 / sigma in double (isg of
    // precision R is not used then); null otherwise
    double *isg64;
};

// core64 applies to single-precision cores only: their Jacobi SVD runs in double.
template <class R>
__host__ __device__ constexpr bool core_in_double(bool core64) {
    return sizeof(R) != 8 && core64;
}

template <class R>
__host__ __device__ inline size_t core_bytes(int mr, int nc, bool stacked, bool core64) {
    const size_t rc = mr < nc ? mr : nc, mx = mr > nc ? mr : nc;
    const bool c64 = core_in_double<R>(core64);
    const size_t nr = (size_t)mr * nc + mx * rc + nc + 3 * rc + (sizeof(R) == 8 ? 0 : rc * rc) +
                      (stacked ? 2 * ((size_t)mr + nc) : 0);
    return 8 * (rc * rc + rc + (c64 ? rc : 0)) + sizeof(R) * nr + 4 * (rc + nc + 8);
}

template <class R>
__device__ CoreBufs<R> carve_core(unsigned char *base, int mr, int nc, bool stacked, bool core64) {
    const int rc = min(mr, nc), mx = max(mr, nc);
    const bool c64 = core_in_double<R>(core64);
    CoreBufs<R> b;
    b.D = reinterpret_cast<double *>(base);
    b.sig = b.D + rc * rc;
    double *dx = b.sig + rc;
    b.isg64 = nullptr;
    if (c64) {
        b.isg64 = dx;
        dx += rc;
    }
    R *x = reinterpret_cast<R *>(dx);
    b.M = x;
    x += (size_t)mr * nc;
    b.C = x;
    x += (size_t)mx * rc;
    b.cn = x;
    x += nc;
    b.tauM = x;
    b.tauC = x + rc;
    b.isg = x + 2 * rc;
    x += 3 * rc;
    if constexpr (sizeof(R) == 8) {
        b.B = b.D;
        b.W = nullptr;
    } else {
        b.B = x;
        x += rc * rc;
        b.W = reinterpret_cast<R *>(b.D);  // r x r floats fit in the rc x rc doubles of D
    }
    b.tauU = b.tauV = b.nrmU = b.nrmV = nullptr;
    if (stacked) {
        b.tauU = x;
        b.nrmU = x + mr;
        x += 2 * mr;
        b.tauV = x;
        b.nrmV = x + nc;
        x += 2 * nc;
    }
    int *ip = reinterpret_cast<int *>(x);
    b.order = ip;
    b.perm = ip + rc;
    b.iflag = ip + rc + nc;
    return b;
}

// Truncated SVD (T_eps of Sec. 3.1) of the mr x nc core M held in b.M, with
// the two QR preconditioning steps of Drmac and Veselic (2008):
//   M P = Q_M [R'; ~0]        pivoted QR in the core precision R, r rows
//   R'^T = Q_C R_C            Householder QR of the nc x r factor, in R
//   R_C^T W = B               one-sided Jacobi on the r x r lower
//                             triangular X = R_C^T; sigma_j = |B_j|
// so that M = (Q_M [B; 0]) (P Q_C W)^T.  Double-precision cores (R = double)
// run the Jacobi in double without forming W: since M^T Q_M [B; 0] = P R'^T B,
// the right factor is P R'^T B Sigma^{-2}.  Single-precision cores run it in
// single precision with W accumulated, and the right factor is P Q_C [W; 0]
// (Sigma^{-2} would amplify the single-precision error of B in the columns
// of small sigma).
// Singular values sigma_i <= eps sigma_1 are dropped.  Returns the kept rank
// (order[0..knew) lists the kept columns of B by decreasing sigma, lowest
// index on ties) and r through r_out; leaves B in precision R (b.B) and
// 1 / sigma (b.isg).  Phase counters (profiling only) go to slots pb + 2 ...
// pb + 7.
// The steps of core_truncate after the pivoted QR (rank r known): the QR of R'^T, the Jacobi SVD,
// ordering and truncation.  Returns the kept rank.
template <class R>
__device__ int core_finish(const CoreBufs<R> &b, int mr, int nc, int r, const TRadd &t, const LaunchArgs &a,
                           int pb, unsigned long long &ph) {
    const bool c64 = core_in_double<R>(a.core64 != 0);
    for (int e = threadIdx.x; e < nc * r; e += blockDim.x) {
        const int c = e % nc, i = e / nc;
        b.C[e] = c >= i ? b.M[i + (size_t)c * mr] : R(0);
    }
    if (threadIdx.x == 0) b.iflag[2] = 0;  // [0]: Jacobi flag, [1]: pivoted-QR flag
    __syncthreads();
    group_householder_qr<R>(b.C, nc, r, b.tauC, b.cn, 0, blockDim.x >> 5, 0);
    // profiling, dense route: the QR of R'^T goes to slot 1 (the stacked route keeps it in its slot 3)
    if (pb == 0) ph = phase_mark(a, 1, ph);
    int sweeps;
    if (c64) {  // the Jacobi SVD of X = R_C^T (single-precision values, exact in double) in double
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
            const int i = e % r, j = e / r;
            b.D[e] = i >= j ? (double)b.C[j + (size_t)i * nc] : 0.0;
        }
        __syncthreads();
        sweeps = block_jacobi(b.D, r, r, b.iflag, b.sig);
        for (int j = threadIdx.x; j < r; j += blockDim.x) {
            double s = 0.0;
            for (int i = 0; i < r; ++i) s += b.D[i + (size_t)j * r] * b.D[i + (size_t)j * r];
            b.sig[j] = sqrt(s);
        }
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) b.B[e] = R(b.D[e]);  // for the left factor
    } else if constexpr (sizeof(R) == 8) {
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) {  // X = R_C^T
            const int i = e % r, j = e / r;
            b.D[e] = i >= j ? b.C[j + (size_t)i * nc] : 0.0;
        }
        __syncthreads();
        sweeps = block_jacobi(b.D, r, r, b.iflag, b.sig);
        for (int j = threadIdx.x; j < r; j += blockDim.x) {
            double s = 0.0;
            for (int i = 0; i < r; ++i) s += b.D[i + (size_t)j * r] * b.D[i + (size_t)j * r];
            b.sig[j] = sqrt(s);
        }
    } else {
        // X = R_C^T and W = I; X is scaled by a power of two 2^-e (exact) that brings its largest
        // entry into [1, 2), so the single-precision squared norms neither overflow nor underflow
        float mx = 0.0f;
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
            const int i = e % r, j = e / r;
            const float v = i >= j ? b.C[j + (size_t)i * nc] : 0.0f;
            b.B[e] = v;
            b.W[e] = i == j ? 1.0f : 0.0f;
            mx = fmaxf(mx, fabsf(v));
        }
        mx = warp_max_f(mx);
        if ((threadIdx.x & 31) == 0 && mx > 0.0f) atomicMax(b.iflag + 2, __float_as_int(mx));
        __syncthreads();
        const float amax = __int_as_float(b.iflag[2]);
        const int ex = (amax > 0.0f && amax <= FLT_MAX) ? ((__float_as_int(amax) >> 23) & 0xff) - 127 : 0;
        const float down = __int_as_float((127 - max(-126, min(126, ex))) << 23);  // 2^-ex
        const float up = __int_as_float((127 + max(-126, min(126, ex))) << 23);    // 2^ex
        if (ex != 0)
            for (int e = threadIdx.x; e < r * r; e += blockDim.x) b.B[e] *= down;
        __syncthreads();
        sweeps = block_jacobi_f(b.B, b.W, r, b.iflag);
        for (int j = threadIdx.x; j < r; j += blockDim.x) {
            float s = 0.0f;
            for (int i = 0; i < r; ++i) s = fmaf(b.B[i + j * r], b.B[i + j * r], s);
            b.sig[j] = (double)sqrtf(s) * (double)up;
        }
        __syncthreads();
        if (ex != 0)
            for (int e = threadIdx.x; e < r * r; e += blockDim.x) b.B[e] *= up;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        int rk = 0;
        for (int l = 0; l < r; ++l) rk += (b.sig[l] > b.sig[j]) || (b.sig[l] == b.sig[j] && l < j);
        b.order[rk] = j;
        if (c64)
            b.isg64[j] = b.sig[j] > 0.0 ? 1.0 / b.sig[j] : 0.0;
        else
            b.isg[j] = b.sig[j] > 0.0 ? R(1.0 / b.sig[j]) : R(0);
    }
    __syncthreads();
    const double s1 = r > 0 ? b.sig[b.order[0]] : 0.0;
    int knew = 0;
    if (!isfinite(s1)) {
        if (threadIdx.x == 0) set_error(a.err, DE_NONFINITE, t.target, s1);
    } else if (s1 > 0.0) {
        const double eps = a.eps_inst ? a.eps_inst[t.inst] : a.eps;
        for (int l = 0; l < r; ++l) knew += b.sig[b.order[l]] > eps * s1;
    }
    if (knew > t.cap) {
        if (threadIdx.x == 0) set_error(a.err, DE_RANKCAP, t.target, (double)knew);
        knew = t.cap;
    }
    ph = phase_mark(a, pb + 3, ph);
    if (a.phase && threadIdx.x == 0) {  // Jacobi sweeps, problem size and task count
        atomicAdd(a.phase + pb + 4, (unsigned long long)sweeps);
        atomicAdd(a.phase + pb + 6, (unsigned long long)r);
        atomicAdd(a.phase + pb + 7, 1ull);
    }
    return knew;
}

template <class R>
__device__ int core_truncate(const CoreBufs<R> &b, int mr, int nc, double delta, const TRadd &t,
                             const LaunchArgs &a, int *r_out, int pb, unsigned long long &ph) {
    const int r = block_qrcp<R>(b.M, mr, nc, b.tauM, b.cn, b.perm, delta, b.iflag);
    ph = phase_mark(a, pb + 2, ph);
    *r_out = r;
    return core_finish<R>(b, mr, nc, r, t, a, pb, ph);
}

// Right factor of the truncated core: V[perm[i], c] = (R'^T B)[i, order[c]] /
// sigma^2 for the nc rows of the core (V of type T, leading dimension ldv).
template <class R, class T>
__device__ void core_write_v(const CoreBufs<R> &b, int mr, int nc, int r, int knew, T *V, int64_t ldv) {
    if (b.isg64) {
        // double Jacobi SVD of a single-precision core: V[perm[i], c] = (R'^T B)[i, order[c]] /
        // sigma^2 in double, R' exact as promoted.  B = X Z comes from the double Jacobi (Z
        // orthogonal to double rounding), so the factor is M^T u_j / sigma_j for the left vectors
        // u_j; its errors (double rounding of B, single-precision rounding of the QR of R'^T) enter
        // the product sigma_j u_j v_j^T at their own level relative to sigma_1, not amplified by
        // sigma_1 / sigma_j.
        for (int e = threadIdx.x; e < nc * knew; e += blockDim.x) {
            const int c = e % knew, i = e / knew;
            const int j = b.order[c];
            const int lmax = min(i, r - 1);
            const double *bj = b.D + (size_t)j * r;
            double sacc = 0.0;
            for (int l = 0; l <= lmax; ++l) sacc = fma((double)b.M[l + (size_t)i * mr], bj[l], sacc);
            V[b.perm[i] + (int64_t)c * ldv] = T((sacc * b.isg64[j]) * b.isg64[j]);
        }
    } else if constexpr (sizeof(R) == 8) {
        for (int e = threadIdx.x; e < nc * knew; e += blockDim.x) {
            const int c = e % knew, i = e / knew;
            const int j = b.order[c];
            const int lmax = min(i, r - 1);
            const R *bj = b.B + (size_t)j * r;
            R s = R(0);
            for (int l = 0; l <= lmax; ++l) s += b.M[l + (size_t)i * mr] * bj[l];
            V[b.perm[i] + (int64_t)c * ldv] = T((s * b.isg[j]) * b.isg[j]);
        }
    } else {
        // V[perm[i], c] = (Q_C [W_sel; 0])[i, c]: the rotations were accumulated in single precision,
        // so the right factor is formed from them (orthonormal columns) rather than through
        // Sigma^{-2}, which would amplify their single-precision error.  One warp per column, the
        // nc <= kVRows entries of y in registers; ends with a barrier (b.C is overwritten next).
        const int lane = threadIdx.x & 31;
        for (int c = threadIdx.x >> 5; c < knew; c += blockDim.x >> 5) {
            const R *wj = b.W + (size_t)b.order[c] * r;
            R y[kVRows / 32];
#pragma unroll
            for (int k = 0; k < kVRows / 32; ++k) {
                const int i = lane + 32 * k;
                y[k] = i < r ? wj[i] : R(0);
            }
            for (int q = r - 1; q >= 0; --q) {  // y := H_q y, H_q = I - tau_q v_q v_q^T, v_q[q] = 1
                const R *v = b.C + (size_t)q * nc;
                R d = R(0);
#pragma unroll
                for (int k = 0; k < kVRows / 32; ++k) {
                    const int i = lane + 32 * k;
                    if (i > q && i < nc) d += v[i] * y[k];
                    if (i == q) d += y[k];
                }
                d = warp_sum_t(d) * b.tauC[q];
#pragma unroll
                for (int k = 0; k < kVRows / 32; ++k) {
                    const int i = lane + 32 * k;
                    if (i > q && i < nc) y[k] -= d * v[i];
                    if (i == q) y[k] -= d;
                }
            }
#pragma unroll
            for (int k = 0; k < kVRows / 32; ++k) {
                const int i = lane + 32 * k;
                if (i < nc) V[b.perm[i] + (int64_t)c * ldv] = T(y[k]);
            }
        }
        __syncthreads();
    }
}

// Output buffer of core_form_u: the buffer of R'^T (no longer read once the Jacobi has started),
// which holds at least mr x knew values of precision R.
template <class R>
__device__ __forceinline__ R *core_out(const CoreBufs<R> &b) {
    return b.C;
}

// Left factor of the truncated core: core_out(b) (mr x knew) := Q_M [B_sel; 0].
// Ends with a barrier.
template <class R>
__device__ void core_form_u(const CoreBufs<R> &b, int mr, int r, int knew) {
    R *C = core_out(b);
    for (int e = threadIdx.x; e < mr * knew; e += blockDim.x) {
        const int i = e % mr, c = e / mr;
        C[e] = i < r ? b.B[i + (size_t)b.order[c] * r] : R(0);
    }
    __syncthreads();
    for (int c = threadIdx.x >> 5; c < knew; c += blockDim.x >> 5)
        warp_apply_q<R>(b.M, mr, r, b.tauM, C + (size_t)c * mr);
    __syncthreads();
}

// Rounded addition (Sec. 3.1): the target's factors and every contribution are
// stacked, U_s = [U_c, c_1 U_1, ...], V_s = [V_c, V_1, ...] (pieces
// zero-padded to the target's index ranges); both stacks are reduced by
// Householder QR (concurrently, one half of the CTA each), and the core
// M = R_u R_v^T is truncated by core_truncate; the new factors are
// U = Q_u [Q_M [B_sel; 0]; 0], V = Q_v [P R'^T B_sel Sigma^{-2}; 0] (double
// factors) or V = Q_v [P Q_C W_sel; 0] (single-precision factors).
// Everything runs in the precision T of the factors.
//
// Shared memory is carved by the task's own core size: the core buffers first
// (core_bytes), then, when they fit in the rest of the CTA's `smem_bytes`,
// the stacked panels themselves; larger panels stay in the global `scratch`.
// The pivoted QR of the core stops at delta times the first pivot: 1e-13 for
// FP64 factors (double rounding level) and 1e-6 for FP32 factors (an order
// above the FP32 rounding of the stacked panels, two below the relative
// tolerances eps the method uses).
// Dense route (targets with m, n <= 128 and m n <= dense_max = 4096; larger dense sums cost more in the
// pivoted QR than the two stacked QRs they replace, measured at n = 20480):
// the sum X = U_c V_c^T + sum_i c_i U_i V_i^T is formed densely and truncated
// by the same core steps, which is the same T_eps of the same sum without the
// two stacked QRs.  Shared memory is carved in two steps: X and the pivoted-QR
// bookkeeping, then, with the rank r of the pivoted QR known, the rank-r
// buffers; when those exceed dense_post_cap bytes the task falls back to the
// stacked route (nothing outside shared memory has been written yet).  Every
// launch provides at least radd_dense_floor bytes, so the route depends on the
// task alone.
template <class R>
__host__ __device__ constexpr int dense_max() {
    return 4096;
}

// Rank-r budget of the dense route: larger when the core SVD of single-precision factors runs in
// double (its R'^T copy and QR are double).
__host__ __device__ constexpr size_t dense_post_cap(bool c64) { return c64 ? 40960 : 24576; }

template <class R>
__host__ __device__ inline size_t dense_pre_bytes(int m, int n) {
    const size_t rc = m < n ? m : n;
    return (sizeof(R) * ((size_t)m * n + n + rc) + sizeof(int) * ((size_t)n + 8) + 15) & ~size_t(15);
}

template <class R>
__host__ __device__ inline size_t dense_post_bytes(int m, int n, int r, bool c64) {
    const size_t mx = m > n ? m : n;
    // D, sig (and 1 / sigma of a double Jacobi in single-precision factors: c64) in double; C, tauC,
    // isg (and B for single precision) in precision R; order
    return 8 * ((size_t)r * r + r + (c64 ? r : 0)) +
           sizeof(R) * (mx * r + 2 * (size_t)r + (sizeof(R) == 8 ? 0 : (size_t)r * r)) + sizeof(int) * (size_t)r;
}

template <class T>
__device__ bool radd_small(const TRadd &t, const Piece *pieces, const LaunchArgs &a, int kself,
                           unsigned char *smem_raw, size_t smem_bytes, double delta) {
    const int m = t.m, n = t.n, rc = min(m, n);
    if (max(m, n) > 128 || (int64_t)m * n > dense_max<T>()) return false;
    T *A = reinterpret_cast<T *>(a.arena);
    int32_t *kd = a.kdyn;
    CoreBufs<T> b;
    b.M = reinterpret_cast<T *>(smem_raw);
    b.cn = b.M + (size_t)m * n;
    b.tauM = b.cn + n;
    b.perm = reinterpret_cast<int *>(b.tauM + rc);
    b.iflag = b.perm + n;
    b.tauU = b.tauV = b.nrmU = b.nrmV = nullptr;
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
        b.M[e] = acc;
    }
    __syncthreads();
    ph = phase_mark(a, 0, ph);
    const int r = block_qrcp<T>(b.M, m, n, b.tauM, b.cn, b.perm, delta, b.iflag);
    ph = phase_mark(a, 2, ph);
    const bool c64 = core_in_double<T>(a.core64 != 0);
    if (dense_post_bytes<T>(m, n, r, c64) > dense_post_cap(c64)) return false;  // uniform over the CTA
    // rank-r buffers after X and the pivot bookkeeping
    b.D = reinterpret_cast<double *>(smem_raw + dense_pre_bytes<T>(m, n));
    b.sig = b.D + r * r;
    b.isg64 = c64 ? b.sig + r : nullptr;
    b.C = reinterpret_cast<T *>(b.sig + r + (c64 ? r : 0));
    b.tauC = b.C + (size_t)max(m, n) * r;
    b.isg = b.tauC + r;
    if constexpr (sizeof(T) == 8) {
        b.B = b.D;
        b.W = nullptr;
        b.order = reinterpret_cast<int *>(b.isg + r);
    } else {
        b.B = b.isg + r;
        b.W = reinterpret_cast<T *>(b.D);  // r x r floats in the r x r doubles of D
        b.order = reinterpret_cast<int *>(b.B + r * r);
    }
    const int knew = core_finish<T>(b, m, n, r, t, a, 0, ph);
    // the target's own factors were read above; every row of V is covered by P
    core_write_v<T, T>(b, m, n, r, knew, A + t.V_off, n);
    // U = Q_M [B_sel; 0], one warp per column in registers (m <= 128)
    for (int c = threadIdx.x >> 5; c < knew; c += blockDim.x >> 5) {
        const T *bc = b.B + (size_t)b.order[c] * r;
        T y[kVRows / 32];
#pragma unroll
        for (int k = 0; k < kVRows / 32; ++k) {
            const int i = (threadIdx.x & 31) + 32 * k;
            y[k] = i < r ? bc[i] : T(0);
        }
        reg_apply_q<T>(b.M, m, m, r, b.tauM, y);
#pragma unroll
        for (int k = 0; k < kVRows / 32; ++k) {
            const int i = (threadIdx.x & 31) + 32 * k;
            if (i < m) A[t.U_off + i + (int64_t)c * m] = y[k];
        }
    }
    if (threadIdx.x == 0) kd[t.kslot] = knew;
    phase_mark(a, 5, ph);
    return true;
}

// When even the core does not fit (K above the CTA's shared-memory capacity),
// it is placed in `core_scratch` (global, radd_smem_bytes(K) bytes).
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
    const int ku = min(m, K), kv = min(n, K);
    const bool c64 = core_in_double<T>(a.core64 != 0);
    const size_t cbytes = (core_bytes<T>(ku, kv, true, c64) + 15) & ~size_t(15);
    const bool core_in_smem = cbytes <= smem_bytes;
    const size_t panel_bytes = (size_t)(m + n) * K * sizeof(T);
    T *WU = core_in_smem && cbytes + panel_bytes <= smem_bytes ? reinterpret_cast<T *>(smem_raw + cbytes) : scratch;
    T *WV = WU + (int64_t)m * K;
    unsigned long long ph = phase_mark(a, 8, 0ull);
    // ---- stack the factors
    for (int64_t e = threadIdx.x; e < (int64_t)(m + n) * K; e += blockDim.x) WU[e] = T(0);
    __syncthreads();
    block_copy<T>(m * kself, [&](int e) { return A[t.U_off + e]; }, [&](int e, T v) { WU[e] = v; });
    block_copy<T>(n * kself, [&](int e) { return A[t.V_off + e]; }, [&](int e, T v) { WV[e] = v; });
    int col = kself;
    for (int q = 0; q < t.npieces; ++q) {
        const Piece pc = pieces[t.piece0 + q];
        const int k = dim_c(pc.U, kd), mu = pc.U.rows, nv = pc.V.rows;
        const T coef = T(pc.coef);
        block_copy<T>(
            mu * k, [&](int e) { return coef * at(A, pc.U, e % mu, e / mu); },
            [&](int e, T v) { WU[pc.roff + e % mu + (int64_t)(col + e / mu) * m] = v; });
        block_copy<T>(
            nv * k, [&](int e) { return at(A, pc.V, e % nv, e / nv); },
            [&](int e, T v) { WV[pc.coff + e % nv + (int64_t)(col + e / nv) * n] = v; });
        col += k;
    }
    __syncthreads();
    ph = phase_mark(a, 8, ph);
    const CoreBufs<T> b = carve_core<T>(core_in_smem ? smem_raw : core_scratch, ku, kv, true, c64);
    // ---- QR of both stacks (one half of the CTA each), core M = R_u R_v^T
    const int half = (blockDim.x >> 5) / 2;
    if ((int)(threadIdx.x >> 5) < half)
        group_householder_qr(WU, m, K, b.tauU, b.nrmU, 0, half, 1);
    else
        group_householder_qr(WV, n, K, b.tauV, b.nrmV, half, half, 2);
    __syncthreads();
    for (int e = threadIdx.x; e < ku * kv; e += blockDim.x) {
        const int i = e % ku, j = e / ku;
        T s = T(0);
        for (int l = max(i, j); l < K; ++l) s += WU[i + (int64_t)l * m] * WV[j + (int64_t)l * n];
        b.M[e] = s;
    }
    __syncthreads();
    ph = phase_mark(a, 9, ph);
    int r = 0;
    const int knew = core_truncate<T>(b, ku, kv, delta, t, a, &r, 8, ph);
    T *Uc = A + t.U_off;
    T *Vc = A + t.V_off;
    // ---- V = Q_v [core right factor; 0] (rows < kv written here)
    core_write_v<T, T>(b, ku, kv, r, knew, Vc, n);
    if (m <= kVRows && n <= kVRows) {
        // ---- U = Q_u [Q_M [B_sel; 0]; 0] and V: one warp per column, the column in registers
        __syncthreads();  // the core rows of V are written
        const int lane = threadIdx.x & 31;
        for (int c = threadIdx.x >> 5; c < 2 * knew; c += blockDim.x >> 5) {
            T y[kVRows / 32];
            if (c < knew) {
                const T *bc = b.B + (size_t)b.order[c] * r;
#pragma unroll
                for (int k = 0; k < kVRows / 32; ++k) {
                    const int i = lane + 32 * k;
                    y[k] = i < r ? bc[i] : T(0);
                }
                reg_apply_q<T>(b.M, ku, ku, r, b.tauM, y);
                reg_apply_q<T>(WU, m, m, ku, b.tauU, y);
                T *dst = Uc + (int64_t)c * m;
#pragma unroll
                for (int k = 0; k < kVRows / 32; ++k)
                    if (lane + 32 * k < m) dst[lane + 32 * k] = y[k];
            } else {
                T *vc = Vc + (int64_t)(c - knew) * n;
#pragma unroll
                for (int k = 0; k < kVRows / 32; ++k) {
                    const int i = lane + 32 * k;
                    y[k] = i < kv ? vc[i] : T(0);
                }
                reg_apply_q<T>(WV, n, n, kv, b.tauV, y);
#pragma unroll
                for (int k = 0; k < kVRows / 32; ++k)
                    if (lane + 32 * k < n) vc[lane + 32 * k] = y[k];
            }
        }
    } else {
        for (int e = threadIdx.x; e < (n - kv) * knew; e += blockDim.x) {
            const int i = kv + e % (n - kv), c = e / (n - kv);
            Vc[i + (int64_t)c * n] = T(0);
        }
        // ---- U = Q_u [Q_M [B_sel; 0]; 0]
        core_form_u<T>(b, ku, r, knew);
        const T *Cu = core_out(b);
        for (int e = threadIdx.x; e < m * knew; e += blockDim.x) {
            const int i = e % m, c = e / m;
            Uc[e] = i < ku ? Cu[i + (size_t)c * ku] : T(0);
        }
        __syncthreads();
        for (int c = threadIdx.x >> 5; c < 2 * knew; c += blockDim.x >> 5) {  // U and V columns together
            if (c < knew)
                warp_apply_q(WU, m, ku, b.tauU, Uc + (int64_t)c * m);
            else
                warp_apply_q(WV, n, kv, b.tauV, Vc + (int64_t)(c - knew) * n);
        }
    }
    if (threadIdx.x == 0) {
        kd[t.kslot] = knew;
        add_flops(a, K_RADD, radd_model_flops(m, n, K, knew));
    }
    phase_mark(a, 13, ph);
}

// Shared memory that every rounded-addition launch provides: the dense route's
// worst case over m, n <= 128, m n <= dense_max, plus its rank-r budget.
template <class R>
size_t radd_dense_floor(bool c64) {
    size_t s = 0;
    for (int m = 1; m <= 128; ++m)
        for (int n = 1; n <= 128 && m * n <= dense_max<R>(); ++n)
            s = std::max(s, dense_pre_bytes<R>(m, n) + dense_post_cap(c64));
    return s;
}

size_t radd_smem_bytes(int kc, int elem, bool core64) {
    if (elem == 8) return std::max(core_bytes<double>(kc, kc, true, false), radd_dense_floor<double>(false));
    return std::max(core_bytes<float>(kc, kc, true, core64), radd_dense_floor<float>(core64));
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
__global__ void __launch_bounds__(kThreads) k_accum(const TAccum *tasks, const Term *terms, LaunchArgs a,
                                                    size_t smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TAccum t = tasks[blockIdx.x];
    dev_accum<T>(t, terms, a, smem_raw, smem_bytes);
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
// successor's in-degree makes it ready.  The first successor it makes ready
// the worker runs itself next (no queue round trip, its inputs are in this
// SM's cache); the others are pushed.  Writes of a task are published with a
// device-scope fence before the release; the consumer reads the slot with an
// acquire load, and a worker that makes a task ready itself fences before
// running it.  Successor lists come with the successor on the longest
// remaining path first (the planner's priority), so that is the one run next
// whenever it becomes ready here.  Successors are released in parallel, one
// thread each.  The worker that completes the last
// task writes an end mark into every queue slot a worker may be waiting on
// (slots that inlining left unfilled).  Every wait has a deadline
// (%globaltimer): on expiry, or when another worker has recorded an error,
// the worker records DE_TIMEOUT (first error wins) and leaves, so the launch
// always ends.
constexpr int kQueueEnd = -3;  // queue slot value: no task will come

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
__global__ void __launch_bounds__(kThreads, 2) k_dataflow(FlowArgs f, LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task, s_next, s_first;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) unsigned long long s_mbar;
    T *scratch = reinterpret_cast<T *>(f.scratch) + (int64_t)blockIdx.x * f.scratch_stride;
    if (threadIdx.x == 0) s_next = -1;
    // tensor cores (single precision, when enabled): this worker's TMEM accumulators (kTcTmemCols
    // columns; at most two workers per SM, 512 columns at most) and the MMA-completion mbarrier.  A CTA of
    // a kernel that holds tcgen05 code keeps the SM's TMEM allocation permit, and with it the SM
    // from a second CTA, until it relinquishes the permit: every single-precision worker does so at
    // once, after its allocation when the tensor cores are on.
    TcState tc{0u, 0u, 0u, false, f.timeout_ns, f.tc_min_inner};
    const bool use_tc = sizeof(T) == 4 && f.tensor;
    int my_tasks = 0;  // tasks this worker ran (profiling: workers that ran any)
    // profiling: the worker's lifetime (slot 14) and its waits on empty queue slots (slot 7); the rest
    // of the lifetime outside the tasks is the executor's own overhead
    const unsigned long long t_life = (f.busy && threadIdx.x == 0) ? global_ns() : 0ull;
    if constexpr (sizeof(T) == 4) {
        if (!use_tc && threadIdx.x < 32) asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (use_tc) {
        const unsigned long long t_alloc = (f.busy && threadIdx.x == 0) ? global_ns() : 0ull;
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                         "r"(kTcTmemCols));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)));
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tc.tmem = s_tmem;
        tc.mbar = smem_u32(&s_mbar);
        tc.on = true;
        if (f.busy && threadIdx.x == 0) atomicAdd(f.busy + 6, global_ns() - t_alloc);  // TMEM allocation wait
    }
    for (;;) {
        if (threadIdx.x == 0) {
            int g = s_next;
            if (g < 0) {
                const int slot = atomicAdd(f.counters, 1);
                if (slot < f.n_tasks) {
                    const unsigned long long t_wait = global_ns();
                    const unsigned long long deadline = t_wait + f.timeout_ns;
                    for (;;) {
                        g = ld_acquire(f.queue + slot);
                        if (g >= 0) break;
                        if (g == kQueueEnd) {  // every task has completed
                            g = -1;
                            break;
                        }
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
                    if (f.busy) atomicAdd(f.busy + 7, global_ns() - t_wait);
                }
            }
            s_task = g;
        }
        __syncthreads();
        const int g = s_task;
        if (g < 0) break;
        const int code = f.code[g];
        const int kind = code >> kCodeShift, idx = code & kCodeMask;
        ++my_tasks;
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
                dev_accum<T, true>(t, f.terms, a, smem_raw, f.smem_bytes, &tc);
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
            s_first = INT_MAX;
        }
        __syncthreads();
        // release the successors in parallel, one thread each: the task's writes (ordered before
        // this point by the barrier) are published by each thread's fence before its decrement
        const int e0 = f.succ_ptr[g], ns = f.succ_ptr[g + 1] - e0;
        for (int c0 = 0; c0 < ns; c0 += blockDim.x) {
            const int e = c0 + threadIdx.x;
            bool ready = false;
            if (e < ns) {
                __threadfence();
                ready = atomicSub(f.indeg + f.succ_idx[e0 + e], 1) == 1;
                if (ready) {
                    __threadfence();
                    atomicMin(&s_first, e);
                }
            }
            __syncthreads();
            // the first ready successor in priority order runs here next; the others are queued
            if (ready && e != s_first) {
                const int pos = atomicAdd(f.counters + 1, 1);
                st_release(f.queue + pos, f.succ_idx[e0 + e]);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_next = s_first < ns ? f.succ_idx[e0 + s_first] : -1;
            // only the sinks are counted: every task precedes a sink, so the last sink to complete is
            // the last task (one global atomic per sink instead of per task)
            if (ns == 0 && atomicAdd(f.counters + 2, 1) == f.n_sinks - 1) {
                // the last task: wake the workers waiting on slots that will stay empty, and
                // those that still claim one (each worker claims at most one more slot)
                __threadfence();
                const int tail = atomicAdd(f.counters + 1, 0), head = atomicAdd(f.counters, 0);
                const int end = min(f.n_tasks, head + (int)gridDim.x);
                for (int pos = tail; pos < end; ++pos) st_release(f.queue + pos, kQueueEnd);
            }
        }
        __syncthreads();
    }
    if (f.busy && threadIdx.x == 0 && my_tasks > 0) atomicAdd(f.busy + 15, 1ull);  // active workers
    if (f.busy && threadIdx.x == 0) atomicAdd(f.busy + 14, global_ns() - t_life);
    if (use_tc) {  // every path out of the loop comes here: the accumulator is given back
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (threadIdx.x < 32)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"(kTcTmemCols));
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
            k_trsm<T><<<count, kThreads, trsm_smem_bytes(aux, sizeof(T)), s>>>(
                reinterpret_cast<const TTrsm *>(tasks) + start, a);
            break;
        case K_PROJECT:
            k_project<T><<<count, kThreads, project_smem_bytes(sizeof(T)), s>>>(
                reinterpret_cast<const TProject *>(tasks) + start, a);
            break;
        case K_ACCUM:
            k_accum<T><<<count, kThreads, accum_smem_bytes(sizeof(T)), s>>>(reinterpret_cast<const TAccum *>(tasks) + start,
                                                                          terms, a, accum_smem_bytes(sizeof(T)));
            break;
        case K_RADD: {
            // includes the dense route's worst case (radd_dense_floor), so that the
            // route a task takes does not depend on the schedule
            const size_t smem = radd_smem_bytes(aux, sizeof(T), a.core64 != 0);
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

template <class K>
static bool max_shared_carveout(K kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared) == cudaSuccess;
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
    ok = allow_dynamic_smem(k_accum<T>, optin) && ok;
    ok = allow_dynamic_smem(k_dataflow<T>, optin) && ok;
    // One split of the unified L1 (all of it as shared memory) for every kernel that runs between
    // or beside data-flow launches: blocks of kernels with different splits do not share an SM, so a
    // small kernel of one handle (permutation, refinement step) would otherwise wait until another
    // handle's persistent launch on another stream has left the SMs.
    ok = max_shared_carveout(k_dataflow<T>) && ok;
    ok = max_shared_carveout(k_reset<T>) && ok;
    ok = max_shared_carveout(k_to_work<T>) && ok;
    ok = max_shared_carveout(k_add_from_work<T>) && ok;
    ok = max_shared_carveout(k_permute<double, double>) && ok;
    ok = max_shared_carveout(k_permute<double, float>) && ok;
    ok = max_shared_carveout(k_permute<float, double>) && ok;
    ok = max_shared_carveout(k_set_slot) && ok;
    ok = max_shared_carveout(k_residual) && ok;
    cudaGetLastError();  // a failure is reported through the return value, not left pending
    return ok;
}

size_t dataflow_smem_bytes(int max_leaf, int elem, int kc, bool core64) {
    size_t s = getrf_smem_bytes(max_leaf, elem);
    s = std::max(s, trsm_smem_bytes(max_leaf, elem));
    s = std::max(s, project_smem_bytes(elem));
    s = std::max(s, accum_smem_bytes(elem));
    s = std::max(s, radd_smem_bytes(kc, elem, core64));
    return s;
}

// Resident workers: the occupancy API counts one CTA per SM for a kernel that holds tcgen05 code
// (it assumes the TMEM allocation permit is kept), but every worker relinquishes the permit at
// start, so the count comes from the registers, the shared memory and the launch bound (two per
// SM) directly; the TMEM of two workers (2 x 128 columns) fits the SM's 512.
template <class T>
int dataflow_workers(size_t smem) {
    int dev = 0, sms = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_dataflow<T>) != cudaSuccess) {
        cudaGetLastError();
        return sms;
    }
    const size_t per_cta = smem + fa.sharedSizeBytes + (size_t)reserved;
    int per = 2;  // __launch_bounds__(kThreads, 2)
    per = std::min<int>(per, (int)((size_t)smem_sm / std::max<size_t>(per_cta, 1)));
    const int regs_cta = ((fa.numRegs * 32 + 255) / 256) * 256 * (kThreads / 32);  // 256-register warp granules
    per = std::min(per, regs_sm / std::max(regs_cta, 1));
    return sms * std::max(per, 1);
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
