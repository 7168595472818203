// Construction of the BEM H-matrix on the device: the leaves of a given block tree for the Laplace
// kernels of Sec. 6.1 (collocation form, one element per degree of freedom).
//
//   dense leaves      A_ij = a_j g(c_i, c_j) (i != j), A_ii = the self-term of element i
//   low-rank leaves   adaptive cross approximation with partial pivoting, then the rounded
//                     truncation T_eps of the cross factors (Sec. 3.1 "Low-rank blocks": the
//                     paper recompresses its interpolation factors by an SVD; the truncation here
//                     is the library's own rounded addition with the cross factors as the only
//                     piece)
//
// g = 1 / (4 pi r) (d = 3), -log r (d = 1), -log r / (2 pi) (d = 2).  Self-terms: sqrt(a / pi) / 2
// (d = 3, a flat disc of area a), a (1 - log(a / 2)) (d = 1) and that over 2 pi (d = 2): the
// integral of -log|t| over a straight element of length a centred at the point.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hlu.h"
#include "kernels.cuh"
#include "tasks.h"

struct hlu_bem {
    int64_t n_leaves = 0;
    std::vector<int32_t> rank;
    std::vector<int64_t> offset;
    int64_t data_len = 0;
    double *data = nullptr;  // device
    // inputs kept for hlu_create_bem
    int32_t n = 0, n_clusters = 0;
    std::vector<int32_t> perm, begin, size, son0, son1, row_cl, col_cl;
    std::vector<int8_t> kind;
};

namespace hlu {
namespace {

constexpr int kBemThreads = 256;
constexpr double kFourPi = 12.566370614359172954, kTwoPi = 6.283185307179586477;

struct BemLeaf {
    int32_t r0, m, c0, n;  // cluster-order row and column ranges
    int64_t D, U, V;       // arena offsets: dense block, or cross factors (cap columns each)
    int32_t kslot;         // kdyn slot of the cross rank (low-rank leaves)
    int32_t pad_;
};

struct BemGeom {
    const double *c;      // n x 3 centroids (original order, row major)
    const double *a;      // n element sizes
    const int32_t *perm;  // cluster order -> original index
    int32_t dim;
};

__device__ __forceinline__ double bem_entry(const BemGeom &g, int i, int j) {
    const double a = g.a[j];
    if (i == j) {
        if (g.dim == 3) return sqrt(a / M_PI) * 0.5;
        const double s = a * (1.0 - log(0.5 * a));
        return g.dim == 1 ? s : s / kTwoPi;
    }
    const double dx = g.c[3 * i] - g.c[3 * j], dy = g.c[3 * i + 1] - g.c[3 * j + 1], dz = g.c[3 * i + 2] - g.c[3 * j + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (g.dim == 3) return a / (kFourPi * r);
    return g.dim == 1 ? -a * log(r) : -a * log(r) / kTwoPi;
}

// Block-wide argmax of (v, idx) with the lowest index among equal values; every thread gets it.
__device__ void block_argmax(double v, int idx, double *sv, int *si, double &ov, int &oi) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        const int wi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (w > v || (w == v && wi < idx)) {
            v = w;
            idx = wi;
        }
    }
    __syncthreads();  // the previous result is no longer read
    if (lane == 0) {
        sv[warp] = v;
        si[warp] = idx;
    }
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sv[lane] : -2.0;
        idx = lane < nw ? si[lane] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            const int wi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (w > v || (w == v && wi < idx)) {
                v = w;
                idx = wi;
            }
        }
        if (lane == 0) {
            sv[32] = v;
            si[32] = idx;
        }
    }
    __syncthreads();
    ov = sv[32];
    oi = si[32];
}

__global__ void __launch_bounds__(kBemThreads) k_bem_dense(const BemLeaf *leaves, BemGeom g, double *arena) {
    const BemLeaf L = leaves[blockIdx.x];
    double *D = arena + L.D;
    for (int64_t e = threadIdx.x; e < (int64_t)L.m * L.n; e += blockDim.x) {
        const int i = (int)(e % L.m), j = (int)(e / L.m);
        D[e] = bem_entry(g, g.perm[L.r0 + i], g.perm[L.c0 + j]);
    }
}

// ACA with partial pivoting (start row 0; column pivot = argmax |residual row|; next row = argmax
// |residual column| over the rows not used yet; lowest index on ties), stopped when
// |u_k| |v_k| <= 0.1 eps |S_k|_F with |S_k|_F^2 updated incrementally, or at min(m, n).  The cross
// factors go to U (m x cap) and V (n x cap); the rank to kdyn[kslot].  Reaching cap < min(m, n)
// without the stopping test is reported as a rank-capacity error of the leaf.
__global__ void __launch_bounds__(kBemThreads) k_bem_aca(const BemLeaf *leaves, BemGeom g, double *arena,
                                                         int32_t *kdyn, int cap, double eps, long long *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double sv[33], dots[2 * 64 + 2];
    __shared__ int si[33];
    __shared__ int s_flag;
    const BemLeaf L = leaves[blockIdx.x];
    const int m = L.m, n = L.n, tid = threadIdx.x, B = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = B >> 5;
    unsigned char *used = smem;
    double *U = arena + L.U, *V = arena + L.V;
    const int kmax = min(min(m, n), cap);
    for (int i = tid; i < m; i += B) used[i] = 0;
    __syncthreads();
    int i = 0, k = 0;
    double s2 = 0.0;  // thread 0
    bool conv = false;
    while (k < kmax) {
        // residual row i into V[:, k]
        const int gi = g.perm[L.r0 + i];
        double best = -1.0;
        int bj = 0x7fffffff;
        for (int j = tid; j < n; j += B) {
            double v = bem_entry(g, gi, g.perm[L.c0 + j]);
            for (int l = 0; l < k; ++l) v -= U[i + (int64_t)l * m] * V[j + (int64_t)l * n];
            V[j + (int64_t)k * n] = v;
            if (fabs(v) > best) {
                best = fabs(v);
                bj = j;
            }
        }
        if (tid == 0) used[i] = 1;
        double pabs;
        int jstar;
        block_argmax(best, bj, sv, si, pabs, jstar);
        const double pv = pabs > 0.0 ? V[jstar + (int64_t)k * n] : 0.0;
        if (pv == 0.0) {  // zero residual row: restart from the first unused row
            double fb = -1.0;
            int fi = 0x7fffffff;
            for (int r = tid; r < m; r += B)
                if (!used[r] && r < fi) {
                    fb = 0.0;
                    fi = r;
                    break;
                }
            double ob;
            int oi;
            block_argmax(fb, fi, sv, si, ob, oi);
            if (ob < 0.0) break;
            i = oi;
            continue;
        }
        const double inv = 1.0 / pv;
        for (int j = tid; j < n; j += B) V[j + (int64_t)k * n] *= inv;
        // residual column jstar into U[:, k]
        const int gj = g.perm[L.c0 + jstar];
        __syncthreads();  // V[jstar, k] is final
        for (int r = tid; r < m; r += B) {
            double u = bem_entry(g, g.perm[L.r0 + r], gj);
            for (int l = 0; l < k; ++l) u -= U[r + (int64_t)l * m] * V[jstar + (int64_t)l * n];
            U[r + (int64_t)k * m] = u;
        }
        __syncthreads();
        // dots: (U_l, u), (V_l, v) for l < k, then |u|^2, |v|^2; one warp per item
        const double *u = U + (int64_t)k * m, *v = V + (int64_t)k * n;
        for (int it = warp; it < 2 * k + 2; it += nw) {
            const bool isu = (it & 1) == 0;
            const int l = it >> 1;
            const double *x = isu ? (l < k ? U + (int64_t)l * m : u) : (l < k ? V + (int64_t)l * n : v);
            const double *y = isu ? u : v;
            const int len = isu ? m : n;
            double s = 0.0;
            for (int r = lane; r < len; r += 32) s += x[r] * y[r];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) dots[it] = s;
        }
        __syncthreads();
        if (tid == 0) {
            double cross = 0.0;
            for (int l = 0; l < k; ++l) cross += dots[2 * l] * dots[2 * l + 1];
            const double uu = dots[2 * k], vv = dots[2 * k + 1];
            s2 += 2.0 * cross + uu * vv;
            s_flag = sqrt(uu * vv) <= 0.1 * eps * sqrt(fmax(s2, 0.0)) ? 1 : 0;
        }
        __syncthreads();
        ++k;
        if (s_flag) {
            conv = true;
            break;
        }
        // next row: argmax |u| over the unused rows
        best = -1.0;
        int bi = 0x7fffffff;
        for (int r = tid; r < m; r += B)
            if (!used[r] && fabs(u[r]) > best) {
                best = fabs(u[r]);
                bi = r;
            }
        double ob;
        int oi;
        block_argmax(best, bi, sv, si, ob, oi);
        if (ob < 0.0) break;
        i = oi;
    }
    if (tid == 0) {
        kdyn[L.kslot] = k;
        if (!conv && k == cap && cap < min(m, n) && atomicAdd(reinterpret_cast<unsigned long long *>(err + 3), 1ull) == 0ull) {
            err[0] = DE_RANKCAP;
            err[1] = blockIdx.x;
            err[2] = k;
        }
    }
}

// Final layout: dense m x n, low-rank U (m x k) then V (n x k), k = kdyn[kslot].
__global__ void __launch_bounds__(kBemThreads) k_bem_pack(const BemLeaf *leaves, const int64_t *out_off,
                                                          const int8_t *kind, const double *arena,
                                                          const int32_t *kdyn, double *out) {
    const BemLeaf L = leaves[blockIdx.x];
    double *o = out + out_off[blockIdx.x];
    if (kind[blockIdx.x] == 0) {
        for (int64_t e = threadIdx.x; e < (int64_t)L.m * L.n; e += blockDim.x) o[e] = arena[L.D + e];
        return;
    }
    const int k = kdyn[L.kslot];
    for (int64_t e = threadIdx.x; e < (int64_t)L.m * k; e += blockDim.x) o[e] = arena[L.U + e];
    for (int64_t e = threadIdx.x; e < (int64_t)L.n * k; e += blockDim.x) o[(int64_t)L.m * k + e] = arena[L.V + e];
}

int cu(cudaError_t e) {
    if (e == cudaSuccess) return HLU_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HLU_ENOMEM : HLU_ECUDA;
}

template <class X>
int dev_copy(X **d, const std::vector<X> &h, std::vector<void *> &owned) {
    *d = nullptr;
    if (h.empty()) return HLU_OK;
    int st = cu(cudaMalloc(reinterpret_cast<void **>(d), sizeof(X) * h.size()));
    if (st) return st;
    owned.push_back(*d);
    return cu(cudaMemcpy(*d, h.data(), sizeof(X) * h.size(), cudaMemcpyHostToDevice));
}

}  // namespace
}  // namespace hlu

using namespace hlu;

extern "C" {

int hlu_bem_build(const hlu_bem_input *in, void *cuda_stream, hlu_bem_t *out) {
    if (!out) return HLU_EINVAL;
    *out = nullptr;
    if (!in || !in->tree || !in->centroid || !in->size || !in->row_cl || !in->col_cl || !in->kind) return HLU_EINVAL;
    const hlu_tree &t = *in->tree;
    if ((in->dim < 1 || in->dim > 3) || t.n < 1 || t.n_clusters < 1 || in->n_leaves < 1 || !(in->eps >= 0.0) ||
        !t.perm || !t.begin || !t.size)
        return HLU_EINVAL;
    const int cap = in->aca_cap > 0 ? in->aca_cap : 48;
    if (cap > 64) return HLU_EINVAL;  // the per-step dot table holds 64 cross vectors
    const int n = t.n;
    for (int c = 0; c < t.n_clusters; ++c)
        if (t.begin[c] < 0 || t.size[c] < 1 || t.begin[c] + t.size[c] > n) return HLU_EINVAL;
    for (int p = 0; p < n; ++p)
        if (t.perm[p] < 0 || t.perm[p] >= n) return HLU_EINVAL;
    for (int p = 0; p < n; ++p)
        if (!(in->size[p] > 0.0) || !std::isfinite(in->centroid[3 * p]) || !std::isfinite(in->centroid[3 * p + 1]) ||
            !std::isfinite(in->centroid[3 * p + 2]))
            return HLU_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    hlu_bem *b = new (std::nothrow) hlu_bem();
    if (!b) return HLU_ENOMEM;
    b->n_leaves = in->n_leaves;
    // arena layout: dense blocks; per low-rank leaf cross factors, truncated factors, workspace
    std::vector<BemLeaf> dense, lowrank;
    std::vector<int64_t> dense_id, lr_id;
    std::vector<TRadd> radd;
    std::vector<Piece> pieces;
    int64_t off = 0;
    int max_m = 1;
    auto a8 = [](int64_t x) { return (x + 7) & ~int64_t(7); };
    for (int64_t l = 0; l < in->n_leaves; ++l) {
        const int rc = in->row_cl[l], cc = in->col_cl[l];
        if (rc < 0 || rc >= t.n_clusters || cc < 0 || cc >= t.n_clusters || (in->kind[l] != 0 && in->kind[l] != 1)) {
            delete b;
            return HLU_EINVAL;
        }
        BemLeaf L{};
        L.r0 = t.begin[rc];
        L.m = t.size[rc];
        L.c0 = t.begin[cc];
        L.n = t.size[cc];
        if (in->kind[l] == 0) {
            L.D = off;
            off = a8(off + int64_t(L.m) * L.n);
            dense.push_back(L);
            dense_id.push_back(l);
        } else {
            const int32_t slot = int32_t(2 * lowrank.size());
            L.U = off;
            L.V = a8(L.U + int64_t(L.m) * cap);
            L.kslot = slot;
            const int64_t Uo = a8(L.V + int64_t(L.n) * cap), Vo = a8(Uo + int64_t(L.m) * cap);
            const int64_t scr = a8(Vo + int64_t(L.n) * cap);
            off = a8(scr + int64_t(L.m + L.n) * cap);
            TRadd r{};
            r.U_off = Uo;
            r.V_off = Vo;
            r.scratch_off = scr;
            r.m = L.m;
            r.n = L.n;
            r.cap = cap;
            r.kslot = slot + 1;
            r.include_self = 0;
            r.piece0 = int32_t(pieces.size());
            r.npieces = 1;
            r.Kcap = cap;
            r.target = int32_t(l);
            r.inst = 0;
            radd.push_back(r);
            pieces.push_back(Piece{1.0, Panel{L.U, L.m, cap, -1, slot, 1, L.m}, Panel{L.V, L.n, cap, -1, slot, 1, L.n}, 0, 0});
            lowrank.push_back(L);
            lr_id.push_back(l);
            max_m = std::max(max_m, L.m);
        }
    }
    std::vector<void *> owned;
    auto fail = [&](int st) {
        for (void *p : owned) cudaFree(p);
        delete b;
        return st;
    };
    std::vector<double> cen(in->centroid, in->centroid + 3 * (int64_t)n), sz(in->size, in->size + n);
    std::vector<int32_t> perm(t.perm, t.perm + n);
    double *d_c, *d_a, *arena;
    int32_t *d_perm, *kdyn;
    BemLeaf *d_dense, *d_lr;
    TRadd *d_radd;
    Piece *d_pieces;
    long long *d_err;
    int st;
    if ((st = dev_copy(&d_c, cen, owned)) || (st = dev_copy(&d_a, sz, owned)) || (st = dev_copy(&d_perm, perm, owned)) ||
        (st = dev_copy(&d_dense, dense, owned)) || (st = dev_copy(&d_lr, lowrank, owned)) ||
        (st = dev_copy(&d_radd, radd, owned)) || (st = dev_copy(&d_pieces, pieces, owned)))
        return fail(st);
    if ((st = cu(cudaMalloc(reinterpret_cast<void **>(&arena), sizeof(double) * std::max<int64_t>(off, 1)))))
        return fail(st);
    owned.push_back(arena);
    const size_t nslots = std::max<size_t>(2 * lowrank.size(), 1);
    if ((st = cu(cudaMalloc(reinterpret_cast<void **>(&kdyn), sizeof(int32_t) * nslots)))) return fail(st);
    owned.push_back(kdyn);
    if ((st = cu(cudaMalloc(reinterpret_cast<void **>(&d_err), sizeof(long long) * 4)))) return fail(st);
    owned.push_back(d_err);
    if ((st = cu(cudaMemsetAsync(kdyn, 0, sizeof(int32_t) * nslots, s))) ||
        (st = cu(cudaMemsetAsync(d_err, 0, sizeof(long long) * 4, s))))
        return fail(st);
    const BemGeom g{d_c, d_a, d_perm, in->dim};
    if (!dense.empty()) k_bem_dense<<<(unsigned)dense.size(), kBemThreads, 0, s>>>(d_dense, g, arena);
    if (!lowrank.empty()) {
        const size_t smem = (size_t)((max_m + 15) & ~15);
        if (smem > 48 * 1024 &&
            (st = cu(cudaFuncSetAttribute(k_bem_aca, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))))
            return fail(st);
        k_bem_aca<<<(unsigned)lowrank.size(), kBemThreads, smem, s>>>(d_lr, g, arena, kdyn, cap, in->eps, d_err);
        if (!set_kernel_attributes<double>()) return fail(HLU_ECUDA);
        LaunchArgs a{};
        a.arena = arena;
        a.kdyn = kdyn;
        a.err = d_err;
        a.eps = in->eps;
        a.kmax = cap;
        a.core64 = 0;
        launch_kind<double>(K_RADD, d_radd, nullptr, d_pieces, 0, (int)radd.size(), cap, a, s);
    }
    if ((st = cu(cudaGetLastError()))) return fail(st);
    long long herr[4];
    std::vector<int32_t> kd(nslots);
    if ((st = cu(cudaMemcpyAsync(herr, d_err, sizeof(herr), cudaMemcpyDeviceToHost, s))) ||
        (st = cu(cudaMemcpyAsync(kd.data(), kdyn, sizeof(int32_t) * nslots, cudaMemcpyDeviceToHost, s))) ||
        (st = cu(cudaStreamSynchronize(s))))
        return fail(st);
    if (herr[0] == DE_RANKCAP) return fail(HLU_ERANKCAP);
    if (herr[0] != DE_OK) return fail(HLU_ENUMERIC);
    // final layout in leaf order
    b->rank.assign(in->n_leaves, 0);
    b->offset.assign(in->n_leaves, 0);
    std::vector<BemLeaf> all(in->n_leaves);
    for (size_t q = 0; q < dense.size(); ++q) all[dense_id[q]] = dense[q];
    for (size_t q = 0; q < lowrank.size(); ++q) {
        BemLeaf L = lowrank[q];
        L.U = radd[q].U_off;  // truncated factors
        L.V = radd[q].V_off;
        L.kslot = radd[q].kslot;
        all[lr_id[q]] = L;
        b->rank[lr_id[q]] = kd[radd[q].kslot];
    }
    int64_t pos = 0;
    for (int64_t l = 0; l < in->n_leaves; ++l) {
        b->offset[l] = pos;
        const BemLeaf &L = all[l];
        pos += in->kind[l] == 0 ? int64_t(L.m) * L.n : int64_t(L.m + L.n) * b->rank[l];
    }
    b->data_len = pos;
    std::vector<int8_t> kinds(in->kind, in->kind + in->n_leaves);
    BemLeaf *d_all;
    int64_t *d_off;
    int8_t *d_kind;
    if ((st = dev_copy(&d_all, all, owned)) || (st = dev_copy(&d_off, b->offset, owned)) ||
        (st = dev_copy(&d_kind, kinds, owned)))
        return fail(st);
    if ((st = cu(cudaMalloc(reinterpret_cast<void **>(&b->data), sizeof(double) * std::max<int64_t>(pos, 1)))))
        return fail(st);
    k_bem_pack<<<(unsigned)in->n_leaves, kBemThreads, 0, s>>>(d_all, d_off, d_kind, arena, kdyn, b->data);
    if ((st = cu(cudaGetLastError())) || (st = cu(cudaStreamSynchronize(s)))) {
        cudaFree(b->data);
        b->data = nullptr;
        return fail(st);
    }
    for (void *p : owned) cudaFree(p);
    b->n = n;
    b->n_clusters = t.n_clusters;
    b->perm.assign(t.perm, t.perm + n);
    b->begin.assign(t.begin, t.begin + t.n_clusters);
    b->size.assign(t.size, t.size + t.n_clusters);
    b->son0.assign(t.son0, t.son0 + t.n_clusters);
    b->son1.assign(t.son1, t.son1 + t.n_clusters);
    b->row_cl.assign(in->row_cl, in->row_cl + in->n_leaves);
    b->col_cl.assign(in->col_cl, in->col_cl + in->n_leaves);
    b->kind = kinds;
    *out = b;
    return HLU_OK;
}

int hlu_bem_result(hlu_bem_t b, int32_t *rank, int64_t *offset, int64_t *data_len, const double **data_dev) {
    if (!b) return HLU_EINVAL;
    if (rank) std::memcpy(rank, b->rank.data(), sizeof(int32_t) * b->n_leaves);
    if (offset) std::memcpy(offset, b->offset.data(), sizeof(int64_t) * b->n_leaves);
    if (data_len) *data_len = b->data_len;
    if (data_dev) *data_dev = b->data;
    return HLU_OK;
}

int hlu_bem_copy_data(hlu_bem_t b, double *host) {
    if (!b || !host) return HLU_EINVAL;
    return cu(cudaMemcpy(host, b->data, sizeof(double) * b->data_len, cudaMemcpyDeviceToHost));
}

int hlu_create_bem(hlu_bem_t b, const hlu_opts *opts, void *cuda_stream, hlu_t *out) {
    if (!out) return HLU_EINVAL;
    *out = nullptr;
    if (!b) return HLU_EINVAL;
    std::vector<double> data(std::max<int64_t>(b->data_len, 1));
    int st = hlu_bem_copy_data(b, data.data());
    if (st) return st;
    const hlu_tree t{b->n, b->n_clusters, b->perm.data(), b->begin.data(), b->size.data(), b->son0.data(),
                     b->son1.data()};
    const hlu_blocks bl{b->n_leaves, b->row_cl.data(), b->col_cl.data(), b->kind.data(), b->rank.data(),
                        b->offset.data(), data.data(), b->data_len};
    return hlu_create(&t, &bl, opts, cuda_stream, out);
}

void hlu_bem_destroy(hlu_bem_t b) {
    if (!b) return;
    if (b->data) cudaFree(b->data);
    delete b;
}

}  // extern "C"
