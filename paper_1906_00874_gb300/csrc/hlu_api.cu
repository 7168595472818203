// C ABI of the H-LU library (declared in include/hlu.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <functional>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hlu.h"
#include "errest.cuh"
#include "gmres.cuh"
#include "kernels.cuh"
#include "plan.h"



using namespace hlu;

namespace {

struct DevPlan {
    TGetrf *getrf = nullptr;
    TTrsm *trsm = nullptr;
    TProject *project = nullptr;
    TAccum *accum = nullptr;
    TRadd *radd = nullptr;
    TSplit *split = nullptr;
    Term *terms = nullptr;
    Piece *pieces = nullptr;
    std::vector<Launch> launches;
    std::vector<int32_t> launch_aux;  // GETRF/TRSM: leaf size for shared memory; RADD: core capacity
    // data-flow execution
    int32_t *code = nullptr, *succ_ptr = nullptr, *succ_idx = nullptr;
    int32_t *indeg0 = nullptr, *indeg = nullptr, *queue = nullptr, *roots = nullptr, *counters = nullptr;
    int32_t n_tasks = 0, n_roots = 0, n_sinks = 0, kc = 1;
    void *scratch = nullptr;
    int64_t scratch_stride = 0;
    void *core_scratch = nullptr;  // cores of rounded additions above kSmemCore (global)
    int64_t core_stride = 0;
    int workers = 0;          // worker CTAs of a launch (at most workers_alloc)
    int workers_alloc = 0;    // workers the per-worker scratch was allocated for
    size_t smem = 0;
};

// Profiling counters: [0, 32) task times and counts of factorisations (see
// FlowArgs::busy), [32, 48) rounded-addition phases (see LaunchArgs::phase),
// [48, 64) task times and counts of solves.
constexpr int kBusyWords = 64;
// Launch-time slots: task kinds (wave schedule), then the data-flow launches of
// factorisations, solves and H-matrix products.
constexpr int kProfSlots = 10;

// Largest stacked rank whose rounded-addition core the data-flow kernel keeps in
// shared memory: sized so that two 256-thread workers fit on one SM.
constexpr int kSmemCore = 64;

struct Pending {
    int kind;
    cudaEvent_t e0, e1;
};

}  // namespace

struct hlu_ctx {
    Planner pl;
    int precision = HLU_FP64;   // storage precision of the factors: HLU_FP64 or HLU_FP32
    bool core64 = true;         // FP32 factors: SVD of each truncation core in FP64 (HLU_FP32_CORE32: FP32)
    bool tensor = false;        // FP32 factors: dense products of the factorisation on the tensor cores
    int max_workers = 0;        // most worker CTAs per data-flow launch (0: all that are resident)
    int schedule = HLU_SCHED_DATAFLOW;
    unsigned long long timeout_ns = 10000000000ull;
    cudaStream_t stream = nullptr;
    void *farena = nullptr;
    double *aarena = nullptr;
    int32_t *kdyn = nullptr;
    long long *err = nullptr;
    double *flops = nullptr;  // [0, 8): factorisation, [8, 16): solves and products
    int32_t *perm = nullptr;
    int64_t *leaf_desc = nullptr;
    double *ir = nullptr;     // refinement work: b, x, r (n x nrhs_max each) and 2 x nrhs_max norms
    double *ir_host = nullptr;  // host copy of the norms (pageable: a pinned allocation would
                                // synchronise the device with the work of every other stream)
    // GMRES: Krylov bases V ((m + 1) panels) and Z = M^{-1} V (m panels) of n x nrhs_max, small state
    int gm_m = 0;
    double *gm_V = nullptr, *gm_Z = nullptr, *gm_small = nullptr, *gm_host = nullptr;
    DevPlan fp, sp, mp;
    int64_t device_bytes = 0;
    int64_t mem_budget = 0;
    bool factored = false;
    double eps = 0.0;
    std::vector<void *> allocs;
    int last_status = HLU_OK;
    long long last_err[4] = {0, 0, 0, 0};
    // profiling
    bool profiling = false;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    double prof_ms[kProfSlots] = {0};
    int64_t prof_count[kProfSlots] = {0};
    int64_t kernels_launched = 0;
    cudaError_t last_cuda = cudaSuccess;
    unsigned long long *busy = nullptr;  // per-kind task time inside the data-flow kernel (profiling)
    bool inject_stall = false;           // next data-flow factorisation: one task never becomes ready
    double *eps_inst = nullptr;          // per-instance tolerances of a batch (device), used when eps_each
    bool eps_each = false;
    double create_ms[2] = {0.0, 0.0};    // host time of hlu_create: validation + planning, device set-up
    // factorisation-error estimate (hlu_factor_error): leaf table and work vectors, made on first use
    ErrLeaf *err_leaves = nullptr;
    double *err_work = nullptr;
    double *err_host = nullptr;
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? HLU_OK : HLU_ECUDA; }

// Device-to-host copy ordered on the handle's stream (not the legacy default stream, which would
// also wait for the work of other handles on other streams).
cudaError_t d2h(hlu_ctx *h, void *dst, const void *src, size_t bytes);

template <class X>
int dalloc(hlu_ctx *h, X **p, size_t count) {
    *p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(X);
    if (h->mem_budget > 0 && h->device_bytes + (int64_t)bytes > h->mem_budget) return HLU_ENOMEM;
    // stream-ordered allocation: a plain cudaMalloc is an implicit synchronisation point between
    // streams, so creating one handle would wait for the kernels of every other handle
    if (cudaMallocAsync(reinterpret_cast<void **>(p), bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return HLU_ENOMEM;
    }
    h->allocs.push_back(*p);
    h->device_bytes += (int64_t)bytes;
    return HLU_OK;
}

template <class X>
int upload(hlu_ctx *h, X **p, const std::vector<X> &v) {
    int st = dalloc(h, p, v.size());
    if (st) return st;
    if (!v.empty())
        return cuda_status(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, h->stream));
    return HLU_OK;
}

int upload_plan(hlu_ctx *h, const Plan &p, DevPlan &d, int kmax) {
    int st;
    if ((st = upload(h, &d.getrf, p.getrf))) return st;
    if ((st = upload(h, &d.trsm, p.trsm))) return st;
    if ((st = upload(h, &d.project, p.project))) return st;
    if ((st = upload(h, &d.accum, p.accum))) return st;
    if ((st = upload(h, &d.radd, p.radd))) return st;
    if ((st = upload(h, &d.split, p.split))) return st;
    if ((st = upload(h, &d.terms, p.terms))) return st;
    if ((st = upload(h, &d.pieces, p.pieces))) return st;
    d.launches = p.launches;
    d.launch_aux.resize(p.launches.size());
    for (size_t i = 0; i < p.launches.size(); ++i) {
        const Launch &L = p.launches[i];
        int aux = h->pl.max_leaf;
        if (L.kind == K_RADD) {
            int kc = 1;
            for (int j = L.start; j < L.start + L.count; ++j) kc = std::max(kc, p.radd[j].Kcap);
            aux = std::min(kc, kmax);
        }
        d.launch_aux[i] = aux;
    }
    // data-flow graph and per-worker workspace
    d.n_tasks = (int32_t)p.n_tasks;
    d.n_roots = (int32_t)p.roots.size();
    d.n_sinks = 0;
    for (int64_t g = 0; g < p.n_tasks; ++g) d.n_sinks += p.succ_ptr[g + 1] == p.succ_ptr[g];
    if ((st = upload(h, &d.code, p.task_code))) return st;
    if ((st = upload(h, &d.succ_ptr, p.succ_ptr))) return st;
    if ((st = upload(h, &d.succ_idx, p.succ_idx))) return st;
    if ((st = upload(h, &d.indeg0, p.indeg))) return st;
    if ((st = upload(h, &d.roots, p.roots))) return st;
    if ((st = dalloc(h, &d.indeg, p.indeg.size()))) return st;
    if ((st = dalloc(h, &d.queue, p.indeg.size()))) return st;
    if ((st = dalloc(h, &d.counters, 3))) return st;
    int kc = 1;
    int64_t stride = 1;
    for (const TRadd &r : p.radd) {
        const int k = std::min(r.Kcap, kmax);
        kc = std::max(kc, k);
        stride = std::max<int64_t>(stride, int64_t(r.m + r.n) * std::max(k, 1));
    }
    d.kc = kc;
    d.scratch_stride = (stride + 31) & ~int64_t(31);
    const int elem = h->precision == HLU_FP64 ? 8 : 4;
    const bool dbl = &d == &h->mp || h->precision == HLU_FP64;
    const bool c64 = !dbl && h->core64;
    d.smem = dataflow_smem_bytes(h->pl.max_leaf, dbl ? 8 : elem, std::min(kc, kSmemCore), c64);
    d.workers = dbl ? dataflow_workers<double>(d.smem) : dataflow_workers<float>(d.smem);
    if (h->max_workers > 0) d.workers = std::min(d.workers, h->max_workers);
    d.workers_alloc = d.workers;
    if (!p.radd.empty()) {
        const size_t bytes = size_t(d.workers) * d.scratch_stride * (dbl ? 8 : elem);
        char *sp = nullptr;
        if ((st = dalloc(h, &sp, bytes))) return st;
        d.scratch = sp;
        if (kc > kSmemCore) {
            d.core_stride = (int64_t)((radd_smem_bytes(kc, dbl ? 8 : elem, c64) + 255) & ~size_t(255));
            char *cp = nullptr;
            if ((st = dalloc(h, &cp, size_t(d.workers) * d.core_stride))) return st;
            d.core_scratch = cp;
        }
    }
    return HLU_OK;
}

const void *task_ptr(const DevPlan &d, int kind) {
    switch (kind) {
        case K_GETRF: return d.getrf;
        case K_TRSM: return d.trsm;
        case K_PROJECT: return d.project;
        case K_ACCUM: return d.accum;
        case K_RADD: return d.radd;
        case K_SPLIT: return d.split;
    }
    return nullptr;
}

cudaEvent_t take_event(hlu_ctx *h) {
    if (!h->free_events.empty()) {
        cudaEvent_t e = h->free_events.back();
        h->free_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Accumulate the durations of the profiled launches (after a synchronisation).
void collect_profile(hlu_ctx *h) {
    for (const Pending &p : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
            h->prof_ms[p.kind] += ms;
            h->prof_count[p.kind] += 1;
        }
        h->free_events.push_back(p.e0);
        h->free_events.push_back(p.e1);
    }
    h->pending.clear();
}

void run_plan(hlu_ctx *h, const DevPlan &d, void *arena, double *flops) {
    LaunchArgs a;
    a.arena = arena;
    a.kdyn = h->kdyn;
    a.err = h->err;
    a.eps = h->eps;
    a.eps_inst = h->eps_each ? h->eps_inst : nullptr;
    a.flops = flops;
    a.phase = (h->profiling && &d == &h->fp) ? h->busy + 32 : nullptr;
    a.kmax = h->pl.opt.kmax_core;
    a.core64 = h->core64 ? 1 : 0;
    const bool dbl = arena == (void *)h->aarena || h->precision == HLU_FP64;
    if (h->schedule == HLU_SCHED_DATAFLOW && d.n_tasks > 0) {
        FlowArgs f;
        f.code = d.code;
        f.succ_ptr = d.succ_ptr;
        f.succ_idx = d.succ_idx;
        f.indeg = d.indeg;
        f.queue = d.queue;
        f.counters = d.counters;
        f.n_tasks = d.n_tasks;
        f.n_sinks = d.n_sinks;
        f.kc = d.kc;
        f.getrf = d.getrf;
        f.trsm = d.trsm;
        f.project = d.project;
        f.accum = d.accum;
        f.radd = d.radd;
        f.split = d.split;
        f.terms = d.terms;
        f.pieces = d.pieces;
        f.smem_bytes = d.smem;
        f.core_scratch = d.core_scratch;
        f.core_stride = d.core_stride;
        f.scratch = d.scratch;
        f.scratch_stride = d.scratch_stride;
        f.timeout_ns = h->timeout_ns;
        f.tensor = (h->tensor && !dbl && &d == &h->fp) ? 1 : 0;
        f.tc_min_inner = 32;
        f.busy = !h->profiling ? nullptr : &d == &h->fp ? h->busy : &d == &h->sp ? h->busy + 48 : nullptr;
        cudaMemcpyAsync(d.indeg, d.indeg0, sizeof(int32_t) * d.n_tasks, cudaMemcpyDeviceToDevice, h->stream);
        cudaMemsetAsync(d.queue, 0xff, sizeof(int32_t) * d.n_tasks, h->stream);
        cudaMemcpyAsync(d.queue, d.roots, sizeof(int32_t) * d.n_roots, cudaMemcpyDeviceToDevice, h->stream);
        if (h->inject_stall && &d == &h->fp && d.n_tasks > 0) {  // test hook: the last task waits forever
            const int32_t last = d.n_tasks - 1;
            launch_set_slot(d.indeg, last, h->pl.fplan.last_indeg + 1, h->stream);
            h->inject_stall = false;
        }
        cudaMemsetAsync(d.counters, 0, 3 * sizeof(int32_t), h->stream);
        launch_set_slot(d.counters, 1, d.n_roots, h->stream);
        // profiling slots 6 / 7 / 8: the data-flow launch of a factorisation / a solve / a product
        Pending pe{&d == &h->fp ? K_NKINDS : &d == &h->sp ? K_NKINDS + 1 : K_NKINDS + 2, nullptr, nullptr};
        if (h->profiling) {
            pe.e0 = take_event(h);
            pe.e1 = take_event(h);
            cudaEventRecord(pe.e0, h->stream);
        }
        if (dbl)
            launch_dataflow<double>(f, a, d.workers, d.smem, h->stream);
        else
            launch_dataflow<float>(f, a, d.workers, d.smem, h->stream);
        if (h->profiling) {
            cudaEventRecord(pe.e1, h->stream);
            h->pending.push_back(pe);
        }
        h->kernels_launched += 2;
        return;
    }
    for (size_t i = 0; i < d.launches.size(); ++i) {
        const Launch &L = d.launches[i];
        Pending pe{L.kind, nullptr, nullptr};
        if (h->profiling) {
            pe.e0 = take_event(h);
            pe.e1 = take_event(h);
            cudaEventRecord(pe.e0, h->stream);
        }
        if (dbl)
            launch_kind<double>(L.kind, task_ptr(d, L.kind), d.terms, d.pieces, L.start, L.count, d.launch_aux[i], a,
                                h->stream);
        else
            launch_kind<float>(L.kind, task_ptr(d, L.kind), d.terms, d.pieces, L.start, L.count, d.launch_aux[i], a,
                               h->stream);
        if (h->profiling) {
            cudaEventRecord(pe.e1, h->stream);
            h->pending.push_back(pe);
        }
    }
    h->kernels_launched += (int64_t)d.launches.size();
}

cudaError_t d2h(hlu_ctx *h, void *dst, const void *src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e;
}

int read_error(hlu_ctx *h) {
    cudaError_t e = cudaGetLastError();  // launch-time errors first
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        h->last_cuda = e;
        return HLU_ECUDA;
    }
    if (h->profiling) collect_profile(h);
    long long w[4];
    if (d2h(h, w, h->err, sizeof(w)) != cudaSuccess) return HLU_ECUDA;
    std::memcpy(h->last_err, w, sizeof(w));
    switch ((int)w[0]) {
        case DE_OK: return HLU_OK;
        case DE_PIVOT: return HLU_EPIVOT;
        case DE_RANKCAP: return HLU_ERANKCAP;
        case DE_NONFINITE: return HLU_ENUMERIC;
        case DE_TIMEOUT: return HLU_ETIMEOUT;
    }
    return HLU_ECUDA;
}

int clear_error(hlu_ctx *h) { return cuda_status(cudaMemsetAsync(h->err, 0, 4 * sizeof(long long), h->stream)); }

template <class T>
int upload_arenas(hlu_ctx *h, const double *data) {
    Planner &pl = h->pl;
    // A_H arena: leaves exactly as given (FP64), then zeroed work panels
    int64_t a_leaf_end = 0;
    for (const Store &s : pl.astore) {
        int64_t end = s.kind == B_DENSE ? s.D_off + int64_t(s.m) * s.n : s.V_off + int64_t(s.n) * s.krank;
        a_leaf_end = std::max(a_leaf_end, end);
    }
    // the staging copy, split over host threads by leaves (panels are packed in leaf order, each
    // followed by at most 7 elements of alignment that are zeroed)
    std::unique_ptr<double[]> a_leaves(new (std::nothrow) double[std::max<int64_t>(a_leaf_end, 1)]);
    if (!a_leaves) return HLU_ENOMEM;
    auto stage = [&](int64_t l0, int64_t l1) {
        auto put = [&](int64_t off, const double *src, int64_t len, int64_t next) {
            std::memcpy(&a_leaves[off], src, sizeof(double) * len);
            for (int64_t i = off + len; i < std::min(next, a_leaf_end); ++i) a_leaves[i] = 0.0;
        };
        for (int64_t l = l0; l < l1; ++l) {
            const Store &s = pl.astore[l];
            const double *src = data + pl.leaf_offset[l];
            if (s.kind == B_DENSE) {
                const int64_t len = int64_t(s.m) * s.n;
                put(s.D_off, src, len, (s.D_off + len + 7) & ~int64_t(7));
            } else {
                const int64_t lu = int64_t(s.m) * s.krank, lv = int64_t(s.n) * s.krank;
                put(s.U_off, src, lu, s.V_off);
                put(s.V_off, src + lu, lv, (s.V_off + lv + 7) & ~int64_t(7));
            }
        }
    };
    const int nthreads = int(std::min<int64_t>(std::max(1u, std::min(8u, std::thread::hardware_concurrency())),
                                                std::max<int64_t>(1, a_leaf_end >> 20)));
    if (nthreads <= 1) {
        stage(0, pl.n_leaves);
    } else {
        run_parts(nthreads, [&](int q) { stage(pl.n_leaves * q / nthreads, pl.n_leaves * (q + 1) / nthreads); });
    }
    std::vector<int64_t> desc(kLeafDesc * pl.n_leaves);
    for (int64_t l = 0; l < pl.n_leaves; ++l) {
        const Store &s = pl.astore[l];
        const Store &f = pl.fstore[l];
        int64_t *d = &desc[kLeafDesc * l];
        d[0] = s.kind == B_DENSE ? 0 : 1;
        d[1] = s.m;
        d[2] = s.n;
        d[3] = s.kind == B_DENSE ? 0 : s.krank;
        d[4] = s.kind == B_DENSE ? s.D_off : s.U_off;
        d[5] = s.kind == B_DENSE ? 0 : s.V_off;
        d[6] = s.kind == B_DENSE ? f.D_off : f.U_off;
        d[7] = s.kind == B_DENSE ? 0 : f.V_off;
        d[8] = s.kind == B_DENSE ? 0 : f.kslot;
    }
    int st;
    if ((st = dalloc(h, &h->aarena, pl.a_elems))) return st;
    if ((st = cuda_status(cudaMemsetAsync(h->aarena, 0, sizeof(double) * pl.a_elems, h->stream)))) return st;
    if ((st = cuda_status(cudaMemcpyAsync(h->aarena, a_leaves.get(), sizeof(double) * a_leaf_end,
                                          cudaMemcpyHostToDevice, h->stream))))
        return st;
    if ((st = upload(h, &h->leaf_desc, desc))) return st;
    T *f = nullptr;
    if ((st = dalloc(h, &f, pl.f_elems))) return st;
    h->farena = f;
    if ((st = cuda_status(cudaMemsetAsync(f, 0, sizeof(T) * pl.f_elems, h->stream)))) return st;
    std::vector<T> ident((size_t)pl.max_leaf * pl.max_leaf, T(0));
    for (int i = 0; i < pl.max_leaf; ++i) ident[i + (size_t)i * pl.max_leaf] = T(1);
    if ((st = cuda_status(cudaMemcpyAsync(f + pl.f_ident_off, ident.data(), sizeof(T) * ident.size(),
                                          cudaMemcpyHostToDevice, h->stream))))
        return st;
    // the host staging vectors die at return: wait for the copies
    return cuda_status(cudaStreamSynchronize(h->stream));
}

// One solve pass on the factor arena's work panel Y (cluster order, nc columns, ld n).
void solve_pass(hlu_ctx *h, int32_t nc) {
    launch_set_slot(h->kdyn, h->pl.nrhs_slot, nc, h->stream);
    h->kernels_launched += 1;
    run_plan(h, h->sp, h->farena, h->flops + 8);
}

// A_H x_c for a cluster-order panel already copied into the A_H arena's X panel; result in its Y panel.
void matvec_pass(hlu_ctx *h, int32_t nc) {
    launch_set_slot(h->kdyn, h->pl.nrhs_slot, nc, h->stream);
    h->kernels_launched += 1;
    run_plan(h, h->mp, h->aarena, h->flops + 8);
}

}  // namespace

namespace {
int factor_impl(hlu_ctx *h);
}  // namespace

extern "C" {

const char *hlu_strerror(int s) {
    switch (s) {
        case HLU_OK: return "ok";
        case HLU_EINVAL: return "invalid argument or malformed H-matrix";
        case HLU_ENOMEM: return "out of device memory (or over the memory budget)";
        case HLU_ESTATE: return "call out of order";
        case HLU_EPIVOT: return "zero or non-finite pivot in a dense diagonal leaf";
        case HLU_ERANKCAP: return "rank capacity exceeded";
        case HLU_ETIMEOUT: return "device-side wait timed out";
        case HLU_ECUDA: return "CUDA runtime error";
        case HLU_ENUMERIC: return "non-finite value during the factorisation";
    }
    return "unknown status";
}

static int create_impl(const hlu_tree *tree, const hlu_blocks *blocks, const hlu_opts *opts, void *cuda_stream,
                       hlu_t *out, const int32_t *inst, int32_t n_inst) {
    if (!out) return HLU_EINVAL;
    *out = nullptr;
    if (!tree || !blocks) return HLU_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    hlu_ctx *h = new (std::nothrow) hlu_ctx();
    if (!h) return HLU_ENOMEM;
    PlanOptions po;
    if (opts) {
        h->precision = opts->precision;
        if (opts->rank_cap > 0) po.rank_cap = opts->rank_cap;
        if (opts->nrhs_max > 0) po.nrhs_max = opts->nrhs_max;
        h->mem_budget = opts->mem_budget;
        h->schedule = opts->schedule;
        if (opts->timeout_s > 0.0) h->timeout_ns = (unsigned long long)(opts->timeout_s * 1e9);
        if (opts->inv_block != 0) po.inv_block = opts->inv_block < 0 ? 0 : opts->inv_block;
        po.temp_reuse = opts->temp_reuse > 0;
        h->tensor = (opts->flags & HLU_FLAG_TENSOR) != 0;
        if (opts->flags & HLU_FLAG_SERIAL_PLAN) po.batch_threads = -1;
        h->max_workers = std::max(0, opts->workers);
    }
    if (h->precision == HLU_FP32_CORE32) {  // FP32 factors, FP32 Jacobi in the truncation cores
        h->precision = HLU_FP32;
        h->core64 = false;
    }
    if ((h->precision != HLU_FP64 && h->precision != HLU_FP32) ||
        (h->schedule != HLU_SCHED_DATAFLOW && h->schedule != HLU_SCHED_WAVES)) {
        delete h;
        return HLU_EINVAL;
    }
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    po.wave_order = h->schedule == HLU_SCHED_WAVES;
    int st = h->pl.build(tree->n, tree->n_clusters, tree->perm, tree->begin, tree->size, tree->son0, tree->son1,
                         blocks->n_leaves, blocks->row_cl, blocks->col_cl, blocks->kind, blocks->rank,
                         blocks->offset, blocks->data, blocks->data_len, po, inst, n_inst);
    if (st == HLU_OK && h->pl.max_leaf > 128) st = HLU_EINVAL;  // a dense leaf column lives in one warp's registers
    if (st == HLU_OK) st = h->pl.plan_all();
    const auto t1 = std::chrono::steady_clock::now();
    if (st == HLU_OK) {
        // the FP64 kernels always run the matrix-vector product on A_H
        const bool attrs = set_kernel_attributes<double>() &&
                           (h->precision == HLU_FP64 || set_kernel_attributes<float>());
        if (!attrs)
            st = HLU_ECUDA;
        else if (h->precision == HLU_FP64)
            st = upload_arenas<double>(h, blocks->data);
        else
            st = upload_arenas<float>(h, blocks->data);
    }
    const int64_t n = h->pl.n, w = h->pl.opt.nrhs_max;
    if (st == HLU_OK) st = upload(h, &h->kdyn, h->pl.slot_init);
    if (st == HLU_OK) st = dalloc(h, &h->err, 4);
    if (st == HLU_OK) st = dalloc(h, &h->flops, 16);
    if (st == HLU_OK) st = dalloc(h, &h->busy, kBusyWords);
    if (st == HLU_OK)
        st = cuda_status(cudaMemsetAsync(h->busy, 0, kBusyWords * sizeof(unsigned long long), h->stream));
    if (st == HLU_OK) st = cuda_status(cudaMemsetAsync(h->flops, 0, 16 * sizeof(double), h->stream));
    if (st == HLU_OK) st = dalloc(h, &h->ir, 3 * n * w + 2 * w);
    if (st == HLU_OK && !(h->ir_host = new (std::nothrow) double[2 * w])) st = HLU_ENOMEM;
    if (st == HLU_OK) st = clear_error(h);
    if (st == HLU_OK) st = upload(h, &h->perm, h->pl.perm);
    const int kmax = h->pl.opt.kmax_core;
    if (st == HLU_OK) st = upload_plan(h, h->pl.fplan, h->fp, kmax);
    if (st == HLU_OK) st = upload_plan(h, h->pl.splan, h->sp, kmax);
    if (st == HLU_OK) st = upload_plan(h, h->pl.mplan, h->mp, kmax);
    if (st == HLU_OK) st = cuda_status(cudaStreamSynchronize(h->stream));
    if (st == HLU_OK) {  // the device holds the graphs now: the host keeps the layout and the figures
        h->pl.release_work();
        for (Plan *p : {&h->pl.fplan, &h->pl.splan, &h->pl.mplan}) p->release_tasks();
    }
    if (st != HLU_OK) {
        hlu_destroy(h);
        return st;
    }
    const auto t2 = std::chrono::steady_clock::now();
    h->create_ms[0] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    h->create_ms[1] = std::chrono::duration<double, std::milli>(t2 - t1).count();
    *out = h;
    return HLU_OK;
}

int hlu_create(const hlu_tree *tree, const hlu_blocks *blocks, const hlu_opts *opts, void *cuda_stream,
               hlu_t *out) {
    return create_impl(tree, blocks, opts, cuda_stream, out, nullptr, 0);
}

}  // extern "C"

namespace {

// Several problems as one block-diagonal H-matrix: count - 1 clusters above the problems (cluster 0
// is the root), then every problem's clusters with indices and ranges shifted; leaves, offsets and
// data concatenated.  inst[c] is the problem of cluster c (-1 above the problems).
struct Forest {
    std::vector<int32_t> perm, begin, size, son0, son1, inst, rc, cc, rk;
    std::vector<int8_t> kd;
    std::vector<int64_t> off;
    std::unique_ptr<double[]> data;
    hlu_tree t{};
    hlu_blocks b{};
};

int make_forest(int32_t count, const hlu_tree *trees, const hlu_blocks *blocks, Forest &f) {
    if (count < 1 || !trees || !blocks) return HLU_EINVAL;
    int64_t N = 0, ncl = count - 1, nl = 0, dl = 0;
    for (int32_t i = 0; i < count; ++i) {
        const hlu_tree &t = trees[i];
        const hlu_blocks &b = blocks[i];
        if (t.n < 1 || t.n_clusters < 1 || !t.perm || !t.begin || !t.size || !t.son0 || !t.son1 || b.n_leaves < 1 ||
            !b.row_cl || !b.col_cl || !b.kind || !b.rank || !b.offset || !b.data || b.data_len < 0)
            return HLU_EINVAL;
        N += t.n;
        ncl += t.n_clusters;
        nl += b.n_leaves;
        dl += b.data_len;
    }
    if (N > INT32_MAX || ncl > INT32_MAX) return HLU_EINVAL;
    // clusters: count - 1 clusters above the instances first (cluster 0 is the root), then every
    // instance's own clusters, indices and ranges shifted; leaves, offsets and data concatenated
    f.perm.assign(N, 0);
    f.begin.assign(ncl, 0);
    f.size.assign(ncl, 0);
    f.son0.assign(ncl, -1);
    f.son1.assign(ncl, -1);
    f.inst.assign(ncl, -1);
    f.rc.assign(nl, 0);
    f.cc.assign(nl, 0);
    f.rk.assign(nl, 0);
    f.kd.assign(nl, 0);
    f.off.assign(nl, 0);
    f.data.reset(new (std::nothrow) double[std::max<int64_t>(dl, 1)]);
    if (!f.data) return HLU_ENOMEM;
    std::vector<int32_t> &perm = f.perm, &begin = f.begin, &size = f.size, &son0 = f.son0, &son1 = f.son1,
                         &inst = f.inst, &rc = f.rc, &cc = f.cc, &rk = f.rk;
    std::vector<int8_t> &kd = f.kd;
    std::vector<int64_t> &off = f.off, cl_off(count);
    std::vector<int64_t> data_at(count);  // where each problem's leaf data starts in the concatenation
    int64_t no = 0, co = count - 1, lo = 0, dof = 0;
    for (int32_t i = 0; i < count; ++i) {
        const hlu_tree &t = trees[i];
        const hlu_blocks &b = blocks[i];
        cl_off[i] = co;
        for (int32_t c = 0; c < t.n_clusters; ++c) {
            begin[co + c] = int32_t(t.begin[c] + no);
            size[co + c] = t.size[c];
            son0[co + c] = t.son0[c] >= 0 ? int32_t(t.son0[c] + co) : -1;
            son1[co + c] = t.son1[c] >= 0 ? int32_t(t.son1[c] + co) : -1;
            inst[co + c] = i;
        }
        for (int32_t k = 0; k < t.n; ++k) perm[no + k] = int32_t(t.perm[k] + no);
        for (int64_t l = 0; l < b.n_leaves; ++l) {
            rc[lo + l] = int32_t(b.row_cl[l] + co);
            cc[lo + l] = int32_t(b.col_cl[l] + co);
            kd[lo + l] = b.kind[l];
            rk[lo + l] = b.rank[l];
            off[lo + l] = b.offset[l] + dof;
        }
        data_at[i] = dof;
        no += t.n;
        co += t.n_clusters;
        lo += b.n_leaves;
        dof += b.data_len;
    }
    // the leaf data, copied problem by problem on up to eight host threads
    {
        std::atomic<int32_t> next{0};
        auto copy = [&] {
            for (int32_t i; (i = next.fetch_add(1)) < count;)
                std::memcpy(f.data.get() + data_at[i], blocks[i].data, sizeof(double) * blocks[i].data_len);
        };
        const int nthreads = int(std::min<int64_t>(std::max(1u, std::min(8u, std::thread::hardware_concurrency())),
                                                    std::min<int64_t>(count, std::max<int64_t>(1, dl >> 20))));
        run_parts(nthreads, [&](int) { copy(); });
    }
    // a balanced binary tree of clusters over the instances, numbered from 0 (the root)
    int32_t next_v = 0;
    std::function<int32_t(int32_t, int32_t)> make = [&](int32_t i0, int32_t i1) -> int32_t {
        if (i1 - i0 == 1) return int32_t(cl_off[i0]);
        const int32_t v = next_v++, mid = (i0 + i1) / 2;
        const int32_t a = make(i0, mid), b = make(mid, i1);
        begin[v] = begin[a];
        size[v] = size[a] + size[b];
        son0[v] = a;
        son1[v] = b;
        return v;
    };
    make(0, count);
    f.t = hlu_tree{int32_t(N), int32_t(ncl), perm.data(), begin.data(), size.data(), son0.data(), son1.data()};
    f.b = hlu_blocks{nl, rc.data(), cc.data(), kd.data(), rk.data(), off.data(), f.data.get(), dl};
    return HLU_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

int plan_only(const hlu_tree *tree, const hlu_blocks *blocks, const hlu_opts *opts, const int32_t *inst,
              int32_t n_inst, hlu_plan_info *out) {
    if (!out || !tree || !blocks) return HLU_EINVAL;
    std::memset(out, 0, sizeof(*out));
    const auto t0 = std::chrono::steady_clock::now();
    PlanOptions po;
    if (opts) {
        if (opts->rank_cap > 0) po.rank_cap = opts->rank_cap;
        if (opts->nrhs_max > 0) po.nrhs_max = opts->nrhs_max;
        if (opts->inv_block != 0) po.inv_block = opts->inv_block < 0 ? 0 : opts->inv_block;
        po.temp_reuse = opts->temp_reuse > 0;
        po.wave_order = opts->schedule == HLU_SCHED_WAVES;
        if (opts->flags & HLU_FLAG_SERIAL_PLAN) po.batch_threads = -1;
    } else {
        po.wave_order = false;
    }
    Planner pl;
    int st = pl.build(tree->n, tree->n_clusters, tree->perm, tree->begin, tree->size, tree->son0, tree->son1,
                      blocks->n_leaves, blocks->row_cl, blocks->col_cl, blocks->kind, blocks->rank, blocks->offset,
                      blocks->data, blocks->data_len, po, inst, n_inst);
    if (st == HLU_OK && pl.max_leaf > 128) st = HLU_EINVAL;
    if (st == HLU_OK) st = pl.plan_all();
    if (st) return st;
    out->factor_tasks = pl.fplan.n_tasks;
    out->factor_edges = pl.fplan.n_edges;
    out->factor_levels = pl.fplan.n_waves;
    out->solve_tasks = pl.splan.n_tasks;
    out->solve_levels = pl.splan.n_waves;
    out->matvec_tasks = pl.mplan.n_tasks;
    out->inverse_blocks = (int64_t)pl.inv_cl.size();
    out->factor_elems = pl.f_elems;
    out->factor_temp_elems = pl.fplan.temp_elems;
    out->factor_temp_peak_elems = pl.fplan.temp_peak_elems;
    out->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    out->factor_critical_us = pl.fplan.critical_us;
    out->solve_critical_us = pl.splan.critical_us;
    return HLU_OK;
}

}  // namespace

extern "C" {

int hlu_plan_info_get(const hlu_tree *tree, const hlu_blocks *blocks, const hlu_opts *opts, hlu_plan_info *out) {
    return plan_only(tree, blocks, opts, nullptr, 0, out);
}

int hlu_plan_info_batch(int32_t count, const hlu_tree *trees, const hlu_blocks *blocks, const hlu_opts *opts,
                        hlu_plan_info *out) {
    Forest f;
    const int st = make_forest(count, trees, blocks, f);
    if (st) return st;
    return plan_only(&f.t, &f.b, opts, f.inst.data(), count, out);
}

int hlu_create_batch(int32_t count, const hlu_tree *trees, const hlu_blocks *blocks, const hlu_opts *opts,
                     void *cuda_stream, hlu_t *out) {
    if (!out) return HLU_EINVAL;
    *out = nullptr;
    Forest f;
    const int st = make_forest(count, trees, blocks, f);
    if (st) return st;
    return create_impl(&f.t, &f.b, opts, cuda_stream, out, f.inst.data(), count);
}

int hlu_factor(hlu_t h, double eps) {
    if (!h || !(eps >= 0.0) || !std::isfinite(eps)) return HLU_EINVAL;
    h->eps = eps;
    h->eps_each = false;
    return factor_impl(h);
}

int hlu_factor_batch(hlu_t h, const double *eps) {
    if (!h || !eps) return HLU_EINVAL;
    const int32_t ni = h->pl.n_inst;
    for (int32_t i = 0; i < ni; ++i)
        if (!(eps[i] >= 0.0) || !std::isfinite(eps[i])) return HLU_EINVAL;
    int st = HLU_OK;
    if (!h->eps_inst && (st = dalloc(h, &h->eps_inst, ni))) return st;
    if ((st = cuda_status(cudaMemcpyAsync(h->eps_inst, eps, sizeof(double) * ni, cudaMemcpyHostToDevice, h->stream))))
        return st;
    if ((st = cuda_status(cudaStreamSynchronize(h->stream)))) return st;  // eps is the caller's memory
    h->eps = eps[0];
    h->eps_each = true;
    return factor_impl(h);
}

int hlu_batch_count(hlu_t h) { return h ? h->pl.n_inst : 0; }

}  // extern "C"

namespace {

int factor_impl(hlu_ctx *h) {
    h->factored = false;
    int st = clear_error(h);
    if (st) return st;
    if ((st = cuda_status(cudaMemsetAsync(h->flops, 0, 16 * sizeof(double), h->stream)))) return st;
    // restore the working copy from A_H (the factorisation overwrites it) and the ranks
    if ((st = cuda_status(cudaMemcpyAsync(h->kdyn, h->pl.slot_init.data(), sizeof(int32_t) * h->pl.n_slots,
                                          cudaMemcpyHostToDevice, h->stream))))
        return st;
    if (h->precision == HLU_FP64)
        launch_reset<double>(h->leaf_desc, h->pl.n_leaves, h->aarena, (double *)h->farena, h->kdyn, h->stream);
    else
        launch_reset<float>(h->leaf_desc, h->pl.n_leaves, h->aarena, (float *)h->farena, h->kdyn, h->stream);
    h->kernels_launched += 1;
    run_plan(h, h->fp, h->farena, h->flops);
    st = read_error(h);
    h->last_status = st;
    h->factored = st == HLU_OK;
    return st;
}

}  // namespace

extern "C" {

int hlu_solve(hlu_t h, double *b, int32_t nrhs, int64_t ldb) {
    if (!h || nrhs < 0 || ldb < h->pl.n) return HLU_EINVAL;
    if (!h->factored) return HLU_ESTATE;
    if (nrhs == 0) return HLU_OK;
    if (!b) return HLU_EINVAL;
    int st = clear_error(h);
    if (st) return st;
    const int32_t n = h->pl.n, w = h->pl.opt.nrhs_max;
    for (int32_t j0 = 0; j0 < nrhs; j0 += w) {
        const int32_t nc = std::min(w, nrhs - j0);
        double *bj = b + (int64_t)j0 * ldb;
        if (h->precision == HLU_FP64) {
            double *Y = (double *)h->farena + h->pl.f_solve_off;
            launch_permute<double, double>(h->perm, n, nc, bj, ldb, Y, n, 1, h->stream);
            solve_pass(h, nc);
            launch_permute<double, double>(h->perm, n, nc, Y, n, bj, ldb, 0, h->stream);
        } else {
            float *Y = (float *)h->farena + h->pl.f_solve_off;
            launch_permute<double, float>(h->perm, n, nc, bj, ldb, Y, n, 1, h->stream);
            solve_pass(h, nc);
            launch_permute<float, double>(h->perm, n, nc, Y, n, bj, ldb, 0, h->stream);
        }
        h->kernels_launched += 2;
    }
    st = read_error(h);
    h->last_status = st;
    return st;
}

int hlu_matvec(hlu_t h, const double *x, double *y, int32_t nrhs, int64_t ld) {
    if (!h || nrhs < 0 || ld < h->pl.n) return HLU_EINVAL;
    if (nrhs == 0) return HLU_OK;
    if (!x || !y) return HLU_EINVAL;
    int st = clear_error(h);
    if (st) return st;
    const int32_t n = h->pl.n, w = h->pl.opt.nrhs_max;
    double *X = h->aarena + h->pl.a_x_off, *Y = h->aarena + h->pl.a_y_off;
    for (int32_t j0 = 0; j0 < nrhs; j0 += w) {
        const int32_t nc = std::min(w, nrhs - j0);
        launch_permute<double, double>(h->perm, n, nc, x + (int64_t)j0 * ld, ld, X, n, 1, h->stream);
        matvec_pass(h, nc);
        launch_permute<double, double>(h->perm, n, nc, Y, n, y + (int64_t)j0 * ld, ld, 0, h->stream);
        h->kernels_launched += 2;
    }
    st = read_error(h);
    return st;
}

int hlu_solve_refined(hlu_t h, const double *b, double *x, int32_t nrhs, int64_t ld, double tol, int32_t max_iter,
                      int32_t *iters_out, double *resid_out) {
    if (!h || nrhs < 0 || ld < h->pl.n || max_iter < 0 || !(tol >= 0.0)) return HLU_EINVAL;
    if (!h->factored) return HLU_ESTATE;
    if (iters_out) *iters_out = 0;
    if (resid_out) *resid_out = 0.0;
    if (nrhs == 0) return HLU_OK;
    if (!b || !x) return HLU_EINVAL;
    int st = clear_error(h);
    if (st) return st;
    const int64_t n = h->pl.n;
    const int32_t w = h->pl.opt.nrhs_max;
    double *bc = h->ir, *xc = bc + n * w, *rc = xc + n * w, *nrm = rc + n * w;
    double *AX = h->aarena + h->pl.a_x_off, *AY = h->aarena + h->pl.a_y_off;
    int32_t iters_max = 0;
    double res_max = 0.0;
    for (int32_t j0 = 0; j0 < nrhs; j0 += w) {
        const int32_t nc = std::min(w, nrhs - j0);
        const size_t bytes = sizeof(double) * n * nc;
        launch_permute<double, double>(h->perm, (int32_t)n, nc, b + (int64_t)j0 * ld, ld, bc, n, 1, h->stream);
        cudaMemsetAsync(xc, 0, bytes, h->stream);
        cudaMemcpyAsync(rc, bc, bytes, cudaMemcpyDeviceToDevice, h->stream);
        int32_t it = 0;
        double res = 0.0;
        if (max_iter == 0) {
            cudaMemsetAsync(nrm, 0, 2 * w * sizeof(double), h->stream);
            launch_residual(bc, xc, rc, n, nc, nrm, nrm + w, h->stream);  // r = b (x = 0)
            cudaMemcpyAsync(h->ir_host, nrm, 2 * w * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if ((st = read_error(h))) return st;
            res = 1.0;
        }
        while (it < max_iter) {
            if (h->precision == HLU_FP64) {
                double *Y = (double *)h->farena + h->pl.f_solve_off;
                launch_to_work<double>(rc, Y, n, nc, h->stream);
                solve_pass(h, nc);
                launch_add_from_work<double>(xc, Y, n, nc, h->stream);
            } else {
                float *Y = (float *)h->farena + h->pl.f_solve_off;
                launch_to_work<float>(rc, Y, n, nc, h->stream);
                solve_pass(h, nc);
                launch_add_from_work<float>(xc, Y, n, nc, h->stream);
            }
            ++it;
            h->kernels_launched += 3;  // to_work, add_from_work, residual
            cudaMemcpyAsync(AX, xc, bytes, cudaMemcpyDeviceToDevice, h->stream);
            matvec_pass(h, nc);
            cudaMemsetAsync(nrm, 0, 2 * w * sizeof(double), h->stream);
            launch_residual(bc, AY, rc, n, nc, nrm, nrm + w, h->stream);
            cudaMemcpyAsync(h->ir_host, nrm, 2 * w * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if ((st = read_error(h))) {
                h->last_status = st;
                return st;
            }
            res = 0.0;
            for (int32_t j = 0; j < nc; ++j) {
                const double bn = std::sqrt(h->ir_host[w + j]);
                const double rj = bn > 0.0 ? std::sqrt(h->ir_host[j]) / bn : std::sqrt(h->ir_host[j]);
                res = std::max(res, rj);
            }
            if (!std::isfinite(res) || res <= tol) break;
        }
        launch_permute<double, double>(h->perm, (int32_t)n, nc, xc, n, x + (int64_t)j0 * ld, ld, 0, h->stream);
        h->kernels_launched += 2;
        iters_max = std::max(iters_max, it);
        res_max = std::max(res_max, res);
    }
    st = read_error(h);
    h->last_status = st;
    if (iters_out) *iters_out = iters_max;
    if (resid_out) *resid_out = res_max;
    return st;
}

int hlu_solve_gmres(hlu_t h, const double *b, double *x, int32_t nrhs, int64_t ld, double tol, int32_t restart,
                    int32_t max_iter, int32_t *iters_out, double *resid_out) {
    if (!h || nrhs < 0 || ld < h->pl.n || max_iter < 0 || !(tol >= 0.0) || restart < 1 || restart > 256)
        return HLU_EINVAL;
    if (!h->factored) return HLU_ESTATE;
    if (iters_out) *iters_out = 0;
    if (resid_out) *resid_out = 0.0;
    if (nrhs == 0) return HLU_OK;
    if (!b || !x) return HLU_EINVAL;
    int st = clear_error(h);
    if (st) return st;
    const int64_t n = h->pl.n;
    const int32_t w = h->pl.opt.nrhs_max, m = restart;
    if (h->gm_m < m) {  // Krylov bases and the small per-column state, kept for later calls
        const int64_t small = int64_t(w) * ((m + 1) * m + 2 * m + 4 * (m + 1) + 4);
        if ((st = dalloc(h, &h->gm_V, size_t(m + 1) * n * w))) return st;
        if ((st = dalloc(h, &h->gm_Z, size_t(m) * n * w))) return st;
        if ((st = dalloc(h, &h->gm_small, size_t(small)))) return st;
        if (!h->gm_host) h->gm_host = new (std::nothrow) double[2 * w];
        if (!h->gm_host) return HLU_ENOMEM;
        h->gm_m = m;
    }
    const int64_t vs = n * w;  // stride between basis panels
    GmState gs;
    gs.m = m;
    gs.H = h->gm_small;
    gs.cs = gs.H + int64_t(w) * (m + 1) * m;
    gs.sn = gs.cs + int64_t(w) * m;
    gs.g = gs.sn + int64_t(w) * m;
    gs.inv = gs.g + int64_t(w) * (m + 1);
    gs.est = gs.inv + w;
    double *t1 = gs.est + w, *t2 = t1 + int64_t(w) * (m + 1), *nrmd = t2 + int64_t(w) * (m + 1);
    double *bc = h->ir, *xc = bc + n * w, *rc = xc + n * w, *nrm = rc + n * w;
    double *AX = h->aarena + h->pl.a_x_off, *AY = h->aarena + h->pl.a_y_off;
    int32_t it_max = 0;
    double res_max = 0.0;
    for (int32_t j0 = 0; j0 < nrhs; j0 += w) {
        const int32_t nc = std::min(w, nrhs - j0);
        const size_t bytes = sizeof(double) * n * nc;
        launch_permute<double, double>(h->perm, (int32_t)n, nc, b + (int64_t)j0 * ld, ld, bc, n, 1, h->stream);
        cudaMemsetAsync(xc, 0, bytes, h->stream);
        int32_t it = 0;
        double res = 0.0;
        std::vector<double> bn(nc, 0.0);
        for (;;) {
            // true residual r = b - A_H x of the cycle's start
            cudaMemcpyAsync(AX, xc, bytes, cudaMemcpyDeviceToDevice, h->stream);
            matvec_pass(h, nc);
            cudaMemsetAsync(nrm, 0, 2 * w * sizeof(double), h->stream);
            launch_residual(bc, AY, rc, n, nc, nrm, nrm + w, h->stream);
            cudaMemcpyAsync(h->ir_host, nrm, 2 * w * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if ((st = read_error(h))) {
                h->last_status = st;
                return st;
            }
            res = 0.0;
            for (int32_t j = 0; j < nc; ++j) {
                bn[j] = std::sqrt(h->ir_host[w + j]);
                const double rj = bn[j] > 0.0 ? std::sqrt(h->ir_host[j]) / bn[j] : std::sqrt(h->ir_host[j]);
                res = std::max(res, rj);
            }
            if (!std::isfinite(res) || res <= tol || it >= max_iter) break;
            // v_0 = r / |r|, g = |r| e_1
            gm_dots(rc, 0, 1, rc, n, nc, nrmd, 1, h->stream);
            gm_start(nrmd, gs, nc, h->stream);
            gm_scale(rc, gs.inv, h->gm_V, n, nc, h->stream);
            int k = 0;
            for (int j = 0; j < m && it < max_iter; ++j) {
                double *Vj = h->gm_V + j * vs, *Zj = h->gm_Z + j * vs;
                // z_j = U^{-1} L^{-1} v_j (the factors in their precision)
                if (h->precision == HLU_FP64) {
                    double *Y = (double *)h->farena + h->pl.f_solve_off;
                    launch_to_work<double>(Vj, Y, n, nc, h->stream);
                    solve_pass(h, nc);
                    cudaMemsetAsync(Zj, 0, bytes, h->stream);
                    launch_add_from_work<double>(Zj, Y, n, nc, h->stream);
                } else {
                    float *Y = (float *)h->farena + h->pl.f_solve_off;
                    launch_to_work<float>(Vj, Y, n, nc, h->stream);
                    solve_pass(h, nc);
                    cudaMemsetAsync(Zj, 0, bytes, h->stream);
                    launch_add_from_work<float>(Zj, Y, n, nc, h->stream);
                }
                // w = A_H z_j, orthogonalised against v_0 .. v_j (two classical Gram-Schmidt passes)
                cudaMemcpyAsync(AX, Zj, bytes, cudaMemcpyDeviceToDevice, h->stream);
                matvec_pass(h, nc);
                gm_dots(h->gm_V, vs, j + 1, AY, n, nc, t1, m + 1, h->stream);
                gm_axpy(h->gm_V, vs, j + 1, t1, m + 1, -1.0, AY, n, nc, h->stream);
                gm_dots(h->gm_V, vs, j + 1, AY, n, nc, t2, m + 1, h->stream);
                gm_axpy(h->gm_V, vs, j + 1, t2, m + 1, -1.0, AY, n, nc, h->stream);
                gm_dots(AY, 0, 1, AY, n, nc, nrmd, 1, h->stream);
                gm_arnoldi(t1, t2, nrmd, gs, j, nc, h->stream);
                gm_scale(AY, gs.inv, h->gm_V + (j + 1) * vs, n, nc, h->stream);
                h->kernels_launched += 11;
                ++it;
                k = j + 1;
                cudaMemcpyAsync(h->gm_host, gs.est, nc * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
                if ((st = read_error(h))) {
                    h->last_status = st;
                    return st;
                }
                bool done = true;
                for (int32_t c = 0; c < nc; ++c) {
                    const double e = h->gm_host[c];
                    if (!std::isfinite(e)) done = true;
                    else if (e > tol * bn[c]) done = false;
                }
                if (done) break;
            }
            // x += Z y, y = R^{-1} g
            gm_hsolve(gs, k, t1, nc, h->stream);
            gm_axpy(h->gm_Z, vs, k, t1, m + 1, 1.0, xc, n, nc, h->stream);
            h->kernels_launched += 6;
        }
        launch_permute<double, double>(h->perm, (int32_t)n, nc, xc, n, x + (int64_t)j0 * ld, ld, 0, h->stream);
        h->kernels_launched += 2;
        it_max = std::max(it_max, it);
        res_max = std::max(res_max, res);
    }
    st = read_error(h);
    h->last_status = st;
    if (iters_out) *iters_out = it_max;
    if (resid_out) *resid_out = res_max;
    return st;
}

int64_t hlu_factor_doubles(hlu_t h) {
    if (!h) return -1;
    int64_t tot = 0;
    for (int64_t l = 0; l < h->pl.n_leaves; ++l) {
        const Store &s = h->pl.fstore[l];
        tot += s.kind == B_DENSE ? int64_t(s.m) * s.n : int64_t(s.m + s.n) * s.cap;
    }
    return tot;
}

int hlu_get_factors(hlu_t h, int32_t *rank_out, int64_t *offsets_out, double *data_out) {
    if (!h || !rank_out || !offsets_out || !data_out) return HLU_EINVAL;
    if (!h->factored) return HLU_ESTATE;
    Planner &pl = h->pl;
    std::vector<int32_t> kd(pl.n_slots);
    int st = cuda_status(cudaStreamSynchronize(h->stream));
    if (st) return st;
    if ((st = cuda_status(d2h(h, kd.data(), h->kdyn, sizeof(int32_t) * pl.n_slots))))
        return st;
    int64_t leaf_end = 0;
    for (int64_t l = 0; l < pl.n_leaves; ++l) {
        const Store &s = pl.fstore[l];
        leaf_end =
            std::max(leaf_end, s.kind == B_DENSE ? s.D_off + int64_t(s.m) * s.n : s.V_off + int64_t(s.n) * s.cap);
    }
    std::vector<double> buf(leaf_end);
    if (h->precision == HLU_FP64) {
        st = cuda_status(d2h(h, buf.data(), h->farena, sizeof(double) * leaf_end));
    } else {
        std::vector<float> fb(leaf_end);
        st = cuda_status(d2h(h, fb.data(), h->farena, sizeof(float) * leaf_end));
        for (int64_t i = 0; i < leaf_end; ++i) buf[i] = fb[i];
    }
    if (st) return st;
    int64_t pos = 0;
    for (int64_t l = 0; l < pl.n_leaves; ++l) {
        const Store &s = pl.fstore[l];
        offsets_out[l] = pos;
        if (s.kind == B_DENSE) {
            rank_out[l] = 0;
            std::memcpy(data_out + pos, &buf[s.D_off], sizeof(double) * s.m * s.n);
            pos += int64_t(s.m) * s.n;
        } else {
            const int32_t k = kd[s.kslot];
            rank_out[l] = k;
            std::memcpy(data_out + pos, &buf[s.U_off], sizeof(double) * s.m * k);
            pos += int64_t(s.m) * k;
            std::memcpy(data_out + pos, &buf[s.V_off], sizeof(double) * s.n * k);
            pos += int64_t(s.n) * k;
        }
    }
    return HLU_OK;
}

int hlu_get_stats(hlu_t h, hlu_stats *o) {
    if (!h || !o) return HLU_EINVAL;
    std::memset(o, 0, sizeof(*o));
    const Plan &f = h->pl.fplan, &s = h->pl.splan;
    o->n_tasks = f.n_tasks;
    o->n_waves = f.n_waves;
    o->n_launches = (int64_t)f.launches.size() + 1;
    o->solve_tasks = s.n_tasks;
    o->solve_waves = s.n_waves;
    o->solve_launches = (int64_t)s.launches.size() + 3;
    o->device_bytes = h->device_bytes;
    for (int k = 0; k < K_NKINDS; ++k) o->tasks_by_kind[k] = f.kind_count[k];
    o->max_stacked = f.max_kcap;
    o->kernels_launched = h->kernels_launched;
    o->create_ms[0] = h->create_ms[0];
    o->create_ms[1] = h->create_ms[1];
    for (int k = 0; k < kProfSlots; ++k) {
        o->kernel_ms[k] = h->prof_ms[k];
        o->kernel_launches[k] = h->prof_count[k];
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HLU_ECUDA;
    double fl[16];
    if (d2h(h, fl, h->flops, sizeof(fl)) != cudaSuccess) return HLU_ECUDA;
    for (int k = 0; k < 8; ++k) {
        o->flops_by_kind[k] = fl[k];
        o->model_flops += fl[k];
        o->solve_flops += fl[8 + k];
    }
    unsigned long long bz[kBusyWords];
    if (d2h(h, bz, h->busy, sizeof(bz)) != cudaSuccess) return HLU_ECUDA;
    for (int k = 0; k < 8; ++k) {
        o->task_busy_ms[k] = bz[k] * 1e-6;
        o->task_count[k] = (int64_t)bz[8 + k];
        o->radd_busy_ms[k] = bz[16 + k] * 1e-6;
        o->radd_count[k] = (int64_t)bz[24 + k];
        o->solve_busy_ms[k] = bz[48 + k] * 1e-6;
        o->solve_task_count[k] = (int64_t)bz[56 + k];
    }
    for (int k = 0; k < 16; ++k) {
        const int s = k & 7;
        o->radd_phase[k] = (s == 4 || s >= 6) ? (double)bz[32 + k] : bz[32 + k] * 1e-6;
    }
    if (h->factored) {
        std::vector<int32_t> kd(h->pl.n_slots);
        if (d2h(h, kd.data(), h->kdyn, sizeof(int32_t) * h->pl.n_slots) == cudaSuccess)
            for (int64_t l = 0; l < h->pl.n_leaves; ++l)
                if (h->pl.fstore[l].kslot >= 0) {
                    const int32_t k = kd[h->pl.fstore[l].kslot];
                    o->max_rank = std::max(o->max_rank, k);
                    o->rank_hist[std::min(std::max(k, 0), 33)] += 1;
                }
    }
    return HLU_OK;
}

int hlu_factor_error(hlu_t h, const double *x0, int32_t iters, double rtol, double *efac, double *norm_a) {
    if (!h || !x0 || !efac || iters < 1 || !(rtol >= 0.0)) return HLU_EINVAL;
    if (!h->factored) return HLU_ESTATE;
    Planner &pl = h->pl;
    const int64_t n = pl.n;
    int st = HLU_OK;
    if (!h->err_leaves) {
        std::vector<ErrLeaf> lv(pl.n_leaves);
        for (int64_t l = 0; l < pl.n_leaves; ++l) {
            const Store &a = pl.astore[l], &f = pl.fstore[l];
            ErrLeaf &e = lv[l];
            e.r0 = pl.cl[a.t].begin;
            e.c0 = pl.cl[a.s].begin;
            e.m = a.m;
            e.n = a.n;
            e.kind = a.kind == B_DENSE ? 0 : 1;
            e.a_off = a.kind == B_DENSE ? a.D_off : a.U_off;
            e.a_voff = a.kind == B_DENSE ? 0 : a.V_off;
            e.ak = a.kind == B_DENSE ? 0 : a.krank;
            e.f_off = f.kind == B_DENSE ? f.D_off : f.U_off;
            e.f_voff = f.kind == B_DENSE ? 0 : f.V_off;
            e.kslot = f.kind == B_DENSE ? -1 : f.kslot;
            e.side = e.r0 == e.c0 ? 0 : e.r0 < e.c0 ? 1 : 2;
        }
        if ((st = upload(h, &h->err_leaves, lv))) return st;
        if ((st = dalloc(h, &h->err_work, 6 * n + 1))) return st;
        if (!(h->err_host = new (std::nothrow) double[1])) return HLU_ENOMEM;
    }
    ErrEstimator e;
    e.n = n;
    e.n_leaves = pl.n_leaves;
    e.leaves = h->err_leaves;
    e.aarena = h->aarena;
    e.farena = h->farena;
    e.kdyn = h->kdyn;
    e.fp64 = h->precision == HLU_FP64;
    e.stream = h->stream;
    e.x0c = h->err_work;
    e.x = e.x0c + n;
    e.z = e.x + n;
    e.w1 = e.z + n;
    e.w2 = e.w1 + n;
    e.w3 = e.w2 + n;
    e.dacc = e.w3 + n;
    e.host_acc = h->err_host;
    st = e.run(x0, h->perm, iters, rtol, efac, norm_a);
    h->kernels_launched += e.launched;
    if (st == HLU_OK) st = read_error(h);
    return st;
}

int hlu_set_launch(hlu_t h, int32_t workers, int32_t flags) {
    if (!h || workers < 0) return HLU_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HLU_ECUDA;
    for (DevPlan *d : {&h->fp, &h->sp, &h->mp})
        d->workers = workers > 0 ? std::min(workers, d->workers_alloc) : d->workers_alloc;
    h->tensor = (flags & HLU_FLAG_TENSOR) != 0;
    return HLU_OK;
}

int hlu_get_launch(hlu_t h, int32_t *workers, int32_t *flags) {
    if (!h) return HLU_EINVAL;
    if (workers) *workers = h->fp.workers;
    if (flags) *flags = h->tensor ? HLU_FLAG_TENSOR : 0;
    return HLU_OK;
}

int hlu_inject_stall(hlu_t h, int32_t on) {
    if (!h) return HLU_EINVAL;
    h->inject_stall = on != 0;
    return HLU_OK;
}

int hlu_set_profiling(hlu_t h, int32_t on) {
    if (!h) return HLU_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HLU_ECUDA;
    collect_profile(h);
    h->profiling = on != 0;
    for (int k = 0; k < kProfSlots; ++k) {
        h->prof_ms[k] = 0.0;
        h->prof_count[k] = 0;
    }
    if (cudaMemsetAsync(h->busy, 0, kBusyWords * sizeof(unsigned long long), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return HLU_ECUDA;
    return HLU_OK;
}

void hlu_destroy(hlu_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    collect_profile(h);
    for (cudaEvent_t e : h->free_events) cudaEventDestroy(e);
    for (void *p : h->allocs)
        if (cudaFreeAsync(p, h->stream) != cudaSuccess) {  // e.g. the caller's stream is gone already
            cudaGetLastError();
            cudaFree(p);
        }
    cudaStreamSynchronize(h->stream);  // the memory is back in the pool (and released) on return
    cudaGetLastError();
    delete[] h->ir_host;
    delete[] h->gm_host;
    delete[] h->err_host;
    delete h;
}

const char *hlu_last_cuda_error(hlu_t h) {
    if (!h || h->last_cuda == cudaSuccess) return "no CUDA error";
    return cudaGetErrorString(h->last_cuda);
}

int hlu_last_error_detail(hlu_t h, int64_t *index, double *value) {
    if (!h) return HLU_EINVAL;
    if (index) *index = h->last_err[1];
    if (value) {
        double v;
        std::memcpy(&v, &h->last_err[2], sizeof(v));
        *value = v;
    }
    return h->last_status;
}

}  // extern "C"
