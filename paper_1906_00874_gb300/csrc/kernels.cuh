// Device kernels of the H-LU task graph (sm_103a).  One CTA executes one task.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tasks.h"

namespace hlu {

constexpr int kThreads = 256;
constexpr int kLeafDesc = 9;  // int64 fields per leaf of the reset descriptor

struct LaunchArgs {
    void *arena;        // T* factor arena (or double* A_H arena)
    int32_t *kdyn;      // dynamic dimensions
    long long *err;     // error word: code, index, value bits, count
    double eps;         // truncation tolerance (rounded addition)
    const double *eps_inst;  // per instance of a batch (device array), else null: eps for all
    double *flops;      // model flops per task kind (K_NKINDS doubles), accumulated
    unsigned long long *phase;  // when profiling: rounded-addition phase counters (16), else null
    int32_t kmax;       // largest stacked rank the core buffers hold
    int32_t core64;     // single-precision factors: SVD of each truncation core in double (1) or single (0)
};

template <class T>
void launch_kind(int kind, const void *tasks, const Term *terms, const Piece *pieces, int start,
                 int count, int kcap, const LaunchArgs &a, cudaStream_t s);

// Opt the task kernels of precision T into the device's largest dynamic shared memory.
template <class T>
bool set_kernel_attributes();

// Persistent data-flow execution of a whole plan (one launch).
struct FlowArgs {
    const int32_t *code;       // per task: (kind << kCodeShift) | index in the kind's array
    const int32_t *succ_ptr;   // successors, CSR
    const int32_t *succ_idx;
    int32_t *indeg;            // working in-degrees (reset before every launch)
    int32_t *queue;            // n_tasks slots, -1 = empty
    int32_t *counters;         // [0] head (next slot to claim), [1] tail (next slot to fill),
                               // [2] completed sinks (tasks without successors)
    int32_t n_tasks;
    int32_t n_sinks;           // every task is done once every sink is (each precedes a sink)
    int32_t kc;                // core capacity of rounded additions (shared memory)
    const TGetrf *getrf;
    const TTrsm *trsm;
    const TProject *project;
    const TAccum *accum;
    const TRadd *radd;
    const TSplit *split;
    const Term *terms;
    const Piece *pieces;
    size_t smem_bytes;         // dynamic shared memory of a worker
    void *core_scratch;        // per-worker global space for rounded-addition cores too big for smem
    int64_t core_stride;       // bytes per worker
    void *scratch;             // per-worker rounded-addition workspace (T elements)
    int64_t scratch_stride;    // elements per worker
    unsigned long long timeout_ns;  // limit of any single wait for a ready task
    int32_t tensor;            // single precision: dense products of ACCUM tasks on the tensor cores
    int32_t tc_min_inner;      // smallest packed inner size a product takes to the tensor cores
    unsigned long long *busy;  // when profiling: [kind] task nanoseconds, [8 + kind] task count,
                               // [16 + b] / [24 + b] the same for rounded additions of size class b; else null
};

size_t dataflow_smem_bytes(int max_leaf, int elem, int kc, bool core64);
template <class T>
int dataflow_workers(size_t smem);
template <class T>
void launch_dataflow(const FlowArgs &f, const LaunchArgs &a, int grid, size_t smem, cudaStream_t s);

// Restore the factor arena from the original matrix (the factorisation works in place).
template <class T>
void launch_reset(const int64_t *leaf_desc, int64_t n_leaves, const double *aarena, T *farena,
                  int32_t *kdyn, cudaStream_t s);

// y[p + j*ld_y] = x[perm[p] + j*ld_x] (gather, to_cluster = 1) or the inverse scatter.
template <class Tin, class Tout>
void launch_permute(const int32_t *perm, int32_t n, int32_t nrhs, const Tin *x, int64_t ldx, Tout *y,
                    int64_t ldy, int to_cluster, cudaStream_t s);

void launch_set_slot(int32_t *kdyn, int32_t slot, int32_t value, cudaStream_t s);

// Iterative-refinement helpers (cluster order, n x nc panels with leading dimension n):
// y (T) = x (double);  x (double) += y (T);  r = b - ax and nrm2[j] += |r_j|^2, bn2[j] += |b_j|^2.
template <class T>
void launch_to_work(const double *x, T *y, int64_t n, int32_t nc, cudaStream_t s);
template <class T>
void launch_add_from_work(double *x, const T *y, int64_t n, int32_t nc, cudaStream_t s);
void launch_residual(const double *b, const double *ax, double *r, int64_t n, int32_t nc, double *nrm2,
                     double *bn2, cudaStream_t s);

// Shared memory of a rounded addition whose stacked rank is at most kcap, with
// factors of elem bytes (also the dense route's worst case); core64: single-precision
// factors whose truncation cores take their SVD in double.
size_t radd_smem_bytes(int kcap, int elem, bool core64);
size_t getrf_smem_bytes(int max_leaf, int elem);

}  // namespace hlu
