// Device kernels of the H-LU task graph (sm_103a).  One CTA executes one task.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tasks.h"

namespace hlu {

constexpr int kThreads = 256;

struct LaunchArgs {
    void *arena;        // T* factor arena (or double* A_H arena)
    int32_t *kdyn;      // dynamic dimensions
    long long *err;     // error word: code, index, value bits, count
    double eps;         // truncation tolerance (rounded addition)
    int32_t kmax;       // largest stacked rank the core buffers hold
};

template <class T>
void launch_kind(int kind, const void *tasks, const Term *terms, const Piece *pieces, int start,
                 int count, int kcap, const LaunchArgs &a, cudaStream_t s);

// Restore the factor arena from the original matrix (the factorisation works in place).
template <class T>
void launch_reset(const int64_t *leaf_desc, int64_t n_leaves, const double *aarena, T *farena,
                  int32_t *kdyn, cudaStream_t s);

// y[p + j*ld_y] = x[perm[p] + j*ld_x] (gather, to_cluster = 1) or the inverse scatter.
template <class Tin, class Tout>
void launch_permute(const int32_t *perm, int32_t n, int32_t nrhs, const Tin *x, int64_t ldx, Tout *y,
                    int64_t ldy, int to_cluster, cudaStream_t s);

void launch_set_slot(int32_t *kdyn, int32_t slot, int32_t value, cudaStream_t s);

size_t radd_smem_bytes(int kcap);
size_t getrf_smem_bytes(int max_leaf, int elem);

}  // namespace hlu
