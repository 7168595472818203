// Device estimate of the factorisation error ||A_H - L U||_2 / ||A_H||_2 (power iteration).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hlu {

// One leaf of the block structure as the estimator applies it: its row and column ranges, its
// storage in the A_H arena (FP64, static rank ak) and in the factor arena (rank in kdyn[kslot]),
// and its side of the diagonal (0 diagonal, 1 above: part of U, 2 below: part of L).
struct ErrLeaf {
    int64_t a_off, a_voff, f_off, f_voff;
    int32_t r0, c0, m, n;
    int32_t kind, ak, kslot, side;
};

struct ErrEstimator {
    int64_t n = 0, n_leaves = 0;
    const ErrLeaf *leaves = nullptr;
    const double *aarena = nullptr;
    const void *farena = nullptr;
    const int32_t *kdyn = nullptr;
    bool fp64 = true;
    cudaStream_t stream = nullptr;
    double *x0c = nullptr, *x = nullptr, *z = nullptr, *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;
    double *dacc = nullptr, *host_acc = nullptr;
    int64_t launched = 0;

    int apply(int which, int trans, const double *x, double *y);
    int normal_apply(bool with_factors, const double *x, double *z);
    int power(bool with_factors, const double *x0, int iters, double rtol, double *out);
    // x0_orig: start vector in the original order (device); perm: cluster position -> original index
    int run(const double *x0_orig, const int32_t *perm, int iters, double rtol, double *efac, double *norm_a);
};

}  // namespace hlu
