// Launchers of the GMRES(m) kernels (gmres.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hlu {

// Small per-column state of a GMRES cycle (device arrays, ncol columns):
// H: (m + 1) x m Hessenberg per column (column major, ld m + 1), cs / sn: m Givens rotations,
// g: m + 1 rotated right-hand side, inv: scale of the next basis vector, est: residual estimate.
struct GmState {
    int m;
    double *H, *cs, *sn, *g, *inv, *est;
};

void gm_dots(const double *X, int64_t xs, int k, const double *Y, int64_t n, int ncol, double *out, int ld,
             cudaStream_t st);
void gm_axpy(const double *X, int64_t xs, int k, const double *h, int ld, double alpha, double *Y, int64_t n,
             int ncol, cudaStream_t st);
void gm_scale(const double *X, const double *f, double *Y, int64_t n, int ncol, cudaStream_t st);
void gm_start(const double *nrm2, const GmState &s, int ncol, cudaStream_t st);
void gm_arnoldi(const double *t1, const double *t2, const double *nrm2, const GmState &s, int j, int ncol,
                cudaStream_t st);
void gm_hsolve(const GmState &s, int k, double *y, int ncol, cudaStream_t st);

}  // namespace hlu
