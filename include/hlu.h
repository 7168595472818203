/*
 * hlu.h - LU factorisation of hierarchical matrices (H-LU) on one GB300 GPU.
 *
 * The operation is the H-LU of Sec. 3.1 of "Exploiting Nested Task-Parallelism
 * in the H-LU Factorization": the 2 x 2 block recursion (LU of the leading
 * diagonal block, triangular solves of the off-diagonal blocks, Schur update,
 * LU of the trailing block) applied at every partitioned diagonal block, with
 * low-rank blocks X = U V^T handled in H-arithmetic (triangular solves on one
 * factor only, factorised products, rounded addition by SVD truncation).  The
 * matrix is described by a cluster tree (Algorithm 1) and the leaves of a
 * block tree (Algorithm 2), as in the `cluster` and `hmatrix` records of Sec. 2.
 *
 * All entry points return an int status (HLU_OK = 0).  No C++ exception and no
 * device trap crosses this interface: device kernels record failures in an
 * error word that the host reads after each call.  All device work of a handle
 * is ordered on the CUDA stream given at creation.  Matrix rows and columns are
 * numbered in cluster order internally; vectors passed to hlu_solve and
 * hlu_matvec are in the ORIGINAL degree-of-freedom order.
 */
#ifndef HLU_H
#define HLU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
enum {
    HLU_OK = 0,
    HLU_EINVAL = 1,    /* malformed tree, leaves not tiling [0,n)^2, low-rank diagonal
                          block, rank > min(m,n), leaf cluster above 128 indices,
                          non-finite input, bad argument */
    HLU_ENOMEM = 2,    /* cudaMalloc failed or the plan exceeds opts.mem_budget */
    HLU_ESTATE = 3,    /* call out of order (a solve or an estimate before hlu_factor) */
    HLU_EPIVOT = 4,    /* zero or non-finite pivot u_kk in a dense diagonal leaf */
    HLU_ERANKCAP = 5,  /* a truncated rank or a stacked rank exceeded its capacity */
    HLU_ETIMEOUT = 6,  /* a device-side wait exceeded its limit */
    HLU_ECUDA = 7,     /* a CUDA runtime call failed */
    HLU_ENUMERIC = 8   /* a non-finite value appeared during the factorisation */
};

/* ------------------------------------------------------------- precision */
enum {
    HLU_FP64 = 0,        /* factors stored and computed in FP64 */
    HLU_FP32 = 1,        /* factors stored and computed in FP32, except the SVD of every
                            truncation core (the one-sided Jacobi of the rounded addition,
                            Sec. 3.1, and the right factor formed from it), which runs in FP64
                            on the FP32 data; the original matrix, hlu_matvec and the
                            refinement stay FP64 */
    HLU_FP32_CORE32 = 2  /* as HLU_FP32, but the truncation cores' Jacobi SVD runs in FP32
                            with the rotations accumulated (faster, singular values to FP32
                            accuracy) */
};

/* Cluster tree (Sec. 2, Algorithm 1), host pointers, clusters numbered so that
 * every cluster's degrees of freedom are the contiguous range
 * [begin[c], begin[c]+size[c]) of the cluster order; cluster 0 is the root.
 * son0/son1 are -1 for a leaf cluster, otherwise the two sons with
 * begin[son0] = begin[c] and begin[son1] = begin[c] + size[son0].
 * perm[p] is the original index of the degree of freedom at cluster position p. */
typedef struct {
    int32_t n;
    int32_t n_clusters;
    const int32_t *perm;
    const int32_t *begin;
    const int32_t *size;
    const int32_t *son0;
    const int32_t *son1;
} hlu_tree;

/* Leaves of the block tree (Sec. 2, Algorithm 2), host pointers.
 * Leaf l covers rows of cluster row_cl[l] and columns of cluster col_cl[l].
 * kind 0 = dense: data[offset[l] ...] holds the m x n block column-major.
 * kind 1 = low rank X = U V^T (Sec. 3.1): data[offset[l] ...] holds U (m x k,
 *          column-major) followed by V (n x k, column-major), k = rank[l].
 * The leaves must tile the matrix exactly, diagonal blocks may not be low rank,
 * 0 <= rank <= min(m, n), and a dense leaf must have a leaf cluster on at least
 * one side (Algorithm 2 partitions a block whose clusters both have sons unless
 * it is stored in low-rank form). */
typedef struct {
    int64_t n_leaves;
    const int32_t *row_cl;
    const int32_t *col_cl;
    const int8_t *kind;
    const int32_t *rank;
    const int64_t *offset;
    const double *data;
    int64_t data_len;    /* number of doubles in data (every leaf must lie inside) */
} hlu_blocks;

/* ------------------------------------------------------------ schedule */
enum {
    HLU_SCHED_DATAFLOW = 0, /* one persistent launch executes the task graph: a task
                               starts as soon as its own predecessors are done */
    HLU_SCHED_WAVES = 1     /* one launch per dependency level and task kind */
};

typedef struct {
    int32_t precision;   /* HLU_FP64, HLU_FP32 or HLU_FP32_CORE32 */
    int32_t rank_cap;    /* capacity of every low-rank block: min(m, n, rank_cap); 0 -> 32 */
    int32_t nrhs_max;    /* widest right-hand-side panel one solve pass takes; 0 -> 64 */
    int32_t schedule;    /* HLU_SCHED_DATAFLOW (default) or HLU_SCHED_WAVES */
    int64_t mem_budget;  /* bytes of device memory the handle may allocate; 0 -> no limit */
    double timeout_s;    /* limit for any device-side wait; 0 -> 10 s.  On expiry the
                            call returns HLU_ETIMEOUT and the device is left usable */
    int32_t inv_block;   /* solve by inverse blocks: the largest diagonal blocks of order
                            <= inv_block (at least the largest leaf) are inverted at the end
                            of hlu_factor, and the solve applies those inverses as dense
                            products above the block substitution of Sec. 3.1 (fewer
                            sequential steps); 0 -> 1024, < 0 -> plain block substitution.
                            The inverses are not counted in the model flops */
    int32_t flags;       /* HLU_FLAG_* bits; 0 for the defaults */
    int32_t workers;     /* most worker CTAs of one data-flow launch of this handle; 0 -> as many
                            as are resident on the GPU at once (two per SM).  A smaller number
                            leaves room for the launches of other handles on other streams to
                            run at the same time (the serving loop gives each group half) */
    int32_t temp_reuse;  /* > 0: the factorisation's product temporaries of one shape (and one
                            problem of a batch) share device regions when their dependency-level
                            intervals do not overlap (tasks of the earlier use precede writers of
                            the later one, cell by cell; the graph keeps its levels).  About half
                            the device memory at n = 20480, for a few percent of factorisation
                            time and a longer planning.  0 (default): every temporary its own region */
} hlu_opts;

/* hlu_opts.flags */
enum {
    /* FP32 factors: compute the dense products of the factorisation (product tasks with >= 32
       rows, >= 16 columns and >= 32 inner columns, data-flow schedule) on the tensor cores
       (tcgen05, three TF32 products per FP32 product, FP32 accumulation in tensor memory) instead
       of CUDA cores.  Off by default: these leaf-sized products (a 64-row leaf cluster, tens of
       inner columns) ran slower on the tensor cores than on CUDA cores in every measured workload */
    HLU_FLAG_TENSOR = 1,
    HLU_FLAG_SERIAL_PLAN = 2  /* plan on one host thread.  hlu_create_batch / hlu_plan_info_batch
                                 with the data-flow schedule: plan the whole batch as one H-matrix.
                                 By default the problems are planned separately on all host threads
                                 and their task graphs joined (the same tasks and dependencies; each
                                 problem keeps its own unused copy of the n x nrhs_max work panels
                                 in the arenas).  hlu_create / hlu_plan_info_get: by default the
                                 dependency analysis of the factorisation runs on a second host
                                 thread beside the expansion of the recursion (the same graph) */
};

typedef struct hlu_ctx *hlu_t;

/* Build the handle: validates and copies the caller's host arrays (they may be
 * freed after the call), plans the task graph of the factorisation and of the
 * solve, and uploads the original matrix A_H (kept in FP64 for hlu_matvec) and
 * the working copy that hlu_factor overwrites.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  On failure *out is NULL. */
int hlu_create(const hlu_tree *tree, const hlu_blocks *blocks, const hlu_opts *opts,
               void *cuda_stream, hlu_t *out);

/* H-LU in place (Sec. 3.1), truncating at relative tolerance eps
 * (singular values sigma_i <= eps * sigma_1 of each rounded addition are dropped).
 * Every call first restores the working copy from A_H on the device, so the
 * handle can be factorised again (e.g. with another eps).  Synchronises the
 * stream and returns the device error status (HLU_EPIVOT, HLU_ERANKCAP,
 * HLU_ENUMERIC with details from hlu_last_error_detail). */
int hlu_factor(hlu_t h, double eps);

/* Batched H-LU: `count` independent problems in one handle.  trees[i] and
 * blocks[i] describe problem i exactly as for hlu_create (indices local to the
 * problem, host pointers).  The handle holds the block-diagonal matrix
 * diag(A_0, ..., A_{count-1}) of order sum n_i: a balanced binary tree of
 * count - 1 clusters joins the problems' roots, and blocks that couple two
 * problems are structurally zero (no leaves, no tasks, no dependencies), so
 * the factorisation and the solve of all problems run in the same launches and
 * no task of one problem waits on another.  Rows and right-hand-side rows of
 * problem i follow those of problems 0..i-1 (offsets sum_{j<i} n_j); every
 * other call (hlu_factor, hlu_solve, hlu_solve_refined, hlu_solve_gmres,
 * hlu_matvec, hlu_get_factors) sees the stacked system of that order.
 * With the data-flow schedule the problems are planned on all host threads,
 * one problem per planner, and their task graphs joined (the same tasks and
 * dependencies as one plan of the whole matrix; HLU_FLAG_SERIAL_PLAN plans it
 * as one on one thread).  The handle keeps no host copy of the task graphs
 * after they are uploaded.  count >= 1; on failure *out is NULL. */
int hlu_create_batch(int32_t count, const hlu_tree *trees, const hlu_blocks *blocks,
                     const hlu_opts *opts, void *cuda_stream, hlu_t *out);

/* hlu_factor with a tolerance per problem: eps[i] (host array of
 * hlu_batch_count(h) values, each finite and >= 0) truncates the rounded
 * additions of problem i.  On a handle from hlu_create it takes eps[0]. */
int hlu_factor_batch(hlu_t h, const double *eps);

/* Number of problems in the handle: count of hlu_create_batch, 1 for
 * hlu_create, 0 for a NULL handle. */
int hlu_batch_count(hlu_t h);

/* ------------------------------------------------ plan without a device */
/* Validation and planning only (host, no CUDA call): the sizes of the task
 * graphs hlu_create would build for these inputs and options. */
typedef struct {
    int64_t factor_tasks;    /* tasks of the factorisation graph */
    int64_t factor_edges;    /* dependencies between them */
    int64_t factor_levels;   /* longest dependency chain (tasks) */
    int64_t solve_tasks;     /* tasks of one solve pass (forward and backward) */
    int64_t solve_levels;
    int64_t matvec_tasks;
    int64_t inverse_blocks;  /* diagonal blocks inverted for the solve (hlu_opts.inv_block) */
    int64_t factor_elems;    /* elements of the factor arena */
    double plan_ms;          /* host time of the planning */
    double factor_critical_us;  /* longest dependency path of the factorisation and of one solve
                                   pass under fixed per-kind task latencies (model, microseconds;
                                   the same weights order the executor's ready tasks) */
    double solve_critical_us;
    int64_t factor_temp_elems;       /* elements of the factorisation's product temporaries */
    int64_t factor_temp_peak_elems;  /* largest sum of them in use at one dependency level */
} hlu_plan_info;

int hlu_plan_info_get(const hlu_tree *tree, const hlu_blocks *blocks, const hlu_opts *opts, hlu_plan_info *out);

/* The same for the batch of hlu_create_batch. */
int hlu_plan_info_batch(int32_t count, const hlu_tree *trees, const hlu_blocks *blocks, const hlu_opts *opts,
                        hlu_plan_info *out);

/* ------------------------------------------------ construction on the GPU */
/* Inputs of hlu_bem_build (host pointers): the Laplace kernel of Sec. 6.1 in
 * dimension dim (3: 1/(4 pi r); 2: -log(r)/(2 pi); 1: -log r), in collocation
 * form with one element per degree of freedom: centroid (n x 3, row major,
 * original order; unused coordinates 0) and size (area or length, n values).
 * The cluster tree and the leaves of the block tree (row_cl, col_cl, kind:
 * 0 dense, 1 low rank) are as for hlu_create; the data are computed here.
 * Low-rank leaves: adaptive cross approximation with partial pivoting to the
 * relative tolerance eps, at most aca_cap cross vectors (0 -> 48, at most 64),
 * then truncated at eps by the rounded addition (Sec. 3.1). */
typedef struct {
    int32_t dim;
    const double *centroid;
    const double *size;
    const hlu_tree *tree;
    int64_t n_leaves;
    const int32_t *row_cl;
    const int32_t *col_cl;
    const int8_t *kind;
    double eps;
    int32_t aca_cap;
    int32_t reserved_;   /* set to 0 */
} hlu_bem_input;

typedef struct hlu_bem *hlu_bem_t;

/* Build the leaf data on the device (stream order, synchronised on return).
 * HLU_ERANKCAP when a cross approximation does not reach eps within aca_cap
 * vectors (the block should be stored dense or partitioned).  On failure *out
 * is NULL. */
int hlu_bem_build(const hlu_bem_input *in, void *cuda_stream, hlu_bem_t *out);

/* The result in the layout of hlu_blocks: rank and offset (host arrays of
 * n_leaves, copied out when non-NULL), the total number of doubles, and the
 * DEVICE pointer to the data (owned by the builder). */
int hlu_bem_result(hlu_bem_t b, int32_t *rank, int64_t *offset, int64_t *data_len, const double **data_dev);

/* Copy the data to host memory (data_len doubles). */
int hlu_bem_copy_data(hlu_bem_t b, double *host);

/* hlu_create on the builder's matrix (its tree, leaves and data). */
int hlu_create_bem(hlu_bem_t b, const hlu_opts *opts, void *cuda_stream, hlu_t *out);

void hlu_bem_destroy(hlu_bem_t b);

/* Solve A x = b with the factors: forward substitution with the unit lower
 * factor, then backward substitution with the upper factor (Sec. 3.1).
 * b is a DEVICE pointer to n x nrhs FP64 values, column-major with leading
 * dimension ldb >= n, in original order; it is overwritten by x. */
int hlu_solve(hlu_t h, double *b_dev, int32_t nrhs, int64_t ldb);

/* y = A_H x with the original (unfactored) H-matrix in FP64 (Sec. 3.1,
 * y = U (V^T x) on low-rank leaves).  x, y: DEVICE pointers, n x nrhs,
 * column-major, leading dimension ld >= n, original order, must not overlap. */
int hlu_matvec(hlu_t h, const double *x_dev, double *y_dev, int32_t nrhs, int64_t ld);

/* Copy the factors back to the host in the input leaf layout: for each leaf,
 * dense leaves as m x n column-major (diagonal leaves hold L below and U on and
 * above the diagonal), low-rank leaves as U then V with rank_out[l] columns.
 * `data_out` must hold hlu_factor_doubles(h) values; offsets_out[l] receives the
 * position of leaf l.  Low-rank factors of L blocks are those of L itself. */
int64_t hlu_factor_doubles(hlu_t h);
int hlu_get_factors(hlu_t h, int32_t *rank_out, int64_t *offsets_out, double *data_out);

/* Iterative refinement (the solve of the mixed-precision form): starting from
 * x = 0, repeat d = U^{-1} L^{-1} r (the factors, in their precision), x += d and
 * r = b - A_H x with the original H-matrix in FP64, until every column meets
 * ||r_j||_2 <= tol ||b_j||_2 or max_iter solves were applied.  b and x are
 * DEVICE pointers to n x nrhs FP64 panels (column-major, leading dimension
 * ld >= n, original order, not overlapping).  *iters_out (may be NULL) gets the
 * number of solves applied (largest over column chunks), *resid_out (may be
 * NULL) the largest relative residual reached.  Returns HLU_OK even when tol is
 * not reached within max_iter; the caller reads *resid_out. */
int hlu_solve_refined(hlu_t h, const double *b_dev, double *x_dev, int32_t nrhs, int64_t ld, double tol,
                      int32_t max_iter, int32_t *iters_out, double *resid_out);

/* Restarted GMRES(m) (Saad and Schultz 1986) in FP64 on A_H x = b with the
 * original H-matrix, right-preconditioned by the factorisation: the Krylov
 * space is built from A_H U^{-1} L^{-1} (the factors in their precision, the
 * solve of Sec. 3.1), orthogonalised by two classical Gram-Schmidt passes, and
 * x = U^{-1} L^{-1} V y with y from the Givens-reduced Hessenberg system.  All
 * columns advance in lockstep from x = 0; a cycle stops after `restart` steps
 * or when every column's residual estimate meets tol ||b_j||_2; each cycle
 * starts from the true FP64 residual.  The preconditioning in the mixed form
 * is the paper's factorisation used for the "GMRES" configuration of the
 * mixed-precision variant (no counterpart in the paper itself, which solves
 * directly).  b and x are DEVICE pointers to n x nrhs FP64 panels (column-major,
 * leading dimension ld >= n, original order, not overlapping); 1 <= restart <= 256.
 * *iters_out (may be NULL) gets the number of Arnoldi steps (one solve and one
 * H-matvec each; largest over column chunks), *resid_out (may be NULL) the largest
 * true relative residual at the end.  The first call allocates the Krylov bases,
 * 2 (restart + 1) n nrhs_max doubles (HLU_ENOMEM beyond opts.mem_budget).
 * Returns HLU_OK even when tol is not reached within max_iter steps. */
int hlu_solve_gmres(hlu_t h, const double *b_dev, double *x_dev, int32_t nrhs, int64_t ld, double tol,
                    int32_t restart, int32_t max_iter, int32_t *iters_out, double *resid_out);

/* Statistics of the plan and of the last calls.  Model flops use the standard
 * operation counts (getrf 2m^3/3, trsm m^2 p, gemm 2mkp, Householder QR
 * 2 a b^2 - 2 b^3/3, Jacobi SVD 21 K^3, Q times a panel 2mKk'), counted on the
 * device from the actual (run-time) ranks. */
typedef struct {
    int64_t n_tasks;          /* tasks of the factorisation plan */
    int64_t n_waves;          /* dependency waves of the factorisation plan */
    int64_t n_launches;       /* kernel launches of one hlu_factor */
    int64_t solve_tasks, solve_waves, solve_launches;
    int64_t device_bytes;     /* device memory held by the handle */
    int64_t tasks_by_kind[8]; /* getrf, trsm, project, accum, radd, split, -, - */
    double model_flops;       /* model flops of the last hlu_factor */
    double flops_by_kind[8];  /* the same, per task kind */
    double solve_flops;       /* model flops of solves and products since the last hlu_factor */
    double kernel_ms[10];     /* with profiling on: summed kernel time per task kind; slots 6 / 7 / 8
                                 hold the data-flow launches of factorisations / of solves / of
                                 H-matrix products */
    int64_t kernel_launches[10];
    double task_busy_ms[8];   /* with profiling on, data-flow factorisations: summed time of the
                                 tasks of each kind (concurrent tasks add up); [6]: summed time the
                                 workers waited for their tensor-memory allocation */
    int64_t task_count[8];    /* the same, task counts; [7]: workers that ran at least one task,
                                 summed over the profiled factorisations */
    double radd_busy_ms[8];   /* the same for rounded additions by target size m + n:
                                 < 128, < 256, < 512, ..., >= 8192 */
    int64_t radd_count[8];
    double solve_busy_ms[8];  /* with profiling on, data-flow solves: summed task time per kind */
    int64_t solve_task_count[8];
    double radd_phase[16];    /* rounded additions, summed ms per phase; [0, 8) dense route
                                 (small targets), [8, 16) stacked route: [0] sum formation or
                                 stacking, [1] QR of the stacks and core product (dense route:
                                 the QR of R'^T of the core), [2] pivoted QR of the core, [3]
                                 Jacobi SVD and truncation (stacked route: with the QR of R'^T), [5] new
                                 factors; counts: [4] Jacobi sweeps, [6] Jacobi sizes r,
                                 [7] tasks */
    int64_t kernels_launched; /* kernels this handle launched since it was created */
    int32_t max_rank;         /* largest rank after the factorisation */
    int32_t max_stacked;      /* largest stacked-rank capacity of a rounded addition */
    int64_t rank_hist[34];    /* low-rank leaves of L and U by rank after the factorisation:
                                 [k] for k = 0 .. 32, [33] for ranks above 32 */
    double create_ms[2];      /* host time of hlu_create: [0] validation and planning of the task
                                 graphs, [1] device allocation, upload and kernel set-up */
} hlu_stats;

int hlu_get_stats(hlu_t h, hlu_stats *out);

/* Factorisation error of the last hlu_factor: E_fac = ||A_H - L U||_2 / ||A_H||_2
 * (the error measure of the H-LU with truncation, Sec. 3.1), both 2-norms
 * estimated by power iteration on M^T M (M = A_H - L U, then M = A_H) with M
 * applied leaf by leaf in FP64 (the factors promoted exactly from their
 * precision), never formed: x = x0 / |x0|, then z = M^T M x, lambda = |z|,
 * x = z / lambda until |lambda - lambda_old| <= rtol lambda or iters products,
 * ||M||_2 ~ sqrt(lambda).  x0: DEVICE pointer to n FP64 values in the original
 * order, not all zero (the same start vector for both norms).  *efac receives
 * the ratio, *norm_a (may be NULL) the estimate of ||A_H||_2.  The first call
 * allocates a leaf table and 6 n + 1 doubles of work space (HLU_ENOMEM beyond
 * opts.mem_budget).  HLU_ESTATE before a successful hlu_factor. */
int hlu_factor_error(hlu_t h, const double *x0_dev, int32_t iters, double rtol, double *efac, double *norm_a);

/* Launch settings of an existing handle (no re-planning): `workers` caps the worker CTAs of
 * every data-flow launch (0 -> as many as the handle was created for; a larger value is
 * clamped to that), `flags` takes HLU_FLAG_TENSOR (the other HLU_FLAG_* bits are ignored).
 * Waits for the handle's stream.  The library's tuner (paper_1906_00874_gb300.autotune) times
 * candidate settings with it.  hlu_get_launch reads the factorisation's settings back. */
int hlu_set_launch(hlu_t h, int32_t workers, int32_t flags);
int hlu_get_launch(hlu_t h, int32_t *workers, int32_t *flags);

/* Failure injection for tests of the timeout path (no counterpart in the paper):
 * with on != 0, the next data-flow factorisation of the handle gets one task
 * (the last of its graph) whose in-degree is one more than its predecessors
 * can clear.  That task never becomes ready, the workers' bounded waits run
 * out after opts.timeout_s, and hlu_factor returns HLU_ETIMEOUT with the
 * device left usable; no memory is touched out of bounds and nothing spins
 * without a limit.  The injection is consumed by that call. */
int hlu_inject_stall(hlu_t h, int32_t on);

/* Profiling: when on, every kernel launch of the handle is bracketed by CUDA
 * events on the handle's stream and its duration is added to kernel_ms of its
 * task kind (read with hlu_get_stats).  Turning it on clears the sums. */
int hlu_set_profiling(hlu_t h, int32_t on);

/* Roofline denominators: FP64 and FP32 fused multiply-add throughput of the
 * current GPU in TFLOP/s, measured with independent FMA chains on every SM
 * (a measurement utility, not part of the factorisation). */
int hlu_probe_alu_peaks(double *fp64_tflops, double *fp32_tflops);

/* Destroy the handle and free its device memory.  NULL-safe. */
void hlu_destroy(hlu_t h);

/* Message for a status code (static string). */
const char *hlu_strerror(int status);

/* y = U (V^T x) for one low-rank block (U: m x k, V: n x k, x: n x nrhs,
 * y: m x nrhs; DEVICE pointers, FP64, column-major with the given leading
 * dimensions), ordered on `cuda_stream`, WITHOUT allocating device memory.
 * The paper has no counterpart of this entry point: it serves callers that
 * may not call cudaMalloc when they compute (a memory budget fixed in advance,
 * a loop that must not stall in the allocator, code that does not own the
 * device's memory).  The k x nrhs intermediate V^T x lives in one fixed array
 * of 65536 doubles (512 KiB) inside the library, held on every GPU that loads
 * the library until the process exits; k * nrhs above 65536 returns
 * HLU_EINVAL.  Every call looks up that array's device address in the
 * current device's context (cudaGetSymbolAddress, with the device current),
 * so no address outlives a context; the first call on a device also loads the
 * library's module there, so make that first call before any stream capture.
 * k = 0 sets y to zero.  Every call uses the same array, so calls
 * that overlap on the GPU (e.g. on two streams at once) race with each other;
 * each call clears the part it accumulates into.  Returns after queueing the
 * work (HLU_OK), HLU_EINVAL for bad sizes or pointers, HLU_ECUDA if a launch
 * fails. */
int hlu_lowrank_apply_noalloc(int32_t m, int32_t n, int32_t k, int32_t nrhs, const double *U, int64_t ldu,
                              const double *V, int64_t ldv, const double *x, int64_t ldx, double *y, int64_t ldy,
                              void *cuda_stream);

/* Message of the CUDA runtime error behind the last HLU_ECUDA of this handle
 * (static string; "no CUDA error" if there was none). */
const char *hlu_last_cuda_error(hlu_t h);

/* Detail of the last device-side failure: the leaf (or task) index involved
 * and a value (the pivot, or the rank that overflowed).  Returns the status. */
int hlu_last_error_detail(hlu_t h, int64_t *index, double *value);

#ifdef __cplusplus
}
#endif
#endif /* HLU_H */
