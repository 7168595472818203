"""Thin ctypes binding of the H-LU C ABI (include/hlu.h).

Every step of the factorisation, the solve and the matrix-vector product runs
in the library's CUDA kernels; this module only marshals arguments.  There is
no CPU path: if libhlu.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhlu.so")

HLU_FP64 = 0
HLU_FP32 = 1          # FP32 factors, FP64 SVD of every truncation core
HLU_FP32_CORE32 = 2   # FP32 factors, FP32 Jacobi in the truncation cores
SCHED_DATAFLOW = 0
SCHED_WAVES = 1
FLAG_TENSOR = 1       # FP32 factors: dense products of the factorisation on the tensor cores
FLAG_SERIAL_PLAN = 2  # plan on one host thread (default: a batch per problem in parallel, one problem on two threads)

STATUS = {0: "HLU_OK", 1: "HLU_EINVAL", 2: "HLU_ENOMEM", 3: "HLU_ESTATE", 4: "HLU_EPIVOT",
          5: "HLU_ERANKCAP", 6: "HLU_ETIMEOUT", 7: "HLU_ECUDA", 8: "HLU_ENUMERIC"}

EXPORTS = ("hlu_create", "hlu_factor", "hlu_solve", "hlu_matvec", "hlu_solve_refined", "hlu_solve_gmres",
           "hlu_factor_doubles",
           "hlu_get_factors", "hlu_get_stats", "hlu_set_profiling", "hlu_destroy", "hlu_strerror",
           "hlu_last_error_detail", "hlu_last_cuda_error", "hlu_probe_alu_peaks", "hlu_inject_stall",
           "hlu_create_batch", "hlu_factor_batch", "hlu_batch_count", "hlu_bem_build", "hlu_bem_result",
           "hlu_bem_copy_data", "hlu_create_bem", "hlu_bem_destroy", "hlu_plan_info_get", "hlu_plan_info_batch",
           "hlu_factor_error", "hlu_lowrank_apply_noalloc", "hlu_set_launch", "hlu_get_launch")
KINDS = ("getrf", "trsm", "project", "accum", "radd", "split", "dataflow_factor", "dataflow_solve",
         "dataflow_matvec")


class HLUError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({_strerror(status)})")


class _Tree(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_clusters", ctypes.c_int32), ("perm", ctypes.c_void_p),
                ("begin", ctypes.c_void_p), ("size", ctypes.c_void_p), ("son0", ctypes.c_void_p),
                ("son1", ctypes.c_void_p)]


class _Blocks(ctypes.Structure):
    _fields_ = [("n_leaves", ctypes.c_int64), ("row_cl", ctypes.c_void_p), ("col_cl", ctypes.c_void_p),
                ("kind", ctypes.c_void_p), ("rank", ctypes.c_void_p), ("offset", ctypes.c_void_p),
                ("data", ctypes.c_void_p), ("data_len", ctypes.c_int64)]


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("rank_cap", ctypes.c_int32), ("nrhs_max", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("mem_budget", ctypes.c_int64), ("timeout_s", ctypes.c_double),
                ("inv_block", ctypes.c_int32), ("flags", ctypes.c_int32), ("workers", ctypes.c_int32),
                ("temp_reuse", ctypes.c_int32)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("factor_tasks", "factor_edges", "factor_levels", "solve_tasks",
                                              "solve_levels", "matvec_tasks", "inverse_blocks", "factor_elems")] + \
               [("plan_ms", ctypes.c_double), ("factor_critical_us", ctypes.c_double),
                ("solve_critical_us", ctypes.c_double), ("factor_temp_elems", ctypes.c_int64),
                ("factor_temp_peak_elems", ctypes.c_int64)]


def plan_info(problems, rank_cap=0, nrhs_max=0, inv_block=0, schedule=SCHED_DATAFLOW, temp_reuse=0, flags=0):
    """Sizes of the task graphs hlu_create (one problem) or hlu_create_batch (a list) would build:
    validation and planning on the host only (hlu_plan_info_get / hlu_plan_info_batch)."""
    lib = load()
    many = isinstance(problems, (list, tuple))
    descs = [_describe(p.n, p.tree.perm, p.tree.begin, p.tree.size, p.tree.son0, p.tree.son1, p.row_cl, p.col_cl,
                       p.kind, p.rank, p.offset, p.data) for p in (problems if many else [problems])]
    opts = _Opts(0, int(rank_cap), int(nrhs_max), int(schedule), 0, 0.0, int(inv_block), int(flags), 0,
                 int(temp_reuse))
    info = _PlanInfo()
    if many:
        trees = (_Tree * len(descs))(*[d[0] for d in descs])
        blocks = (_Blocks * len(descs))(*[d[1] for d in descs])
        st = lib.hlu_plan_info_batch(len(descs), trees, blocks, ctypes.byref(opts), ctypes.byref(info))
    else:
        st = lib.hlu_plan_info_get(ctypes.byref(descs[0][0]), ctypes.byref(descs[0][1]), ctypes.byref(opts),
                                   ctypes.byref(info))
    if st != 0:
        raise HLUError(st, "hlu_plan_info")
    return {f: getattr(info, f) for f, _ in info._fields_}


class _BemInput(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("centroid", ctypes.c_void_p), ("size", ctypes.c_void_p),
                ("tree", ctypes.POINTER(_Tree)), ("n_leaves", ctypes.c_int64), ("row_cl", ctypes.c_void_p),
                ("col_cl", ctypes.c_void_p), ("kind", ctypes.c_void_p), ("eps", ctypes.c_double),
                ("aca_cap", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n_tasks", ctypes.c_int64), ("n_waves", ctypes.c_int64), ("n_launches", ctypes.c_int64),
                ("solve_tasks", ctypes.c_int64), ("solve_waves", ctypes.c_int64),
                ("solve_launches", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("tasks_by_kind", ctypes.c_int64 * 8), ("model_flops", ctypes.c_double),
                ("flops_by_kind", ctypes.c_double * 8), ("solve_flops", ctypes.c_double),
                ("kernel_ms", ctypes.c_double * 10), ("kernel_launches", ctypes.c_int64 * 10),
                ("task_busy_ms", ctypes.c_double * 8), ("task_count", ctypes.c_int64 * 8),
                ("radd_busy_ms", ctypes.c_double * 8), ("radd_count", ctypes.c_int64 * 8),
                ("solve_busy_ms", ctypes.c_double * 8), ("solve_task_count", ctypes.c_int64 * 8),
                ("radd_phase", ctypes.c_double * 16),
                ("kernels_launched", ctypes.c_int64), ("max_rank", ctypes.c_int32), ("max_stacked", ctypes.c_int32),
                ("rank_hist", ctypes.c_int64 * 34), ("create_ms", ctypes.c_double * 2)]

    def as_dict(self):
        per_kind = ("tasks_by_kind", "flops_by_kind", "kernel_ms", "kernel_launches", "task_busy_ms", "task_count",
                    "solve_busy_ms", "solve_task_count")
        per_size = ("radd_busy_ms", "radd_count")
        d = {f: getattr(self, f) for f, _ in self._fields_
             if f not in per_kind + per_size + ("radd_phase", "rank_hist", "create_ms")}
        d["rank_hist"] = list(self.rank_hist)
        d["create_ms"] = {"plan": self.create_ms[0], "device_setup": self.create_ms[1]}
        ph = list(self.radd_phase)
        d["radd_phase"] = {}
        for route, b in (("dense", 0), ("stacked", 8)):
            d["radd_phase"][route] = {"form_ms": ph[b], "stack_qr_ms": ph[b + 1], "qrcp_ms": ph[b + 2],
                                      "jacobi_ms": ph[b + 3], "factors_ms": ph[b + 5],
                                      "mean_jacobi_sweeps": ph[b + 4] / max(ph[b + 7], 1),
                                      "mean_jacobi_r": ph[b + 6] / max(ph[b + 7], 1), "tasks": ph[b + 7]}
        for f in per_kind:
            d[f] = dict(zip(KINDS, list(getattr(self, f))[:len(KINDS)]))
        # profiling of the factorisation's workers (summed over workers): lifetime, and waits on
        # queue slots that no ready task had filled yet
        d["worker_life_ms"] = self.task_count[6] * 1e-6
        d["worker_wait_ms"] = self.task_busy_ms[7]
        sizes = ("<128", "<256", "<512", "<1024", "<2048", "<4096", "<8192", ">=8192")
        for f in per_size:
            d[f] = dict(zip(sizes, list(getattr(self, f))))
        return d


_lib = None


def load(path=LIB_PATH):
    """Load libhlu.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhlu.so not found at {path}: build it with paper_1906_00874_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.hlu_create.argtypes = [ctypes.POINTER(_Tree), ctypes.POINTER(_Blocks), ctypes.POINTER(_Opts), vp,
                               ctypes.POINTER(vp)]
    lib.hlu_factor.argtypes = [vp, dbl]
    lib.hlu_plan_info_get.argtypes = [ctypes.POINTER(_Tree), ctypes.POINTER(_Blocks), ctypes.POINTER(_Opts),
                                      ctypes.POINTER(_PlanInfo)]
    lib.hlu_plan_info_batch.argtypes = [i32, ctypes.POINTER(_Tree), ctypes.POINTER(_Blocks), ctypes.POINTER(_Opts),
                                        ctypes.POINTER(_PlanInfo)]
    lib.hlu_bem_build.argtypes = [ctypes.POINTER(_BemInput), vp, ctypes.POINTER(vp)]
    lib.hlu_bem_result.argtypes = [vp, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(vp)]
    lib.hlu_bem_copy_data.argtypes = [vp, vp]
    lib.hlu_create_bem.argtypes = [vp, ctypes.POINTER(_Opts), vp, ctypes.POINTER(vp)]
    lib.hlu_bem_destroy.argtypes = [vp]
    lib.hlu_bem_destroy.restype = None
    lib.hlu_create_batch.argtypes = [i32, ctypes.POINTER(_Tree), ctypes.POINTER(_Blocks), ctypes.POINTER(_Opts), vp,
                                     ctypes.POINTER(vp)]
    lib.hlu_factor_batch.argtypes = [vp, ctypes.POINTER(dbl)]
    lib.hlu_batch_count.argtypes = [vp]
    lib.hlu_solve.argtypes = [vp, vp, i32, i64]
    lib.hlu_matvec.argtypes = [vp, vp, vp, i32, i64]
    lib.hlu_solve_refined.argtypes = [vp, vp, vp, i32, i64, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl)]
    lib.hlu_solve_gmres.argtypes = [vp, vp, vp, i32, i64, dbl, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl)]
    lib.hlu_factor_error.argtypes = [vp, vp, i32, dbl, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.hlu_set_launch.argtypes = [vp, i32, i32]
    lib.hlu_get_launch.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.hlu_set_profiling.argtypes = [vp, i32]
    lib.hlu_inject_stall.argtypes = [vp, i32]
    lib.hlu_probe_alu_peaks.argtypes = [ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.hlu_factor_doubles.argtypes = [vp]
    lib.hlu_factor_doubles.restype = i64
    lib.hlu_get_factors.argtypes = [vp, vp, vp, vp]
    lib.hlu_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.hlu_destroy.argtypes = [vp]
    lib.hlu_destroy.restype = None
    lib.hlu_strerror.argtypes = [ctypes.c_int]
    lib.hlu_strerror.restype = ctypes.c_char_p
    lib.hlu_last_error_detail.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(dbl)]
    lib.hlu_last_cuda_error.argtypes = [vp]
    lib.hlu_last_cuda_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _strerror(status):
    try:
        return load().hlu_strerror(int(status)).decode()
    except Exception:
        return "?"


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr_and_ld(t, n, what):
    """(pointer, nrhs, ld) of a CUDA float64 tensor holding an n x nrhs column-major panel:
    shape (n,) or (n, nrhs) with stride(0) == 1 (any stride(0) when n == 1: one row)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{what} must be a CUDA float64 tensor")
    if t.dim() == 1:
        if t.shape[0] != n or (n > 1 and t.stride(0) != 1):
            raise ValueError(f"{what}: expected a contiguous vector of length {n}")
        return t.data_ptr(), 1, n
    if t.dim() != 2 or t.shape[0] != n or (n > 1 and t.stride(0) != 1):
        raise ValueError(f"{what}: expected shape ({n}, nrhs) in column-major layout (stride(0) == 1)")
    ld = n if t.shape[1] <= 1 else t.stride(1)
    if ld < n:
        raise ValueError(f"{what}: columns overlap (stride(1) < {n})")
    return t.data_ptr(), t.shape[1], ld


def to_device_panel(a, device="cuda"):
    """CUDA float64 tensor of shape (n, nrhs) in column-major layout from a host array."""
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.tensor(a, device=device)
    return torch.tensor(np.ascontiguousarray(a.T), device=device).t()


def _describe(n, perm, begin, size, son0, son1, row_cl, col_cl, kind, rank, offset, data):
    """(_Tree, _Blocks, arrays they point into) of one problem; the arrays must outlive the structs."""
    keep = [np.ascontiguousarray(a, dtype=t) for a, t in (
        (perm, np.int32), (begin, np.int32), (size, np.int32), (son0, np.int32), (son1, np.int32),
        (row_cl, np.int32), (col_cl, np.int32), (kind, np.int8), (rank, np.int32), (offset, np.int64),
        (data, np.float64))]
    perm_, begin_, size_, son0_, son1_, row_, col_, kind_, rank_, off_, data_ = keep
    tree = _Tree(int(n), int(begin_.shape[0]), _ptr(perm_), _ptr(begin_), _ptr(size_), _ptr(son0_), _ptr(son1_))
    blocks = _Blocks(int(row_.shape[0]), _ptr(row_), _ptr(col_), _ptr(kind_), _ptr(rank_), _ptr(off_),
                     _ptr(data_), int(data_.shape[0]))
    return tree, blocks, keep


def probe_alu_peaks():
    """(FP64, FP32) FMA throughput of the current GPU in TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = load().hlu_probe_alu_peaks(ctypes.byref(a), ctypes.byref(b))
    if st != 0:
        raise HLUError(st, "hlu_probe_alu_peaks")
    return a.value, b.value


class HLU:
    """One H-matrix on the GPU: factorise once, solve many times."""

    def __init__(self, n, perm, begin, size, son0, son1, row_cl, col_cl, kind, rank, offset, data,
                 precision=HLU_FP64, rank_cap=0, nrhs_max=0, mem_budget=0, stream=None,
                 schedule=SCHED_DATAFLOW, timeout_s=0.0, inv_block=0, flags=0, workers=0, temp_reuse=0):
        tree, blocks, keep = _describe(n, perm, begin, size, son0, son1, row_cl, col_cl, kind, rank, offset, data)
        self._open(1, ctypes.byref(tree), ctypes.byref(blocks), [int(n)], int(blocks.n_leaves), precision, rank_cap,
                   nrhs_max, mem_budget, stream, schedule, timeout_s, inv_block, flags, workers, temp_reuse)

    def _open(self, count, trees, blocks, sizes, n_leaves, precision, rank_cap, nrhs_max, mem_budget, stream,
              schedule, timeout_s, inv_block=0, flags=0, workers=0, temp_reuse=0):
        lib = load()
        self._h = ctypes.c_void_p()
        opts = _Opts(int(precision), int(rank_cap), int(nrhs_max), int(schedule), int(mem_budget), float(timeout_s),
                     int(inv_block), int(flags), int(workers), int(temp_reuse))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.n = int(sum(sizes))
        self.sizes = tuple(sizes)
        self.n_leaves = n_leaves
        self.precision = int(precision)
        if count == 1:
            st = lib.hlu_create(trees, blocks, ctypes.byref(opts), ctypes.c_void_p(stream), ctypes.byref(self._h))
        else:
            st = lib.hlu_create_batch(count, trees, blocks, ctypes.byref(opts), ctypes.c_void_p(stream),
                                      ctypes.byref(self._h))
        if st != 0:
            self._h = ctypes.c_void_p()
            raise HLUError(st, "hlu_create" if count == 1 else "hlu_create_batch")

    @classmethod
    def batch(cls, problems, precision=HLU_FP64, rank_cap=0, nrhs_max=0, mem_budget=0, stream=None,
              schedule=SCHED_DATAFLOW, timeout_s=0.0, inv_block=0, flags=0, workers=0, temp_reuse=0):
        """One handle for several independent problems (hlu_create_batch): the block-diagonal
        system whose rows are the problems' rows in turn (offsets of self.sizes)."""
        descs = [_describe(p.n, p.tree.perm, p.tree.begin, p.tree.size, p.tree.son0, p.tree.son1, p.row_cl,
                           p.col_cl, p.kind, p.rank, p.offset, p.data) for p in problems]
        if not descs:
            raise ValueError("batch needs at least one problem")
        trees = (_Tree * len(descs))(*[d[0] for d in descs])
        blocks = (_Blocks * len(descs))(*[d[1] for d in descs])
        self = cls.__new__(cls)
        self._open(len(descs), trees, blocks, [p.n for p in problems], sum(int(d[1].n_leaves) for d in descs),
                   precision, rank_cap, nrhs_max, mem_budget, stream, schedule, timeout_s, inv_block, flags, workers,
                   temp_reuse)
        return self

    @property
    def count(self):
        """Number of problems in the handle (hlu_batch_count)."""
        return load().hlu_batch_count(self._h)

    @classmethod
    def from_problem(cls, p, **kw):
        t = p.tree
        return cls(p.n, t.perm, t.begin, t.size, t.son0, t.son1, p.row_cl, p.col_cl, p.kind, p.rank, p.offset,
                   p.data, **kw)

    def _check(self, st, what):
        if st != 0:
            if st == 7:  # HLU_ECUDA: say which CUDA error
                what = f"{what} [{load().hlu_last_cuda_error(self._h).decode()}]"
            raise HLUError(st, what)

    def factor(self, eps):
        """H-LU with tolerance eps; a sequence gives one tolerance per problem of a batch."""
        if np.ndim(eps) == 0:
            self._check(load().hlu_factor(self._h, float(eps)), "hlu_factor")
            return
        e = np.ascontiguousarray(eps, dtype=np.float64)
        if e.shape != (self.count,):
            raise ValueError(f"expected {self.count} tolerances, got shape {e.shape}")
        self._check(load().hlu_factor_batch(self._h, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "hlu_factor_batch")

    def solve(self, b):
        """Overwrite the CUDA float64 panel b (n,) or (n, nrhs) column-major with A^{-1} b."""
        ptr, nrhs, ld = _dev_ptr_and_ld(b, self.n, "b")
        self._check(load().hlu_solve(self._h, ctypes.c_void_p(ptr), nrhs, ld), "hlu_solve")
        return b

    def matvec(self, x, y):
        """y = A_H x (original H-matrix, FP64) for CUDA float64 panels."""
        px, nrhs, ldx = _dev_ptr_and_ld(x, self.n, "x")
        py, nrhs2, ldy = _dev_ptr_and_ld(y, self.n, "y")
        if nrhs != nrhs2 or ldx != ldy:
            raise ValueError("x and y must have the same shape and leading dimension")
        self._check(load().hlu_matvec(self._h, ctypes.c_void_p(px), ctypes.c_void_p(py), nrhs, ldx), "hlu_matvec")
        return y

    def solve_refined(self, b, x, tol=1e-10, max_iter=20):
        """x = refined solution of A_H x = b (CUDA float64 panels, same layout);
        returns (solves applied, largest relative residual)."""
        pb, nrhs, ldb = _dev_ptr_and_ld(b, self.n, "b")
        px, nrhs2, ldx = _dev_ptr_and_ld(x, self.n, "x")
        if nrhs != nrhs2 or ldb != ldx:
            raise ValueError("b and x must have the same shape and leading dimension")
        it = ctypes.c_int32()
        res = ctypes.c_double()
        self._check(load().hlu_solve_refined(self._h, ctypes.c_void_p(pb), ctypes.c_void_p(px), nrhs, ldb,
                                             float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(res)),
                    "hlu_solve_refined")
        return it.value, res.value

    def solve_gmres(self, b, x, tol=1e-10, restart=30, max_iter=300):
        """x = GMRES(restart) solution of A_H x = b in FP64, right-preconditioned by the factors
        (CUDA float64 panels, same layout); returns (Arnoldi steps, largest relative residual)."""
        pb, nrhs, ldb = _dev_ptr_and_ld(b, self.n, "b")
        px, nrhs2, ldx = _dev_ptr_and_ld(x, self.n, "x")
        if nrhs != nrhs2 or ldb != ldx:
            raise ValueError("b and x must have the same shape and leading dimension")
        it = ctypes.c_int32()
        res = ctypes.c_double()
        self._check(load().hlu_solve_gmres(self._h, ctypes.c_void_p(pb), ctypes.c_void_p(px), nrhs, ldb,
                                           float(tol), int(restart), int(max_iter), ctypes.byref(it),
                                           ctypes.byref(res)), "hlu_solve_gmres")
        return it.value, res.value

    def factor_error(self, x0=None, seed=1, iters=30, rtol=1e-3):
        """E_fac = ||A_H - L U||_2 / ||A_H||_2 of the last factorisation, estimated on the device
        (hlu_factor_error); x0: start vector in the original order (CUDA float64, n values), by
        default N(0,1) from `seed`.  Returns (E_fac, estimate of ||A_H||_2)."""
        import torch
        if x0 is None:
            x0 = torch.from_numpy(np.random.default_rng(seed).standard_normal(self.n)).to("cuda")
        ptr, nrhs, _ = _dev_ptr_and_ld(x0, self.n, "x0")
        if nrhs != 1:
            raise ValueError("x0 must be one vector of n values")
        e, a = ctypes.c_double(), ctypes.c_double()
        self._check(load().hlu_factor_error(self._h, ctypes.c_void_p(ptr), int(iters), float(rtol), ctypes.byref(e),
                                            ctypes.byref(a)), "hlu_factor_error")
        return e.value, a.value

    def set_launch(self, workers=0, flags=0):
        """Launch settings without re-planning (hlu_set_launch): worker cap and HLU_FLAG_TENSOR."""
        self._check(load().hlu_set_launch(self._h, int(workers), int(flags)), "hlu_set_launch")

    def get_launch(self):
        """(workers of a factorisation launch, flags) of the handle (hlu_get_launch)."""
        w, f = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().hlu_get_launch(self._h, ctypes.byref(w), ctypes.byref(f)), "hlu_get_launch")
        return w.value, f.value

    def inject_stall(self, on=True):
        """Test hook: the next factorisation stalls on one task until the wait limit (HLU_ETIMEOUT)."""
        self._check(load().hlu_inject_stall(self._h, int(bool(on))), "hlu_inject_stall")

    def set_profiling(self, on):
        self._check(load().hlu_set_profiling(self._h, 1 if on else 0), "hlu_set_profiling")

    def get_factors(self):
        """(rank, offset, data) of the factors in the input leaf layout (host numpy)."""
        lib = load()
        tot = lib.hlu_factor_doubles(self._h)
        rank = np.zeros(self.n_leaves, dtype=np.int32)
        off = np.zeros(self.n_leaves, dtype=np.int64)
        data = np.zeros(max(int(tot), 1), dtype=np.float64)
        self._check(lib.hlu_get_factors(self._h, _ptr(rank), _ptr(off), _ptr(data)), "hlu_get_factors")
        return rank, off, data

    def stats(self):
        s = Stats()
        self._check(load().hlu_get_stats(self._h, ctypes.byref(s)), "hlu_get_stats")
        return s.as_dict()

    def error_detail(self):
        idx = ctypes.c_int64()
        val = ctypes.c_double()
        st = load().hlu_last_error_detail(self._h, ctypes.byref(idx), ctypes.byref(val))
        return st, idx.value, val.value

    def close(self):
        if self._h:
            load().hlu_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BEMBuild:
    """The leaves of an H-matrix built on the GPU (hlu_bem_build): the Laplace kernel of dimension
    `dim` on the elements (centroid, size) for the given cluster tree and block-tree leaves."""

    def __init__(self, dim, centroid, size, perm, begin, csize, son0, son1, row_cl, col_cl, kind, eps,
                 aca_cap=0, stream=None):
        lib = load()
        keep = [np.ascontiguousarray(a, dtype=t) for a, t in (
            (centroid, np.float64), (size, np.float64), (perm, np.int32), (begin, np.int32), (csize, np.int32),
            (son0, np.int32), (son1, np.int32), (row_cl, np.int32), (col_cl, np.int32), (kind, np.int8))]
        c_, a_, perm_, begin_, size_, s0_, s1_, r_, cc_, k_ = keep
        self.n, self.n_leaves = int(a_.shape[0]), int(r_.shape[0])
        tree = _Tree(self.n, int(begin_.shape[0]), _ptr(perm_), _ptr(begin_), _ptr(size_), _ptr(s0_), _ptr(s1_))
        inp = _BemInput(int(dim), _ptr(c_), _ptr(a_), ctypes.pointer(tree), self.n_leaves, _ptr(r_), _ptr(cc_),
                        _ptr(k_), float(eps), int(aca_cap), 0)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._b = ctypes.c_void_p()
        st = lib.hlu_bem_build(ctypes.byref(inp), ctypes.c_void_p(stream), ctypes.byref(self._b))
        if st != 0:
            self._b = ctypes.c_void_p()
            raise HLUError(st, "hlu_bem_build")
        self.rank = np.zeros(self.n_leaves, dtype=np.int32)
        self.offset = np.zeros(self.n_leaves, dtype=np.int64)
        n_data = ctypes.c_int64()
        dev = ctypes.c_void_p()
        lib.hlu_bem_result(self._b, _ptr(self.rank), _ptr(self.offset), ctypes.byref(n_data), ctypes.byref(dev))
        self.data_len = n_data.value

    @classmethod
    def from_problem(cls, p, eps=None, **kw):
        """The GPU build of a problem's matrix: its geometry, trees and leaf kinds."""
        t = p.tree
        return cls(getattr(p, "dim", 3), p.centroid, p.area, t.perm, t.begin, t.size, t.son0, t.son1, p.row_cl,
                   p.col_cl, p.kind, p.eps if eps is None else eps, **kw)

    def data(self):
        """The leaf data copied to host memory (layout of hlu_blocks)."""
        out = np.empty(max(self.data_len, 1))
        st = load().hlu_bem_copy_data(self._b, _ptr(out))
        if st != 0:
            raise HLUError(st, "hlu_bem_copy_data")
        return out[:self.data_len]

    def create(self, precision=HLU_FP64, rank_cap=0, nrhs_max=0, mem_budget=0, stream=None,
               schedule=SCHED_DATAFLOW, timeout_s=0.0, inv_block=0, flags=0, workers=0, temp_reuse=0):
        """An HLU handle on this matrix (hlu_create_bem)."""
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        opts = _Opts(int(precision), int(rank_cap), int(nrhs_max), int(schedule), int(mem_budget), float(timeout_s),
                     int(inv_block), int(flags), int(workers), int(temp_reuse))
        h = HLU.__new__(HLU)
        h._h = ctypes.c_void_p()
        h.n, h.sizes, h.n_leaves, h.precision = self.n, (self.n,), self.n_leaves, int(precision)
        st = load().hlu_create_bem(self._b, ctypes.byref(opts), ctypes.c_void_p(stream), ctypes.byref(h._h))
        if st != 0:
            h._h = ctypes.c_void_p()
            raise HLUError(st, "hlu_create_bem")
        return h

    def close(self):
        if self._b:
            load().hlu_bem_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
