"""The planner's task lists, run on the CPU in double precision (tests/plan_executor.cpp) in random
dependency-respecting orders, reproduce the oracle's factorisation and solve.  This checks the
expansion of the recursion (operands, dependencies, truncation points) on the host, independently of
the GPU kernels."""
import copy
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import HLUOracle, build_hmatrix, densify
from oracle.errors import lu_solve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1906_00874_gb300", "csrc")


@pytest.fixture(scope="module")
def executor(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    so = str(tmp_path_factory.mktemp("exec") / "plan_executor.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-fPIC", "-shared", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "plan_executor.cpp"), os.path.join(CSRC, "plan.cpp"), "-o", so],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(so)
    lib.plan_execute.restype = ctypes.c_int
    return lib


def _run(lib, p, eps, inv_block, seed):
    t = p.tree
    keep = []

    def ptr(a, tp):
        x = np.ascontiguousarray(a, dtype=tp)
        keep.append(x)
        return x.ctypes.data_as(ctypes.c_void_p)
    out = np.zeros(4 * p.data.size + 16)
    off = np.zeros(p.n_leaves, dtype=np.int64)
    rank = np.zeros(p.n_leaves, dtype=np.int32)
    b = np.asfortranarray(p.b_perm()).copy(order="F")
    st = lib.plan_execute(
        ctypes.c_int32(p.n), ctypes.c_int32(t.n_clusters), ptr(t.perm, np.int32), ptr(t.begin, np.int32),
        ptr(t.size, np.int32), ptr(t.son0, np.int32), ptr(t.son1, np.int32), ctypes.c_int64(p.n_leaves),
        ptr(p.row_cl, np.int32), ptr(p.col_cl, np.int32), ptr(p.kind, np.int8), ptr(p.rank, np.int32),
        ptr(p.offset, np.int64), ptr(p.data, np.float64), ctypes.c_int64(p.data.size), ctypes.c_double(eps),
        ctypes.c_int32(inv_block), ctypes.c_uint64(seed), out.ctypes.data_as(ctypes.c_void_p),
        off.ctypes.data_as(ctypes.c_void_p), rank.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p),
        ctypes.c_int32(b.shape[1]))
    assert st == 0, st
    q = copy.copy(p)
    q.rank, q.offset, q.data = rank, off, out
    return q, b


@pytest.fixture(scope="module")
def oracle1280(prob1280):
    return HLUOracle(prob1280, prob1280.eps).factor()


@pytest.mark.parametrize("inv_block,seed", [(-1, 1), (0, 2), (64, 3)])
def test_task_lists_reproduce_the_oracle(executor, prob1280, oracle1280, inv_block, seed):
    p, o = prob1280, oracle1280
    q, x = _run(executor, p, p.eps, inv_block, seed)
    ranks_o = {l.leaf_id: l.rank for l in o.A.leaves() if l.kind == "lowrank"}
    assert all(int(q.rank[i]) == k for i, k in ranks_o.items())
    amax = np.max(np.abs(densify(build_hmatrix(p))))
    assert np.max(np.abs(densify(build_hmatrix(q)) - densify(o.A))) <= 1e-12 * amax
    xo = lu_solve(o.A, p.b_perm())
    assert np.max(np.abs(x - xo)) <= 1e-12 * np.max(np.abs(xo))
