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
                    os.path.join(ROOT, "tests", "plan_executor.cpp"), os.path.join(CSRC, "plan.cpp"),
                    os.path.join(CSRC, "plan_batch.cpp"), "-o", so],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(so)
    lib.plan_execute.restype = ctypes.c_int
    return lib


def _run(lib, p, eps, inv_block, seed, inst=None, temp_reuse=0, batch_threads=0):
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
        ctypes.c_int32(b.shape[1]), None if inst is None else ptr(inst, np.int32),
        ctypes.c_int32(0 if inst is None else int(np.max(inst)) + 1), ctypes.c_int32(temp_reuse),
        ctypes.c_int32(batch_threads))
    assert st == 0, st
    q = copy.copy(p)
    q.rank, q.offset, q.data = rank, off, out
    return q, b


@pytest.fixture(scope="module")
def oracle1280(prob1280):
    return HLUOracle(prob1280, prob1280.eps).factor()


@pytest.mark.parametrize("inv_block,seed,temp_reuse", [(-1, 1, 0), (0, 2, 0), (64, 3, 0), (0, 4, 1), (-1, 5, 1)])
def test_task_lists_reproduce_the_oracle(executor, prob1280, oracle1280, inv_block, seed, temp_reuse):
    """With temp_reuse the product temporaries share regions by dependency-level intervals; a missing
    order between two uses of a region would corrupt the factors in some random order."""
    p, o = prob1280, oracle1280
    q, x = _run(executor, p, p.eps, inv_block, seed, temp_reuse=temp_reuse)
    ranks_o = {l.leaf_id: l.rank for l in o.A.leaves() if l.kind == "lowrank"}
    assert all(int(q.rank[i]) == k for i, k in ranks_o.items())
    amax = np.max(np.abs(densify(build_hmatrix(p))))
    assert np.max(np.abs(densify(build_hmatrix(q)) - densify(o.A))) <= 1e-12 * amax
    xo = lu_solve(o.A, p.b_perm())
    assert np.max(np.abs(x - xo)) <= 1e-12 * np.max(np.abs(xo))


class _Forest:
    """Several problems as one block-diagonal H-matrix: a balanced tree of count - 1 clusters above
    the problems' roots (cluster 0 the root), then each problem's clusters, leaves and data shifted
    (the layout hlu_create_batch builds)."""

    def __init__(self, probs):
        count = len(probs)
        ncl = count - 1 + sum(p.tree.begin.size for p in probs)
        self.n = sum(p.n for p in probs)
        begin, size = np.zeros(ncl, np.int64), np.zeros(ncl, np.int64)
        son0, son1 = -np.ones(ncl, np.int64), -np.ones(ncl, np.int64)
        inst = -np.ones(ncl, np.int64)
        perm, rows, cols, kinds, ranks, offs, datas = [], [], [], [], [], [], []
        co, no, do, cl_off = count - 1, 0, 0, []
        for i, p in enumerate(probs):
            t = p.tree
            k = t.begin.size
            cl_off.append(co)
            begin[co:co + k] = t.begin + no
            size[co:co + k] = t.size
            son0[co:co + k] = np.where(t.son0 >= 0, t.son0 + co, -1)
            son1[co:co + k] = np.where(t.son1 >= 0, t.son1 + co, -1)
            inst[co:co + k] = i
            perm.append(t.perm + no)
            rows.append(p.row_cl + co)
            cols.append(p.col_cl + co)
            kinds.append(p.kind)
            ranks.append(p.rank)
            offs.append(p.offset + do)
            datas.append(p.data)
            co, no, do = co + k, no + p.n, do + p.data.size
        nxt = [0]

        def make(i0, i1):
            if i1 - i0 == 1:
                return cl_off[i0]
            v = nxt[0]
            nxt[0] += 1
            mid = (i0 + i1) // 2
            a, b = make(i0, mid), make(mid, i1)
            begin[v], size[v], son0[v], son1[v] = begin[a], size[a] + size[b], a, b
            return v
        make(0, count)

        class T:
            pass
        self.tree = T()
        self.tree.perm, self.tree.begin, self.tree.size = np.concatenate(perm), begin, size
        self.tree.son0, self.tree.son1 = son0, son1
        self.tree.n_clusters = ncl
        self.row_cl, self.col_cl = np.concatenate(rows), np.concatenate(cols)
        self.kind, self.rank = np.concatenate(kinds), np.concatenate(ranks)
        self.offset, self.data = np.concatenate(offs), np.concatenate(datas)
        self.n_leaves = self.row_cl.size
        self.inst = inst
        self._b = np.concatenate([p.b_perm() for p in probs], axis=0)
        self.leaf0 = np.cumsum([0] + [p.n_leaves for p in probs])

    def b_perm(self):
        return self._b


@pytest.mark.parametrize("batch_threads", [-1, 0, 2])
def test_batch_task_lists_equal_the_problems_own(executor, batch_threads):
    """A batch's task lists, executed, give every problem exactly the factors and solve of its own
    task lists (no task couples two problems), with and without the inverse blocks, planned as one
    forest (batch_threads < 0) or per problem on several threads and joined."""
    from bem_inputs import build_problem
    probs = [build_problem(3, 32, 2.0, 1e-4, nrhs=2), build_problem(2, 32, 2.0, 1e-4, nrhs=2, seed=1,
                                                                    axes=(1.0, 0.6, 0.4)),
             build_problem(2, 32, 2.0, 1e-4, nrhs=2, seed=2, axes=(1.0, 0.8, 0.5))]
    f = _Forest(probs)
    for inv_block, reuse in ((-1, 0), (0, 0), (0, 1)):
        qb, xb = _run(executor, f, 1e-4, inv_block, 7, inst=f.inst, temp_reuse=reuse, batch_threads=batch_threads)
        row = 0
        for i, p in enumerate(probs):
            q, x = _run(executor, p, 1e-4, inv_block, 11 + i, temp_reuse=reuse)
            lo = f.leaf0[i]
            assert np.array_equal(qb.rank[lo:lo + p.n_leaves], q.rank)
            for l in range(p.n_leaves):
                m, n = p.leaf_shape(l)
                k = int(q.rank[l])
                ln = m * n if p.kind[l] == 0 else (m + n) * k
                a = qb.data[qb.offset[lo + l]:qb.offset[lo + l] + ln]
                assert np.array_equal(a, q.data[q.offset[l]:q.offset[l] + ln]), (i, l)
            assert np.array_equal(xb[row:row + p.n], x)
            row += p.n


def test_batch_with_clusters_out_of_problem_order_is_planned_as_one_forest(executor):
    """A forest whose clusters are numbered out of problem order (not the layout hlu_create_batch
    builds, so the per-problem planning does not apply) is planned as one forest and gives the same
    factors and solve as the forest in problem order."""
    from bem_inputs import build_problem
    probs = [build_problem(2, 32, 2.0, 1e-4, nrhs=1), build_problem(2, 32, 2.0, 1e-4, nrhs=1, seed=1,
                                                                    axes=(1.0, 0.6, 0.4))]
    f = _Forest(probs)
    ref_q, ref_x = _run(executor, f, 1e-4, 0, 3, inst=f.inst)
    # renumber every cluster but the root with a seeded permutation
    ncl = f.tree.n_clusters
    pi = np.concatenate([[0], 1 + np.random.default_rng(5).permutation(ncl - 1)])
    g = copy.copy(f)
    g.tree = copy.copy(f.tree)
    for name in ("begin", "size"):
        a = np.empty_like(getattr(f.tree, name))
        a[pi] = getattr(f.tree, name)
        setattr(g.tree, name, a)
    for name in ("son0", "son1"):
        src = getattr(f.tree, name)
        a = np.empty_like(src)
        a[pi] = np.where(src >= 0, pi[np.maximum(src, 0)], -1)
        setattr(g.tree, name, a)
    inst = np.empty_like(f.inst)
    inst[pi] = f.inst
    g.inst = inst
    g.row_cl, g.col_cl = pi[f.row_cl], pi[f.col_cl]
    q, x = _run(executor, g, 1e-4, 0, 4, inst=g.inst)
    assert np.array_equal(q.rank, ref_q.rank)
    for l in range(f.n_leaves):
        assert q.offset[l] == ref_q.offset[l]
    assert np.array_equal(q.data, ref_q.data)
    assert np.array_equal(x, ref_x)


@pytest.mark.parametrize("inv_block,temp_reuse", [(-1, 0), (0, 0), (0, 1)])
def test_piped_analysis_builds_the_serial_graphs(executor, inv_block, temp_reuse):
    """The factorisation's dependency analysis on a second host thread (the default for one problem)
    builds exactly the graphs of the one-thread planner: task codes, waves, predecessor and successor
    lists, roots and priorities of the factorisation, solve and matvec plans, and the arena sizes."""
    from bem_inputs import build_problem
    lib = executor
    lib.plan_graphs_equal.restype = ctypes.c_int
    for p in (build_problem(3, 32, 2.0, 1e-4, nrhs=1),
              build_problem(4, 32, 2.0, 1e-6, nrhs=1, seed=3, axes=(1.0, 0.7, 0.5))):
        t = p.tree
        keep = []

        def ptr(a, tp):
            x = np.ascontiguousarray(a, dtype=tp)
            keep.append(x)
            return x.ctypes.data_as(ctypes.c_void_p)
        st = lib.plan_graphs_equal(
            ctypes.c_int32(p.n), ctypes.c_int32(t.n_clusters), ptr(t.perm, np.int32), ptr(t.begin, np.int32),
            ptr(t.size, np.int32), ptr(t.son0, np.int32), ptr(t.son1, np.int32), ctypes.c_int64(p.n_leaves),
            ptr(p.row_cl, np.int32), ptr(p.col_cl, np.int32), ptr(p.kind, np.int8), ptr(p.rank, np.int32),
            ptr(p.offset, np.int64), ptr(p.data, np.float64), ctypes.c_int64(p.data.size),
            ctypes.c_int32(inv_block), ctypes.c_int32(temp_reuse))
        assert st == 0, (p.n, st)
