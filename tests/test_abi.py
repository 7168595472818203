"""The C-ABI library loads, exports every declared entry point, and rejects
malformed H-matrices during host-side validation (no GPU needed: validation
happens before any device call)."""
import copy
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_00874_gb300 import build, hlu
    build.build()
    return hlu.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hlu.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|int64_t|const char \*)\s*\*?\s*(hlu_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    from paper_1906_00874_gb300.hlu import EXPORTS
    assert set(EXPORTS) <= set(names)


def test_strerror_covers_all_codes(lib):
    for code in range(9):
        assert lib.hlu_strerror(code).decode() != "unknown status"


def _create(prob, **mut):
    from paper_1906_00874_gb300.hlu import HLU
    t = prob.tree
    args = dict(n=prob.n, perm=t.perm, begin=t.begin, size=t.size, son0=t.son0, son1=t.son1,
                row_cl=prob.row_cl, col_cl=prob.col_cl, kind=prob.kind, rank=prob.rank,
                offset=prob.offset, data=prob.data)
    args.update(mut)
    return HLU(stream=0, **args)


def _expect_einval(prob, **mut):
    from paper_1906_00874_gb300.hlu import HLUError
    with pytest.raises(HLUError) as e:
        _create(prob, **mut)
    assert e.value.status == 1


def test_rejects_missing_leaf(lib, prob1280):
    keep = np.arange(1, prob1280.n_leaves)
    _expect_einval(prob1280, row_cl=prob1280.row_cl[keep], col_cl=prob1280.col_cl[keep],
                   kind=prob1280.kind[keep], rank=prob1280.rank[keep], offset=prob1280.offset[keep])


def test_rejects_lowrank_diagonal(lib, prob1280):
    kind = prob1280.kind.copy()
    d = np.flatnonzero(prob1280.row_cl == prob1280.col_cl)[0]
    kind[d] = 1
    _expect_einval(prob1280, kind=kind)


def test_rejects_rank_above_min_dims(lib, prob1280):
    rank = prob1280.rank.copy()
    l = np.flatnonzero(prob1280.kind == 1)[0]
    rank[l] = 10 ** 6
    _expect_einval(prob1280, rank=rank)


def test_rejects_non_finite_data(lib, prob1280):
    data = prob1280.data.copy()
    data[prob1280.offset[3]] = np.nan
    _expect_einval(prob1280, data=data)


def test_rejects_bad_permutation(lib, prob1280):
    perm = prob1280.tree.perm.copy()
    perm[0] = perm[1]
    _expect_einval(prob1280, perm=perm)


def test_rejects_broken_son_ranges(lib, prob1280):
    size = prob1280.tree.size.copy()
    size[1] += 1
    _expect_einval(prob1280, size=size)


def test_rejects_data_out_of_range(lib, prob1280):
    off = prob1280.offset.copy()
    off[-1] = prob1280.data.shape[0]
    _expect_einval(prob1280, offset=off)


def test_rejects_dense_block_between_split_clusters(lib, prob1280):
    """A low-rank leaf whose clusters both have sons may not be declared dense."""
    t = prob1280.tree
    cand = [l for l in range(prob1280.n_leaves) if prob1280.kind[l] == 1
            and t.son0[prob1280.row_cl[l]] >= 0 and t.son0[prob1280.col_cl[l]] >= 0]
    assert cand
    l = cand[0]
    m, n = prob1280.leaf_shape(l)
    kind = prob1280.kind.copy()
    kind[l] = 0
    data = np.concatenate([prob1280.data, np.zeros(m * n)])
    off = prob1280.offset.copy()
    off[l] = prob1280.data.shape[0]
    _expect_einval(prob1280, kind=kind, data=data, offset=off)


def test_rejects_leaf_cluster_above_128(lib):
    """One dense 200 x 200 leaf: the leaf kernels handle at most 128 rows."""
    from paper_1906_00874_gb300.hlu import HLU, HLUError
    n = 200
    with pytest.raises(HLUError) as e:
        HLU(n, np.arange(n), [0], [n], [-1], [-1], [0], [0], [0], [0], [0], np.eye(n).ravel(order="F"), stream=0)
    assert e.value.status == 1


def test_batch_rejects_bad_count_and_bad_problem(lib, prob1280):
    """hlu_create_batch validates every problem of the batch (and count >= 1)
    before any device call."""
    from paper_1906_00874_gb300.hlu import HLU, HLUError, _Blocks, _Opts, _Tree
    h = ctypes.c_void_p(1)
    st = lib.hlu_create_batch(0, ctypes.POINTER(_Tree)(), ctypes.POINTER(_Blocks)(), ctypes.byref(_Opts()),
                              ctypes.c_void_p(0), ctypes.byref(h))
    assert st == 1 and not h.value
    assert lib.hlu_batch_count(None) == 0
    bad = copy.copy(prob1280)
    keep = np.arange(1, prob1280.n_leaves)
    bad.row_cl, bad.col_cl = prob1280.row_cl[keep], prob1280.col_cl[keep]
    bad.kind, bad.rank, bad.offset = prob1280.kind[keep], prob1280.rank[keep], prob1280.offset[keep]
    with pytest.raises(HLUError) as e:
        HLU.batch([prob1280, bad], stream=0)
    assert e.value.status == 1


def test_bem_build_validates_before_any_device_call(lib, prob1280):
    """hlu_bem_build rejects a bad dimension, a cross-approximation capacity above 64, a bad
    permutation and a non-positive element size on the host."""
    from paper_1906_00874_gb300.hlu import BEMBuild, HLUError
    p = prob1280
    t = p.tree
    good = dict(dim=3, centroid=p.centroid, size=p.area, perm=t.perm, begin=t.begin, csize=t.size, son0=t.son0,
                son1=t.son1, row_cl=p.row_cl, col_cl=p.col_cl, kind=p.kind, eps=1e-4, stream=0)
    bad_perm = t.perm.copy()
    bad_perm[0] = p.n
    bad_size = p.area.copy()
    bad_size[3] = 0.0
    for mut in (dict(dim=4), dict(aca_cap=65), dict(perm=bad_perm), dict(size=bad_size), dict(eps=-1.0)):
        with pytest.raises(HLUError) as e:
            BEMBuild(**{**good, **mut})
        assert e.value.status == 1, mut
