"""H-matrix construction on the GPU (hlu_bem_build): the leaves of a problem's
block tree built on the device from its geometry, against the host generator
and the kernel itself.

Dense leaves are the kernel entries (equal to the host's to rounding); every
low-rank leaf approximates its exact kernel block to the tolerance; ranks are
those of the host's ACA + SVD up to pivoting differences; and the GPU-built
matrix factorised and refined solves the host-built system to the truncation
level (residual checked with the oracle's FP64 H-matvec)."""
import numpy as np
import pytest

from bem_inputs import build_problem, kernel_block
from oracle import build_hmatrix
from oracle.errors import solve_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    from paper_1906_00874_gb300 import build
    build.build()
    assert torch.cuda.is_available()


CASES = [dict(r=3, leaf=32, eta=2.0, eps=1e-4, dim=3), dict(r=3, leaf=32, eta=1.0, eps=1e-6, dim=3),
         dict(r=3, leaf=32, eta=0.5, eps=1e-4, dim=1), dict(r=3, leaf=32, eta=0.5, eps=1e-4, dim=2)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"d{c['dim']}_eta{c['eta']}_eps{c['eps']:g}")
def test_leaves_match_kernel_and_host_build(case):
    from paper_1906_00874_gb300.hlu import BEMBuild
    p = build_problem(nrhs=2, **case)
    g = BEMBuild.from_problem(p)
    data = g.data()
    perm = p.tree.perm
    worst, rank_diff = 0.0, []
    for l in range(p.n_leaves):
        r0, m, c0, n = p.leaf_ranges(l)
        rows, cols = perm[r0:r0 + m], perm[c0:c0 + n]
        o = int(g.offset[l])
        if p.kind[l] == 0:
            D = data[o:o + m * n].reshape((m, n), order="F")
            assert np.max(np.abs(D - p.leaf_dense(l))) <= 1e-14 * np.max(np.abs(p.leaf_dense(l))), l
            continue
        k = int(g.rank[l])
        U = data[o:o + m * k].reshape((m, k), order="F")
        V = data[o + m * k:o + (m + n) * k].reshape((n, k), order="F")
        exact = kernel_block(p.centroid, p.area, rows, cols, case["dim"])
        err = np.linalg.norm(U @ V.T - exact) / np.linalg.norm(exact)
        worst = max(worst, err)
        rank_diff.append(abs(k - int(p.rank[l])))
    assert worst <= 10 * case["eps"], worst
    assert max(rank_diff) <= 2 and np.mean(rank_diff) <= 0.5
    g.close()


def test_gpu_built_matrix_solves_host_system():
    import torch
    from paper_1906_00874_gb300 import HLU_FP32
    from paper_1906_00874_gb300.hlu import BEMBuild, to_device_panel
    p = build_problem(3, 32, 2.0, 1e-4, nrhs=2)
    g = BEMBuild.from_problem(p)
    h = g.create(precision=HLU_FP32)
    h.factor(p.eps)
    b = to_device_panel(p.b)
    x = torch.zeros_like(b)
    it, res = h.solve_refined(b, x, tol=1e-10, max_iter=30)
    assert res <= 1e-10
    A = build_hmatrix(p)  # the host-built H-matrix
    xh = x.cpu().numpy()[p.tree.perm]
    assert np.all(solve_error(A, xh, p.b_perm()) <= 10 * p.eps)
    h.close()
    g.close()


def test_rank_capacity_is_reported():
    from paper_1906_00874_gb300.hlu import BEMBuild, HLUError
    p = build_problem(3, 32, 2.0, 1e-4, nrhs=1)
    with pytest.raises(HLUError) as e:
        BEMBuild.from_problem(p, eps=1e-12, aca_cap=2)
    assert e.value.status == 5
