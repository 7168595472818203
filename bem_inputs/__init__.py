"""Seeded synthetic inputs: BEM H-matrices on refined icosahedra / ellipsoids.

This package generates data only (mesh, cluster tree, block tree, compressed
leaves, right-hand sides).  It holds none of the H-LU arithmetic and is the one
module that both the CPU oracle and the GPU library consume.
"""
from .problem import Problem, build_problem, build_structure  # noqa: F401
from .assemble import kernel_block  # noqa: F401
from .mesh import icosphere, ellipsoid, triangle_data  # noqa: F401

# Named workloads (icosphere refinement r, leaf size, eta, eps, rhs count).
WORKLOADS = {
    "sphere1280": dict(r=3, leaf=32, eta=2.0, eps=1e-4, nrhs=1),
    "sphere5120": dict(r=4, leaf=32, eta=2.0, eps=1e-4, nrhs=1),
    "sphere20480": dict(r=5, leaf=64, eta=2.0, eps=1e-4, nrhs=16),
    "sphere81920": dict(r=6, leaf=64, eta=2.0, eps=1e-6, nrhs=64),
    # variants of Table 1 (Sec. 6.3): other eta values, the d = 1, 2 log kernels, and the
    # dense-only recursive structure of Sec. 6.2 (eta = 0: no admissible block)
    "sphere20480_eta1": dict(r=5, leaf=64, eta=1.0, eps=1e-4, nrhs=16),
    "sphere20480_eta0.5": dict(r=5, leaf=64, eta=0.5, eps=1e-4, nrhs=16),
    "line20480_eta0.5": dict(r=5, leaf=64, eta=0.5, eps=1e-4, nrhs=16, dim=1),
    "line20480_eta0.25": dict(r=5, leaf=64, eta=0.25, eps=1e-4, nrhs=16, dim=1),
    "circle20480_eta1": dict(r=5, leaf=64, eta=1.0, eps=1e-4, nrhs=16, dim=2),
    "circle20480_eta0.25": dict(r=5, leaf=64, eta=0.25, eps=1e-4, nrhs=16, dim=2),
    "dense5120": dict(r=4, leaf=64, eta=0.0, eps=1e-4, nrhs=16),
}

# Batches of independent problems: `count` ellipsoids, instance i drawn from seed i.
BATCHES = {
    "ellipsoids64": dict(count=64, levels=(3, 4), eps=(1e-4, 1e-6), leaf=32, eta=2.0),
    # 256 ellipsoids refined 3 to 5 times (n = 1280 .. 20480), all three axes uniform in [0.5, 2],
    # leaf 32 at every size
    "ellipsoids256": dict(count=256, levels=(3, 4, 5), eps=(1e-4, 1e-6), leaf=32, eta=2.0, leaf_large=32,
                          axes_range=(0.5, 2.0)),
}


def batch_specs(count, levels=(3, 4), eps=(1e-4, 1e-6), leaf=32, eta=2.0, leaf_large=64, axes_range=None):
    """Keyword arguments of build_problem for each instance of a batch.

    Instance i uses default_rng(i): refinement r uniform in `levels`, tolerance
    uniform in `eps`, ellipsoid axes (1, a, b) with a, b uniform in [0.4, 1]
    (or, with axes_range = (lo, hi), all three axes uniform in [lo, hi]), one
    right-hand side drawn from seed i.  Problems with r >= 5 (n >= 20480) use
    the leaf size `leaf_large`."""
    import numpy as np
    out = []
    for i in range(count):
        g = np.random.default_rng(i)
        r = int(g.choice(levels))
        e = float(g.choice(eps))
        if axes_range is None:
            a, b = (float(v) for v in g.uniform(0.4, 1.0, 2))
            axes = (1.0, round(a, 6), round(b, 6))
        else:
            axes = tuple(round(float(v), 6) for v in g.uniform(axes_range[0], axes_range[1], 3))
        out.append(dict(r=r, leaf=leaf_large if r >= 5 else leaf, eta=eta, eps=e, nrhs=1, seed=i, axes=axes))
    return out


# Request streams for the serving loop.
STREAMS = {
    "serve64": dict(requests=64, repeat=0.3, nrhs=(1, 64), levels=(3, 4), eps=(1e-4, 1e-6), leaf=32, eta=2.0),
    # with n = 20480 problems too (r = 5, leaf 64 as the single-problem workloads of that size use)
    "serve64r5": dict(requests=64, repeat=0.3, nrhs=(1, 64), levels=(3, 4, 5), eps=(1e-4, 1e-6), leaf=32, eta=2.0),
    # n from 1280 to 81920 (r uniform in 3..6), all three axes uniform in [0.5, 2]; the groups share
    # their product temporaries (temp_reuse) so that n = 81920 problems fit the budget several at a time
    "serve64r6": dict(requests=64, repeat=0.3, nrhs=(1, 64), levels=(3, 4, 5, 6), eps=(1e-4, 1e-6), leaf=32,
                      eta=2.0, axes_range=(0.5, 2.0), temp_reuse=1),
}


def stream_specs(requests, repeat=0.3, nrhs=(1, 64), seed=0, **batch_kw):
    """A seeded request stream: a list of (problem index, nrhs, rhs seed) and the build_problem
    keyword arguments of every distinct problem.  Each request repeats an earlier problem with
    probability `repeat` (uniform over those seen), else names a new one (problem i of
    batch_specs); nrhs is uniform in the closed range `nrhs`.  Arrival times are the caller's."""
    import numpy as np
    g = np.random.default_rng(seed)
    reqs, n_prob = [], 0
    for i in range(requests):
        if n_prob and g.random() < repeat:
            k = int(g.integers(n_prob))
        else:
            k, n_prob = n_prob, n_prob + 1
        reqs.append((k, int(g.integers(nrhs[0], nrhs[1] + 1)), 1000 + i))
    return reqs, batch_specs(n_prob, **batch_kw)
