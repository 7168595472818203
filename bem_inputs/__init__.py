"""Seeded synthetic inputs: BEM H-matrices on refined icosahedra / ellipsoids.

This package generates data only (mesh, cluster tree, block tree, compressed
leaves, right-hand sides).  It holds none of the H-LU arithmetic and is the one
module that both the CPU oracle and the GPU library consume.
"""
from .problem import Problem, build_problem  # noqa: F401
from .assemble import kernel_block  # noqa: F401
from .mesh import icosphere, ellipsoid, triangle_data  # noqa: F401

# Named workloads (icosphere refinement r, leaf size, eta, eps, rhs count).
WORKLOADS = {
    "sphere1280": dict(r=3, leaf=32, eta=2.0, eps=1e-4, nrhs=1),
    "sphere5120": dict(r=4, leaf=32, eta=2.0, eps=1e-4, nrhs=1),
    "sphere20480": dict(r=5, leaf=64, eta=2.0, eps=1e-4, nrhs=16),
    "sphere81920": dict(r=6, leaf=64, eta=2.0, eps=1e-6, nrhs=64),
}
