"""Plain FP64 CPU oracle for the H-LU factorisation (test infrastructure only).

This package is the independent reference that the GPU library is checked
against.  Only the tests, the package's smoke check and the benchmark's CPU
baseline use it; the GPU library neither imports it nor shares any code with
it.  It is written for clarity, not speed: numpy arrays, recursion over the
block tree as the recursive 2 x 2 block LU of Sec. 3.1,
and library primitives (matmul, QR, SVD, triangular solve) as single steps.

Modules
  hmatrix   block tree built from the shared leaf arrays; densify, H x dense
  dense     hand-written unpivoted LU and triangular solves (Sec. 3.1 "Dense blocks")
  hlu       the H-LU recursion, triangular solves on H-matrices, truncated
            products and rounded addition (Sec. 3.1 "Low-rank blocks")
  errors    factorisation and solve error estimates (power iteration)
"""
from .hmatrix import HBlock, build_hmatrix, densify  # noqa: F401
from .hlu import HLUOracle, Counters  # noqa: F401
