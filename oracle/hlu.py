"""The H-LU factorisation of Sec. 3.1, written as the textbook recursive block
LU (test infrastructure only).

A partitioned diagonal block [[A00, A01], [A10, A11]] is factorised by the
standard 2 x 2 block LU recursion: factor A00, solve the two off-diagonal
panels with its triangular factors (L00^{-1} A01 and A10 U00^{-1}), subtract
the Schur product L10 U01 from A11 and factor what remains.  A dense leaf is
factorised by unpivoted LU.  The triangular solves recurse the same way
through the structure of the solved block: a low-rank block is solved on one
of its factors only (U for L^{-1} X, V for X U^{-1}), a dense block by
substitution through the H-structure of the triangular factor, and a
partitioned block by the block substitution first son, Schur update, second
son.

Products and additions (Sec. 3.1): a product with a low-rank factor stays
factorised, Z (U V^T) = (Z U) V^T and (U V^T) Z = U (Z^T V)^T.  Adding to a
low-rank target is rounded addition: stack the factors, take the SVD of the
sum and drop the small singular values.  A product of two dense or partitioned
blocks is written in factorised form too (an identity factor on the side of
its leaf cluster), so a dense contribution to a low-rank target is converted
by the same rounded addition.

Readings where the paper is silent (each one is listed in the design notes):
  * truncation rule: keep sigma_i > eps * sigma_1 (strict), rank 0 if sigma_1 = 0;
  * one truncation per (addmul call, low-rank target leaf): addmul recurses while
    A and B are both partitioned; otherwise the exact product A B is formed
    (factorised when A or B is low rank, dense otherwise), restricted to each
    leaf of C, and added once;
  * a low-rank target C with two partitioned factors is split into a temporary
    2 x 2 block of low-rank sons (restrictions of its factors), the recursion
    continues on the sons, and the sons are merged back into C by one rounded
    addition of their zero-padded factors ("split" reading, the default);
  * the same target under the plain definition (reading="plain"): the exact
    product A B is formed densely, restricted to C, and C := T_eps(C + alpha A B)
    is the truncated SVD of the exact dense sum, one truncation per target leaf;
  * the factor Sigma of a truncated block is kept in U (U <- Q_u X Sigma, V <- Q_v Y).
"""
from __future__ import annotations

import collections

import numpy as np

from .dense import lu_nopiv, solve_unit_lower, solve_upper_right
from .hmatrix import HBlock, build_hmatrix, densify, hmul, hmul_t


def qr_flops(m, K):
    """Model flops of a Householder QR of an m x K panel: 2 a b^2 - 2 b^3 / 3 with
    a = max(m, K), b = min(m, K) (Golub and Van Loan)."""
    a, b = max(m, K), min(m, K)
    return 2.0 * a * b * b - 2.0 * b ** 3 / 3.0


class Counters:
    """Model flop counts (standard operation counts) and event statistics."""

    def __init__(self):
        self.flops = collections.Counter()
        self.events = collections.Counter()
        self.trunc_K = collections.Counter()
        self.trunc_rank = collections.Counter()
        self.min_pivot = np.inf

    def total(self):
        return float(sum(self.flops.values()))


class HLUOracle:
    """Plain FP64 H-LU of a shared-input problem.  After factor(), self.A holds
    L (strictly below the diagonal, unit diagonal implied) and U (on and above)
    in the block structure of the input."""

    def __init__(self, problem, eps, hm=None, reading="split"):
        if reading not in ("split", "plain"):
            raise ValueError(f"unknown reading {reading!r}")
        self.problem = problem
        self.eps = float(eps)
        self.reading = reading
        self.A = build_hmatrix(problem) if hm is None else hm
        self.c = Counters()

    # ----------------------------------------------------------- recursion
    def factor(self):
        self.lu(self.A)
        return self

    def lu(self, b):
        if b.kind == "dense":
            m = b.m
            piv = lu_nopiv(b.D)
            self.c.flops["getrf"] += 2.0 * m ** 3 / 3.0
            self.c.events["getrf"] += 1
            if not np.all(np.isfinite(piv)) or np.any(piv == 0.0):
                raise FloatingPointError(f"zero or non-finite pivot in leaf {b.leaf_id}")
            self.c.min_pivot = min(self.c.min_pivot, float(np.min(piv)))
            return
        if b.kind != "part":
            raise ValueError("low-rank diagonal block")
        (a00, a01), (a10, a11) = b.sons
        self.lu(a00)
        self.trsm_l(a00, a01)
        self.trsm_u(a00, a10)
        self.addmul(a11, -1.0, a10, a01)
        self.lu(a11)

    # ------------------------------------------------ triangular solves
    def trsm_l(self, L, X):
        """X := L^{-1} X, L the unit lower part of the factored diagonal block."""
        if X.kind == "lowrank":
            self.trsm_l_panel(L, X.U)
        elif X.kind == "dense":
            self.trsm_l_panel(L, X.D)
        else:
            (l00, _), (l10, l11) = L.sons
            for j in (0, 1):
                self.trsm_l(l00, X.sons[0][j])
            for j in (0, 1):
                self.addmul(X.sons[1][j], -1.0, l10, X.sons[0][j])
            for j in (0, 1):
                self.trsm_l(l11, X.sons[1][j])

    def trsm_u(self, U, X):
        """X := X U^{-1}, U the upper part of the factored diagonal block."""
        if X.kind == "lowrank":
            self.trsm_u_panel(U, X.V.T)  # (U_x V_x^T) U^{-1} = U_x (V_x^T U^{-1})
        elif X.kind == "dense":
            self.trsm_u_panel(U, X.D)
        else:
            (u00, u01), (_, u11) = U.sons
            for i in (0, 1):
                self.trsm_u(u00, X.sons[i][0])
            for i in (0, 1):
                self.addmul(X.sons[i][1], -1.0, X.sons[i][0], u01)
            for i in (0, 1):
                self.trsm_u(u11, X.sons[i][1])

    def trsm_l_panel(self, L, P):
        """P := L^{-1} P for a dense panel P (rows = L's rows), in place."""
        if L.kind == "dense":
            solve_unit_lower(L.D, P)
            self.c.flops["trsm"] += float(L.m) ** 2 * (P.shape[1] if P.ndim > 1 else 1)
            self.c.events["trsm"] += 1
            return
        (l00, _), (l10, l11) = L.sons
        m0 = l00.m
        self.trsm_l_panel(l00, P[:m0])
        P[m0:] -= self._hmul(l10, P[:m0])
        self.trsm_l_panel(l11, P[m0:])

    def trsm_u_panel(self, U, P):
        """P := P U^{-1} for a dense panel P (columns = U's columns), in place."""
        if U.kind == "dense":
            solve_upper_right(U.D, P)
            self.c.flops["trsm"] += float(U.m) ** 2 * P.shape[0]
            self.c.events["trsm"] += 1
            return
        (u00, u01), (_, u11) = U.sons
        n0 = u00.n
        self.trsm_u_panel(u00, P[:, :n0])
        P[:, n0:] -= self._hmul_t(u01, P[:, :n0].T).T
        self.trsm_u_panel(u11, P[:, n0:])

    # ---------------------------------------------------------- products
    def _hmul(self, b, x):
        self._count_hmul(b, x.shape[1] if x.ndim > 1 else 1)
        return hmul(b, x)

    def _hmul_t(self, b, x):
        self._count_hmul(b, x.shape[1] if x.ndim > 1 else 1)
        return hmul_t(b, x)

    def _count_hmul(self, b, p):
        for leaf in b.leaves():
            if leaf.kind == "dense":
                self.c.flops["gemm"] += 2.0 * leaf.m * leaf.n * p
            else:
                self.c.flops["lrmul"] += 2.0 * (leaf.m + leaf.n) * leaf.rank * p

    def product(self, A, B):
        """Exact A B for aligned blocks as factors (U, V), A B = U V^T.

        Sec. 3.1: a product with a low-rank factor stays factorised,
        (U_a V_a^T) B = U_a (B^T V_a)^T and A (U_b V_b^T) = (A U_b) V_b^T.  A
        product of two non-low-rank blocks is written with an identity factor
        on the side of a leaf cluster (or as the pair of dense factors when
        the inner dimension is the smallest), so every contribution reaches
        its target in factorised form."""
        if A.kind == "lowrank":
            self.c.events["prod_lr_left"] += 1
            return A.U, self._hmul_t(B, A.V)
        if B.kind == "lowrank":
            self.c.events["prod_lr_right"] += 1
            return self._hmul(A, B.U), B.V
        t, r, s = A.m, A.n, B.n
        if A.kind == "dense" and B.kind == "dense" and r <= min(t, s):
            self.c.events["prod_dense_dense"] += 1
            return A.D, B.D.T
        if A.kind == "dense" and (B.kind == "part" or t <= s):
            self.c.events["prod_dense_left"] += 1
            return np.eye(t), self._hmul_t(B, A.D.T)
        self.c.events["prod_dense_right"] += 1
        return self._hmul(A, B.D), np.eye(s)

    def addmul(self, C, alpha, A, B):
        """C := C + alpha A B with truncation at low-rank leaves of C."""
        if self.reading == "plain" and A.kind == "part" and B.kind == "part":
            # plain definition: the exact product, formed densely, is distributed over the
            # leaves of C; each low-rank leaf is truncated once, by the SVD of its exact sum
            P = densify(A) @ densify(B)
            self.c.flops["gemm"] += 2.0 * A.m * A.n * B.n
            self.c.events["prod_dense_exact"] += 1
            self.add_dense_into(C, alpha, P)
            return
        if A.kind == "part" and B.kind == "part":
            if C.kind == "part":
                for i in (0, 1):
                    for j in (0, 1):
                        for k in (0, 1):
                            self.addmul(C.sons[i][j], alpha, A.sons[i][k], B.sons[k][j])
                return
            if C.kind == "lowrank":
                # low-rank target, both factors partitioned: descend into a
                # temporary 2 x 2 split of the target and merge it back
                S = self.split_lowrank(C, A, B)
                for i in (0, 1):
                    for j in (0, 1):
                        for k in (0, 1):
                            self.addmul(S.sons[i][j], alpha, A.sons[i][k], B.sons[k][j])
                C.U, C.V = self.merge_lowrank(C, S)
                return
        P = self.product(A, B)
        self.add_into(C, alpha, P, 0, 0)

    def split_lowrank(self, C, A, B):
        """Temporary partitioned copy of a low-rank block: son (i, j) holds the
        restriction U[rows_i] V[cols_j]^T of its factors."""
        S = HBlock(C.t, C.s, C.r0, C.m, C.c0, C.n)
        S.kind = "part"
        S.sons = [[None, None], [None, None]]
        for i in (0, 1):
            for j in (0, 1):
                a, b = A.sons[i][0], B.sons[0][j]
                s = HBlock(a.t, b.s, a.r0, a.m, b.c0, b.n)
                s.kind = "lowrank"
                s.U = C.U[a.r0 - C.r0:a.r0 - C.r0 + a.m].copy()
                s.V = C.V[b.c0 - C.c0:b.c0 - C.c0 + b.n].copy()
                S.sons[i][j] = s
        self.c.events["split"] += 1
        return S

    def merge_lowrank(self, C, S):
        """Rounded addition of the four zero-padded sons back into one block."""
        us, vs = [], []
        for row in S.sons:
            for s in row:
                u = np.zeros((C.m, s.rank))
                v = np.zeros((C.n, s.rank))
                u[s.r0 - C.r0:s.r0 - C.r0 + s.m] = s.U
                v[s.c0 - C.c0:s.c0 - C.c0 + s.n] = s.V
                us.append(u)
                vs.append(v)
        self.c.events["merge"] += 1
        return self.rounded_add(np.hstack(us), np.hstack(vs))

    def add_dense_into(self, C, alpha, P):
        """C := C + alpha P for a dense C.m x C.n array P: added exactly to dense leaves, and to a
        low-rank leaf as T_eps(C + alpha P) of the dense sum."""
        if C.kind == "part":
            for row in C.sons:
                for s in row:
                    self.add_dense_into(s, alpha, P[s.r0 - C.r0:s.r0 - C.r0 + s.m, s.c0 - C.c0:s.c0 - C.c0 + s.n])
        elif C.kind == "dense":
            C.D += alpha * P
            self.c.events["add_dense"] += 1
        else:
            C.U, C.V = self.truncate_dense(C.U @ C.V.T + alpha * P)

    def add_into(self, C, alpha, P, r, c):
        """Add alpha * (U V^T)[r:r+C.m, c:c+C.n] to C (exact product restricted to C)."""
        U, V = P
        if C.kind == "part":
            for row in C.sons:
                for s in row:
                    self.add_into(s, alpha, P, r + s.r0 - C.r0, c + s.c0 - C.c0)
            return
        Up = U[r:r + C.m]
        Vp = V[c:c + C.n]
        if C.kind == "dense":
            C.D += alpha * (Up @ Vp.T)
            self.c.flops["lrexpand"] += 2.0 * C.m * C.n * Up.shape[1]
            self.c.events["add_dense"] += 1
        else:
            C.U, C.V = self.rounded_add(np.hstack([C.U, alpha * Up]), np.hstack([C.V, Vp]))

    # ------------------------------------------------ rounded addition
    def _keep(self, sig):
        if sig.size == 0 or sig[0] == 0.0:
            return 0
        return int(np.count_nonzero(sig > self.eps * sig[0]))

    def truncate_dense(self, X):
        """T_eps of a dense block by its SVD (the plain definition of the rounded addition):
        X = Q_1 diag(sigma) Q_2^T, keep the sigma_i > eps * sigma_1, U = Q_1 Sigma, V = Q_2."""
        m, n = X.shape
        x, sig, yt = np.linalg.svd(X, full_matrices=False)
        k = self._keep(sig)
        self.c.flops["svd"] += 21.0 * max(m, n) * min(m, n) ** 2
        self.c.events["truncate_dense"] += 1
        self.c.trunc_K[min(m, n)] += 1
        self.c.trunc_rank[k] += 1
        return x[:, :k] * sig[:k], yt[:k].T.copy()

    def rounded_add(self, Us, Vs):
        """Truncated SVD of Us Vs^T from the stacked factors (Sec. 3.1):
        QR of both stacks, SVD of the small core R_u R_v^T, drop sigma_i <= eps*sigma_1."""
        m, K = Us.shape
        n = Vs.shape[0]
        qu, ru = np.linalg.qr(Us)
        qv, rv = np.linalg.qr(Vs)
        x, sig, yt = np.linalg.svd(ru @ rv.T)
        k = self._keep(sig)
        ku, kv = ru.shape[0], rv.shape[0]
        self.c.flops["qr"] += qr_flops(m, K) + qr_flops(n, K)
        self.c.flops["svd"] += 21.0 * max(ku, kv) ** 3
        self.c.flops["qx"] += 2.0 * (m * ku + n * kv) * k
        self.c.events["rounded_add"] += 1
        self.c.trunc_K[K] += 1
        self.c.trunc_rank[k] += 1
        return qu @ (x[:, :k] * sig[:k]), qv @ yt[:k].T
