"""Shared set-up of the GPU parity tests: run the library on a problem and
rebuild the oracle's block tree from the factors it returns."""
import copy

import numpy as np


def gpu_factor(p, eps=None, **kw):
    from paper_1906_00874_gb300 import HLU
    h = HLU.from_problem(p, **kw)
    h.factor(p.eps if eps is None else eps)
    return h


def factors_as_problem(p, h):
    rank, off, data = h.get_factors()
    q = copy.copy(p)
    q.rank, q.offset, q.data = rank, off, data
    return q


def rank_agreement(o, q):
    lr = [l for l in o.A.leaves() if l.kind == "lowrank"]
    same = sum(int(q.rank[l.leaf_id] == l.rank) for l in lr)
    return same, len(lr)
