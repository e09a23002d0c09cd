"""Exact combinatorial solvers for tiny graphs (TEST INFRASTRUCTURE ONLY).

Used to pin the oracle (brute-force enumeration over {0,1}^N) and for the
behavioural check that CPRA reaches the exact MIS on small RRGs (the N = 30,
d = 3 instances of the variation-diversified MIS experiment).  Only tests/
may import this module.
"""
from __future__ import annotations

import itertools

import numpy as np


def adjacency_sets(rowptr, col):
    N = len(rowptr) - 1
    return [set(int(c) for c in col[rowptr[i]:rowptr[i + 1]]) for i in range(N)]


def mis_qubo_direct(adj, x, lam):
    """-sum_i x_i + lam * #{edges with both ends 1}; edges read from the
    adjacency sets, each unordered pair once."""
    N = len(adj)
    size = sum(x)
    inside = 0
    for i in range(N):
        for j in adj[i]:
            if i < j and x[i] and x[j]:
                inside += 1
    return -size + lam * inside


def cut_size_direct(adj, x):
    N = len(adj)
    cut = 0
    for i in range(N):
        for j in adj[i]:
            if i < j and x[i] != x[j]:
                cut += 1
    return cut


def all_binary(N):
    for bits in itertools.product((0, 1), repeat=N):
        yield np.array(bits, dtype=np.int64)


def max_independent_set_size(adj):
    """Branch and bound on the highest-degree vertex (exact, N <= ~60)."""
    best = [0]

    def rec(cand: frozenset, size: int):
        if not cand:
            best[0] = max(best[0], size)
            return
        if size + len(cand) <= best[0]:
            return
        # vertex of maximum degree inside cand
        v = max(cand, key=lambda u: len(adj[u] & cand))
        if len(adj[v] & cand) == 0:
            # cand is independent
            best[0] = max(best[0], size + len(cand))
            return
        # branch 1: take v
        rec(cand - {v} - adj[v], size + 1)
        # branch 2: drop v
        rec(cand - {v}, size)

    rec(frozenset(range(len(adj))), 0)
    return best[0]


def max_cut_brute(adj):
    N = len(adj)
    best = 0
    for bits in itertools.product((0, 1), repeat=N - 1):
        x = (0,) + bits                  # fix x_0 = 0 (cut is symmetric)
        best = max(best, cut_size_direct(adj, x))
    return best
