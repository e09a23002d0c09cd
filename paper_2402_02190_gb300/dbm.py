"""Diverse bipartite matching runs (App. problem specification, Eq.
matching-cost-function): the penalty-grid run on one instance (the DBM
experiment of the penalty-diversified section, S = 11 x 11 penalty vectors)
and multi-instance CPRA (App. multi-instance: one instance per shot, one
penalty vector), with the exact optimum that their approximation ratio
(ApR = reward of the best feasible matching found / optimal reward) is
measured against.  The library does the work; this module arranges the
shots and solves the reference problem with scipy's mixed-integer solver.
"""
from __future__ import annotations

import time

import numpy as np

from . import cpra
from . import inputs as I


def best_diverse_matching(C, M, N1: int, N2: int, p: float, q: float, time_limit: float = 120.0):
    """Optimal reward of the matching problem behind Eq. matching-cost-function
    with its constraints kept hard: maximise sum C x over x in {0,1}^(N1 x N2)
    with at most one pair per row and per column, at least a share p of the
    pairs across fields (sum M x >= p sum x) and at least a share q within a
    field (sum (1 - M) x >= q sum x).  C, M: [N1 * N2] in node order i*N2 + j.
    Returns (value, x) with x int [N1 * N2]."""
    from scipy.optimize import Bounds, LinearConstraint, milp
    from scipy.sparse import lil_matrix

    N = N1 * N2
    C = np.asarray(C, np.float64)
    M = np.asarray(M, np.float64)
    A = lil_matrix((N1 + N2 + 2, N))
    for i in range(N1):
        A[i, i * N2:(i + 1) * N2] = 1.0
    for j in range(N2):
        A[N1 + j, j::N2] = 1.0
    A[N1 + N2, :] = M - p                # sum (M - p) x >= 0
    A[N1 + N2 + 1, :] = (1.0 - M) - q    # sum (1 - M - q) x >= 0
    lb = np.concatenate([np.full(N1 + N2, -np.inf), [0.0, 0.0]])
    ub = np.concatenate([np.ones(N1 + N2), [np.inf, np.inf]])
    res = milp(-C, constraints=LinearConstraint(A.tocsr(), lb, ub), integrality=np.ones(N),
               bounds=Bounds(0, 1), options={"time_limit": time_limit})
    if res.x is None:
        raise RuntimeError(f"MILP failed: {res.message}")
    x = np.round(res.x).astype(np.int64)
    return float((C * x).sum()), x


def penalty_grid_shots(N1: int, N2: int, C, M, p: float, q: float, n: int = 11):
    """Shots of the penalty-grid run: one instance, lambda_s = (a, a, b, b) with
    a, b in {2^0, ..., 2^(n-1)}.  Returns (C, M, lam4, pq) for cpra_set_dbm."""
    return I.dbm_shots(N1, N2, [(C, M)], I.dbm_lambda_grid(n), (p, q))


def multi_instance_shots(N1: int, N2: int, instances, lam=(2.0, 2.0, 12.0, 12.0), pq=(0.25, 0.25)):
    """Shots of multi-instance CPRA: shot s solves instance s with one penalty
    vector (the App. multi-instance run uses (2, 2, 12, 12))."""
    S = len(instances)
    return I.dbm_shots(N1, N2, instances, np.tile(np.asarray(lam, np.float32), (S, 1)), pq)


def run(rp, col, N1: int, N2: int, shots, H: int, max_steps: int, eval_every: int,
        precision: int = cpra.BF16, seed: int = 1, preset: dict | None = None):
    """One CPRA run over the given shots (C, M, lam4, pq) with the paper's
    optimiser and schedule (cpra.paper_preset) unless `preset` overrides it.
    Returns the per-shot best feasible records, the early-stopping step and
    the wall time."""
    import torch
    C, M, lam4, pq = shots
    S = lam4.shape[0]
    kw = cpra.paper_preset(cpra.DBM, max_steps)
    if preset:
        kw.update(preset)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = cpra.Solver(rp, col, problem=cpra.DBM, S=S, H0=H, H1=H, precision=precision, seed=seed, **kw)
    s.set_dbm(N1, C, M, lam4, pq)
    best, best_step = s.solve(max_steps, eval_every)
    stop = s.early_stop_step()
    steps_run = int(s.get(cpra.T_STEP)[0])
    s.close()
    torch.cuda.synchronize()
    return dict(best=best, best_step=best_step, stop=stop, steps_applied=steps_run,
                seconds=time.perf_counter() - t0)


def apr(best, optimum):
    """Per-shot ApR of cpra_solve's best records (nan where no feasible
    matching was seen) against per-shot optima."""
    v = np.where(best["objective"] >= 0, best["value"], np.nan)
    return v / np.asarray(optimum, np.float64)
