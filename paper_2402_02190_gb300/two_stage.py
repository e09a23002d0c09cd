"""Two-stage S' -> S schedule of the paper (Related work / continuous tensor
relaxation discussion and App. two-stage): a warm-up network with S' heads is
trained on the first S' tasks; its encoder (layer 1 and the node
embeddings) is then frozen and a fresh S-way head is trained alone on all S
tasks.  Both phases stop once the annealing term falls below a threshold.
The library does the work (weighted MIS, head-only training, the stopping
rule, graph-replayed steps); this module arranges the two contexts.
"""
from __future__ import annotations

import time

import numpy as np

from . import cpra


def _weighted_best(rec):
    """cpra_solve's best feasible weight per task (value -1: none seen) -> nan."""
    return np.where(rec["value"] >= 0.0, rec["value"], np.nan)


def _solve(s, steps, eval_every):
    best, best_step = s.solve(steps, eval_every)
    return best, best_step


def encoder_slice(H0: int, H1: int) -> int:
    """Length of the encoder block [Wcat1 | b1] at the front of the flat parameters."""
    return 2 * H1 * H0 + H1


def run_two_stage(rp, col, W, lam, S_pre: int, pre_steps: int, ft_steps: int, H: int = 64,
                  precision: int = cpra.BF16, eval_every: int = 100, ann_below: float = 1e-4,
                  lr: float = 1e-3, seed: int = 1):
    """W: node weights [N, S] of the S tasks; lam: penalty per task [S].
    Returns a dict with the per-task best feasible weight, phase times and
    the stopping steps."""
    import torch
    N, S = W.shape
    h0 = encoder_slice(H, H)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pre = cpra.Solver(rp, col, lam=lam[:S_pre], problem=cpra.WMIS, S=S_pre, H0=H, H1=H,
                      precision=precision, gamma0=-2.0, gamma1=2.0, schedule_steps=pre_steps,
                      es_ann_below=ann_below, lr=lr, seed=seed)
    pre.set_node_weights(W[:, :S_pre])
    pre_best, _ = _solve(pre, pre_steps, eval_every)
    pre_stop = pre.early_stop_step()
    enc = pre.get(cpra.T_THETA)[:h0].copy()
    emb = pre.get(cpra.T_EMB)
    pre.close()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ft = cpra.Solver(rp, col, lam=lam, problem=cpra.WMIS, S=S, H0=H, H1=H, precision=precision,
                     gamma0=0.1, gamma1=0.0, schedule_steps=ft_steps, es_ann_below=ann_below,
                     train_encoder=0, lr=lr, seed=seed + 1)
    th = ft.get(cpra.T_THETA)
    th[:h0] = enc                      # the trained encoder; the head stays fresh
    ft.set(cpra.T_THETA, th)
    ft.set(cpra.T_EMB, emb)
    ft.set_node_weights(W)
    ft_best, _ = _solve(ft, ft_steps, eval_every)
    ft_stop = ft.early_stop_step()
    enc_after = ft.get(cpra.T_THETA)[:h0]
    ft.close()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    v = _weighted_best(ft_best)
    return dict(pre_seconds=t1 - t0, ft_seconds=t2 - t1, total_seconds=t2 - t0,
                pre_stop=pre_stop, ft_stop=ft_stop, best=v,
                avg_weight=float(np.nanmean(v)) if np.isfinite(v).any() else float("nan"),
                feasible_tasks=int(np.isfinite(v).sum()),
                encoder_unchanged=bool(np.array_equal(enc_after, enc)),
                pre_best=_weighted_best(pre_best))


def run_scratch(rp, col, W, lam, steps: int, H: int = 64, precision: int = cpra.BF16,
                eval_every: int = 100, ann_below: float = 1e-4, lr: float = 1e-3, seed: int = 1):
    """The baseline: one network with all S heads trained from scratch with the
    warm-up schedule."""
    import torch
    N, S = W.shape
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = cpra.Solver(rp, col, lam=lam, problem=cpra.WMIS, S=S, H0=H, H1=H, precision=precision,
                    gamma0=-2.0, gamma1=2.0, schedule_steps=steps, es_ann_below=ann_below, lr=lr,
                    seed=seed)
    s.set_node_weights(W)
    best, _ = _solve(s, steps, eval_every)
    stop = s.early_stop_step()
    s.close()
    torch.cuda.synchronize()
    v = _weighted_best(best)
    return dict(total_seconds=time.perf_counter() - t0, stop=stop, best=v,
                avg_weight=float(np.nanmean(v)) if np.isfinite(v).any() else float("nan"),
                feasible_tasks=int(np.isfinite(v).sum()))
