"""Warm-start pipeline around the library's warm-start network (cpra_ws_*):
CPRA solves on seeded training graphs give rounded targets, the network is
fitted to them on disjoint unions of graphs, and its logits seed new CPRA
runs through cpra_set_init_logits.  Everything on the GPU runs in the
library's kernels; this module only arranges graphs and tensors.
"""
from __future__ import annotations

import time

import numpy as np

from . import cpra
from . import inputs as I


def disjoint_union(graphs):
    """CSR of the disjoint union of [(rowptr, col), ...] (node ids offset)."""
    rps, cols, off, eoff = [], [], 0, 0
    for k, (rp, col) in enumerate(graphs):
        rps.append((np.asarray(rp[:-1] if k < len(graphs) - 1 else rp, dtype=np.int64)) + eoff)
        cols.append(np.asarray(col, dtype=np.int64) + off)
        off += len(rp) - 1
        eoff += int(rp[-1])
    return np.concatenate(rps), np.concatenate(cols)


def training_graphs(n_graphs: int, seed: int, n_min: int = 1000, n_max: int = 10000,
                    degrees=(3, 5, 10)):
    """Seeded random d-regular graphs with N uniform in [n_min, n_max] (N d even)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_graphs):
        d = int(rng.choice(degrees))
        N = int(rng.integers(n_min, n_max + 1))
        if (N * d) % 2:
            N += 1
        rp, col = I.random_regular_graph(N, d, seed=seed * 100003 + k)
        out.append((rp, col, d))
    return out


def cpra_targets(rp, col, S: int, lam, steps: int, precision: int = cpra.BF16, H: int = 64,
                 seed: int = 1, problem: int = cpra.MIS):
    """Runs plain CPRA for `steps` steps and returns its rounded solution bits
    (uint32 [N, ceil(S/32)]) and the per-shot evaluation."""
    s = cpra.Solver(rp, col, lam=lam if problem == cpra.MIS else None, problem=problem, S=S,
                    H0=H, H1=H, precision=precision, gamma0=-2.0, gamma1=0.1,
                    schedule_steps=steps, seed=seed)
    for t in range(steps):
        s.step(t)
    rec, _, bits = s.round_eval(want_bits=True)
    s.close()
    return bits, rec


def cpra_targets_union(graphs, S: int, lam, steps: int, precision: int = cpra.BF16, H: int = 64,
                       seed: int = 1, max_nodes: int = 200_000, problem: int = cpra.MIS):
    """Plain CPRA on many graphs at once (the paper's multi-instance form):
    the graphs, in order, are packed into disjoint unions of at most
    `max_nodes` nodes, one CPRA run of `steps` steps solves each union (one
    network, one embedding row per node; union u uses seed + u), and the
    union's rounded bits are split back per graph.  Returns
    [bits (uint32 [N_k, ceil(S/32)])]."""
    out, group, nodes, unions = [], [], 0, [0]

    def flush():
        if not group:
            return
        rp, col = disjoint_union([(g[0], g[1]) for g in group])
        bits, _ = cpra_targets(rp, col, S, lam, steps, precision, H=H, seed=seed + unions[0],
                               problem=problem)
        unions[0] += 1
        off = 0
        for g in group:
            n = len(g[0]) - 1
            out.append(np.ascontiguousarray(bits[off:off + n]))
            off += n

    for g in graphs:
        n = len(g[0]) - 1
        if group and nodes + n > max_nodes:
            flush()
            group, nodes = [], 0
        group.append(g)
        nodes += n
    flush()
    return out


def mis_best_from_bits(rp, col, bits, S: int) -> int:
    """Largest MIS size among the shots of packed solution bits that have no
    violated edge (host arithmetic, for reports on small graphs)."""
    bits = np.asarray(bits).view(np.uint32)
    x = np.zeros((bits.shape[0], S), dtype=bool)
    for s in range(S):
        x[:, s] = (bits[:, s // 32] >> np.uint32(s % 32)) & np.uint32(1)
    ei, ej = I.csr_to_edges(np.asarray(rp), np.asarray(col))
    viol = (x[ei] & x[ej]).sum(axis=0)
    size = x.sum(axis=0)
    ok = viol == 0
    return int(size[ok].max()) if ok.any() else -1


def train_network(net, dataset, epochs: int, batch_graphs: int, seed: int = 0, device="cuda"):
    """Fits the network on disjoint unions of `batch_graphs` training graphs.
    dataset: [(rowptr, col, bits, graph_seed)].  Returns the per-epoch mean loss."""
    import torch
    rng = np.random.default_rng(seed)
    losses = []
    # features of each graph are fixed by its graph seed (computed once)
    feats = []
    for rp, col, bits, gs in dataset:
        rpd = torch.from_numpy(rp.astype(np.int32)).to(device)
        feats.append(net.features(rpd, gs).cpu())
    for ep in range(epochs):
        order = rng.permutation(len(dataset))
        ep_loss = []
        for b in range(0, len(order), batch_graphs):
            idx = order[b:b + batch_graphs]
            rp, col = disjoint_union([(dataset[k][0], dataset[k][1]) for k in idx])
            X = torch.cat([feats[k] for k in idx]).to(device)
            bits = np.concatenate([dataset[k][2] for k in idx])
            t = dict(rp=torch.from_numpy(rp.astype(np.int32)).to(device),
                     col=torch.from_numpy(col.astype(np.int32)).to(device),
                     bits=torch.from_numpy(np.ascontiguousarray(bits).view(np.int32)).to(device))
            ep_loss.append(net.train_step(t["rp"], t["col"], X, t["bits"]))
        losses.append(float(np.mean(ep_loss)))
    return losses


def predict_logits(net, rp, col, graph_seed: int, device="cuda"):
    import torch
    rpd = torch.from_numpy(np.asarray(rp, dtype=np.int32)).to(device)
    cold = torch.from_numpy(np.asarray(col, dtype=np.int32)).to(device)
    X = net.features(rpd, graph_seed)
    return net.predict(rpd, cold, X)


def best_feasible(rec, problem=cpra.MIS) -> int:
    """Largest objective over shots (MIS: among shots without violations)."""
    if problem == cpra.MAXCUT:
        return int(rec["objective"].max())
    ok = rec["violations"] == 0
    return int(rec["objective"][ok].max()) if ok.any() else -1


def run_trace(rp, col, S: int, lam, steps: int, eval_every: int, precision: int,
              init_logits=None, gamma0: float = -2.0, gamma1: float = 0.1, H: int = 64,
              seed: int = 1, problem: int = cpra.MIS, t0=None, final_terms=None):
    """A CPRA run that records (wall seconds since t0, step, running best
    feasible objective) at every evaluation.  Context creation and the
    warm-start offset upload are inside the timed span.  If `final_terms`
    is a list, the last step's loss terms (cost_s, pen_s, ann_s per shot,
    then Psi) are appended to it."""
    import torch
    if t0 is None:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
    s = cpra.Solver(rp, col, lam=lam if problem == cpra.MIS else None, problem=problem, S=S,
                    H0=H, H1=H, precision=precision, gamma0=gamma0, gamma1=gamma1,
                    schedule_steps=steps, seed=seed, recompute=1 if len(rp) > 100_001 else 0)
    if init_logits is not None:
        s.set_init_logits(init_logits)
    trace = []
    best = -1
    for t in range(steps):
        terms = s.step(t, want_terms=final_terms is not None and t == steps - 1)
        if terms is not None and final_terms is not None:
            final_terms.append(terms)
        if (t + 1) % eval_every == 0 or t == steps - 1:
            rec, _, _ = s.round_eval()
            best = max(best, best_feasible(rec, problem))
            trace.append((time.perf_counter() - t0, t + 1, best))
    s.close()
    return trace


def time_to_reach(trace, target):
    """First (seconds, steps) at which the running best reaches target, or None."""
    for sec, step, best in trace:
        if best >= target:
            return sec, step
    return None


def binarised_fraction(terms, N: int, S: int) -> float:
    """How far a run has binarised, from its annealing terms: 1 minus the mean
    of 1 - (2P-1)^2 over all N x S entries (1 = every P at 0 or 1, 0 = every P
    at 1/2).  terms: cpra_step's loss terms (ann_s at [2S, 3S))."""
    ann = np.asarray(terms, dtype=np.float64)[2 * S:3 * S]
    return float(1.0 - ann.sum() / (N * S))
