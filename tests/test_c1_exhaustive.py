"""Config 1's exhaustive check (reading c-14): the induced subgraph on the
first 16 nodes reached by BFS from node 0 of the seeded 100-node 3-regular
graph.  Its independence number is fixed two independent ways (enumeration
of all 2^16 binary points of the MIS QUBO, and branch and bound), and the
FP64 oracle's own CPRA run of config 1's settings (S = 8 penalty shots
lambda = 1..8, width 16, Adam 1e-3, gamma -2 -> 0.1 over 3000 steps,
alpha = 2) reaches it.  The GPU run on the same subgraph is in
test_gpu_c1.py."""
import numpy as np

from oracle import cpra_oracle as O
from oracle import exact as X
from paper_2402_02190_gb300 import inputs as I


def c1_subgraph():
    rp, col = I.random_regular_graph(100, 3, seed=1)
    return I.bfs_induced_subgraph(rp, col, 16, root=0)


def test_c1_subgraph_independence_number_two_ways():
    rp, col = c1_subgraph()
    assert len(rp) - 1 == 16
    adj = X.adjacency_sets(rp, col)
    # every binary point: the QUBO with lambda = 1 equals -|x| exactly when x
    # is independent, so the largest such |x| is alpha(G)
    enum = max(int(x.sum()) for x in X.all_binary(16) if X.mis_qubo_direct(adj, x, 1.0) == -x.sum())
    assert enum == X.max_independent_set_size(adj) == 10


def oracle_cpra_run(rp, col, T=3000, seed=1, eval_every=50):
    """Config 1's CPRA run in FP64 (plain oracle steps); returns the best
    feasible set size seen at the evaluations and the last evaluation."""
    g = O.Graph(rp, col)
    N, S, H = len(rp) - 1, 8, 16
    lam = I.lambda_linspace(1.0, 8.0, S).astype(np.float64)
    theta, X0 = I.seeded_params(N, H, H, S, seed=seed)
    th, x0, st = theta.astype(np.float64), X0.astype(np.float64), None
    best = -1
    for t in range(T):
        cfg = dict(H0=H, H1=H, S=S, problem=O.MIS, alpha=2, lam=lam,
                   gamma=O.gamma_schedule(t, T, -2.0, 0.1), nu=0.0, div_kind=O.DIV_STD,
                   lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, train_embedding=True)
        out = O.step(g, th, x0, cfg, t=t + 1, adam_state=st)
        th, x0, st = out["theta_next"], out["X0_next"], out["adam_next"]
        if (t + 1) % eval_every == 0:
            ev = out["eval"]
            ok = ev["violations"] == 0
            if ok.any():
                best = max(best, int(ev["objective"][ok].max()))
    return best, out


def test_oracle_cpra_reaches_the_independence_number_of_the_c1_subgraph():
    rp, col = c1_subgraph()
    adj = X.adjacency_sets(rp, col)
    best, out = oracle_cpra_run(rp, col)
    assert best == 10
    # every rounded shot without violations is an independent set (edge by edge)
    X_ = out["X"]
    for s in np.flatnonzero(out["eval"]["violations"] == 0):
        assert all(not (X_[i, s] and X_[j, s]) for i in range(16) for j in adj[i])
