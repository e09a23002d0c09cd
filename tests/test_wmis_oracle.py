"""Pins of the oracle's weighted MIS (the task family of the paper's
two-stage experiment) and of its head-only step (the fine-tuning stage)."""
import itertools

import numpy as np
import pytest

from oracle import cpra_oracle as O
from oracle import exact as X
from paper_2402_02190_gb300 import inputs as I


def _g(N, d, seed):
    rp, col = I.random_regular_graph(N, d, seed)
    return O.Graph(rp, col), rp, col


@pytest.mark.parametrize("N,d,seed", [(10, 3, 1), (12, 4, 3)])
def test_weighted_relaxation_equals_direct_qubo(N, d, seed):
    g, rp, col = _g(N, d, seed)
    adj = X.adjacency_sets(rp, col)
    xs = np.array(list(X.all_binary(N))).T.astype(np.float64)       # N x 2^N
    S = xs.shape[1]
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.0, 1.0, size=(N, S))
    lam = np.resize([0.5, 2.0, 7.0], S)
    t = O.loss_terms(g, xs, lam, O.WMIS, 2, weights=W)
    assert np.all(t["ann"] == 0.0)
    for s in range(0, S, 7):
        x = xs[:, s].astype(int)
        viol = sum(1 for i in range(N) for j in adj[i] if i < j and x[i] and x[j])
        want = -float((W[:, s] * x).sum()) + lam[s] * viol
        assert t["cost"][s] + lam[s] * t["pen"][s] == pytest.approx(want, abs=1e-12)


@pytest.mark.parametrize("N,d,seed", [(12, 3, 2), (13, 4, 6)])
def test_min_weighted_qubo_is_minus_max_weight_independent_set(N, d, seed):
    """With lambda above every weight the QUBO minimum is minus the heaviest
    independent set, found here by enumerating node subsets directly."""
    g, rp, col = _g(N, d, seed)
    adj = X.adjacency_sets(rp, col)
    w = np.random.default_rng(seed).uniform(0.1, 1.0, size=N)
    best = 0.0
    for r in range(N + 1):
        for sub in itertools.combinations(range(N), r):
            ss = set(sub)
            if all(j not in ss for i in sub for j in adj[i]):
                best = max(best, float(w[list(sub)].sum()))
    xs = np.array(list(X.all_binary(N))).T.astype(np.float64)
    S = xs.shape[1]
    W = np.repeat(w[:, None], S, axis=1)
    lam = np.full(S, 2.0)
    t = O.loss_terms(g, xs, lam, O.WMIS, 2, weights=W)
    assert (t["cost"] + lam * t["pen"]).min() == pytest.approx(-best, abs=1e-12)
    ev = O.integer_eval(g, xs.astype(np.int64), lam, O.WMIS, weights=W)
    ok = ev["violations"] == 0
    assert ev["value"][ok].max() == pytest.approx(best, abs=1e-12)


def test_unit_weights_reduce_to_mis():
    g, rp, col = _g(30, 3, 4)
    rng = np.random.default_rng(1)
    P = rng.uniform(0.05, 0.95, size=(30, 6))
    lam = np.linspace(1, 3, 6)
    W = np.ones_like(P)
    a = O.loss_terms(g, P, lam, O.MIS, 2)
    b = O.loss_terms(g, P, lam, O.WMIS, 2, weights=W)
    for k in ("cost", "pen", "ann"):
        assert np.allclose(a[k], b[k], rtol=0, atol=1e-12)
    assert np.allclose(O.grad_P(g, P, lam, O.MIS, 2, 0.3, 0.2),
                       O.grad_P(g, P, lam, O.WMIS, 2, 0.3, 0.2, weights=W), rtol=0, atol=1e-12)
    x = (P > 0.5).astype(np.int64)
    ea, eb = O.integer_eval(g, x, lam, O.MIS), O.integer_eval(g, x, lam, O.WMIS, weights=W)
    assert np.array_equal(ea["objective"], eb["objective"])
    assert np.allclose(ea["qubo"], eb["qubo"]) and np.allclose(eb["value"], ea["objective"])


def test_weighted_grad_matches_finite_differences():
    rp, col = I.erdos_renyi_graph(15, 0.3, seed=8)
    g = O.Graph(rp, col)
    rng = np.random.default_rng(3)
    S = 5
    P = rng.uniform(0.05, 0.95, size=(15, S))
    W = rng.uniform(0.0, 2.0, size=(15, S))
    lam = np.linspace(1, 4, S)

    def R(Pm):
        t = O.loss_terms(g, Pm, lam, O.WMIS, 4, O.DIV_STD, W)
        return O.total_loss(t, lam, 0.7, 0.4, O.WMIS)

    G = O.grad_P(g, P, lam, O.WMIS, 4, 0.7, 0.4, O.DIV_STD, W)
    h = 1e-6
    fd = np.zeros_like(P)
    for idx in np.ndindex(*P.shape):
        a = P.copy(); a[idx] += h
        b = P.copy(); b[idx] -= h
        fd[idx] = (R(a) - R(b)) / (2 * h)
    assert np.linalg.norm(G - fd) <= 1e-7 * np.linalg.norm(fd)


def test_head_only_step_keeps_the_encoder():
    rp, col = I.random_regular_graph(40, 3, seed=5)
    g = O.Graph(rp, col)
    N, H, S = 40, 8, 6
    theta, X0 = I.seeded_params(N, H, H, S, seed=2)
    W = np.random.default_rng(0).uniform(0, 1, size=(N, S))
    cfg = dict(H0=H, H1=H, S=S, problem=O.WMIS, alpha=2, lam=np.full(S, 2.0), gamma=0.1, nu=0.0,
               div_kind=O.DIV_STD, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0,
               weights=W)
    full = O.step(g, theta, X0, cfg, t=1)
    head = O.step(g, theta, X0, dict(cfg, train_encoder=False), t=1)
    h0 = 2 * H * H + H
    assert np.array_equal(head["theta_next"][:h0], theta[:h0].astype(np.float64))
    assert np.array_equal(head["theta_next"][h0:], full["theta_next"][h0:])
    assert np.array_equal(head["X0_next"], np.asarray(X0, np.float64))
