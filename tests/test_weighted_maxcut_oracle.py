"""Pins of the oracle's weighted max-cut (Table objective-functions: the
MaxCut QUBO sum_{i<j} A_ij (2 x_i x_j - x_i - x_j) with edge weights A_ij),
checked against what the mathematics fixes: at every binary point the
relaxed cost is minus the cut weight counted edge by edge, its minimum over
{0,1}^N is minus the maximum cut weight found by enumeration, the integer
evaluation returns that cut weight, and the gradients match central finite
differences -- with positive and with signed (+-1) weights."""
import itertools

import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I


def _weighted_graph(N, d, seed, kind):
    rp, col = I.random_regular_graph(N, d, seed)
    w = I.seeded_edge_weights(rp, col, seed + 1, kind)
    return rp, col, w, O.Graph(rp, col, weights=w)


def _cut_weight(rp, col, w, x):
    """Weight of the cut of x, from the CSR rows (each edge once, i < j)."""
    total = 0.0
    for i in range(len(rp) - 1):
        for e in range(rp[i], rp[i + 1]):
            j = col[e]
            if i < j and x[i] != x[j]:
                total += float(w[e])
    return total


@pytest.mark.parametrize("kind", ["uniform", "pm1"])
def test_weights_are_symmetric(kind):
    rp, col, w, _ = _weighted_graph(40, 5, 3, kind)
    for i in range(40):
        for e in range(rp[i], rp[i + 1]):
            j = col[e]
            back = rp[j] + np.flatnonzero(col[rp[j]:rp[j + 1]] == i)[0]
            assert w[back] == w[e]


@pytest.mark.parametrize("kind", ["uniform", "pm1"])
def test_relaxation_is_minus_cut_weight_and_its_minimum_the_max_cut(kind):
    N = 10
    rp, col, w, g = _weighted_graph(N, 3, 5, kind)
    xs = np.array(list(itertools.product((0, 1), repeat=N)), dtype=np.float64).T  # N x 2^N
    t = O.loss_terms(g, xs, np.zeros(xs.shape[1]), O.MAXCUT, alpha=2)
    direct = np.array([_cut_weight(rp, col, w, xs[:, k]) for k in range(xs.shape[1])])
    assert np.allclose(t["cost"], -direct, rtol=0, atol=1e-12)
    assert t["cost"].min() == pytest.approx(-direct.max())
    assert np.all(t["ann"] == 0.0)
    ev = O.integer_eval(g, xs.astype(np.int64), None, O.MAXCUT)
    assert np.allclose(ev["value"], direct, rtol=0, atol=1e-12)
    assert np.array_equal(ev["qubo"], -ev["value"])
    cnt = np.array([sum(1 for i in range(N) for e in range(rp[i], rp[i + 1])
                        if i < col[e] and xs[i, k] != xs[col[e], k]) for k in range(xs.shape[1])])
    assert np.array_equal(ev["objective"], cnt)


@pytest.mark.parametrize("kind", ["uniform", "pm1"])
@pytest.mark.parametrize("div_kind", [O.DIV_STD, O.DIV_VAR])
def test_weighted_grad_P_matches_finite_differences(kind, div_kind):
    rp, col, w, g = _weighted_graph(14, 4, 9, kind)
    rng = np.random.default_rng(4)
    S = 4
    P = rng.uniform(0.05, 0.95, size=(14, S))
    lam = np.zeros(S)

    def R(Pm):
        t = O.loss_terms(g, Pm, lam, O.MAXCUT, 2, div_kind)
        return O.total_loss(t, lam, 0.7, 0.3, O.MAXCUT)

    G = O.grad_P(g, P, lam, O.MAXCUT, 2, 0.7, 0.3, div_kind)
    h = 1e-6
    fd = np.zeros_like(P)
    for idx in np.ndindex(*P.shape):
        a = P.copy(); a[idx] += h
        b = P.copy(); b[idx] -= h
        fd[idx] = (R(a) - R(b)) / (2 * h)
    assert np.linalg.norm(G - fd) <= 1e-7 * np.linalg.norm(fd)


def test_unit_weights_reduce_to_the_unweighted_graph():
    rp, col = I.random_regular_graph(30, 3, 2)
    g0 = O.Graph(rp, col)
    g1 = O.Graph(rp, col, weights=np.ones(len(col)))
    P = np.random.default_rng(1).uniform(size=(30, 6))
    a = O.loss_terms(g0, P, np.zeros(6), O.MAXCUT, 2)
    b = O.loss_terms(g1, P, np.zeros(6), O.MAXCUT, 2)
    assert np.array_equal(a["cost"], b["cost"])
    assert np.array_equal(O.grad_P(g0, P, np.zeros(6), O.MAXCUT, 2, 0.5, 0.0),
                          O.grad_P(g1, P, np.zeros(6), O.MAXCUT, 2, 0.5, 0.0))
