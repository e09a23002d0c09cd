"""Pins of the oracle's diverse bipartite matching loss (Eq.
matching-cost-function): direct formula at binary points, brute-force
optimum, finite differences, violation counts, and the constraint graph."""
import itertools

import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I


def _inst(N1, N2, S, seed, p=0.25, q=0.25):
    rng = np.random.default_rng(seed)
    C = rng.random((N1 * N2, S))
    M = (rng.random((N1 * N2, S)) < 0.5).astype(np.float64)
    lam4 = rng.uniform(0.5, 4.0, size=(S, 4))
    pq = np.tile([p, q], (S, 1))
    return dict(N1=N1, N2=N2, C=C, M=M, lam4=lam4, pq=pq)


def _direct(x, C, M, lam, p, q, N1, N2):
    """l(x) of Eq. matching-cost-function written with explicit loops."""
    r = lambda v: v if v > 0 else 0.0
    X = [[x[i * N2 + j] for j in range(N2)] for i in range(N1)]
    val = -sum(C[i * N2 + j] * X[i][j] for i in range(N1) for j in range(N2))
    val += lam[0] * sum(r(sum(X[i]) - 1) for i in range(N1))
    val += lam[1] * sum(r(sum(X[i][j] for i in range(N1)) - 1) for j in range(N2))
    T = sum(sum(row) for row in X)
    U = sum(M[i * N2 + j] * X[i][j] for i in range(N1) for j in range(N2))
    val += lam[2] * r(p * T - U) + lam[3] * r(q * T - (T - U))
    return val


def _graph(N1, N2):
    rp, col = I.dbm_graph(N1, N2)
    return O.Graph(rp, col)


@pytest.mark.parametrize("N1,N2", [(2, 3), (3, 3)])
def test_relaxation_equals_direct_formula_at_binary_points(N1, N2):
    N = N1 * N2
    xs = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.float64).T   # N x 2^N
    S = xs.shape[1]
    inst = _inst(N1, N2, S, seed=N)
    g = _graph(N1, N2)
    t = O.loss_terms(g, xs, np.ones(S), O.DBM, 2, inst=inst)
    assert np.all(t["ann"] == 0.0)
    for s in range(0, S, 5):
        want = _direct(xs[:, s], inst["C"][:, s], inst["M"][:, s], inst["lam4"][s], 0.25, 0.25, N1, N2)
        assert t["cost"][s] + t["pen"][s] == pytest.approx(want, abs=1e-12)
    ev = O.integer_eval(g, xs.astype(np.int64), np.ones(S), O.DBM, inst=inst)
    assert np.allclose(ev["qubo"], t["cost"] + t["pen"], rtol=0, atol=1e-12)


def test_large_penalties_give_the_best_diverse_matching():
    """With large lambdas the QUBO minimum is minus the heaviest matching that
    meets both diversity constraints, found by enumerating matchings."""
    N1, N2 = 3, 3
    rng = np.random.default_rng(4)
    C = rng.random(N1 * N2)
    M = np.array([0, 1, 1, 1, 0, 1, 1, 1, 0], dtype=np.float64)
    p, q = 0.25, 0.25
    best = 0.0
    for xbits in itertools.product([0, 1], repeat=9):
        X = np.array(xbits).reshape(3, 3)
        if (X.sum(axis=1) > 1).any() or (X.sum(axis=0) > 1).any():
            continue
        T, U = X.sum(), (M.reshape(3, 3) * X).sum()
        if p * T - U > 0 or q * T - (T - U) > 0:
            continue
        best = max(best, float((C.reshape(3, 3) * X).sum()))
    xs = np.array(list(itertools.product([0, 1], repeat=9)), dtype=np.float64).T
    S = xs.shape[1]
    inst = dict(N1=3, N2=3, C=np.repeat(C[:, None], S, 1), M=np.repeat(M[:, None], S, 1),
                lam4=np.full((S, 4), 50.0), pq=np.tile([p, q], (S, 1)))
    t = O.loss_terms(_graph(3, 3), xs, np.ones(S), O.DBM, 2, inst=inst)
    assert (t["cost"] + t["pen"]).min() == pytest.approx(-best, abs=1e-12)


def test_gradient_matches_finite_differences():
    N1, N2, S = 3, 4, 5
    inst = _inst(N1, N2, S, seed=9)
    g = _graph(N1, N2)
    rng = np.random.default_rng(1)
    P = rng.uniform(0.05, 0.95, size=(N1 * N2, S))

    def R(Pm):
        t = O.loss_terms(g, Pm, np.ones(S), O.DBM, 4, O.DIV_STD, inst=inst)
        return O.total_loss(t, np.ones(S), 0.6, 0.3, O.DBM)

    G = O.grad_P(g, P, np.ones(S), O.DBM, 4, 0.6, 0.3, O.DIV_STD, inst=inst)
    h = 1e-7
    fd = np.zeros_like(P)
    for idx in np.ndindex(*P.shape):
        a = P.copy(); a[idx] += h
        b = P.copy(); b[idx] -= h
        fd[idx] = (R(a) - R(b)) / (2 * h)
    # no ReLU kink lies within h of this P
    parts = O.dbm_parts(P, inst)
    assert np.abs(parts["R"] - 1).min() > 1e-4 and np.abs(parts["K"] - 1).min() > 1e-4
    assert np.linalg.norm(G - fd) <= 1e-6 * np.linalg.norm(fd)


def test_violation_counts():
    N1, N2 = 2, 3
    inst = dict(N1=2, N2=3, C=np.ones((6, 1)), M=np.array([[0], [1], [1], [1], [0], [1]], float),
                lam4=np.ones((1, 4)), pq=np.array([[0.6, 0.5]]))
    x = np.array([[1], [1], [0], [0], [1], [0]])     # row 0 has two pairs, column 1 two pairs
    ev = O.integer_eval(_graph(2, 3), x, np.ones(1), O.DBM, inst=inst)
    # T = 3, U = M.x = 1: p T - U = 0.8 > 0 (violated), q T - (T - U) = -0.5 (met)
    assert ev["objective"][0] == 3 and ev["violations"][0] == 1 + 1 + 1
    assert ev["value"][0] == 3.0


def test_constraint_graph():
    rp, col = I.dbm_graph(4, 5)
    assert np.all(np.diff(rp) == 4 + 5 - 2)
    edges = set(zip(np.repeat(np.arange(20), np.diff(rp)).tolist(), col.tolist()))
    assert all((j, i) in edges for i, j in edges)
    assert (0 * 5 + 1, 0) in edges and (1 * 5 + 0, 0) in edges and (1 * 5 + 1, 0) not in edges


@pytest.mark.parametrize("N1,N2,seed", [(3, 3, 1), (3, 4, 2), (4, 3, 5)])
def test_reference_optimum_matches_enumeration(N1, N2, seed):
    """The exact optimum the DBM runs are scored against (scipy's MILP) equals
    enumeration of all pair sets on tiny instances."""
    pytest.importorskip("scipy.optimize", minversion=None)
    from scipy import optimize
    if not hasattr(optimize, "milp"):
        pytest.skip("scipy without milp")
    from paper_2402_02190_gb300 import dbm
    Cv, Mv, p, q = I.dbm_instance(N1, N2, seed=seed, n_fields=2)
    C, M = Cv.astype(np.float64), Mv.astype(np.float64)
    best = 0.0
    for xbits in itertools.product([0, 1], repeat=N1 * N2):
        X = np.array(xbits).reshape(N1, N2)
        if (X.sum(axis=1) > 1).any() or (X.sum(axis=0) > 1).any():
            continue
        T, U = X.sum(), (M.reshape(N1, N2) * X).sum()
        if p * T - U > 0 or q * T - (T - U) > 0:
            continue
        best = max(best, float((C.reshape(N1, N2) * X).sum()))
    val, x = dbm.best_diverse_matching(C, M, N1, N2, p, q)
    assert val == pytest.approx(best, abs=1e-9)
    # the returned matching is feasible and has that reward
    inst = dict(N1=N1, N2=N2, C=C[:, None], M=M[:, None], lam4=np.ones((1, 4)), pq=np.array([[p, q]]))
    ev = O.integer_eval(_graph(N1, N2), x[:, None], np.ones(1), O.DBM, inst=inst)
    assert ev["violations"][0] == 0 and ev["value"][0] == pytest.approx(best, abs=1e-9)


def test_run_layouts():
    """The shot layouts of the DBM runs: the 11 x 11 grid of (a, a, b, b) over
    powers of two on one instance, and one instance per shot with the fixed
    (2, 2, 12, 12) of the multi-instance run."""
    from paper_2402_02190_gb300 import dbm
    Cv, Mv, p, q = I.dbm_instance(5, 4, seed=3)
    C, M, lam4, pq = dbm.penalty_grid_shots(5, 4, Cv, Mv, p, q)
    assert C.shape == M.shape == (20, 121) and lam4.shape == (121, 4) and pq.shape == (121, 2)
    assert np.array_equal(C, np.repeat(Cv[:, None], 121, axis=1))
    vals = 2.0 ** np.arange(11)
    assert set(lam4[:, 0]) == set(vals) and np.array_equal(lam4[:, 0], lam4[:, 1])
    assert np.array_equal(lam4[:, 2], lam4[:, 3])
    assert len({(a, b) for a, _, b, _ in lam4}) == 121
    insts = [I.dbm_instance(5, 4, seed=k)[:2] for k in range(7)]
    C, M, lam4, pq = dbm.multi_instance_shots(5, 4, insts, pq=(0.05, 0.05))
    assert C.shape == (20, 7)
    for s in range(7):
        assert np.array_equal(C[:, s], insts[s][0]) and np.array_equal(M[:, s], insts[s][1])
    assert np.all(lam4 == np.array([2, 2, 12, 12], np.float32)) and np.all(pq == 0.05)
    # field indicators are 0/1 and rewards lie in [0, 1)
    assert set(np.unique(Mv)) <= {0.0, 1.0} and Cv.min() >= 0 and Cv.max() < 1


def test_apr_marks_shots_without_a_feasible_matching():
    from paper_2402_02190_gb300 import dbm
    best = np.zeros(3, dtype=[("objective", "i8"), ("violations", "i8"), ("qubo", "f8"), ("value", "f8")])
    best["objective"] = [4, -1, 0]
    best["value"] = [9.0, -1.0, 0.0]
    a = dbm.apr(best, [10.0, 10.0, 10.0])
    assert a[0] == pytest.approx(0.9) and np.isnan(a[1]) and a[2] == 0.0


@pytest.mark.parametrize("N1,N2", [(1, 4), (3, 5), (6, 2)])
def test_constraint_graph_aggregation_by_line_sums(N1, N2):
    """On the matching's constraint graph the neighbour sum of pair (r, k) is
    its row line's sum plus its column line's sum minus twice its own value
    (the identity the line-sum aggregation of the library relies on), and the
    adjoint aggregation equals the forward one (constant degree, symmetric A)."""
    g = _graph(N1, N2)
    rng = np.random.default_rng(N1 * 10 + N2)
    X = rng.normal(size=(N1 * N2, 7))
    Xr = X.reshape(N1, N2, 7)
    R = Xr.sum(axis=1)      # N1 x 7
    K = Xr.sum(axis=0)      # N2 x 7
    nb = (R[:, None, :] + K[None, :, :] - 2.0 * Xr).reshape(N1 * N2, 7)
    deg = N1 + N2 - 2
    want = nb / deg if deg else np.zeros_like(nb)
    assert np.allclose(O.mean_aggregate(g, X), want, rtol=0, atol=1e-12)
    assert np.allclose(O.mean_aggregate_adjoint(g, X), want, rtol=0, atol=1e-12)


def test_early_stop_monitors_the_dbm_penalty_unweighted():
    """For DBM the monitored loss is sum_s (cost_s + pen_s): the penalty term
    already carries its lambdas, so the per-shot lambda vector is not applied."""
    S = 3
    seq = []
    for t in range(6):
        cost = np.full(S, -1.0 - 0.5 * t)     # falls by 0.5 per shot and step
        pen = np.full(S, 2.0 + 0.25 * t)      # rises by 0.25
        seq.append((cost, pen, np.zeros(S)))
    lam = np.full(S, 7.0)
    # unweighted, cost + pen falls by 0.25 per shot and step: never stale
    assert O.early_stop_step(seq, [1.0] * 6, lam, O.DBM, 1e-9, 3) == -1
    # weighted by lambda = 7 it would rise by 1.25 (stale from step 1 on)
    assert O.early_stop_step(seq, [1.0] * 6, lam, O.MIS, 1e-9, 3) == 3
