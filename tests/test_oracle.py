"""Pins for the FP64 oracle itself (no GPU).

Each test ties the oracle to something other than itself: numbers printed in
the paper, brute-force enumeration, closed forms, textbook special cases,
independent library routines (networkx, torch.optim) and central finite
differences.  A plausible slip in the oracle (dropped term, wrong sign or
index, transposed operand) fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import cpra_oracle as O
from oracle import exact as X
from paper_2402_02190_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _graph(N, d, seed):
    rp, col = I.random_regular_graph(N, d, seed)
    return O.Graph(rp, col), rp, col


# ---------------------------------------------------------------- paper pins
def test_param_counts_match_paper_tables():
    rows = []
    with open(os.path.join(GOLDEN, "param_counts.txt")) as f:
        for line in f:
            line = line.split("--")[0].strip()
            if not line or line.startswith("#"):
                continue
            H0, H1, S, count = (int(v) for v in line.split())
            rows.append((H0, H1, S, count))
    assert len(rows) == 4
    for H0, H1, S, count in rows:
        assert O.param_count(H0, H1, S) == count
        # the flat layout the oracle unpacks has exactly that many entries
        assert I.param_layout(H0, H1, S)["_total"][0] == count
    # H0 = int(N^0.8) for N = 10,000 (App. C.1)
    assert int(10000 ** 0.8) == 1584


# ---------------------------------------------------------- brute-force pins
@pytest.mark.parametrize("N,d,seed", [(10, 3, 1), (12, 3, 7), (12, 4, 3)])
def test_relaxation_equals_qubo_at_binary_points(N, d, seed):
    g, rp, col = _graph(N, d, seed)
    adj = X.adjacency_sets(rp, col)
    lam = np.array([0.5, 2.0, 7.0])
    xs = np.array(list(X.all_binary(N))).T          # N x 2^N, every binary x
    S = xs.shape[1]
    for problem in (O.MIS, O.MAXCUT):
        lam_s = np.resize(lam, S)
        t = O.loss_terms(g, xs.astype(np.float64), lam_s, problem, alpha=2)
        # annealing term vanishes at every vertex of the hypercube (Lemma A.1)
        assert np.all(t["ann"] == 0.0)
        for s in range(S):
            x = xs[:, s]
            if problem == O.MIS:
                want = X.mis_qubo_direct(adj, x, lam_s[s])
                got = t["cost"][s] + lam_s[s] * t["pen"][s]
            else:
                want = -X.cut_size_direct(adj, x)
                got = t["cost"][s]
            assert got == pytest.approx(want, abs=1e-12)


@pytest.mark.parametrize("N,d,seed", [(12, 3, 2), (14, 3, 5), (12, 5, 9)])
def test_min_mis_qubo_is_minus_independence_number(N, d, seed):
    """For lambda > 1 the MIS QUBO minimum equals -alpha(G) (textbook
    reduction); alpha(G) from networkx's exact max clique of the complement."""
    nx = pytest.importorskip("networkx")
    g, rp, col = _graph(N, d, seed)
    G = nx.Graph()
    G.add_nodes_from(range(N))
    G.add_edges_from(zip(g.ei.tolist(), g.ej.tolist()))
    _, alpha_nx = nx.max_weight_clique(nx.complement(G), weight=None)
    adj = X.adjacency_sets(rp, col)
    assert X.max_independent_set_size(adj) == alpha_nx
    xs = np.array(list(X.all_binary(N))).T.astype(np.float64)
    lam = np.full(xs.shape[1], 2.0)
    t = O.loss_terms(g, xs, lam, O.MIS, alpha=2)
    assert (t["cost"] + lam * t["pen"]).min() == pytest.approx(-alpha_nx)
    ev = O.integer_eval(g, xs.astype(np.int64), lam, O.MIS)
    feasible = ev["violations"] == 0
    assert ev["objective"][feasible].max() == alpha_nx


@pytest.mark.parametrize("N,d,seed", [(10, 3, 4), (12, 4, 6)])
def test_min_cut_qubo_is_minus_maxcut(N, d, seed):
    g, rp, col = _graph(N, d, seed)
    adj = X.adjacency_sets(rp, col)
    xs = np.array(list(X.all_binary(N))).T.astype(np.float64)
    t = O.loss_terms(g, xs, np.zeros(xs.shape[1]), O.MAXCUT, alpha=2)
    assert t["cost"].min() == pytest.approx(-X.max_cut_brute(adj))
    ev = O.integer_eval(g, xs.astype(np.int64), None, O.MAXCUT)
    assert ev["objective"].max() == X.max_cut_brute(adj)
    assert np.array_equal(-ev["qubo"], ev["objective"].astype(np.float64))


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("alpha", [2, 4, 6])
def test_annealing_term_closed_forms(alpha):
    g, _, _ = _graph(20, 3, 11)
    N, S = 20, 7
    half = np.full((N, S), 0.5)
    t = O.loss_terms(g, half, np.ones(S), O.MIS, alpha)
    assert np.all(t["ann"] == N)                   # phi(1/2) = 1 (Lemma A.1)
    gamma = 1.7
    Gh = O.grad_P(g, half, np.zeros(S), O.MIS, alpha, gamma, 0.0)
    # MIS with lambda = 0: dR/dP = -1 + gamma * phi'(1/2) = -1
    assert np.allclose(Gh, -1.0, atol=0, rtol=0)
    # at binary points phi' = -2 alpha (2p - 1)^(alpha-1) = -+2 alpha
    for p, sgn in ((0.0, -1.0), (1.0, 1.0)):
        Pb = np.full((N, S), p)
        Gb = O.grad_P(g, Pb, np.zeros(S), O.MIS, alpha, gamma, 0.0)
        assert np.allclose(Gb, -1.0 - 2.0 * alpha * gamma * sgn)
    # symmetry phi(p) = phi(1 - p)
    rng = np.random.default_rng(0)
    P = rng.uniform(size=(N, S))
    a1 = O.loss_terms(g, P, np.ones(S), O.MIS, alpha)["ann"]
    a2 = O.loss_terms(g, 1.0 - P, np.ones(S), O.MIS, alpha)["ann"]
    assert np.allclose(a1, a2)


def test_prop32_variance_equals_pairwise_hamming():
    """S^2 sum_i VAR_s[x_is] = sum_{s<l} d_H(x_s, x_l) (Prop. 3.2), against an
    O(S^2 N) loop over pairs."""
    rng = np.random.default_rng(3)
    for N, S in ((1, 2), (5, 3), (17, 8), (30, 33)):
        Xb = rng.integers(0, 2, size=(N, S))
        lhs = S * S * O.shot_variance(Xb.astype(np.float64)).sum()
        rhs = 0
        for s in range(S):
            for l in range(s + 1, S):
                rhs += int(np.sum(Xb[:, s] != Xb[:, l]))
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-9)
        g = O.Graph(*I.edges_to_csr(N, np.zeros(0, int), np.zeros(0, int)))
        ev = O.integer_eval(g, Xb, np.ones(S), O.MIS)
        assert ev["pair_hamming"] == rhs
        # Psi in VAR form is minus the same quantity
        t = O.loss_terms(g, Xb.astype(np.float64), np.ones(S), O.MIS, 2, O.DIV_VAR)
        assert t["psi"] == pytest.approx(-rhs, rel=1e-12, abs=1e-9)


def test_psi_std_closed_form():
    """Two shots at 0 and 1 on every node: STD = 1/2, Psi = -S N / 2."""
    N = 9
    P = np.zeros((N, 2))
    P[:, 1] = 1.0
    g = O.Graph(*I.edges_to_csr(N, np.zeros(0, int), np.zeros(0, int)))
    t = O.loss_terms(g, P, np.ones(2), O.MIS, 2, O.DIV_STD)
    assert t["psi"] == pytest.approx(-2 * N * 0.5)
    # constant rows have zero variance and zero Psi gradient
    P2 = np.full((N, 4), 0.3)
    G = O.grad_P(g, P2, np.zeros(4), O.MIS, 2, 0.0, 1.0, O.DIV_STD)
    assert np.allclose(G, -1.0)


# ------------------------------------------------------------- aggregation
def test_mean_aggregate_matches_dense_row_normalised_adjacency():
    rp, col = I.erdos_renyi_graph(40, 0.06, seed=5)   # has isolated nodes
    g = O.Graph(rp, col)
    N = g.N
    A = np.zeros((N, N))
    for i, j in zip(g.ei, g.ej):
        A[i, j] = A[j, i] = 1.0
    deg = A.sum(axis=1)
    assert (deg == 0).any()
    Dinv = np.diag(np.where(deg > 0, 1.0 / np.maximum(deg, 1), 0.0))
    rng = np.random.default_rng(1)
    Xm = rng.standard_normal((N, 6))
    assert np.allclose(O.mean_aggregate(g, Xm), Dinv @ A @ Xm, atol=1e-14)
    Y = rng.standard_normal((N, 6))
    assert np.allclose(O.mean_aggregate_adjoint(g, Y), (Dinv @ A).T @ Y, atol=1e-14)
    # adjoint identity <A_hat X, Y> = <X, A_hat^T Y>
    lhs = np.sum(O.mean_aggregate(g, Xm) * Y)
    rhs = np.sum(Xm * O.mean_aggregate_adjoint(g, Y))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_forward_reduces_to_mlp_without_neighbour_weights():
    """With W1 = W2 = 0 each node is an independent 2-layer MLP (textbook)."""
    g, _, _ = _graph(16, 3, 2)
    H0, H1, S = 5, 6, 4
    theta, X0 = I.seeded_params(16, H0, H1, S, seed=4)
    p = O.unpack(theta, H0, H1, S)
    th = O.pack(p["B1"], 0 * p["W1"], p["b1"], p["B2"], 0 * p["W2"], p["b2"])
    out = O.forward(g, th, X0, H0, H1, S)["P"]
    for v in range(16):
        h = np.zeros(H1)
        for o in range(H1):
            h[o] = max(0.0, sum(p["B1"][o, k] * X0[v, k] for k in range(H0)) + p["b1"][o])
        for s in range(S):
            z = sum(p["B2"][s, o] * h[o] for o in range(H1)) + p["b2"][s]
            assert out[v, s] == pytest.approx(1.0 / (1.0 + np.exp(-z)), rel=1e-13)


def test_init_logits_offset_of_the_head():
    """The warm-start offset L0 enters the head's pre-activation: with every
    weight and bias zero P = sigmoid(L0) exactly, and an offset that is
    constant per shot is the same as adding it to b2."""
    rp, col = I.random_regular_graph(30, 3, seed=2)
    g = O.Graph(rp, col)
    N, H, S = 30, 16, 5
    rng = np.random.default_rng(0)
    L0 = rng.normal(size=(N, S)) * 3
    theta0 = np.zeros(O.param_count(H, H, S))
    X0 = rng.normal(size=(N, H))
    P = O.forward(g, theta0, X0, H, H, S, init_logits=L0)["P"]
    assert np.array_equal(P, 1.0 / (1.0 + np.exp(-L0)))
    theta, X0 = I.seeded_params(N, H, H, S, seed=4)
    c = rng.normal(size=S)
    lay = I.param_layout(H, H, S)
    off, shape = lay["b2"]
    theta_b = theta.astype(np.float64).copy()
    theta_b[off:off + S] += c
    Pa = O.forward(g, theta, X0, H, H, S, init_logits=np.tile(c, (N, 1)))["P"]
    Pb = O.forward(g, theta_b, X0, H, H, S)["P"]
    assert np.allclose(Pa, Pb, rtol=0, atol=1e-15)


def test_forward_on_complete_graph_closed_form():
    """On K_n the neighbour mean is (sum of all rows - own row) / (n - 1)."""
    n = 6
    ei, ej = zip(*itertools.combinations(range(n), 2))
    g = O.Graph(*I.edges_to_csr(n, np.array(ei), np.array(ej)))
    rng = np.random.default_rng(2)
    Xm = rng.standard_normal((n, 3))
    want = (Xm.sum(axis=0)[None, :] - Xm) / (n - 1)
    assert np.allclose(O.mean_aggregate(g, Xm), want, atol=1e-14)


# -------------------------------------------------------- finite differences
def _fd_case(problem, div_kind, alpha, seed):
    N, H0, H1, S = 12, 4, 5, 6
    rp, col = I.random_regular_graph(N, 3, seed)
    g = O.Graph(rp, col)
    theta, X0 = I.seeded_params(N, H0, H1, S, seed=seed + 100, weight_scale=2.0)
    cfg = dict(H0=H0, H1=H1, S=S, problem=problem, alpha=alpha,
               lam=np.linspace(0.5, 3.0, S), gamma=-0.7, nu=0.35, div_kind=div_kind)
    return g, theta.astype(np.float64), X0.astype(np.float64), cfg


def _loss(g, theta, X0, cfg):
    c = O.forward(g, theta, X0, cfg["H0"], cfg["H1"], cfg["S"])
    t = O.loss_terms(g, c["P"], cfg["lam"], cfg["problem"], cfg["alpha"], cfg["div_kind"])
    return O.total_loss(t, cfg["lam"], cfg["gamma"], cfg["nu"], cfg["problem"])


@pytest.mark.parametrize("problem", [O.MIS, O.MAXCUT])
@pytest.mark.parametrize("div_kind", [O.DIV_STD, O.DIV_VAR])
@pytest.mark.parametrize("alpha", [2, 4])
def test_gradients_match_central_finite_differences(problem, div_kind, alpha):
    g, theta, X0, cfg = _fd_case(problem, div_kind, alpha, seed=3 + alpha)
    c = O.forward(g, theta, X0, cfg["H0"], cfg["H1"], cfg["S"])
    # stay away from ReLU kinks so central differences are valid
    assert np.min(np.abs(c["Z1"])) > 1e-4
    GP = O.grad_P(g, c["P"], cfg["lam"], problem, alpha, cfg["gamma"], cfg["nu"], div_kind)
    gr = O.backward(g, theta, c, GP, cfg["H0"], cfg["H1"], cfg["S"])
    h = 1e-6
    fd_t = np.zeros_like(theta)
    for k in range(len(theta)):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd_t[k] = (_loss(g, tp, X0, cfg) - _loss(g, tm, X0, cfg)) / (2 * h)
    fd_x = np.zeros_like(X0)
    for idx in np.ndindex(*X0.shape):
        xp = X0.copy(); xp[idx] += h
        xm = X0.copy(); xm[idx] -= h
        fd_x[idx] = (_loss(g, theta, xp, cfg) - _loss(g, theta, xm, cfg)) / (2 * h)
    lay = I.param_layout(cfg["H0"], cfg["H1"], cfg["S"])
    for name in ("Wcat1", "b1", "Wcat2", "b2"):
        off, shape = lay[name]
        n = int(np.prod(shape))
        a, b = gr["theta"][off:off + n], fd_t[off:off + n]
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b) + 1e-9, name
    assert np.linalg.norm(gr["X0"] - fd_x) <= 1e-6 * np.linalg.norm(fd_x)


@pytest.mark.parametrize("problem", [O.MIS, O.MAXCUT])
@pytest.mark.parametrize("div_kind", [O.DIV_STD, O.DIV_VAR])
def test_grad_P_matches_finite_differences(problem, div_kind):
    rp, col = I.erdos_renyi_graph(15, 0.3, seed=8)
    g = O.Graph(rp, col)
    rng = np.random.default_rng(9)
    S = 5
    P = rng.uniform(0.05, 0.95, size=(15, S))
    lam = np.linspace(1, 4, S)
    args = (lam, problem, 4, 0.9, 0.6, div_kind)

    def R(Pm):
        t = O.loss_terms(g, Pm, lam, problem, 4, div_kind)
        return O.total_loss(t, lam, 0.9, 0.6, problem)

    G = O.grad_P(g, P, *args)
    h = 1e-6
    fd = np.zeros_like(P)
    for idx in np.ndindex(*P.shape):
        a = P.copy(); a[idx] += h
        b = P.copy(); b[idx] -= h
        fd[idx] = (R(a) - R(b)) / (2 * h)
    assert np.linalg.norm(G - fd) <= 1e-7 * np.linalg.norm(fd)


# ----------------------------------------------------------------- optimiser
def test_adam_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    n = 50
    th = rng.standard_normal(n)
    for wd, cls in ((0.0, torch.optim.Adam), (1e-2, torch.optim.AdamW)):
        pt = torch.tensor(th.copy(), dtype=torch.float64, requires_grad=True)
        opt = cls([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=wd)
        m = np.zeros(n); v = np.zeros(n); cur = th.copy()
        for t in range(1, 6):
            gt = rng.standard_normal(n)
            pt.grad = torch.tensor(gt, dtype=torch.float64)
            opt.step()
            cur, m, v = O.adam(cur, m, v, gt, t, lr=1e-3, wd=wd)
            assert np.allclose(cur, pt.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_bf16_round_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(10000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 10000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, 1e-40],
                                 dtype=np.float32)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.bf16_round(x), want)


def test_relu_decision_in_bf16_only_moves_near_zero_signs():
    g, theta, X0, cfg = _fd_case(O.MIS, O.DIV_STD, 2, seed=2)
    a = O.forward(g, theta, X0, cfg["H0"], cfg["H1"], cfg["S"])
    b = O.forward(g, theta, X0, cfg["H0"], cfg["H1"], cfg["S"], relu_decision="bf16")
    differ = a["relu_on"] != b["relu_on"]
    assert np.all(np.abs(a["Z1"][differ]) < 0.05)
    assert np.array_equal(a["relu_on"], a["Z1"] > 0)


def test_relu_decision_in_bf16_flips_only_within_the_rounding_bound():
    """The BF16 reading of the ReLU sign (operands rounded to bfloat16, unit
    roundoff u = 2^-8) may only disagree with the FP64 sign where |Z1| is
    within the worst-case error that rounding X0, the neighbour mean and the
    layer-1 weights can put into Z1:
      |dX0| |B1|^T + |bf(X0)| |dB1|^T + |dM1| |W1|^T + |bf(M1)| |dW1|^T,
    with |dX0| <= u|X0|, |dB1| <= u|B1|, |dW1| <= u|W1|, and
    |dM1| <= u mean|X0| + (u + 2^-23) |mean bf(X0)| (the mean of rounded
    rows, rounded once more through float32).  A decision taken on the wrong
    operand, transposed weights or a missing term flips signs outside it."""
    N, H0, H1, S = 600, 32, 32, 8
    rp, col = I.random_regular_graph(N, 5, 7)
    g = O.Graph(rp, col)
    theta, X0 = I.seeded_params(N, H0, H1, S, seed=11)
    theta = theta.astype(np.float64)
    X0 = X0.astype(np.float64)
    a = O.forward(g, theta, X0, H0, H1, S)
    b = O.forward(g, theta, X0, H0, H1, S, relu_decision="bf16")
    p = O.unpack(theta, H0, H1, S)
    u = 2.0 ** -8
    aB, aW = np.abs(p["B1"]), np.abs(p["W1"])
    xb = np.abs(O.bf16_round(X0))
    mx = O.mean_aggregate(g, O.bf16_round(X0))
    bound = (u * np.abs(X0) @ aB.T + xb @ (u * aB).T
             + (u * O.mean_aggregate(g, np.abs(X0)) + (u + 2.0 ** -23) * np.abs(mx)) @ aW.T
             + np.abs(O.bf16_round(mx)) @ (u * aW).T)
    bound = bound * (1 + 1e-9) + 1e-300
    flipped = a["relu_on"] != b["relu_on"]
    assert flipped.sum() > 0                      # the case exercises the reading
    assert np.all(np.abs(a["Z1"][flipped]) <= bound[flipped])
    # and it is a rounding-level reading: few entries are that close to 0
    assert (np.abs(a["Z1"]) <= bound).mean() < 0.05


def test_adam_first_step_closed_form():
    g = np.array([3.0, -2e-3, 0.0, 1e-12])
    th, m, v = O.adam(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, lr=0.1)
    assert np.allclose(th, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_gamma_schedule_endpoints():
    assert O.gamma_schedule(0, 3000, -2.0, 0.1) == -2.0
    assert O.gamma_schedule(2999, 3000, -2.0, 0.1) == pytest.approx(0.1)
    assert O.gamma_schedule(1500, 3001, -2.0, 0.1) == pytest.approx(-0.95)


# ------------------------------------------------------ early stopping
def _es_terms(ls, phis, S=3, lam=(1.0, 2.0, 0.5)):
    """Per-step terms whose monitored sums are exactly ls[t] and phis[t]
    (gamma_t = 1): cost carries l_t in shot 0, pen = 0, ann carries phi_t."""
    seq = []
    for l_t, p_t in zip(ls, phis):
        cost = np.zeros(S); pen = np.zeros(S); ann = np.zeros(S)
        cost[0] = l_t
        ann[0] = p_t
        seq.append((cost, pen, ann))
    return seq, [1.0] * len(ls), np.array(lam)


def test_early_stop_constant_run_stops_after_patience():
    seq, g, lam = _es_terms([5.0] * 10, [2.0] * 10)
    # steps 1, 2, 3 are stale: patience 3 completes at step 3
    assert O.early_stop_step(seq, g, lam, O.MIS, 1e-5, 3) == 3
    assert O.early_stop_step(seq, g, lam, O.MIS, 1e-5, 9) == 9
    assert O.early_stop_step(seq, g, lam, O.MIS, 1e-5, 10) == -1


def test_early_stop_needs_both_values_stale():
    # the loss keeps falling by more than tol while phi is flat: never stale
    ls = [10.0 - t for t in range(12)]
    seq, g, lam = _es_terms(ls, [1.0] * 12)
    assert O.early_stop_step(seq, g, lam, O.MIS, 1e-5, 2) == -1
    # and the other way round
    seq, g, lam = _es_terms([1.0] * 12, ls)
    assert O.early_stop_step(seq, g, lam, O.MIS, 1e-5, 2) == -1


def test_early_stop_rise_counts_and_improvement_resets():
    # rises count as stale; a drop larger than tol resets the count
    ls = [5.0, 5.5, 6.0, 4.0, 4.0 + 5e-6, 4.0 + 1e-5, 4.1]
    seq, g, lam = _es_terms(ls, [0.0] * len(ls))
    assert O.early_stop_step(seq, g, lam, O.MIS, 1e-5, 2) == 2
    assert O.early_stop_step(seq, g, lam, O.MIS, 1e-5, 3) == 6
    assert O.early_stop_step(seq, g, lam, O.MIS, 1e-5, 4) == -1
    # a drop of exactly tol is still stale (|change| <= tol)
    seq, g, lam = _es_terms([1.0, 1.0 - 2.0 ** -20, 1.0 - 2.0 ** -19], [0.0] * 3)
    assert O.early_stop_step(seq, g, lam, O.MIS, 2.0 ** -20, 2) == 2


def test_early_stop_monitored_sums():
    """The penalty weights enter the MIS loss and not the MaxCut one, and
    gamma scales the annealing term."""
    S = 3
    lam = np.array([1.0, 2.0, 0.5])
    cost = np.array([-1.0, -2.0, -3.0])
    pen = np.array([0.5, 0.25, 1.0])
    ann = np.array([1.0, 2.0, 3.0])
    # MIS: l = -6 + (0.5 + 0.5 + 0.5) = -4.5; an identical second step is stale
    seq = [(cost, pen, ann), (cost, pen, ann)]
    assert O.early_stop_step(seq, [1.0, 1.0], lam, O.MIS, 0.0, 1) == 1
    # the pen entries change by +1 in step 2: MIS loss rises (stale), MaxCut
    # loss is unchanged (stale); phi falls by 6 with gamma 1 -> not stale
    seq = [(cost, pen, ann), (cost, pen + 1.0, ann)]
    assert O.early_stop_step(seq, [1.0, -1.0], lam, O.MIS, 1e-5, 1) == -1
    assert O.early_stop_step(seq, [1.0, 1.0], lam, O.MIS, 1e-5, 1) == 1
    # MIS loss falls when pen falls; MaxCut ignores pen
    seq = [(cost, pen, ann), (cost, pen - 0.25, ann)]
    assert O.early_stop_step(seq, [1.0, 1.0], lam, O.MIS, 1e-5, 1) == -1
    assert O.early_stop_step(seq, [1.0, 1.0], lam, O.MAXCUT, 1e-5, 1) == 1


# ------------------------------------------------------ integer evaluation
@pytest.mark.parametrize("seed", [0, 1])
def test_integer_eval_invariants(seed):
    rp, col = I.erdos_renyi_graph(60, 0.08, seed=seed)
    g = O.Graph(rp, col)
    adj = X.adjacency_sets(rp, col)
    rng = np.random.default_rng(seed)
    S = 37
    P = I.seeded_P(60, S, seed)
    Xr = O.round_solutions(P)
    assert np.array_equal(Xr, (P > np.float32(0.5)).astype(np.int64))
    assert Xr[3].sum() == 0                      # row of exact 0.5 rounds to 0
    lam = rng.uniform(0.5, 3, S)
    ev = O.integer_eval(g, Xr, lam, O.MIS)
    for s in range(S):
        x = Xr[:, s]
        inside = sum(1 for i in range(60) for j in adj[i] if i < j and x[i] and x[j])
        assert ev["violations"][s] == inside
        assert ev["objective"][s] == x.sum()
        assert ev["qubo"][s] == pytest.approx(-x.sum() + lam[s] * inside)
        if inside == 0:                           # an independent set
            assert all(not (x[i] and x[j]) for i in range(60) for j in adj[i])
    ev2 = O.integer_eval(g, Xr, None, O.MAXCUT)
    for s in range(S):
        assert ev2["objective"][s] == X.cut_size_direct(adj, Xr[:, s])
    # bit packing round trip
    bits = O.pack_bits(Xr)
    assert bits.shape == (60, 2)
    un = np.zeros_like(Xr)
    for s in range(S):
        un[:, s] = (bits[:, s // 32] >> (s % 32)) & 1
    assert np.array_equal(un, Xr)


# ---------------------------------------------------------- Theorem 3.1
def test_theorem31_gamma_limits_on_P():
    """Projected gradient descent on P alone: large negative gamma drives
    every entry to 1/2 (convex limit); large positive gamma drives entries to
    {0, 1} (binary limit)."""
    g, _, _ = _graph(16, 3, 1)
    S = 4
    lam = np.full(S, 2.0)
    rng = np.random.default_rng(0)
    P0 = rng.uniform(0.1, 0.9, size=(16, S))
    P = P0.copy()
    for _ in range(4000):
        P = np.clip(P - 1e-3 * O.grad_P(g, P, lam, O.MIS, 2, -200.0, 0.0), 0, 1)
    assert np.allclose(P, 0.5, atol=1e-2)
    P = P0.copy()
    for _ in range(4000):
        P = np.clip(P - 1e-3 * O.grad_P(g, P, lam, O.MIS, 2, 200.0, 0.0), 0, 1)
    assert np.all((P == 0.0) | (P == 1.0))


def test_full_step_shapes_and_consistency():
    g, theta, X0, cfg = _fd_case(O.MIS, O.DIV_STD, 2, seed=1)
    cfg.update(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, train_embedding=True)
    out = O.step(g, theta, X0, cfg, t=1)
    assert out["P"].shape == (12, cfg["S"])
    assert np.all((out["P"] > 0) & (out["P"] < 1))
    # first Adam step moves every parameter with non-zero gradient by ~lr
    d = np.abs(out["theta_next"] - theta)
    nz = np.abs(out["grads"]["theta"]) > 1e-6
    assert np.allclose(d[nz], 1e-3, rtol=1e-3)
