"""Diverse bipartite matching (Eq. matching-cost-function) on the GPU
against the FP64 oracle: a full training step with one instance per shot
(multi-instance CPRA, App. multi-instance), the exact evaluation of the
rounded matchings, graph replay, and cpra_solve on a tiny instance whose
best diverse matching is found by enumeration."""
import itertools

import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402


def _mixed_shots(N1, N2, S, seed):
    """Shots with their own instance: field-difference densities 0.1 / 0.5 /
    0.9 (so each diversity constraint is active in some shots and not in
    others), rewards in [0, 1), lambdas and (p, q) varying per shot."""
    rng = np.random.default_rng(seed)
    N = N1 * N2
    dens = np.array([0.1, 0.5, 0.9])[np.arange(S) % 3]
    # the shots with a negative offset (T near 0) get one field class only, so
    # their diversity decisions do not hinge on which few pairs dominate T
    low = np.arange(S) % 4 == 0
    dens[low] = (np.arange(S)[low] // 4) % 2
    C = rng.random((N, S)).astype(np.float32)
    M = (rng.random((N, S)) < dens[None, :]).astype(np.float32)
    lam4 = rng.uniform(0.5, 4.0, size=(S, 4)).astype(np.float32)
    pq = np.where((np.arange(S) % 2 == 0)[:, None], 0.25, 0.05).astype(np.float32) * np.ones((S, 2), np.float32)
    # shots with a strongly negative offset start with every line sum below 1
    L0 = rng.normal(size=(N, S)) * 0.5 + np.where(low, -9.0, 0.0)[None, :]
    return C, M, lam4, pq, L0.astype(np.float32)


def _inst(N1, N2, C, M, lam4, pq):
    return dict(N1=N1, N2=N2, C=C.astype(np.float64), M=M.astype(np.float64),
                lam4=lam4.astype(np.float64), pq=pq.astype(np.float64))


def _run_step(precision, N1=30, N2=20, S=40, H=32, nu=0.25, seed=2, graph="constraint"):
    N = N1 * N2
    # the constraint graph takes the line-sum aggregations; any other graph
    # the gathered ones
    rp, col = I.dbm_graph(N1, N2) if graph == "constraint" else I.random_regular_graph(N, 6, seed)
    g = O.Graph(rp, col)
    C, M, lam4, pq, L0 = _mixed_shots(N1, N2, S, seed)
    theta, X0 = I.seeded_params(N, H, H, S, seed=seed + 1, weight_scale=1.5)
    mt, vt = I.seeded_adam_state(len(theta), seed=seed + 2)
    mx, vx = I.seeded_adam_state(N * H, seed=seed + 3)
    T, t_idx, t_prev = 9, 4, 2
    s = cpra.Solver(rp, col, problem=cpra.DBM, S=S, H0=H, H1=H, precision=precision, nu=nu,
                    gamma0=-1.0, gamma1=1.0, schedule_steps=T, keep_emb_grad=1)
    for which, arr in ((cpra.T_THETA, theta), (cpra.T_EMB, X0), (cpra.T_THETA_M, mt),
                       (cpra.T_THETA_V, vt), (cpra.T_EMB_M, mx), (cpra.T_EMB_V, vx),
                       (cpra.T_STEP, np.array([t_prev]))):
        s.set(which, arr)
    s.set_dbm(N1, C, M, lam4, pq)
    s.set_init_logits(L0)
    terms = s.step(t_idx, want_terms=True).astype(np.float64)
    out = dict(P=s.P(), grad=s.get(cpra.T_GRAD), gX0=s.get(cpra.T_EMB_GRAD),
               theta=s.get(cpra.T_THETA), X0=s.get(cpra.T_EMB), terms=terms)
    rec, ham, bits = s.round_eval(want_bits=True)
    s.close()
    inst = _inst(N1, N2, C, M, lam4, pq)
    gamma = O.gamma_schedule(t_idx, T, -1.0, 1.0)
    cfg = dict(H0=H, H1=H, S=S, problem=O.DBM, alpha=2, lam=np.ones(S), gamma=gamma, nu=nu,
               div_kind=O.DIV_STD, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0, dbm=inst)
    if precision == cpra.BF16:
        cfg["relu_decision"] = "bf16"
        cfg["init_logits"] = O.bf16_round(L0)
    else:
        cfg["init_logits"] = L0.astype(np.float64)
    ref = O.step(g, theta, X0, cfg, t=t_prev + 1,
                 adam_state=dict(m_theta=mt, v_theta=vt, m_X0=mx.reshape(N, H), v_X0=vx.reshape(N, H)))
    return out, ref, rec, ham, bits, inst, g, theta, X0, gamma, S, H


@pytest.mark.parametrize("graph", ["constraint", "random"])
@pytest.mark.parametrize("precision,tol,margin,rel", [(cpra.FP32, 1e-5, 1e-3, 1e-3),
                                                     (cpra.BF16, 2e-2, 0.2, 1e-2)])
def test_step_matches_oracle(precision, tol, margin, rel, graph):
    out, ref, rec, ham, bits, inst, g, theta, X0, gamma, S, H = _run_step(precision, graph=graph)
    # every ReLU of the penalty is decided with room to spare, and both
    # branches occur (rows, columns and each diversity constraint)
    parts = O.dbm_parts(ref["P"], inst)
    pq = inst["pq"]
    g3 = pq[:, 0] * parts["T"] - parts["U"]
    g4 = pq[:, 1] * parts["T"] - (parts["T"] - parts["U"])
    for v in (parts["R"] - 1, parts["K"] - 1):
        assert np.abs(v).min() > margin and (v > 0).any() and (v < 0).any()
    for v in (g3, g4):   # relative to T: the shots with a negative offset have T near 0
        assert (np.abs(v) / parts["T"]).min() > rel and (v > 0).any() and (v < 0).any()

    assert np.abs(out["P"] - ref["P"]).max() <= tol
    t, rt = out["terms"], ref["terms"]
    norm = np.abs(rt["cost"]) + np.abs(rt["pen"]) + abs(gamma) * rt["ann"]
    for k, a in (("cost", t[:S]), ("pen", t[S:2 * S]), ("ann", t[2 * S:3 * S])):
        assert np.max(np.abs(a - rt[k]) / norm) <= tol, k
    assert abs(t[3 * S] - rt["psi"]) <= tol * abs(rt["psi"])
    lay = I.param_layout(H, H, S)
    for name in ("Wcat1", "b1", "Wcat2", "b2"):
        off, shape = lay[name]
        n = int(np.prod(shape))
        a, b = out["grad"][off:off + n], ref["grads"]["theta"][off:off + n]
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), name
    gx = out["gX0"].reshape(X0.shape)
    assert np.linalg.norm(gx - ref["grads"]["X0"]) <= tol * np.linalg.norm(ref["grads"]["X0"])
    dref = ref["theta_next"] - theta
    assert np.linalg.norm(out["theta"] - ref["theta_next"]) <= 10 * tol * np.linalg.norm(dref)

    # exact evaluation of the returned matchings
    x = I.unpack_bits(bits, S).astype(np.int64)
    ev = O.integer_eval(g, x, np.ones(S), O.DBM, inst=inst)
    assert np.array_equal(rec["objective"], ev["objective"])
    assert np.array_equal(rec["violations"], ev["violations"])
    assert np.allclose(rec["value"], ev["value"], rtol=1e-12, atol=1e-9)
    assert np.allclose(rec["qubo"], ev["qubo"], rtol=1e-12, atol=1e-9)
    assert ham == ev["pair_hamming"]
    if precision == cpra.FP32:
        decided = np.abs(ref["P"] - 0.5) > 1e-5
        assert np.array_equal(x[decided], ref["X"][decided])


def test_graph_replay_equals_single_steps():
    N1, N2, S = 12, 9, 27
    rp, col = I.dbm_graph(N1, N2)
    inst = [I.dbm_instance(N1, N2, seed=k) for k in range(S)]
    C, M, lam4, pq = I.dbm_shots(N1, N2, [(c, m) for c, m, _, _ in inst],
                                 np.tile([2.0, 2.0, 12.0, 12.0], (S, 1)), (0.25, 0.25))
    kw = dict(problem=cpra.DBM, S=S, H0=32, H1=32, precision=cpra.BF16, nu=0.1,
              schedule_steps=20, seed=4)
    a = cpra.Solver(rp, col, **kw)
    a.set_dbm(N1, C, M, lam4, pq)
    for t in range(12):
        a.step(t)
    b = cpra.Solver(rp, col, **kw)
    b.set_dbm(N1, C, M, lam4, pq)
    b.steps(0, 5)
    b.steps(5, 7)
    ra, _, xa = a.round_eval(want_bits=True)
    rb, _, xb = b.round_eval(want_bits=True)
    assert np.array_equal(a.P(), b.P())
    assert np.array_equal(a.get(cpra.T_THETA), b.get(cpra.T_THETA))
    assert np.array_equal(xa, xb)
    assert np.array_equal(ra, rb)
    a.close()
    b.close()


def _best_diverse_matching(C, M, N1, N2, p, q):
    best = 0.0
    for xbits in itertools.product([0, 1], repeat=N1 * N2):
        X = np.array(xbits).reshape(N1, N2)
        if (X.sum(axis=1) > 1).any() or (X.sum(axis=0) > 1).any():
            continue
        T, U = X.sum(), (M.reshape(N1, N2) * X).sum()
        if p * T - U > 0 or q * T - (T - U) > 0:
            continue
        best = max(best, float((C.reshape(N1, N2) * X).sum()))
    return best


def test_solve_on_a_tiny_penalty_grid():
    """A 3 x 4 instance on a 4 x 4 penalty grid: cpra_solve keeps, per shot,
    the feasible matching of largest reward; none exceeds the enumerated
    optimum, and the best found over the grid reaches it."""
    N1, N2 = 3, 4
    rp, col = I.dbm_graph(N1, N2)
    Cv, Mv, p, q = I.dbm_instance(N1, N2, seed=7, n_fields=3)
    opt = _best_diverse_matching(Cv.astype(np.float64), Mv.astype(np.float64), N1, N2, p, q)
    grid = np.array([(a, a, b, b) for a in (1.0, 2.0, 4.0, 8.0) for b in (1.0, 2.0, 4.0, 8.0)])
    C, M, lam4, pq = I.dbm_shots(N1, N2, [(Cv, Mv)], grid, (p, q))
    s = cpra.Solver(rp, col, problem=cpra.DBM, S=len(grid), H0=16, H1=16, lr=1e-2,
                    gamma0=-2.0, gamma1=0.5, schedule_steps=600, seed=1)
    s.set_dbm(N1, C, M, lam4, pq)
    best, best_step = s.solve(600, 20)
    s.close()
    assert (best["objective"] >= 0).all()          # the empty matching is feasible
    assert (best["violations"] == 0).all()
    assert (best["value"] <= opt + 1e-6).all()
    assert best["value"].max() >= opt - 1e-6


def test_errors():
    rp, col = I.dbm_graph(4, 5)
    s = cpra.Solver(rp, col, problem=cpra.DBM, S=8, H0=16, H1=16)
    with pytest.raises(cpra.CpraError) as e:
        s.step(0)
    assert e.value.status == cpra.CPRA_ESTATE
    C = np.zeros((20, 8), np.float32)
    lam4 = np.ones((8, 4), np.float32)
    pq = np.full((8, 2), 0.25, np.float32)
    with pytest.raises(cpra.CpraError):
        s.set_dbm(3, C, C, lam4, pq)                 # 3 does not divide 20
    with pytest.raises(cpra.CpraError):
        s.set_dbm(4, C, C + 2.0, lam4, pq)           # M outside [0, 1]
    s.set_dbm(4, C, C, lam4, pq)
    s.step(0)
    # a different N1 reallocates the instance buffers; the 4 x 5 constraint
    # graph is not the 5 x 4 one, so the aggregations gather again
    s.set_dbm(5, C, C, lam4, pq)
    s.step(1)
    assert np.isfinite(s.P()).all()
    s.close()
    m = cpra.Solver(rp, col, lam=np.ones(8, np.float32), problem=cpra.MIS, S=8, H0=16, H1=16)
    with pytest.raises(cpra.CpraError):
        m.set_dbm(4, C, C, lam4, pq)
    m.close()


def test_step_at_the_papers_width_matches_oracle():
    """The paper's DBM network is 2500 wide (H0 = H1; here 2512, the next
    multiple of 16) on the 11 x 11 penalty grid: wide aggregations in column
    slices and the dense layers with streamed weights, BF16 form."""
    out, ref, rec, ham, bits, inst, g, theta, X0, gamma, S, H = _run_step(
        cpra.BF16, N1=20, N2=25, S=121, H=2512, seed=3)
    tol = 2e-2
    assert np.abs(out["P"] - ref["P"]).max() <= tol
    t, rt = out["terms"], ref["terms"]
    norm = np.abs(rt["cost"]) + np.abs(rt["pen"]) + abs(gamma) * rt["ann"]
    L = t[:S] + t[S:2 * S] + gamma * t[2 * S:3 * S]
    Lr = rt["cost"] + rt["pen"] + gamma * rt["ann"]
    assert np.max(np.abs(L - Lr) / norm) <= tol
    lay = I.param_layout(H, H, S)
    for name in ("Wcat1", "b1", "Wcat2", "b2"):
        off, shape = lay[name]
        n = int(np.prod(shape))
        a, b = out["grad"][off:off + n], ref["grads"]["theta"][off:off + n]
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), name
    x = I.unpack_bits(bits, S).astype(np.int64)
    ev = O.integer_eval(g, x, np.ones(S), O.DBM, inst=inst)
    assert np.array_equal(rec["violations"], ev["violations"])
    assert np.allclose(rec["qubo"], ev["qubo"], rtol=1e-12, atol=1e-9)


def test_device_early_stop_matches_oracle_rule():
    """The device monitor on a DBM context (lambda vector of ones, the
    penalty carrying its own lambdas) stops where the oracle's rule does on
    the same per-step terms."""
    N1, N2, S, T = 8, 6, 12, 200
    rp, col = I.dbm_graph(N1, N2)
    C, M, lam4, pq, _ = _mixed_shots(N1, N2, S, seed=5)
    s = cpra.Solver(rp, col, problem=cpra.DBM, S=S, H0=16, H1=16, lr=1e-3, gamma0=-2.0,
                    gamma1=0.1, schedule_steps=T, es_tol=1e-2, es_patience=4, seed=3)
    s.set_dbm(N1, C, M, lam4, pq)
    seq, gammas = [], []
    for t in range(60):
        terms = s.step(t, want_terms=True).astype(np.float32)
        seq.append((terms[:S], terms[S:2 * S], terms[2 * S:3 * S]))
        gammas.append(float(np.float32(O.gamma_schedule(t, T, -2.0, float(np.float32(0.1))))))
    got = s.early_stop_step()
    s.close()
    want = O.early_stop_step(seq, gammas, np.full(S, 7.0), O.DBM, float(np.float32(1e-2)), 4)
    assert got == want
