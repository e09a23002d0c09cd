"""Early stopping of the Implementation paragraph on the GPU: the device
monitor stops at the step the oracle's rule picks from the same per-step loss
terms, freezes the parameters from that step on, and ends cpra_solve."""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402


def _run(problem, lr, tol, patience, steps=60, precision=cpra.FP32):
    N, S, T = 300, 16, 400
    rp, col = I.random_regular_graph(N, 3, seed=4)
    lam = I.lambda_linspace(1.0, 4.0, S)
    g0, g1 = -2.0, 0.1
    s = cpra.Solver(rp, col, lam=lam if problem == cpra.MIS else None, problem=problem, S=S,
                    H0=16, H1=16, precision=precision, lr=lr, gamma0=g0, gamma1=g1,
                    schedule_steps=T, es_tol=tol, es_patience=patience, seed=3)
    seq, gammas, thetas = [], [], []
    for t in range(steps):
        terms = s.step(t, want_terms=True).astype(np.float32)
        seq.append((terms[:S], terms[S:2 * S], terms[2 * S:3 * S]))
        gammas.append(float(np.float32(O.gamma_schedule(t, T, float(np.float32(g0)),
                                                        float(np.float32(g1))))))
        thetas.append(s.get(cpra.T_THETA))
    want = O.early_stop_step(seq, gammas, lam.astype(np.float64), problem,
                             float(np.float32(tol)), patience)
    got = s.early_stop_step()
    steps_applied = int(s.get(cpra.T_STEP)[0])
    emb = s.get(cpra.T_EMB)
    s.close()
    return want, got, thetas, steps_applied, emb


@pytest.mark.parametrize("problem", [cpra.MIS, cpra.MAXCUT])
@pytest.mark.parametrize("lr,tol,patience", [(1e-7, 1e-5, 4), (1e-3, 2.0, 3), (1e-3, 1e-5, 5)])
def test_device_stop_step_equals_oracle_rule(problem, lr, tol, patience):
    want, got, thetas, applied, _ = _run(problem, lr, tol, patience)
    assert got == want
    if want >= 0:
        # the stopping step and every later one leave the parameters alone
        for t in range(want, len(thetas)):
            assert np.array_equal(thetas[t], thetas[want - 1]), t
        assert applied == want
    else:
        assert applied == len(thetas)


def test_tiny_learning_rate_stops_at_patience():
    """With a negligible learning rate every step after the first is stale
    (both monitored values move by far less than the tolerance)."""
    want, got, thetas, applied, _ = _run(cpra.MIS, 1e-9, 1e-2, 6, steps=20)
    assert want == got == 6
    assert applied == 6


def test_solve_ends_at_the_evaluation_after_stopping():
    N, S = 300, 16
    rp, col = I.random_regular_graph(N, 3, seed=4)
    lam = I.lambda_linspace(1.0, 4.0, S)
    s = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=S, H0=16, H1=16, lr=1e-9,
                    es_tol=1e-2, es_patience=7, seed=3)
    best, best_step = s.solve(10_000, 5)
    stop = s.early_stop_step()
    assert stop == 7
    assert int(s.get(cpra.T_STEP)[0]) == 7
    # the loop ended at the first evaluation after the stop (step 10), so no
    # recorded evaluation is later than that
    assert best_step.max() <= 10
    s.close()


def test_state_round_trip_keeps_the_stop():
    N, S = 300, 16
    rp, col = I.random_regular_graph(N, 3, seed=4)
    lam = I.lambda_linspace(1.0, 4.0, S)
    kw = dict(lam=lam, problem=cpra.MIS, S=S, H0=16, H1=16, lr=1e-9, es_tol=1e-2, es_patience=3,
              seed=3)
    a = cpra.Solver(rp, col, **kw)
    for t in range(8):
        a.step(t)
    blob = cpra.cpra_get_state(a.ctx)
    b = cpra.Solver(rp, col, **kw)
    cpra.cpra_set_state(b.ctx, blob)
    assert b.early_stop_step() == a.early_stop_step() == 3
    th = b.get(cpra.T_THETA)
    b.step(8)
    assert np.array_equal(b.get(cpra.T_THETA), th)
    a.close()
    b.close()
