"""cpra_steps replays one captured training step as a CUDA graph: the steps
it runs are bit-identical to the same number of cpra_step calls (per-step
gamma and Adam bias corrections come from the device in both paths)."""
import numpy as np
import pytest

from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402


def _state(s):
    rec, ham, bits = s.round_eval(want_bits=True)
    return dict(P=s.P(), theta=s.get(cpra.T_THETA), emb=s.get(cpra.T_EMB),
                m=s.get(cpra.T_EMB_M), step=s.get(cpra.T_STEP), bits=bits,
                obj=rec["objective"], viol=rec["violations"], ham=ham)


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", [cpra.FP32, cpra.BF16])
@pytest.mark.parametrize("extra", [dict(), dict(recompute=1, nu=0.3),
                                   dict(problem=cpra.MAXCUT, diversity_kind=cpra.DIV_VAR, nu=0.1)])
def test_graph_replay_equals_single_steps(precision, extra):
    rp, col = I.random_regular_graph(1500, 4, seed=12)
    S = 40
    kw = dict(problem=cpra.MIS, S=S, H0=32, H1=48, precision=precision, schedule_steps=30, seed=4)
    kw.update(extra)
    lam = I.lambda_geomspace(0.5, 10, S) if kw["problem"] == cpra.MIS else None
    a = cpra.Solver(rp, col, lam=lam, **kw)
    for t in range(25):
        a.step(t)
    b = cpra.Solver(rp, col, lam=lam, **kw)
    b.steps(0, 10)        # first call: direct step + capture + 9 replays
    b.steps(10, 15)       # replays only
    _same(_state(a), _state(b))
    a.close()
    b.close()


def test_graph_replay_with_offset_and_early_stopping():
    """The warm-start offset set between calls (the captured step is rebuilt)
    and the device-side early stop behave as in the single-step path."""
    rp, col = I.random_regular_graph(800, 3, seed=2)
    S = 16
    lam = I.lambda_linspace(1, 4, S)
    kw = dict(problem=cpra.MIS, S=S, H0=16, H1=16, lr=1e-9, es_tol=1e-2, es_patience=5, seed=9)
    L0 = np.random.default_rng(3).normal(size=(800, S)).astype(np.float32)
    a = cpra.Solver(rp, col, lam=lam, **kw)
    for t in range(4):
        a.step(t)
    a.set_init_logits(L0)
    for t in range(4, 20):
        a.step(t)
    b = cpra.Solver(rp, col, lam=lam, **kw)
    b.steps(0, 4)
    b.set_init_logits(L0)
    b.steps(4, 16)
    assert a.early_stop_step() == b.early_stop_step() >= 0
    _same(_state(a), _state(b))
    a.close()
    b.close()
