"""The two-stage S' -> S schedule end to end on a small weighted-MIS case:
the warm-up network's encoder is carried into the fine-tuning context,
stays frozen there, and the fresh head finds feasible weighted sets."""
import numpy as np
import pytest

from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402
from paper_2402_02190_gb300 import two_stage as TS  # noqa: E402


def test_two_stage_carries_and_freezes_the_encoder():
    rp, col = I.random_regular_graph(200, 5, seed=11)
    S, Sp = 24, 8
    W = np.random.default_rng(2).uniform(0.0, 1.0, size=(200, S)).astype(np.float32)
    lam = np.full(S, 2.0, np.float32)
    r = TS.run_two_stage(rp, col, W, lam, Sp, 1200, 400, H=32, precision=cpra.BF16,
                         eval_every=50, lr=1e-2)
    assert r["encoder_unchanged"]
    assert r["feasible_tasks"] > S // 2
    ok = np.isfinite(r["best"])
    assert np.all(r["best"][ok] >= 0.0) and r["avg_weight"] > 0.0   # the empty set is feasible
    # a feasible weight never exceeds the sum of the task's weights
    assert np.all(r["best"][ok] <= W.sum(axis=0)[ok] + 1e-6)
    sc = TS.run_scratch(rp, col, W, lam, 1600, H=32, precision=cpra.BF16, eval_every=50, lr=1e-2)
    assert sc["feasible_tasks"] > 0
