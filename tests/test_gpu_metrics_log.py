"""The JSON-lines metrics log of cpra_solve: one line per evaluation with
the step index, gamma_t, the loss terms, the rounded shots' records and
sum_i k_i (S - k_i), consistent with what the solve returns and with the
oracle's evaluation of the final step's rounding."""
import json

import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402


def test_metrics_log_one_line_per_evaluation(tmp_path):
    N, S, steps, every = 2000, 24, 250, 100
    rp, col = I.random_regular_graph(N, 4, seed=21)
    lam = I.lambda_geomspace(0.5, 4.0, S)
    s = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=S, H0=32, H1=32, precision=cpra.BF16,
                    gamma0=-1.0, gamma1=0.5, schedule_steps=steps, nu=0.1)
    log = tmp_path / "metrics.jsonl"
    s.set_metrics_log(str(log))
    best, best_step = s.solve(steps, every)
    # the last evaluation is the context's current state
    rec, ham, bits = s.round_eval(want_bits=True)
    terms = s.get(cpra.T_TERMS)
    s.set_metrics_log(None)
    s.close()
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    # evaluations at step 0, every `every` steps, and the last step
    assert [x["t"] for x in lines] == [0, 100, 200, 249]
    assert [x["steps"] for x in lines] == [1, 100, 100, 49]
    elapsed = [x["elapsed"] for x in lines]
    assert elapsed == sorted(elapsed) and all(x["seconds"] > 0 for x in lines)
    for x in lines:
        assert x["gamma"] == pytest.approx(O.gamma_schedule(x["t"], steps, -1.0, 0.5), rel=1e-6)
        for k in ("cost", "pen", "ann", "objective", "violations", "value"):
            assert len(x[k]) == S
        assert np.all(np.isfinite(x["cost"])) and np.isfinite(x["psi"])
    last = lines[-1]
    assert np.array_equal(last["objective"], rec["objective"])
    assert np.array_equal(last["violations"], rec["violations"])
    assert last["pair_hamming"] == ham
    t = terms.astype(np.float64)
    assert np.array_equal(np.float32(last["cost"]), np.float32(t[:S]))
    assert np.array_equal(np.float32(last["ann"]), np.float32(t[2 * S:3 * S]))
    assert np.float32(last["psi"]) == np.float32(t[3 * S])
    # the logged records are the oracle's evaluation of the rounded shots
    ev = O.integer_eval(O.Graph(rp, col), _unpack(bits, S), lam.astype(np.float64), O.MIS)
    assert np.array_equal(last["objective"], ev["objective"])
    assert last["pair_hamming"] == ev["pair_hamming"]
    # the solve's best per shot is the best feasible logged evaluation
    for sh in range(S):
        feas = [(x["objective"][sh], x["t"]) for x in lines if x["violations"][sh] == 0]
        if feas:
            assert best["objective"][sh] == max(o for o, _ in feas)
        else:
            assert best["objective"][sh] == -1 and best_step[sh] == -1


def _unpack(bits, S):
    x = np.zeros((bits.shape[0], S), dtype=np.int64)
    for sh in range(S):
        x[:, sh] = (bits[:, sh // 32] >> (sh % 32)) & 1
    return x


def test_metrics_log_bad_path_is_rejected():
    rp, col = I.random_regular_graph(100, 3, seed=2)
    s = cpra.Solver(rp, col, lam=np.ones(8, np.float32), problem=cpra.MIS, S=8)
    with pytest.raises(cpra.CpraError) as e:
        s.set_metrics_log("/nonexistent-dir/metrics.jsonl")
    assert e.value.status == cpra.CPRA_EINVAL
    s.close()
