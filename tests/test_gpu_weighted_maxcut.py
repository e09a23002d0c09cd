"""MaxCut with edge weights A_ij (Table objective-functions: the QUBO
sum_ij A_ij (2 x_i x_j - x_i - x_j)) on the GPU: one full step against the
FP64 oracle holding the same weights (FP32 1e-5, BF16 2e-2, the same
measures as the unweighted step tests), through both loss kernels (S <= 64
in registers, S > 64 staged through shared memory), and the records of the
rounded step against the oracle's evaluation: cut edge counts bit-exact, cut
weights (summed in FP64 on both sides) to 1e-12 relative."""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402
from test_gpu_parity import _check_step, _run_step_case, unpack_bits  # noqa: E402

WEIGHTED_CASES = [
    # problem, div, alpha, nu, S, H, N, graph; edge weights
    ((O.MAXCUT, O.DIV_STD, 2, 0.2, 40, 32, 900, ("er", 8)), "uniform"),
    ((O.MAXCUT, O.DIV_VAR, 2, 0.1, 64, 32, 1202, ("rrg", 5)), "pm1"),
    ((O.MAXCUT, O.DIV_STD, 2, 0.2, 100, 48, 700, ("rrg", 6)), "uniform"),
    ((O.MAXCUT, O.DIV_STD, 2, 0.0, 256, 32, 1500, ("er", 12)), "pm1"),
]


def _check_records(out, ref, S, tol):
    x_gpu = unpack_bits(out["bits"], S)
    decided = np.abs(ref["P"] - 0.5) > tol
    assert np.array_equal(x_gpu[decided], ref["X"][decided])
    if decided.all():
        ev = ref["eval"]
        assert np.array_equal(out["rec"]["objective"], ev["objective"])
        assert np.array_equal(out["rec"]["violations"], ev["violations"])
        assert np.allclose(out["rec"]["value"], ev["value"], rtol=1e-12, atol=1e-9)
        assert out["ham"] == ev["pair_hamming"]
    assert np.array_equal(out["rec"]["qubo"], -out["rec"]["value"])


@pytest.mark.parametrize("precision,tol", [(cpra.FP32, 1e-5), (cpra.BF16, 2e-2)])
@pytest.mark.parametrize("case,weights", WEIGHTED_CASES)
def test_weighted_maxcut_step_matches_oracle(case, weights, precision, tol):
    out, ref, g, lam, gamma, theta, X0 = _run_step_case(case, precision, weights=weights)
    _check_step(out, ref, g, lam, gamma, theta, X0, case[4], case[5], tol, case[0])
    _check_records(out, ref, case[4], 1e-5 if precision == cpra.FP32 else 2e-2)


def test_weighted_records_of_the_gpu_rounding():
    """Whatever the step's P, the records of its rounding equal the oracle's
    evaluation of the GPU's own bits (no tolerance band at P = 0.5)."""
    rp, col = I.random_regular_graph(3000, 7, seed=41)
    w = I.seeded_edge_weights(rp, col, seed=42, kind="pm1")
    s = cpra.Solver(rp, col, problem=cpra.MAXCUT, S=70, H0=16, H1=16, precision=cpra.BF16,
                    weights=w)
    s.step(0)
    rec, ham, bits = s.round_eval(want_bits=True)
    s.close()
    x = unpack_bits(bits, 70)
    ev = O.integer_eval(O.Graph(rp, col, weights=w), x, np.zeros(70), O.MAXCUT)
    assert np.array_equal(rec["objective"], ev["objective"])
    assert np.allclose(rec["value"], ev["value"], rtol=1e-12, atol=1e-9)
    assert np.array_equal(rec["qubo"], -rec["value"])
    assert ham == ev["pair_hamming"]


def test_weighted_maxcut_solve_keeps_the_heaviest_cut():
    """With signed weights the heaviest cut need not cut the most edges:
    cpra_solve keeps, per shot, the evaluation with the largest cut weight,
    which no cut can push past the total positive weight."""
    rp, col = I.random_regular_graph(600, 4, seed=31)
    w = I.seeded_edge_weights(rp, col, seed=32, kind="pm1")
    s = cpra.Solver(rp, col, problem=cpra.MAXCUT, S=16, H0=16, H1=16, precision=cpra.FP32,
                    schedule_steps=300, weights=w)
    best, step = s.solve(300, 50)
    s.close()
    g = O.Graph(rp, col, weights=w)
    assert np.all(step >= 0)
    assert np.all(best["value"] > 0)
    assert np.all(best["value"] <= g.ew[g.ew > 0].sum())
    assert np.array_equal(best["qubo"], -best["value"])
