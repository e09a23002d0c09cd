"""Config 1 on the GPU: the exhaustive check on the 16-node BFS subgraph
(reading c-14) and the end-to-end run of the 100-node graph beside the FP64
oracle's own run of the same settings (S = 8, lambda = 1..8, width 16, FP32,
Adam 1e-3, gamma -2 -> 0.1 over 3000 steps).  The two trajectories are not
expected to agree step for step after thousands of steps (the iteration is
chaotic); both must return valid independent sets, and on the subgraph the
CUDA path must reach the independence number found by enumeration."""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from oracle import exact as X
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402

from test_c1_exhaustive import c1_subgraph, oracle_cpra_run  # noqa: E402


def gpu_c1_run(rp, col, T=3000, seed=1, eval_every=50):
    N, S, H = len(rp) - 1, 8, 16
    lam = I.lambda_linspace(1.0, 8.0, S)
    theta, X0 = I.seeded_params(N, H, H, S, seed=seed)
    s = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=S, H0=H, H1=H, precision=cpra.FP32,
                    gamma0=-2.0, gamma1=0.1, schedule_steps=T, seed=seed)
    s.set(cpra.T_THETA, theta)
    s.set(cpra.T_EMB, X0)
    best, best_step = s.solve(T, eval_every)
    P = s.P()
    rec, ham, bits = s.round_eval(want_bits=True)
    s.close()
    return best, P, rec, ham, bits, lam


def _check_records(rp, col, P, rec, ham, bits, lam):
    """The records of the GPU's own final P equal the oracle's integer
    evaluation, bit for bit; shots without violations are independent sets."""
    g = O.Graph(rp, col)
    Xg = O.round_solutions(P)
    ev = O.integer_eval(g, Xg, lam.astype(np.float64), O.MIS)
    assert np.array_equal(bits, O.pack_bits(Xg))
    assert np.array_equal(rec["objective"], ev["objective"])
    assert np.array_equal(rec["violations"], ev["violations"])
    assert np.array_equal(rec["qubo"], ev["qubo"]) and ham == ev["pair_hamming"]
    adj = X.adjacency_sets(rp, col)
    for s in np.flatnonzero(rec["violations"] == 0):
        assert all(not (Xg[i, s] and Xg[j, s]) for i in range(len(adj)) for j in adj[i])


def test_gpu_cpra_reaches_the_independence_number_of_the_c1_subgraph():
    rp, col = c1_subgraph()
    adj = X.adjacency_sets(rp, col)
    alpha = X.max_independent_set_size(adj)
    best, P, rec, ham, bits, lam = gpu_c1_run(rp, col)
    feasible = best["violations"] == 0
    assert feasible.any() and int(best["objective"][feasible].max()) == alpha == 10
    _check_records(rp, col, P, rec, ham, bits, lam)


def test_gpu_c1_end_to_end_beside_the_oracle_run():
    import json
    import os
    import time
    rp, col = I.random_regular_graph(100, 3, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, P, rec, ham, bits, lam = gpu_c1_run(rp, col)
    t_gpu = time.perf_counter() - t0
    _check_records(rp, col, P, rec, ham, bits, lam)
    feasible = best["violations"] == 0
    gpu_best = int(best["objective"][feasible].max())
    t0 = time.perf_counter()
    ref_best, _ = oracle_cpra_run(rp, col)
    t_ref = time.perf_counter() - t0
    print(f"config 1 (N=100): GPU FP32 best feasible {gpu_best} in {t_gpu:.2f} s, "
          f"FP64 oracle {ref_best} in {t_ref:.2f} s")
    path = os.environ.get("CPRA_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": "c1_end_to_end", "gpu_fp32_best": gpu_best,
                                "gpu_seconds": t_gpu, "oracle_fp64_best": ref_best,
                                "oracle_seconds": t_ref, "gpu_final_objective":
                                [int(v) for v in rec["objective"]],
                                "gpu_final_violations": [int(v) for v in rec["violations"]]}) + "\n")
    # alpha(G) = 45 (exact MILP); both runs land within a few nodes of it
    assert 40 <= gpu_best <= 45 and 40 <= ref_best <= 45
