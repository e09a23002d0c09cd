"""Parity at the benchmark's full size, in the launch configuration bench.py
times: MIS on a seeded random 5-regular graph with N = 10^6 nodes, S = 256
shots, H0 = H1 = 128, BF16 dense layers (and the all-FP32 form).

* Sampled outputs the oracle computes one by one: for a sample of nodes v,
  the oracle runs on the induced 3-hop ball around v.  A two-layer GCN's
  output at v depends only on nodes within two hops and the loss gradient at
  v on P within one hop, so P_v and dR/dZ2_v from the ball are exact.
* Properties that hold at any size, evaluated in FP64 from the exported P and
  rounded bits: the per-shot cost, penalty and annealing sums, and the exact
  integer evaluation (set sizes, violated edges, pairwise Hamming sum).
"""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402

N, D, S, H = 10**6, 5, 256, 128


@pytest.fixture(scope="module")
def graph():
    return I.random_regular_graph(N, D, seed=5)


def ball(rowptr, col, v, radius):
    seen = {v: 0}
    order = [v]
    frontier = [v]
    for r in range(radius):
        nxt = []
        for u in frontier:
            for w in col[rowptr[u]:rowptr[u + 1]]:
                w = int(w)
                if w not in seen:
                    seen[w] = len(order)
                    order.append(w)
                    nxt.append(w)
        frontier = nxt
    return order, seen


def induced(rowptr, col, order, seen):
    ei, ej = [], []
    for u in order:
        lu = seen[u]
        for w in col[rowptr[u]:rowptr[u + 1]]:
            lw = seen.get(int(w))
            if lw is not None and lu < lw:
                ei.append(lu)
                ej.append(lw)
    return I.edges_to_csr(len(order), np.array(ei), np.array(ej))


@pytest.mark.parametrize("precision,tol", [(cpra.BF16, 2e-2), (cpra.FP32, 1e-5)])
def test_full_size_step_sampled_and_properties(graph, precision, tol):
    rp, col = graph
    lam = I.lambda_geomspace(0.5, 10.0, S)
    theta, X0 = I.seeded_params(N, H, H, S, seed=21)
    gamma = -1.3
    solver = cpra.Solver(rp, col, lam=lam, problem=cpra.MIS, S=S, H0=H, H1=H,
                         precision=precision, gamma0=gamma, gamma1=gamma, schedule_steps=1)
    solver.set(cpra.T_THETA, theta)
    solver.set(cpra.T_EMB, X0)
    terms = solver.step(0, want_terms=True).astype(np.float64)
    P = solver.P()
    GZ2 = solver.get(cpra.T_GZ2).reshape(N, S)
    rec, ham, bits = solver.round_eval(want_bits=True)
    solver.close()

    # ---- sampled nodes against the oracle on their 3-hop balls ----
    rng = np.random.default_rng(7)
    decision = "bf16" if precision == cpra.BF16 else None
    for v in rng.choice(N, size=24, replace=False):
        order, seen = ball(rp, col, int(v), 3)
        srp, scol = induced(rp, col, order, seen)
        g = O.Graph(srp, scol)
        c = O.forward(g, theta, X0[order], H, H, S, relu_decision=decision)
        GP = O.grad_P(g, c["P"], lam.astype(np.float64), O.MIS, 2, gamma, 0.0)
        p_ref = c["P"][0]
        gz_ref = GP[0] * p_ref * (1.0 - p_ref)
        assert np.abs(P[v] - p_ref).max() <= tol
        assert np.linalg.norm(GZ2[v] - gz_ref) <= tol * np.linalg.norm(gz_ref) + 1e-30
        x_ref = (p_ref > 0.5)
        decided = np.abs(p_ref - 0.5) > tol
        x_gpu = np.array([(bits[v, s // 32] >> (s % 32)) & 1 for s in range(S)], dtype=bool)
        assert np.array_equal(x_gpu[decided], x_ref[decided])

    # ---- whole-graph sums as properties of the exported P (FP64) ----
    P64 = P.astype(np.float64)
    cost = -P64.sum(axis=0)
    ann = (1.0 - (2.0 * P64 - 1.0) ** 2).sum(axis=0)
    ei, ej = I.csr_to_edges(rp, col)
    pen = np.zeros(S)
    for a in range(0, len(ei), 200_000):
        pen += (P64[ei[a:a + 200_000]] * P64[ej[a:a + 200_000]]).sum(axis=0)
    norm = np.abs(cost) + lam * np.abs(pen) + abs(gamma) * ann
    Lg = terms[:S] + lam * terms[S:2 * S] + gamma * terms[2 * S:3 * S]
    Lr = cost + lam * pen + gamma * ann
    assert np.max(np.abs(Lg - Lr) / norm) <= 1e-5
    assert np.max(np.abs(terms[2 * S:3 * S] - ann) / ann) <= 1e-5

    # ---- exact integer evaluation as a property of the returned bits ----
    b8 = bits.view(np.uint8)                       # N x 32 bytes, little-endian bit order
    size = np.unpackbits(b8, axis=1, bitorder="little").sum(axis=0, dtype=np.int64)
    viol = np.zeros(S, dtype=np.int64)
    for a in range(0, len(ei), 500_000):
        both = b8[ei[a:a + 500_000]] & b8[ej[a:a + 500_000]]
        viol += np.unpackbits(both, axis=1, bitorder="little").sum(axis=0, dtype=np.int64)
    assert np.array_equal(rec["objective"], size[:S])
    assert np.array_equal(rec["violations"], viol[:S])
    assert np.array_equal(rec["qubo"], -size[:S].astype(np.float64) + lam.astype(np.float64) * viol[:S])
    k = np.unpackbits(b8, axis=1, bitorder="little").sum(axis=1, dtype=np.int64)
    assert ham == int((k * (S - k)).sum())
    # bits agree with the exported P everywhere (same FP32 decision)
    x_from_P = np.packbits(P > np.float32(0.5), axis=1, bitorder="little")
    assert np.array_equal(x_from_P, b8)
