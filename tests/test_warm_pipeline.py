"""Host logic of the warm-start pipeline: graph batching and seeded graph
sets (no GPU)."""
import numpy as np

from paper_2402_02190_gb300 import inputs as I
from paper_2402_02190_gb300 import warm as WM


def test_disjoint_union_is_the_block_diagonal_graph():
    a = I.random_regular_graph(10, 3, seed=1)
    b = I.erdos_renyi_graph(7, 0.4, seed=2)
    c = I.random_regular_graph(6, 2, seed=3)
    rp, col = WM.disjoint_union([a, b, c])
    assert len(rp) == 10 + 7 + 6 + 1 and rp[-1] == a[0][-1] + b[0][-1] + c[0][-1]
    assert np.all(np.diff(rp) >= 0)
    ei, ej = I.csr_to_edges(rp, col)
    want = set()
    for off, (r, cc) in zip((0, 10, 17), (a, b, c)):
        for i, j in zip(*I.csr_to_edges(r, cc)):
            want.add((i + off, j + off))
    assert set(zip(ei.tolist(), ej.tolist())) == want
    # rows stay sorted and inside their own block
    for i in range(23):
        row = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0)
        blk = 0 if i < 10 else (1 if i < 17 else 2)
        lo, hi = (0, 10) if blk == 0 else ((10, 17) if blk == 1 else (17, 23))
        assert np.all((row >= lo) & (row < hi))


def test_training_graphs_are_seeded_and_valid():
    g1 = WM.training_graphs(5, seed=4, n_min=50, n_max=80)
    g2 = WM.training_graphs(5, seed=4, n_min=50, n_max=80)
    for (r1, c1, d1), (r2, c2, d2) in zip(g1, g2):
        assert d1 == d2 and np.array_equal(r1, r2) and np.array_equal(c1, c2)
        N = len(r1) - 1
        assert 50 <= N <= 81 and (N * d1) % 2 == 0
        assert np.all(np.diff(r1) == d1)


def test_time_to_reach_and_best_feasible():
    tr = [(0.1, 50, 3), (0.2, 100, 9), (0.3, 150, 10)]
    assert WM.time_to_reach(tr, 9) == (0.2, 100)
    assert WM.time_to_reach(tr, 11) is None
    rec = np.zeros(3, dtype=[("objective", "<i8"), ("violations", "<i8"), ("qubo", "<f8")])
    rec["objective"] = [5, 9, 7]
    rec["violations"] = [0, 2, 0]
    assert WM.best_feasible(rec) == 7
    assert WM.best_feasible(rec, problem=1) == 9


def test_union_targets_pack_in_order_and_split_back(monkeypatch):
    """Multi-instance target solves: graphs are packed in order into unions of
    at most max_nodes nodes, each union is solved once, and each graph gets
    back exactly its own rows of the union's bits."""
    graphs = [(r, c) for r, c, _ in WM.training_graphs(6, seed=3, n_min=20, n_max=40)]
    sizes = [len(r) - 1 for r, _ in graphs]
    solved = []

    def fake_solve(rp, col, S, lam, steps, precision, H=64, seed=1, problem=0):
        # row i of the union carries its union row index, so a graph's slice
        # tells where it was cut from
        solved.append((len(rp) - 1, seed))
        assert np.all(np.diff(rp) >= 0)
        N = len(rp) - 1
        return np.arange(N, dtype=np.uint32)[:, None].repeat((S + 31) // 32, 1), None

    monkeypatch.setattr(WM, "cpra_targets", fake_solve)
    out = WM.cpra_targets_union(graphs, 64, None, 10, max_nodes=70, seed=5)
    # greedy packing in order, never above the budget
    unions, cur = [], 0
    for n in sizes:
        if cur and cur + n > 70:
            unions.append(cur)
            cur = 0
        cur += n
    unions.append(cur)
    assert [u for u, _ in solved] == unions
    assert [s for _, s in solved] == [5 + k for k in range(len(unions))]
    assert [o.shape for o in out] == [(n, 2) for n in sizes]
    k = 0
    for u in unions:
        off = 0
        while off < u:
            assert np.array_equal(out[k][:, 0], np.arange(off, off + sizes[k]))
            off += sizes[k]
            k += 1
    assert k == len(graphs)
