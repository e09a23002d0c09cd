"""C-ABI library checks that need no GPU: it builds, loads, exports every
symbol include/cpra.h declares, and rejects bad graphs / configurations on
the host before touching the device."""
import os
import re

import numpy as np
import pytest

from paper_2402_02190_gb300 import build as B
from paper_2402_02190_gb300 import cpra
from paper_2402_02190_gb300 import inputs as I

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "cpra.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return cpra.lib()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^CPRA_API\s+[\w\s\*]*?\b(cpra_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cpra_init_graph", "cpra_step", "cpra_round_eval", "cpra_solve",
                 "cpra_op_loss", "cpra_op_round_eval", "cpra_destroy"):
        assert must in names
    assert set(names) == set(cpra.ABI_FUNCTIONS)


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_checked_library_exports_every_declared_symbol(L):
    """The checked build (in-kernel CSR checks) is the same ABI."""
    import ctypes
    Lc = ctypes.CDLL(cpra.LIB_CHECKED_PATH)
    for name in declared_functions():
        assert hasattr(Lc, name), name


def test_release_build_reports_no_csr_checks(L):
    """cpra_csr_check answers -1 from the release build (no device call)."""
    assert cpra.cpra_csr_check() == (-1, -1, -1)


def test_config_default_and_param_counts(L):
    cfg = cpra.cpra_config_default()
    assert (cfg.problem, cfg.S, cfg.H0, cfg.H1, cfg.alpha) == (cpra.MIS, 8, 16, 16, 2)
    assert cfg.lr == pytest.approx(1e-3) and cfg.beta2 == pytest.approx(0.999)
    assert cfg.gamma0 == pytest.approx(-2.0) and cfg.gamma1 == pytest.approx(0.1)
    assert (cfg.train_embedding, cfg.keep_emb_grad) == (1, 0)
    golden = os.path.join(os.path.dirname(__file__), "golden", "param_counts.txt")
    for line in open(golden):
        line = line.split("--")[0].strip()
        if line and not line.startswith("#"):
            H0, H1, S, count = (int(v) for v in line.split())
            assert cpra.cpra_param_count_for(H0, H1, S) == count


def test_workspace_bytes_valid_and_invalid(L):
    cfg = cpra.make_config(S=256, H0=128, H1=128, precision=cpra.BF16, problem=cpra.MAXCUT)
    nb = cpra.cpra_workspace_bytes(10**6, 5 * 10**6, cfg)
    # P alone is N * S * 4 bytes
    assert nb > 10**6 * 256 * 4
    bad = cpra.make_config(S=0)
    assert cpra.cpra_workspace_bytes(100, 300, bad) == 0
    bad = cpra.make_config(H0=24)
    assert cpra.cpra_workspace_bytes(100, 300, bad) == 0


def test_recompute_shares_activation_and_gradient_blocks(L):
    """recompute = 1 keeps no layer activations for the backward: [X0|M1]
    and [H1|M2] share memory with the same-shaped gradient blocks, and only
    the N x H1 ReLU mask bits are added."""
    N, nnz, H0, H1 = 10**6, 5 * 10**6, 128, 128
    for prec, act in ((cpra.BF16, 2), (cpra.FP32, 4)):
        kw = dict(S=256, H0=H0, H1=H1, precision=prec, problem=cpra.MAXCUT)
        full = cpra.cpra_workspace_bytes(N, nnz, cpra.make_config(recompute=0, **kw))
        lean = cpra.cpra_workspace_bytes(N, nnz, cpra.make_config(recompute=1, **kw))
        saved = 2 * N * (H0 + H1) * act - N * (H1 // 16) * 2
        assert abs((full - lean) - saved) <= 4 * 256
    rp, col = I.random_regular_graph(20, 3, seed=1)
    st, msg = _init_status(rp, col, recompute=2)
    assert st == cpra.CPRA_EINVAL and "recompute" in msg


def _init_status(rowptr, col, **kw):
    cfg = cpra.make_config(problem=cpra.MAXCUT, **kw)
    try:
        cpra.cpra_init_graph(rowptr, col, cfg, workspace=None)
    except cpra.CpraError as e:
        return e.status, str(e)
    return cpra.CPRA_OK, ""


@pytest.mark.parametrize("case", ["selfloop", "unsorted", "asym", "range", "rowptr0", "dup"])
def test_invalid_graphs_rejected_on_host(L, case):
    rp, col = I.random_regular_graph(20, 3, seed=1)
    rp = rp.copy()
    col = col.copy()
    if case == "selfloop":
        col[0] = 0
    elif case == "unsorted":
        col[0], col[1] = col[1], col[0]
    elif case == "asym":
        # 0 -> 1 and 1 -> 2 without the reverse entries
        rp, col = np.array([0, 1, 2, 2, 2]), np.array([1, 2], dtype=np.int32)
    elif case == "range":
        col[5] = 99
    elif case == "rowptr0":
        rp[0] = 1
    elif case == "dup":
        col[1] = col[0]
    st, msg = _init_status(rp, col)
    assert st == cpra.CPRA_EINVAL, msg


@pytest.mark.parametrize("first,second", [("range", "selfloop"), ("selfloop", "range"),
                                          ("asym", "range")])
def test_large_graph_reports_its_lowest_failing_row(L, first, second):
    """Graphs with at least 2^18 entries are checked on several host threads
    over row ranges; the message is the lowest failing row's, whatever the
    thread count.  Each planted defect replaces the entry (r, k) of the row's
    largest neighbour k > r, so the rows it unbalances lie above r."""
    N, d = 100_000, 6
    rp, col = I.random_regular_graph(N, d, seed=3)
    col = col.copy()

    def row_with_higher_neighbour(start):
        return next(r for r in range(start, N) if col[rp[r + 1] - 1] > r)

    def plant(kind, row):
        e0, e1 = int(rp[row]), int(rp[row + 1])
        if kind == "range":
            col[e1 - 1] = N + 7
            return "column index out of range"
        if kind == "selfloop":
            col[e1 - 1] = row
            col[e0:e1].sort()
            return f"self-loop at node {row}"
        nb = set(col[e0:e1].tolist())
        c = next(v for v in range(row + 1, N) if v not in nb)
        col[e1 - 1] = c
        col[e0:e1].sort()
        return f"not symmetric: ({row},{c})"

    r1 = row_with_higher_neighbour(20_000)
    r2 = row_with_higher_neighbour(90_000)
    want = plant(first, r1)
    plant(second, r2)
    st, msg = _init_status(rp, col)
    assert st == cpra.CPRA_EINVAL and want in msg, msg


def test_invalid_config_rejected_on_host(L):
    rp, col = I.random_regular_graph(20, 3, seed=1)
    st, _ = _init_status(rp, col, alpha=3)
    assert st == cpra.CPRA_EINVAL
    st, msg = _init_status(rp, col, keep_emb_grad=2)
    assert st == cpra.CPRA_EINVAL and "keep_emb_grad" in msg
    cfg = cpra.make_config(problem=cpra.MIS)   # MIS without lambda
    with pytest.raises(cpra.CpraError) as ei:
        cpra.cpra_init_graph(rp, col, cfg, workspace=None)
    assert ei.value.status == cpra.CPRA_EINVAL
    assert "lambda" in str(ei.value)


def test_memory_cap_fault_injection(L):
    """A configured allocation cap makes init fail with ENOMEM, on the host,
    before any device allocation."""
    rp, col = I.random_regular_graph(200, 3, seed=2)
    st, msg = _init_status(rp, col, mem_cap_bytes=1024)
    assert st == cpra.CPRA_ENOMEM, msg
    assert "mem_cap_bytes" in msg


def _init_weighted(rowptr, col, w, problem):
    lam = np.ones(8, np.float32) if problem == cpra.MIS else None
    cfg = cpra.make_config(problem=problem, S=8)
    try:
        cpra.cpra_init_graph(rowptr, col, cfg, lam=lam, workspace=None, weights=w)
    except cpra.CpraError as e:
        return e.status, str(e)
    return cpra.CPRA_OK, ""


@pytest.mark.parametrize("case", ["mis", "asym", "nan"])
def test_invalid_edge_weights_rejected_on_host(L, case):
    """Edge weights (the MaxCut QUBO's A_ij) are rejected before any device
    work when they are given for another problem, differ between the two
    CSR entries of an edge, or are not finite."""
    rp, col = I.random_regular_graph(20, 3, seed=1)
    w = I.seeded_edge_weights(rp, col, 2)
    problem = cpra.MAXCUT
    if case == "mis":
        problem = cpra.MIS
    elif case == "asym":
        w = w.copy()
        w[0] += 1.0
    else:
        w = w.copy()
        w[3] = np.nan
    st, msg = _init_weighted(rp, col, w, problem)
    assert st == cpra.CPRA_EINVAL
    assert {"mis": "CPRA_MAXCUT only", "asym": "symmetric", "nan": "finite"}[case] in msg
