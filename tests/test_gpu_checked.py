"""The checked build (libcpra_checked.so: every kernel that walks the graph
tests each CSR row range and column index before using it) on the GPU.

1. On valid graphs it computes what the release build computes: a full step
   in both forms against the FP64 oracle with the usual bars, the op-level
   loss and evaluation bit-equal to the release library's, and no failed
   check.
2. On device CSR arrays outside the op-level contract -- a column index out
   of range, row offsets that decrease, go negative or pass rowptr[N] -- the
   kernels read the failing row as empty and the failing index as node 0
   (so every access stays inside the arrays) and count the failure;
   cpra_csr_check reports the smallest failing row / CSR position, and the
   next valid call reports none.

The out-of-contract inputs go to the checked build only: the fixture selects
it and asserts that it answers cpra_csr_check with a count (the release
build answers -1) before any test runs."""
import numpy as np
import pytest

from oracle import cpra_oracle as O
from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402
from test_gpu_parity import _check_step, _run_step_case, dev_csr, rup  # noqa: E402


@pytest.fixture
def checked():
    prev = cpra.use_library("checked")
    try:
        assert cpra.lib()._name.endswith("libcpra_checked.so")
        n, _, _ = cpra.cpra_csr_check()  # also clears anything left over
        assert n >= 0, "the selected library is not the checked build"
        yield
    finally:
        cpra.use_library(prev)


def _op_buffers(N, S, seed):
    P = I.seeded_P(N, S, seed=seed)
    ld = rup(S, 16)
    Pd = torch.full((N, ld), 0.75, device="cuda")
    Pd[:, :S] = torch.from_numpy(P).cuda()
    lam = torch.from_numpy(I.lambda_geomspace(0.5, 10.0, S)).cuda()
    return P, Pd, lam, ld


def _op_loss(rpd, cold, Pd, lam, S, ld):
    """cpra_op_loss (MIS) and cpra_op_round_eval on one device graph; returns
    G, terms, bits, the records and the Hamming sum as host arrays."""
    N = Pd.shape[0]
    W = (S + 31) // 32
    G = torch.zeros((N, ld), device="cuda")
    bits = torch.zeros((N, W), dtype=torch.int32, device="cuda")
    terms = torch.zeros(4 * S + 1, device="cuda")
    scratch = torch.empty(cpra.cpra_op_loss_scratch_bytes(N, S), dtype=torch.uint8, device="cuda")
    cpra.cpra_op_loss(rpd, cold, Pd, lam, O.MIS, 2, -0.8, 0.37, O.DIV_STD, 0, G, bits, terms,
                      scratch)
    rec = torch.zeros(S * 4, dtype=torch.float64, device="cuda")
    ham = torch.zeros(1, dtype=torch.int64, device="cuda")
    cnt = torch.empty(cpra.cpra_op_round_eval_scratch_bytes(S), dtype=torch.uint8, device="cuda")
    bits2 = torch.zeros((N, W), dtype=torch.int32, device="cuda")
    cpra.cpra_op_round_eval(rpd, cold, Pd, S, lam, O.MIS, bits2, rec, ham, cnt)
    torch.cuda.synchronize()
    return (G.cpu().numpy(), terms.cpu().numpy(), bits.cpu().numpy(), rec.cpu().numpy(),
            int(ham.item()))


CASES = [
    (O.MIS, O.DIV_STD, 4, 0.3, 24, 32, 700, ("er", 5)),
    (O.MAXCUT, O.DIV_STD, 2, 0.2, 100, 48, 517, ("rrg", 20)),
]


@pytest.mark.parametrize("precision,tol", [(cpra.FP32, 1e-5), (cpra.BF16, 2e-2)])
@pytest.mark.parametrize("case", CASES)
def test_checked_full_step_matches_oracle(checked, case, precision, tol):
    out, ref, g, lam, gamma, theta, X0 = _run_step_case(case, precision)
    _check_step(out, ref, g, lam, gamma, theta, X0, case[4], case[5], tol, case[0])
    assert cpra.cpra_csr_check() == (0, -1, -1)


@pytest.mark.parametrize("S", [24, 100])
def test_checked_op_calls_equal_the_release_build(checked, S):
    """Both loss kernels (S = 24 in registers, S = 100 staged) and the
    evaluation: the checks change no result."""
    N = 1500
    rp, col = I.random_regular_graph(N, 6, seed=S)
    rpd, cold = dev_csr(rp, col)
    _, Pd, lam, ld = _op_buffers(N, S, seed=4)
    got = _op_loss(rpd, cold, Pd, lam, S, ld)
    assert cpra.cpra_csr_check() == (0, -1, -1)
    cpra.use_library("release")
    try:
        want = _op_loss(rpd, cold, Pd, lam, S, ld)
    finally:
        cpra.use_library("checked")
    for a, b in zip(got[:4], want[:4]):
        assert np.array_equal(a, b)
    assert got[4] == want[4]


@pytest.mark.parametrize("S", [24, 100])
def test_checked_build_records_bad_column_indices(checked, S):
    N = 2000
    rp, col = I.random_regular_graph(N, 4, seed=9)
    nnz = len(col)
    e0, e1 = nnz // 3, (2 * nnz) // 3
    bad = col.astype(np.int32).copy()
    bad[e0] = N          # one past the last node
    bad[e1] = -7
    rpd, _ = dev_csr(rp, col)
    badd = torch.from_numpy(bad).cuda()
    _, Pd, lam, ld = _op_buffers(N, S, seed=5)
    _op_loss(rpd, badd, Pd, lam, S, ld)
    n, row, ent = cpra.cpra_csr_check()
    assert n > 0 and row == -1 and ent == e0
    # a valid call afterwards finds nothing
    _op_loss(rpd, torch.from_numpy(col.astype(np.int32)).cuda(), Pd, lam, S, ld)
    assert cpra.cpra_csr_check() == (0, -1, -1)


@pytest.mark.parametrize("kind", ["past_nnz", "decreasing", "negative"])
@pytest.mark.parametrize("S", [24, 100])
def test_checked_build_records_bad_row_offsets(checked, kind, S):
    N = 2000
    rp, col = I.random_regular_graph(N, 4, seed=10)
    nnz = len(col)
    k = N // 2
    bad = rp.astype(np.int32).copy()
    if kind == "past_nnz":      # rows k-1 (end > nnz) and k (beg > end) fail
        bad[k] = nnz + 5
        first = k - 1
    elif kind == "decreasing":  # row k starts after it ends; row k-1 stays in range
        bad[k] = bad[k + 1] + 1
        first = k
    else:                       # rows k-1 (end < beg) and k (beg < 0) fail
        bad[k] = -3
        first = k - 1
    badd = torch.from_numpy(bad).cuda()
    cold = torch.from_numpy(col.astype(np.int32)).cuda()
    _, Pd, lam, ld = _op_buffers(N, S, seed=6)
    _op_loss(badd, cold, Pd, lam, S, ld)
    n, row, ent = cpra.cpra_csr_check()
    assert n > 0 and row == first and ent == -1
    _op_loss(torch.from_numpy(rp.astype(np.int32)).cuda(), cold, Pd, lam, S, ld)
    assert cpra.cpra_csr_check() == (0, -1, -1)


def test_checked_build_covers_the_aggregations(checked):
    """The row-gather SpMM (here the warm-start network's mean aggregations,
    which take a device CSR as given) records a bad column index too."""
    N, S = 1200, 8
    rp, col = I.random_regular_graph(N, 3, seed=12)
    bad = col.astype(np.int32).copy()
    e0 = len(col) // 2
    bad[e0] = N + 100
    net = cpra.WarmStartNet(N, len(col), F=16, H=32, S=S)
    try:
        rpd = torch.from_numpy(rp.astype(np.int32)).cuda()
        X = net.features(rpd, 3)
        net.predict(rpd, torch.from_numpy(bad).cuda(), X)
        n, row, ent = cpra.cpra_csr_check()
        assert n > 0 and row == -1 and ent == e0
        net.predict(rpd, torch.from_numpy(col.astype(np.int32)).cuda(), X)
        assert cpra.cpra_csr_check() == (0, -1, -1)
    finally:
        net.close()
