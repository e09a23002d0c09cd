"""The allocation-free loss entry point (cpra_op_loss_noalloc).

It serves callers that cannot call cudaMalloc (a host application that owns
all device memory, or a latency-critical path where an allocation is not
acceptable): its scratch lives in a fixed device array inside the library.
These checks call it through the C ABI and compare it with cpra_op_loss,
which takes caller-allocated scratch, on two calls in a row with different
inputs, so a stale counter or partial row from the first call would show in
the second.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402

TOL = 1e-5  # the FP32 tolerance of the parity tests


def _inputs(N, S, d, seed):
    rp, col = I.random_regular_graph(N, d, seed)
    P = I.seeded_P(N, S, seed)
    ld = (S + 15) // 16 * 16
    Pd = torch.zeros((N, ld), device="cuda")
    Pd[:, :S] = torch.from_numpy(P).cuda()
    lam = torch.from_numpy(I.lambda_geomspace(0.5, 10.0, S)).cuda()
    return (torch.tensor(rp.astype(np.int32), device="cuda"),
            torch.tensor(col.astype(np.int32), device="cuda"), Pd, lam, ld)


def _run(entry, N, S, d, seed, problem, div, with_bits=True, stream=None):
    rpd, cold, Pd, lam, ld = _inputs(N, S, d, seed)
    G = torch.full((N, ld), float("nan"), device="cuda")
    bits = torch.zeros((N, (S + 31) // 32), dtype=torch.int32, device="cuda") if with_bits else None
    terms = torch.zeros(4 * S + 1, device="cuda")
    args = (rpd, cold, Pd, lam, problem, 2, -0.6, 0.25, div, 0, G, bits, terms)
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())  # the inputs are ready
    if entry == "noalloc":
        cpra.cpra_op_loss_noalloc(*args, stream=stream)
    else:
        scratch = torch.empty(cpra.cpra_op_loss_scratch_bytes(N, S), dtype=torch.uint8,
                              device="cuda")
        cpra.cpra_op_loss(*args, scratch, stream=stream)
    torch.cuda.synchronize()
    return (G.cpu().numpy(), bits.cpu().numpy() if with_bits else None,
            terms.cpu().numpy().astype(np.float64))


def _close(a, b):
    scale = max(np.abs(b).max(), 1e-30)
    return np.abs(a - b).max() <= TOL * scale


def _compare(a, b, S):
    G1, b1, t1 = a
    G0, b0, t0 = b
    assert _close(G1, G0)
    if b0 is not None:
        assert np.array_equal(b1, b0)
    for q in range(3):                       # cost, pen, ann per shot
        assert _close(t1[q * S:(q + 1) * S], t0[q * S:(q + 1) * S])
    assert abs(t1[3 * S] - t0[3 * S]) <= TOL * abs(t0[3 * S])       # Psi
    assert _close(t1[3 * S + 1:], t0[3 * S + 1:])                    # column sums


def test_noalloc_matches_allocating_entry_on_two_calls_in_a_row():
    calls = [(200_002, 256, 5, 1, cpra.MIS, cpra.DIV_STD),
             (5_000, 37, 3, 2, cpra.MAXCUT, cpra.DIV_VAR)]
    for N, S, d, seed, problem, div in calls:
        _compare(_run("noalloc", N, S, d, seed, problem, div),
                 _run("alloc", N, S, d, seed, problem, div), S)


def test_noalloc_small_call_after_a_large_one_and_on_a_side_stream():
    """A call whose grid is set by its rows (fewer blocks than the cap) right
    after one that filled the whole array, at the same S, so a partial row
    left by the first call would be read by the second; then a call on a
    torch side stream without rounding bits."""
    S = 256
    _compare(_run("noalloc", 200_002, S, 5, 1, cpra.MIS, cpra.DIV_STD),
             _run("alloc", 200_002, S, 5, 1, cpra.MIS, cpra.DIV_STD), S)
    _compare(_run("noalloc", 700, S, 5, 4, cpra.MIS, cpra.DIV_STD),
             _run("alloc", 700, S, 5, 4, cpra.MIS, cpra.DIV_STD), S)
    side = torch.cuda.Stream()
    _compare(_run("noalloc", 3_001, S, 4, 5, cpra.MAXCUT, cpra.DIV_STD, with_bits=False,
                  stream=side),
             _run("alloc", 3_001, S, 4, 5, cpra.MAXCUT, cpra.DIV_STD, with_bits=False), S)


def test_noalloc_rejects_more_shots_than_its_scratch_holds():
    S = cpra.NOALLOC_MAX_S + 1
    N = 64
    rpd, cold, Pd, lam, ld = _inputs(N, S, 3, 3)
    G = torch.zeros((N, ld), device="cuda")
    terms = torch.zeros(4 * S + 1, device="cuda")
    st = cpra.lib().cpra_op_loss_noalloc(
        N, S, C.c_void_p(rpd.data_ptr()), C.c_void_p(cold.data_ptr()), C.c_void_p(Pd.data_ptr()),
        Pd.stride(0), C.c_void_p(lam.data_ptr()), cpra.MIS, 2, C.c_float(0.0), C.c_float(0.0), 0,
        0, C.c_void_p(G.data_ptr()), G.stride(0), None, C.c_void_p(terms.data_ptr()), None)
    assert st == cpra.CPRA_EINVAL
    with pytest.raises(cpra.CpraError):
        cpra.cpra_op_loss_noalloc(rpd, cold, Pd, lam, cpra.MIS, 2, 0.0, 0.0, 0, 0, G, None, terms)
