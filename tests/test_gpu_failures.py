"""Failure detection without a GPU fault: the device error word that the
kernels set when a bounded wait gives up (CPRA_ETIMEOUT) or a loss term is
not finite (CPRA_ENUMERIC) is written from the host through the
fault-injection hook, and the calls that read it must report the status,
clear the word and leave the context usable."""
import numpy as np
import pytest

from paper_2402_02190_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2402_02190_gb300 import cpra  # noqa: E402

ETIMEOUT, ENUMERIC, EINVAL = 5, 4, 1


def _solver():
    rp, col = I.random_regular_graph(300, 3, seed=21)
    return cpra.Solver(rp, col, lam=I.lambda_linspace(1, 4, 8), problem=cpra.MIS, S=8, H0=16,
                       H1=16, precision=cpra.FP32, schedule_steps=100)


@pytest.mark.parametrize("bits,status", [(2, ETIMEOUT), (1, ENUMERIC), (3, ETIMEOUT)])
def test_injected_error_word_is_reported_once_and_cleared(bits, status):
    s = _solver()
    s.step(0, want_terms=True)
    cpra.cpra_inject_error_flag(s.ctx, bits)
    s.step(1)                       # asynchronous: does not read the word
    with pytest.raises(cpra.CpraError) as e:
        s.step(2, want_terms=True)
    assert e.value.status == status
    terms = s.step(3, want_terms=True)  # cleared: the context is usable again
    assert np.all(np.isfinite(terms))
    s.close()


def test_injected_timeout_ends_cpra_solve():
    s = _solver()
    cpra.cpra_inject_error_flag(s.ctx, 2)
    with pytest.raises(cpra.CpraError) as e:
        s.solve(40, 10)
    assert e.value.status == ETIMEOUT
    rec, step = s.solve(20, 10)        # and the next solve runs normally
    assert len(rec) == 8 and len(step) == 8
    s.close()


def test_injection_rejects_other_bits():
    s = _solver()
    for bits in (0, 4, -1):
        with pytest.raises(cpra.CpraError) as e:
            cpra.cpra_inject_error_flag(s.ctx, bits)
        assert e.value.status == EINVAL
    s.close()
