"""NVTX ranges (tracing): the library opens a range in the "cpra" domain for
each ABI call that launches work and for each kernel region of a step.  The
ranges are recorded through an NVTX injection library of the tests' own
(tests/nvtx_record.c, loaded through NVTX_INJECTION64_PATH in a child
process).  On the CPU an op-level call that is rejected on the host still
opens and closes its range; on the GPU one step shows every kernel region of
the schedule in order."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _recorder(tmp_path):
    so = str(tmp_path / "nvtx_record.so")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["gcc", "-shared", "-fPIC", "-O2", "-I", cuda_inc, "-o", so,
                    os.path.join(HERE, "nvtx_record.c")], check=True)
    return so


def _run_recorded(tmp_path, code):
    log = tmp_path / "nvtx.log"
    env = dict(os.environ, NVTX_INJECTION64_PATH=_recorder(tmp_path), CPRA_NVTX_LOG=str(log),
               PYTHONPATH=ROOT)
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=ROOT, timeout=600)
    return log.read_text().split("\n")[:-1]


def test_rejected_op_call_opens_and_closes_its_range(tmp_path):
    from paper_2402_02190_gb300 import build as B
    B.build()
    code = ("from paper_2402_02190_gb300 import cpra\n"
            "L = cpra.lib()\n"
            "st = L.cpra_op_loss(0, 1, None, None, None, 4, None, 0, 2, 0.0, 0.0, 0, 0, None, 4,"
            " None, None, None, 0, None)\n"
            "assert st == cpra.CPRA_EINVAL, st\n")
    assert _run_recorded(tmp_path, code) == ["cpra_op_loss", "<pop>"]


# the step's schedule: forward, fused loss, evaluation of the rounded shots,
# adjoint, embedding update fused into the last aggregation, Adam
STEP_REGIONS = ["spmm_agg1", "gemm_layer1", "spmm_agg2", "gemm_layer2", "loss_fused",
                "loss_finalize", "round_eval", "wgrad2", "gemm_dgrad2", "spmm_bwd2", "wgrad1",
                "gemm_dgrad1", "spmm_bwd1_adam_embedding", "adam"]


@pytest.mark.gpu
def test_step_shows_every_kernel_region(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("needs a GPU")
    code = ("from paper_2402_02190_gb300 import cpra, inputs as I\n"
            "rp, col = I.random_regular_graph(3000, 5, seed=1)\n"
            "s = cpra.Solver(rp, col, lam=I.lambda_geomspace(0.5, 10.0, 100), problem=cpra.MIS,"
            " S=100, H0=64, H1=64, precision=cpra.BF16)\n"
            "s.step(0, want_terms=True)\n"
            "s.round_eval()\n"
            "s.close()\n")
    lines = _run_recorded(tmp_path, code)
    names = [x for x in lines if x != "<pop>"]
    assert lines.count("<pop>") == len(names)          # every range closed
    i = names.index("cpra_step")
    step = names[i + 1:]
    # the schedule's kernel regions, in order, inside the step
    pos = [step.index(r) for r in STEP_REGIONS]
    assert pos == sorted(pos), list(zip(STEP_REGIONS, pos))
    assert "cpra_round_eval" in names
