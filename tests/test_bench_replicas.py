"""The multi-GPU path of bench.py is independent replicas (one per rank, no
data-path collective); its only exchange is the max-over-ranks time.  This
checks that host logic with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # rank r "took" 10 + r seconds for its replica's 5 units
        t = bench.max_over_ranks(10.0 + rank, dist, device="cpu")
        out[rank] = (t, bench.replica_throughput(world, 5.0, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (11.0, 2 * 5.0 / 11.0)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(1, 10.0, 2.0) == 5.0


def test_roofline_byte_counts():
    """The loss kernel's algorithmic and compulsory bytes at the default
    workload (N = 10^6, nnz = 5*10^6, S = 256, BF16 G), from their parts."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    N, nnz, S = 10**6, 5 * 10**6, 256
    gather = nnz * S * 4            # every neighbour row of P, FP32
    own = N * S * 4                 # each row's own P row
    g_out = N * S * 2               # G_Z2 in BF16
    csr = 4 * (N + 1) + 4 * nnz
    bits = N * (S // 32) * 4
    assert bench.loss_kernel_bytes(N, nnz, S, 2) == gather + own + g_out + csr + bits == 6_712_000_004
    assert bench.loss_compulsory_bytes(N, nnz, S, 2) == own + g_out + csr + bits
    assert bench.loss_kernel_bytes(N, nnz, S, 4) - bench.loss_kernel_bytes(N, nnz, S, 2) == N * S * 2
