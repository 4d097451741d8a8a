"""The benchmark's multi-rank host logic on CPU with two gloo ranks: each
rank runs its own condition (weak scaling, no data-path collective) and the
step time reported is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1503_03806_gb300 import synth
    w = synth.WORKLOADS["medium"]
    T = bench.rank_temperature(w, rank, world)
    local = 10.0 + rank * 5.0
    m = bench.max_over_ranks(local, dist, "cpu")
    out.put((rank, T, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, T0, m0), (r1, T1, m1) = res
    assert T0 != T1 and {T0, T1} == {500.0, 3000.0}
    assert m0 == m1 == 15.0


def test_single_rank_uses_the_workload_condition():
    import bench
    from paper_1503_03806_gb300 import synth
    w = synth.WORKLOADS["medium"]
    assert bench.rank_temperature(w, 0, 1) == w["T"][0]
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
