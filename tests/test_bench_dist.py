"""The multi-rank path of the benchmark on CPU: two gloo ranks agree on the
slowest rank's time and on the whole-job throughput (replicas, weak
scaling); and the benchmark's argument checks."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx = bench.max_over_ranks(10.0 + 5.0 * rank)
    val = bench.whole_job_value(world, 1000, 3, mx)
    out.put((rank, mx, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    expect = 2 * 1000 * 3 / (15.0 * 1e-3) / 1e9
    assert all(abs(r[2] - expect) < 1e-15 for r in res)


def test_single_process_is_its_own_max():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_value(1, 2000, 2, 4.0) == pytest.approx(2000 * 2 / 4e-3 / 1e9)


def test_edge_option_only_with_the_profiling_modes():
    """--edge (another box size) is accepted by the solve and ax modes only,
    so that the bench line always measures the stated workload."""
    import bench
    a = bench.parse(["--mode", "solve", "--edge", "24", "--order", "7"])
    assert (a.edge, a.order) == (24, 7)
    assert bench.parse([]).edge == 0
    for mode in ("full", "sweep", "batched"):
        with pytest.raises(SystemExit):
            bench.parse(["--mode", mode, "--edge", "24"])
