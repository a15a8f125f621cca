"""Multi-rank logic of bench.py on CPU (gloo, world size 2): each rank gets the
same voxel grid with its own easy-axis angle (no data exchanged), the step
time is the maximum over ranks, and the job throughput counts every rank's
instances."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    args = type("A", (), {"instances": 0, "warmup_periods": 1})()
    _, inst = bench.workload_for_rank(rank, args)
    ms = 100.0 + 50.0 * rank                      # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    q.put((rank, float(inst["phi"][0]), inst["h_off"].copy(), ms_max,
           bench.job_throughput(world, len(inst), 2, ms_max)))
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, phi0, off0, ms0, v0), (r1, phi1, off1, ms1, v1) = res
    assert phi0 == 0.0 and abs(phi1 - np.deg2rad(15.0)) < 1e-15
    np.testing.assert_array_equal(off0, off1)
    assert ms0 == ms1 == 150.0
    assert v0 == v1 == pytest.approx(2 * 1024 * 2 / 0.150)
