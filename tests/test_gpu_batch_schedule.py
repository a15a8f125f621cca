"""Scheduling of fp_solve_batch: CTAs take instances from the context's work
counter (two CTAs per SM with five stages, their factors in per-CTA global
slots; one CTA per SM with three).  Every instance must be solved exactly once
on every call, whatever n is against the number of CTAs, and the result of an
instance must not depend on which CTA (and factor slot) took it: the batch
outputs equal, bit for bit, those of the instance solved alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_08040_gb300 import build, workloads      # noqa: E402

pytestmark = pytest.mark.gpu

DSPEC = workloads.DriveSpec(amp=(0.010, 0.006, 0.0), freq=(50e3, 60e3, 0.0), phase=(0.0, 0.0, 0.0),
                            period=1e-4, samples_per_period=64, warmup_periods=0, output_periods=1)


@pytest.fixture(scope="module")
def fp():
    build.build()
    from paper_2106_08040_gb300 import fp as fpmod
    return fpmod


def solve(fp, ctx, inst):
    dev = torch.device("cuda")
    n, S = len(inst), ctx.num_samples()
    d_inst = fp.instances_to_device(inst, dev)
    m = torch.full((n, S, 3), np.nan, dtype=torch.float64, device=dev)
    dm = torch.full((n, S, 3), np.nan, dtype=torch.float64, device=dev)
    st = torch.full((n,), -1, dtype=torch.int32, device=dev)
    stats = torch.full((n, 4), -1, dtype=torch.int32, device=dev)
    fp.fp_solve_batch(ctx, d_inst, n, m, dm, st, stats)
    torch.cuda.synchronize()
    return m.cpu().numpy(), dm.cpu().numpy(), st.cpu().numpy(), stats.cpu().numpy()


@pytest.mark.parametrize("stages", [5, 3])
def test_every_instance_once_on_repeated_calls(fp, stages):
    """n = 1, one more than two CTAs per SM, and a ragged multiple: all statuses
    and outputs written on each of two consecutive calls (a counter that were
    not reset would leave the second call's buffers untouched), identical across
    the calls and equal to single-instance solves."""
    ctx = fp.Context(fp.Material(), fp.Drive(**DSPEC.__dict__), fp.Tol(rtol=1e-9, stages=stages), 10)
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    inst_all = workloads.random_instances(2 * n_sms + 1, 10, seed=5, max_offset=0.004, K_range=(5e2, 3e3))
    try:
        for n in (1, 2 * n_sms + 1):
            inst = inst_all[:n]
            first = solve(fp, ctx, inst)
            second = solve(fp, ctx, inst)
            for out in (first, second):
                assert (out[2] == 0).all()
                assert (out[3][:, 0] > 0).all()
                assert np.isfinite(out[0]).all() and np.isfinite(out[1]).all()
            for a, b in zip(first, second):
                np.testing.assert_array_equal(a, b)
            for i in sorted({0, n // 2, n - 1}):
                alone = solve(fp, ctx, inst[i:i + 1])
                np.testing.assert_array_equal(alone[0][0], first[0][i])
                np.testing.assert_array_equal(alone[1][0], first[1][i])
                np.testing.assert_array_equal(alone[3][0], first[3][i])
    finally:
        ctx.close()
