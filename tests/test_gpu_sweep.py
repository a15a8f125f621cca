"""Uneven sweeps (fp_sweep_*): bucketed, cost-ordered, work-counter launches
captured in a CUDA graph, and the per-bucket autotuner.

A sweep runs the same per-instance solve as fp_solve_batch (only the launch
degree, the order and the CTA that takes an instance differ), so with the
context's settings its outputs equal fp_solve_batch's bit for bit.  After
autotuning a bucket may use another Radau stage count or refactorisation
interval; both runs then converge to the same trajectory within the
integrator tolerance (rtol 1e-10 here), checked at 1e-8 relative L2.
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


def uneven(fp, n=300):
    inst = workloads.random_instances(n, 16, seed=21, max_offset=0.004, K_range=(5e2, 3e3))
    inst["L"] = fp.truncation_degree(inst, drive=fp.Drive(**DSPEC.__dict__), L_min=8, L_max=16)
    return inst


def buffers(n, S):
    dev = torch.device("cuda")
    return (torch.full((n, S, 3), np.nan, dtype=torch.float64, device=dev),
            torch.full((n, S, 3), np.nan, dtype=torch.float64, device=dev),
            torch.full((n,), -1, dtype=torch.int32, device=dev),
            torch.zeros((n, 4), dtype=torch.int32, device=dev))


def test_sweep_matches_solve_batch_and_replays(fp):
    ctx = fp.Context(fp.Material(), fp.Drive(**DSPEC.__dict__), fp.Tol(rtol=1e-10, stages=3), 16)
    inst = uneven(fp)
    assert len(set(inst["L"].tolist())) >= 3
    m_ref, dm_ref, st_ref, _ = fp.solve(ctx, inst)
    torch.cuda.synchronize()
    assert (st_ref.cpu().numpy() == 0).all()
    sw = fp.Sweep(ctx, inst, bucket_width=1)
    info = sw.info()
    assert sum(b["count"] for b in info) == len(inst)
    assert [b["L"] for b in info] == sorted([b["L"] for b in info], reverse=True)
    d_inst = fp.instances_to_device(inst, torch.device("cuda"))
    s = torch.cuda.Stream()
    m, dm, st, stats = buffers(len(inst), ctx.num_samples())
    for _ in range(2):                       # capture, then graph replay
        m.fill_(np.nan); dm.fill_(np.nan); st.fill_(-1)
        with torch.cuda.stream(s):
            sw.run(d_inst, m, dm, st, stats, stream=s)
        s.synchronize()
        assert (st.cpu().numpy() == 0).all()
        np.testing.assert_array_equal(m.cpu().numpy(), m_ref.cpu().numpy())
        np.testing.assert_array_equal(dm.cpu().numpy(), dm_ref.cpu().numpy())
    sw.close()
    ctx.close()


def test_autotuned_sweep_converges_to_the_same_trajectories(fp):
    ctx = fp.Context(fp.Material(), fp.Drive(**DSPEC.__dict__), fp.Tol(rtol=1e-10, stages=3), 16)
    inst = uneven(fp, 200)
    m_ref, _, st_ref, _ = fp.solve(ctx, inst)
    sw = fp.Sweep(ctx, inst, bucket_width=2)
    d_inst = fp.instances_to_device(inst, torch.device("cuda"))
    s = torch.cuda.Stream()
    m, dm, st, stats = buffers(len(inst), ctx.num_samples())
    with torch.cuda.stream(s):
        sw.autotune(d_inst, m, dm, st, sample=16, stream=s)
        sw.run(d_inst, m, dm, st, stats, stream=s)
    s.synchronize()
    info = sw.info()
    assert all(b["tuned_ms"] > 0 for b in info), info
    assert all(b["stages"] in (3, 5) and b["refactor_every"] in (8, 16) for b in info)
    assert (st.cpu().numpy() == 0).all()
    a, r = m.cpu().numpy(), m_ref.cpu().numpy()
    err = np.linalg.norm((a - r).reshape(len(inst), -1), axis=1) / np.linalg.norm(r.reshape(len(inst), -1), axis=1)
    assert err.max() < 1e-8, err.max()
    sw.close()
    ctx.close()
