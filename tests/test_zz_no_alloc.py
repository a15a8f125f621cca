"""fp_grad_noalloc: the adjoint on the library's fixed scratch array.

Some callers may not allocate device memory when they call (a host program that
fixes this library's device-memory footprint, a service that must not grow or
fragment its memory); fp_grad_noalloc serves them from a static device array
instead of a caller-supplied workspace.  These checks call it through the C ABI
and compare it with fp_grad on the same inputs, twice in a row on different
instances (the second call reuses the array the first one left behind), with
a step budget that lets only two CTAs fit in the array so that each CTA takes
several instances in turn.  A request whose single instance cannot fit is
refused before any launch.

This file is collected last so that a stop-at-first-failure run has already
run every other test before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_08040_gb300 import build, workloads      # noqa: E402

pytestmark = pytest.mark.gpu

DSPEC = workloads.DriveSpec(amp=(0.010, 0.0, 0.0), freq=(50e3, 50e3, 50e3), phase=(0.0, 0.0, 0.0),
                            period=2e-5, samples_per_period=64, warmup_periods=0, output_periods=1)
CH = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
KMAX = 20
L = 8
RTOL = 1e-9          # the tolerance the adjoint tests hold fp_grad's autograd wrapper to


@pytest.fixture(scope="module")
def fp():
    build.build()
    from paper_2106_08040_gb300 import fp as fpmod
    return fpmod


def context(fp, max_steps):
    return fp.Context(fp.Material(), fp.Drive(**DSPEC.__dict__),
                      fp.Tol(rtol=1e-10, stages=3, max_steps=max_steps), L)


def inputs(fp, seed, n=3):
    inst = workloads.random_instances(n, L, seed=seed, max_offset=0.004, K_range=(5e2, 3e3))
    G = np.random.default_rng(seed + 100).normal(size=(n, 2, KMAX + 1, 2))
    dev = torch.device("cuda")
    return fp.instances_to_device(inst, dev), torch.from_numpy(G).to(dev), n


def outputs(n):
    dev = torch.device("cuda")
    return (torch.full((n, 4), np.nan, dtype=torch.float64, device=dev),
            torch.full((n,), -7, dtype=torch.int32, device=dev),
            torch.zeros((n, 4), dtype=torch.int32, device=dev))


def with_workspace(fp, ctx, d_inst, dJ, n):
    grad, st, stats = outputs(n)
    work = torch.empty(fp.fp_grad_workspace_bytes(ctx, n), dtype=torch.uint8, device=dJ.device)
    fp.fp_grad(ctx, d_inst, n, KMAX, CH, dJ, grad, st, work, d_stats=stats)
    torch.cuda.synchronize()
    return grad.cpu().numpy(), st.cpu().numpy(), stats.cpu().numpy()


def without_workspace(fp, ctx, d_inst, dJ, n):
    grad, st, stats = outputs(n)
    fp.fp_grad_noalloc(ctx, d_inst, n, KMAX, CH, dJ, grad, st, d_stats=stats)
    torch.cuda.synchronize()
    return grad.cpu().numpy(), st.cpu().numpy(), stats.cpu().numpy()


def test_noalloc_matches_fp_grad_on_two_calls(fp):
    ctx = context(fp, max_steps=300_000)
    # 15.2 MB of scratch per CTA at this step budget: two CTAs fit in 32 MiB
    per_cta = fp.fp_grad_workspace_bytes(ctx, 1)
    assert 2 * per_cta <= (32 << 20) < 3 * per_cta
    for seed in (5, 6):
        d_inst, dJ, n = inputs(fp, seed)
        g_ref, st_ref, stats_ref = with_workspace(fp, ctx, d_inst, dJ, n)
        g, st, stats = without_workspace(fp, ctx, d_inst, dJ, n)
        assert (st_ref == 0).all(), (st_ref, stats_ref)
        assert (st == 0).all(), (st, stats)
        np.testing.assert_array_equal(stats, stats_ref)
        np.testing.assert_allclose(g, g_ref, rtol=RTOL, atol=0)
    ctx.close()


def test_noalloc_calls_allocate_no_device_memory(fp):
    """Free device memory (driver view) is the same after a first and after a
    second fp_grad_noalloc call: the calls allocate nothing.  Every buffer the
    test needs exists before the first reading, so torch's caching allocator
    does not move either."""
    ctx = context(fp, max_steps=300_000)
    d_inst, dJ, n = inputs(fp, 7)
    grad, st, stats = outputs(n)
    fp.fp_grad_noalloc(ctx, d_inst, n, KMAX, CH, dJ, grad, st, d_stats=stats)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    fp.fp_grad_noalloc(ctx, d_inst, n, KMAX, CH, dJ, grad, st, d_stats=stats)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert (st.cpu().numpy() == 0).all()
    assert free1 == free0, (free0, free1)
    ctx.close()


def test_noalloc_refuses_an_instance_larger_than_the_array(fp):
    ctx = context(fp, max_steps=2_000_000)
    assert fp.fp_grad_workspace_bytes(ctx, 1) > (32 << 20)
    d_inst, dJ, n = inputs(fp, 5, n=1)
    grad, st, _ = outputs(n)
    with pytest.raises(RuntimeError, match="fixed buffer holds"):
        fp.fp_grad_noalloc(ctx, d_inst, n, KMAX, CH, dJ, grad, st)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == -7          # nothing was launched
    ctx.close()
