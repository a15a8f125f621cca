"""The trained surrogate against the method that trained it.

Fresh draws of the training domain (uneven-sweep distribution, barrier
sigma <= 12, L = 16) are solved by fp_solve_batch + fp_signal (the reference) and
answered by the two-member surrogate ensemble.  The stated accuracy comes from
the held-out evaluation at training time (median relative L2 error of the 400
complex harmonics about 1.5e-2, 90th percentile about 6e-2), checked here with
margin; the gain is the time per answer: one solve of one instance against one
surrogate query in a large batch.
"""
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_08040_gb300 import build, workloads      # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    build.build()
    from paper_2106_08040_gb300 import fp, surrogate, surrogate_train
    base, ext = os.path.splitext(surrogate_train.DEFAULT_OUT)
    if not os.path.exists(base + ".m0" + ext):
        pytest.skip("no trained surrogate weights in the package")
    return fp, surrogate, surrogate_train


def test_trained_surrogate_error_and_gain(mods):
    fp, surrogate, stt = mods
    draw = workloads.uneven_sweep_instances(512, 16, seed=99)
    inst = draw[fp.Material().sigma(draw["K"], draw["d"]) <= 12.0][:96]
    ctx = stt.solver_context(16, 1e-7)
    torch.cuda.synchronize()
    t0 = time.time()
    y, st = stt.solve_signals(ctx, inst)
    t_solver = (time.time() - t0) / len(inst)            # seconds per instance (one batch, all SMs)
    ctx.close()
    ok = st == 0
    assert ok.mean() > 0.9
    ens = stt.Ensemble.load(stt.DEFAULT_OUT)
    x = torch.from_numpy(surrogate.features(inst).astype(np.float32)).cuda()
    mean, spread = ens.infer(x)
    err = stt.relative_errors(mean.cpu().numpy().astype(np.float64)[ok], y[ok])
    assert np.median(err) < 4e-2, np.median(err)
    assert np.quantile(err, 0.9) < 0.15, np.quantile(err, 0.9)
    assert ens.members[0].error_flag() == 0 and ens.members[1].error_flag() == 0
    # the member spread ranks the errors: accepted answers are better than rejected ones
    spr = spread.cpu().numpy()[ok]
    thr = np.median(spr)
    assert np.median(err[spr <= thr]) < np.median(err[spr > thr])
    # gain: time per answer
    xb = x.repeat(65536 // len(inst) + 1, 1)[:65536].contiguous()
    ens.infer(xb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        ens.infer(xb)
    e1.record()
    torch.cuda.synchronize()
    t_query = e0.elapsed_time(e1) * 1e-3 / 5 / xb.shape[0]
    assert t_solver / t_query > 1e3, (t_solver, t_query)


def test_fused_ensemble_matches_two_member_passes(mods):
    """fp_surrogate_infer_ensemble (mean and spread folded into the second
    member's last epilogue) against two fp_surrogate_infer passes combined on
    the host in FP64, on a query count that is not a multiple of the 128-row
    tiles: the mean to FP32 rounding of (y0 + y1) / 2, the spread to 1e-5
    (FP32 sums of 800 squares in a different order)."""
    fp, surrogate, stt = mods
    ens = stt.Ensemble.load(stt.DEFAULT_OUT)
    rng = np.random.default_rng(4)
    draw = workloads.uneven_sweep_instances(1000, 16, seed=17)
    x = torch.from_numpy(surrogate.features(draw).astype(np.float32)).cuda()
    mean, spread = ens.infer(x)
    y0 = ens.members[0].infer(x).cpu().numpy().astype(np.float64)
    y1 = ens.members[1].infer(x).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    m_ref = 0.5 * (y0 + y1)
    s_ref = np.linalg.norm(y0 - y1, axis=1) / (2 * np.linalg.norm(m_ref, axis=1))
    mm = mean.cpu().numpy().astype(np.float64)
    assert np.abs(mm - m_ref).max() <= 2e-7 * np.abs(m_ref).max()
    assert np.abs(spread.cpu().numpy() - s_ref).max() <= 1e-5 * s_ref.max()
    assert ens.members[0].error_flag() == 0 and ens.members[1].error_flag() == 0
