"""Host-side pieces of the uneven sweep: the per-instance truncation degree
rule and the Fibonacci easy-axis directions (CPU only)."""
import numpy as np

from paper_2106_08040_gb300 import workloads


def test_fibonacci_directions():
    th, ph = workloads.fibonacci_directions(16)
    z = np.cos(th)
    np.testing.assert_allclose(z, 1.0 - (2 * np.arange(16) + 1) / 16, atol=1e-15)
    assert np.all((ph >= 0) & (ph < 2 * np.pi))
    # distinct, and z symmetric about the equator (the set spans the sphere evenly)
    np.testing.assert_allclose(np.sort(z), -np.sort(z)[::-1], atol=1e-15)


def test_truncation_degree_rule():
    from paper_2106_08040_gb300 import fp
    inst = workloads.make_instances(5)
    inst["K"] = [1e2, 1e3, 3e3, 1e4, 1e4]
    inst["d"] = 20e-9
    inst["h_off"][:, 0] = [0.0, 0.0, 0.0, 0.0, 0.02]
    L = fp.truncation_degree(inst, L_min=8, L_max=16)
    assert L.min() >= 8 and L.max() <= 16
    assert np.all(np.diff(L[:4]) >= 0)                   # larger barrier, larger degree
    assert L[4] >= L[3]                                   # larger field, larger degree
    # the formula itself at one point: sigma and xi by hand
    kT = 1.380649e-23 * 293.0
    V = np.pi * (20e-9) ** 3 / 6
    sig = 1e3 * V / kT
    assert fp.truncation_degree(inst[1:2], L_min=2, L_max=64)[0] == int(np.ceil(2 + 5.5 * np.sqrt(sig)))


def test_sweep_order_buckets_and_cost_order():
    """fp_sweep_order (host part of fp_sweep_plan): a permutation, buckets of
    decreasing launch degree (L rounded up to the bucket width, capped at
    L_max), each queued by decreasing sigma + b_T (|B_off| + |B_drive|)."""
    import pytest
    from paper_2106_08040_gb300 import build
    build.build()
    from paper_2106_08040_gb300 import fp
    inst = workloads.random_instances(200, 8, seed=4, max_offset=0.01, K_range=(5e2, 1e4))
    inst["L"] = np.random.default_rng(4).integers(3, 17, size=200)
    dspec = workloads.drive_lissajous()
    drv = fp.Drive(**dspec.__dict__)
    mat = fp.Material()
    for width in (1, 3):
        order, buckets = fp.sweep_order(inst, mat, drv, 16, bucket_width=width)
        assert sorted(order.tolist()) == list(range(200))
        assert sum(c for _, c in buckets) == 200
        Ls = [L for L, _ in buckets]
        assert Ls == sorted(Ls, reverse=True) and len(set(Ls)) == len(Ls)
        kT = 1.380649e-23 * mat.T_B
        V = np.pi * inst["d"] ** 3 / 6
        cost = inst["K"] * V / kT + V * mat.Ms / kT * (np.linalg.norm(inst["h_off"], axis=1) + np.linalg.norm(drv.amp))
        s = 0
        for L, c in buckets:
            idx = order[s:s + c]
            launch = np.minimum(16, (inst["L"][idx] + width - 1) // width * width)
            assert (launch == L).all()
            assert (np.diff(cost[idx]) <= 1e-9 * cost[idx][:-1]).all()
            s += c
    bad = inst.copy()
    bad["L"][5] = 17
    with pytest.raises(RuntimeError, match="outside"):
        fp.sweep_order(bad, mat, drv, 16)
