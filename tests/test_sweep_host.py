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
