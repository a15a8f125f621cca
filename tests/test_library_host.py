"""Host-side checks of libfp.so (no GPU work): it loads, exports every entry
point declared in include/fp.h, and its closed-form coupling tables reproduce
the oracle's quadrature-built weak-form matrices (Sec. 2.1, Eq. FP-general and
Eq. convection in the easy-axis frame)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fp():
    from paper_2106_08040_gb300 import build
    build.build()
    from paper_2106_08040_gb300 import fp as fpmod
    return fpmod


def declared_entry_points():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(fp_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(fp):
    from paper_2106_08040_gb300 import _lib
    L = _lib.lib()
    names = declared_entry_points()
    assert "fp_solve_batch" in names and "fp_setup" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(_lib.EXPORTED) >= set(names)


@pytest.mark.parametrize("L", [2, 7, 16])
def test_closed_form_tables_match_oracle_weak_form(fp, L):
    from oracle import galerkin, physics
    K, d = 3.5e3, 18e-9
    B = np.array([0.007, -0.004, 0.009])
    A = fp.fp_operator_dense(fp.Material(), L, K, d, B)
    P = physics.derive(physics.Material(), K, d)
    A0, A1 = galerkin.weak_form_matrices(L, P, np.array([0.0, 0.0, 1.0]))
    ref = A0 + np.einsum("k,kij->ij", B, A1)
    assert np.abs(A - ref).max() <= 1e-13 * np.abs(ref).max()


def test_bad_arguments_return_errors(fp):
    with pytest.raises(RuntimeError, match="L=1"):
        fp.fp_operator_dense(fp.Material(), 1, 1e3, 2e-8, [0, 0, 0])


def test_missing_library_fails_loudly(tmp_path):
    """Without libfp.so the binding raises at the first call; there is no
    fallback path (checked in a child process so the loaded library of this
    session is untouched)."""
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_2106_08040_gb300 import _lib, fp\n"
        "_lib.LIB_PATH = %r\n"
        "try:\n"
        "    fp.fp_max_degree()\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e); sys.exit(0)\n"
        "sys.exit(3)\n"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))), str(tmp_path / "libfp.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "not built" in r.stdout
