"""Host-side entry points of the Sec. 2.3 distance measures (no GPU): the
mixing orders of Eq. mix and the frequency index set I_freq, bit-exact against
the oracle."""
import numpy as np
import pytest

from oracle import models


@pytest.fixture(scope="module")
def fp():
    from paper_2106_08040_gb300 import build
    build.build()
    from paper_2106_08040_gb300 import fp as fpmod
    return fpmod


@pytest.mark.parametrize("n_dens", [16, 5, 1])
def test_mixing_order_matches_oracle(fp, n_dens):
    for k in list(range(0, 817)) + [-1, -17, -400, 5000]:
        assert fp.fp_mixing_order(k, n_dens) == models.mixing_order(k, n_dens), k


def test_freq_index_set_matches_oracle(fp):
    for mx, my in ((3, 2), (20, 20), (0, 5), (1, 1)):
        ref = models.freq_index_set(mx, my, 16)
        ref = ref[ref <= 816]
        np.testing.assert_array_equal(fp.fp_freq_index_set(mx, my, 16, 816), ref)
