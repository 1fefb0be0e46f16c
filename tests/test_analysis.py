"""FWHM and rebinning of population histograms (Sec. 4)."""
import math

import numpy as np
import pytest

from paper_1704_01888_gb300 import analysis


def test_fwhm_of_gaussian_histogram():
    x = np.arange(-200, 201, dtype=np.float64)
    for sigma in (5.0, 17.0, 40.0):
        h = np.exp(-x**2 / (2 * sigma**2)) * 1e6
        assert analysis.fwhm(x, h) == pytest.approx(2 * math.sqrt(2 * math.log(2)) * sigma, rel=2e-3)


def test_fwhm_outermost_crossings_and_edges():
    x = np.arange(10.0)
    h = np.array([0, 1, 4, 2, 1, 2, 4, 1, 0, 0], dtype=float)  # two peaks of 4, valley 1 < 2
    # outermost crossings of the line at 2: between x=1,2 (at 1 + 1/3) and x=6,7 (at 6 + 2/3)
    assert analysis.fwhm(x, h) == pytest.approx((6 + 2 / 3) - (1 + 1 / 3))
    assert analysis.peaks(h) == [2, 6]
    assert analysis.fwhm(x, np.zeros(10)) == 0.0
    assert analysis.fwhm(x, np.eye(10)[0]) == pytest.approx(0.5)  # a peak on the edge


def test_rebin_energy_histogram():
    N = 16
    hist = np.zeros(2 * N + 1, dtype=np.int32)
    hist[[0, 1, 2, 3, 4, 32]] = [1, 2, 3, 4, 5, 6]
    e, c = analysis.rebin_energy_histogram(hist, N, width=4)
    assert c.sum() == hist.sum() and c[0] == 10 and c[1] == 5 and c[-1] == 6
    assert e[0] == pytest.approx((-32 + 1.5) / 16)
    e1, c1 = analysis.rebin_energy_histogram(hist, N)
    assert np.array_equal(c1, hist) and e1[0] == -2.0 and e1[-1] == 0.0
