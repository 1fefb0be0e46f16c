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
    # the peak holding the maximum alone: crossings at 1 + 1/3 and 3 + 0 (h[3] = 2 is at half)
    h2 = np.array([0, 1, 4, 2, 1, 2, 3, 1, 0, 0], dtype=float)
    assert analysis.fwhm(x, h2, main_peak=True) == pytest.approx(3.0 - (1 + 1 / 3))
    assert analysis.fwhm(x, h2) == pytest.approx((6 + 1 / 2) - (1 + 1 / 3))
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


def test_magnetisation_and_energy_histogram():
    q, L = 10, 8
    N = L * L
    Mt = np.array([N, N // q + 0, 40])
    m = analysis.magnetisation(q, N, Mt)
    assert m[0] == pytest.approx(1.0)              # ordered: every site in one state
    assert m[1] == pytest.approx((q * (N // q) / N - 1) / (q - 1))
    assert m[2] == pytest.approx((10 * 40 / 64 - 1) / 9)
    assert analysis.magnetisation(q, N, [N / q])[0] == pytest.approx(0.0)  # equal occupations
    E = np.array([-2 * N, -2 * N, -3, 0])
    h = analysis.energy_histogram(E, N)
    assert h.size == 2 * N + 1 and h[0] == 2 and h[2 * N - 3] == 1 and h[2 * N] == 1 and h.sum() == 4


def test_widths_of_gaussian_populations():
    rng = np.random.default_rng(5)
    q, L = 8, 32
    N = L * L
    R = 400000
    E = np.clip(np.round(rng.normal(-1.2 * N, 40.0, R)), -2 * N, 0).astype(np.int32)
    m_target = rng.normal(0.5, 0.08, R)
    Mt = np.round((m_target * (q - 1) + 1) * N / q).astype(np.int32)
    we, wm = analysis.widths(q, L, E, Mt, e_bin=4, m_bins=100)
    c = 2 * math.sqrt(2 * math.log(2))
    assert we == pytest.approx(c * 40.0 / N, rel=0.05)
    assert wm == pytest.approx(c * 0.08, rel=0.05)


def test_ranged_widths_resolve_narrow_and_wide_populations():
    """The bins follow the population's range: the FWHM of Gaussian E and m
    is recovered at a small and at a large lattice alike."""
    rng = np.random.default_rng(11)
    c = 2 * math.sqrt(2 * math.log(2))
    q = 10
    for L, sd_E, sd_m, R in ((16, 6.0, 0.05, 200000), (256, 900.0, 0.004, 200000)):
        N = L * L
        E = np.clip(np.round(rng.normal(-1.0 * N, sd_E, R)), -2 * N, 0).astype(np.int32)
        Mt = np.round((rng.normal(0.3, sd_m, R) * (q - 1) + 1) * N / q).astype(np.int32)
        we, wm = analysis.ranged_widths(q, L, E, Mt, bins=60)
        assert we == pytest.approx(c * sd_E / N, rel=0.08)
        assert wm == pytest.approx(c * sd_m, rel=0.08)
    # a population of identical replicas has zero width
    assert analysis.ranged_widths(q, 16, np.full(5, -300), np.full(5, 40)) == (0.0, 0.0)


def test_table1_schedule_follows_the_caption():
    from paper_1704_01888_gb300 import workloads as wl

    for q, (a, b, c, d) in wl.TABLE_I_WINDOWS.items():
        for n_beta in (1000, 2000, 200):
            beta = wl.table1_betas(q, n_beta)
            k = np.round(beta * 10000).astype(int)
            steps = np.diff(k)
            a4, b4, c4, d4, f = 10 * a, 10 * b, 10 * c, 10 * d, 10000 // n_beta
            assert k[0] == 0 and k[-1] == d4 and np.all(steps > 0)
            assert np.all(steps[k[1:] <= a4] <= 500) and np.all(steps[(k[:-1] >= a4) & (k[1:] <= b4)] == 100)
            assert np.all(steps[(k[:-1] >= b4) & (k[1:] <= c4)] == f) and np.all(steps[k[:-1] >= c4] == 100)
            assert np.count_nonzero((k[:-1] >= b4) & (k[1:] <= c4)) == (c4 - b4) // f
    assert len(wl.TABLE_I) == 22 and {q for q, _ in wl.TABLE_I} == {6, 8, 10, 20}
    assert sorted(wl.TABLE_II) == [10, 25, 50, 100, 200, 500, 1000] and sorted(wl.TABLE_III) == [100, 200, 500, 1000, 2000]


def test_crossing_of_two_branches():
    from paper_1704_01888_gb300 import analysis

    x = np.linspace(0.0, 2.0, 21)
    f = 1.0 - 0.5 * x          # crosses g at x = 4/3
    g = 0.25 * x
    assert analysis.crossing(x, f, g) == pytest.approx(4.0 / 3.0, rel=1e-12)
    assert analysis.crossing(x, f + 10.0, g) is None
    assert analysis.crossing(x, g, g) == 0.0


def test_crossings_prefer_separated_branches():
    from paper_1704_01888_gb300 import analysis

    x = np.linspace(0.0, 3.0, 301)
    noise = 1e-4 * np.sin(37.0 * x)                  # branches that coincide below x = 1
    f = np.where(x < 1.0, noise, 0.3 * (2.0 - x) * (x - 1.0))
    g = np.zeros_like(x)
    cs = analysis.crossings(x, f, g)
    best = max(cs, key=lambda c: c[1])
    assert best[0] == pytest.approx(2.0, abs=0.01)
    assert len(cs) > 3


def test_modes_ignore_noise_and_find_two_phases():
    from paper_1704_01888_gb300 import analysis

    rng = np.random.default_rng(3)
    x = np.arange(400)
    one = rng.poisson(200 * np.exp(-0.5 * ((x - 200) / 30.0) ** 2))
    assert len(analysis.modes(one)) == 1
    two = rng.poisson(150 * np.exp(-0.5 * ((x - 120) / 20.0) ** 2) + 90 * np.exp(-0.5 * ((x - 290) / 25.0) ** 2))
    m = analysis.modes(two)
    assert len(m) == 2 and abs(m[0] - 120) < 8 and abs(m[1] - 290) < 10
    # a shoulder without a dip is one mode
    sh = 200 * np.exp(-0.5 * ((x - 200) / 30.0) ** 2) + 150 * np.exp(-0.5 * ((x - 240) / 30.0) ** 2)
    assert len(analysis.modes(sh)) == 1
