"""Post-processing of population histograms (Sec. 4 of arXiv:1704.01888).

The energy histogram of a population (hist[k] = number of replicas with
E = k - 2N, as returned by the library) and the histogram of the replicas'
magnetisations m_j = (q Mt_j / N - 1) / (q - 1) (Eq. 5, from the occupations
Mt_j of the most common state) are reduced to their full widths at half
maximum, which the paper uses to follow the broadening of the distributions
near a first-order transition: the distance between the two intersections of
the histogram with the line at half its maximum.  Reading: the intersections
are the outermost half-maximum crossings, located by linear interpolation
between neighbouring bins.  Plain numpy on data already copied to the host;
nothing here touches the device.
"""
from __future__ import annotations

import numpy as np


def rebin_energy_histogram(hist: np.ndarray, N: int, width: int = 1):
    """Energy histogram in bins of `width` energy units, as (e_centres, counts)
    with e = E / N per site.  Bins start at E = -2N."""
    h = np.asarray(hist, dtype=np.int64)
    if h.size != 2 * N + 1:
        raise ValueError("hist must have 2N + 1 bins")
    nb = -(-h.size // width)
    padded = np.zeros(nb * width, dtype=np.int64)
    padded[: h.size] = h
    counts = padded.reshape(nb, width).sum(axis=1)
    E_lo = -2 * N + width * np.arange(nb)
    centres = (E_lo + (width - 1) / 2.0) / N
    return centres, counts


def fwhm(x: np.ndarray, h: np.ndarray, main_peak: bool = False) -> float:
    """Full width at half maximum of a histogram h over equally spaced bin
    centres x, by linear interpolation between bins: between the outermost
    half-maximum crossings, or (main_peak) the crossings nearest to the
    maximum on either side, i.e. the width of the peak that holds the
    maximum when the histogram has several."""
    x = np.asarray(x, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    if h.size == 0 or h.max() <= 0:
        return 0.0
    half = h.max() / 2.0
    if main_peak:
        top = int(np.argmax(h))
        below_l = np.nonzero(h[:top] < half)[0]
        below_r = np.nonzero(h[top:] < half)[0]
        lo = int(below_l[-1]) + 1 if below_l.size else 0
        hi = top + int(below_r[0]) - 1 if below_r.size else h.size - 1
    else:
        above = np.nonzero(h >= half)[0]
        lo, hi = int(above[0]), int(above[-1])
    if lo > 0:
        x_left = x[lo - 1] + (half - h[lo - 1]) * (x[lo] - x[lo - 1]) / (h[lo] - h[lo - 1])
    else:
        x_left = x[0]
    if hi < h.size - 1:
        x_right = x[hi] + (h[hi] - half) * (x[hi + 1] - x[hi]) / (h[hi] - h[hi + 1])
    else:
        x_right = x[-1]
    return float(x_right - x_left)


def peaks(h: np.ndarray, min_separation: int = 2, rel_height: float = 0.2):
    """Indices of local maxima higher than rel_height * max, at least
    min_separation bins apart (a coarse test for two-peak coexistence)."""
    h = np.asarray(h, dtype=np.float64)
    if h.size < 3 or h.max() <= 0:
        return [int(np.argmax(h))] if h.size else []
    cand = [i for i in range(h.size)
            if h[i] >= rel_height * h.max() and (i == 0 or h[i] >= h[i - 1]) and (i == h.size - 1 or h[i] > h[i + 1])]
    out = []
    for i in sorted(cand, key=lambda k: -h[k]):
        if all(abs(i - j) >= min_separation for j in out):
            out.append(i)
    return sorted(out)


def modes(h: np.ndarray, smooth_frac: float = 0.03, rel_height: float = 0.1, min_dip: float = 0.25):
    """The modes of a histogram, robust to bin-to-bin noise: the occupied
    range is smoothed with a Gaussian of standard deviation smooth_frac of
    its width (at least one bin); local maxima of the smoothed counts above
    rel_height of the highest are candidates; two candidates are separate
    modes when the smoothed counts between them dip below (1 - min_dip) of the
    lower one (otherwise the lower is dropped).  Returns the mode indices (into
    h) in ascending order: two or more mean coexisting phases (Sec. 4)."""
    h = np.asarray(h, dtype=np.float64)
    nz = np.flatnonzero(h > 0)
    if nz.size == 0:
        return []
    lo, hi = int(nz[0]), int(nz[-1]) + 1
    x = h[lo:hi]
    sigma = max(1.0, smooth_frac * x.size)
    r = int(np.ceil(3 * sigma))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / sigma) ** 2)
    sm = np.convolve(np.pad(x, r), k / k.sum(), mode="valid")
    cand = [i for i in range(sm.size)
            if sm[i] >= rel_height * sm.max() and (i == 0 or sm[i] > sm[i - 1]) and (i == sm.size - 1 or sm[i] >= sm[i + 1])]
    kept = []
    for i in sorted(cand, key=lambda c: -sm[c]):
        if all(sm[min(i, j):max(i, j) + 1].min() <= (1.0 - min_dip) * min(sm[i], sm[j]) for j in kept):
            kept.append(i)
    return sorted(lo + i for i in kept)


def magnetisation(q: int, N: int, Mt: np.ndarray) -> np.ndarray:
    """m_j = (q Mt_j / N - 1) / (q - 1), the magnetisation of Eq. 5 per replica."""
    return (q * np.asarray(Mt, dtype=np.float64) / N - 1.0) / (q - 1.0)


def energy_histogram(E: np.ndarray, N: int) -> np.ndarray:
    """hist[k] = number of replicas with E = k - 2N (the library's layout)."""
    E = np.asarray(E, dtype=np.int64)
    return np.bincount(E + 2 * N, minlength=2 * N + 1)


def widths(q: int, L: int, E: np.ndarray, Mt: np.ndarray, e_bin: int = 4, m_bins: int = 60):
    """(omega_e, omega_m): FWHM of the energy-per-site histogram (bins of
    e_bin energy units) and of the magnetisation histogram (m_bins equal bins
    spanning the population's range of m, so that the bins stay narrower than
    the distribution at every L) of one population."""
    N = L * L
    x, h = rebin_energy_histogram(energy_histogram(E, N), N, e_bin)
    # m takes the discrete values of Mt = 1..N: bins of a whole number of Mt
    # values avoid the aliasing of bins that straddle a varying count of them
    Mt = np.asarray(Mt, dtype=np.int64)
    lo, hi = int(Mt.min()), int(Mt.max())
    if hi <= lo:
        return fwhm(x, h), 0.0
    width = max(1, -(-(hi - lo + 1) // m_bins))
    counts = np.bincount((Mt - lo) // width)
    centres = magnetisation(q, N, lo + width * np.arange(counts.size) + (width - 1) / 2.0)
    return fwhm(x, h), fwhm(centres, counts)


def ranged_widths(q: int, L: int, E: np.ndarray, Mt: np.ndarray, bins: int = 40, main_peak: bool = False):
    """(omega_e, omega_m): FWHM of the energy-per-site and magnetisation
    histograms of one population, each in about `bins` bins of a whole
    number of its integer units (E, Mt) spanning the population's range, so
    that the resolution follows the distribution's width at every L
    (main_peak as for fwhm)."""
    N = L * L

    def binned(v):
        v = np.asarray(v, dtype=np.int64)
        lo, hi = int(v.min()), int(v.max())
        width = max(1, -(-(hi - lo + 1) // bins))
        counts = np.bincount((v - lo) // width)
        return lo + width * np.arange(counts.size) + (width - 1) / 2.0, counts

    if np.asarray(E).size == 0:
        return 0.0, 0.0
    ue, he = binned(E)
    um, hm = binned(Mt)
    return fwhm(ue / N, he, main_peak), fwhm(magnetisation(q, N, um), hm, main_peak)


def crossings(x: np.ndarray, f: np.ndarray, g: np.ndarray, window: int = 6):
    """Every change of sign of d = f - g as (x_cross, score), x_cross by
    linear interpolation and score = the smaller of max |d| over the `window`
    points before and after it: a crossing between two clearly separated
    branches scores high, one in the noise where the branches coincide low."""
    x = np.asarray(x, dtype=np.float64)
    d = np.asarray(f, dtype=np.float64) - np.asarray(g, dtype=np.float64)
    out = []
    for i in range(d.size - 1):
        if (d[i] > 0.0) != (d[i + 1] > 0.0):
            xc = float(x[i] + d[i] * (x[i + 1] - x[i]) / (d[i] - d[i + 1]))
            score = min(np.abs(d[max(0, i - window + 1): i + 1]).max(), np.abs(d[i + 1: i + 1 + window]).max())
            out.append((xc, float(score)))
    return out


def crossing(x: np.ndarray, f: np.ndarray, g: np.ndarray):
    """The x at which f - g changes sign (the first change of sign, located
    by linear interpolation), or None.  Used for the free-energy branches of
    cooling and heating runs (Sec. 6: -beta F = ln Z of the two branches
    cross at the transition)."""
    x = np.asarray(x, dtype=np.float64)
    d = np.asarray(f, dtype=np.float64) - np.asarray(g, dtype=np.float64)
    for i in range(d.size - 1):
        if d[i] == 0.0:
            return float(x[i])
        if (d[i] > 0.0) != (d[i + 1] > 0.0):
            return float(x[i] + d[i] * (x[i + 1] - x[i]) / (d[i] - d[i + 1]))
    return None
