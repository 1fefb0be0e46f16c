"""Post-processing of population histograms (Sec. 4 of arXiv:1704.01888).

The energy histogram of a population (hist[k] = number of replicas with
E = k - 2N, as returned by the library) is rebinned and reduced to the full
width at half maximum, which the paper uses to follow the broadening of the
distribution near a first-order transition: the distance between the two
intersections of the histogram with the line at half its maximum.  Reading:
the intersections are the outermost half-maximum crossings, located by linear
interpolation between neighbouring bins.  Plain numpy on data already copied
to the host; nothing here touches the device.
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


def fwhm(x: np.ndarray, h: np.ndarray) -> float:
    """Full width at half maximum of a histogram h over equally spaced bin
    centres x (outermost half-maximum crossings, linear interpolation)."""
    x = np.asarray(x, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    if h.size == 0 or h.max() <= 0:
        return 0.0
    half = h.max() / 2.0
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
