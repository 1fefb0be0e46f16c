"""Seeded synthetic workloads: the population-annealing configurations that the
tests and the benchmark run, as plain parameters and inverse-temperature
schedules.  This module holds no step of the method; both the CUDA path and
the CPU oracle take these values as inputs.

The schedules are constant steps beta_i = beta_end * i / K (Sec. 2 of
arXiv:1704.01888 uses constant steps), evaluated in that order so that both
sides see the same doubles.  beta_t = ln(1 + sqrt(q)) (Sec. 3) only places
histograms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    q: int
    L: int
    R: int
    K: int
    beta_end: float
    theta: int
    seed: int = 1
    hist_bin: int = 1
    hist_steps: tuple = field(default_factory=tuple)
    track_families: bool = False
    stream: int = 0

    @property
    def N(self) -> int:
        return self.L * self.L

    def betas(self) -> np.ndarray:
        return np.array([self.beta_end * i / self.K for i in range(self.K + 1)], dtype=np.float64)

    def attempts_per_step(self, R_i: int | None = None) -> int:
        return (self.R if R_i is None else R_i) * self.N * self.theta


def beta_t(q: int) -> float:
    return math.log(1.0 + math.sqrt(q))


def nearest_step(wl: Workload, beta: float) -> int:
    b = wl.betas()
    return int(np.argmin(np.abs(b - beta)))


def splitmix64(x: int) -> int:
    """SplitMix64 output for state x (Steele, Lea & Flood, OOPSLA 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


# Plain PA, q = 10, L = 16, R = 1000, beta 0 -> 1.6 in 100 steps, theta = 10.
C1 = Workload("plain-q10-L16-R1000", q=10, L=16, R=1000, K=100, beta_end=1.6, theta=10)

# Plain PA at scale, q = 10, L = 64, R = 100000, 200 steps to 1.6, theta = 10;
# energy histogram (bin width 4) at the grid point nearest beta_t = 1.42606.
C2 = Workload("plain-q10-L64-R100000", q=10, L=64, R=100000, K=200, beta_end=1.6, theta=10, hist_bin=4)
C2.hist_steps = (nearest_step(C2, beta_t(10)),)

# Differentiable / adaptive case, q = 8, L = 128, R = 200000 (beta range and
# theta are not given; 1.1 * beta_t and theta = 10 are the reading taken here).
C4 = Workload("adaptive-q8-L128-R200000", q=8, L=128, R=200000, K=200, beta_end=1.1 * beta_t(8), theta=10)

# Strong first-order case, q = 20, L = 256, R = 100000, 300 steps to 1.9,
# theta = 20, histograms around beta_t = 1.69967 and family entropy per step.
C5 = Workload("strong-q20-L256-R100000", q=20, L=256, R=100000, K=300, beta_end=1.9, theta=20, hist_bin=4,
              track_families=True)
C5.hist_steps = (nearest_step(C5, beta_t(20)), nearest_step(C5, beta_t(20)) + 1)


def batched_runs(M: int = 64, seed: int = 1):
    """M independent runs: q from {5, 6, 8, 10}, L from {16, 32, 48, 64},
    R uniform in [10000, 50000] via SplitMix64, 150 steps to 1.1 beta_t(q),
    theta = 10; all runs share the seed and run m has stream m."""
    runs = []
    for m in range(M):
        q = (5, 6, 8, 10)[m % 4]
        L = (16, 32, 48, 64)[(m // 4) % 4]
        R = 10000 + splitmix64(seed * 0x100000000 + m) % 40001
        runs.append(Workload(f"batch{m}", q=q, L=L, R=int(R), K=150, beta_end=1.1 * beta_t(q), theta=10,
                             seed=seed, stream=m))
    return runs


def scaled(wl: Workload, R: int | None = None, K: int | None = None, name: str | None = None) -> Workload:
    """The same workload with fewer replicas or steps (same beta grid spacing
    when K is cut: beta_end scales with K)."""
    K2 = wl.K if K is None else K
    return Workload(name or wl.name + "-scaled", q=wl.q, L=wl.L, R=wl.R if R is None else R, K=K2,
                    beta_end=wl.beta_end * K2 / wl.K, theta=wl.theta, seed=wl.seed, hist_bin=wl.hist_bin,
                    track_families=wl.track_families)


def width_study_runs(seed: int = 1, qs=(6, 8, 10, 20), Ls=(16, 32, 64, 128, 256), R: int = 1000,
                     theta: int = 100, K: int = 100):
    """Histogram-width study in the style of the paper's Table I (Sec. 4): for
    each q and L a population of R = 1000 replicas, theta = 100 sweeps per
    step, cooled in K equal steps from beta = 0 to beta_t(q) = ln(1 + sqrt q);
    the energy and magnetisation histograms are taken at the last step.  All
    runs share the seed; run m has stream m."""
    runs = []
    m = 0
    for q in qs:
        for L in Ls:
            runs.append(Workload(f"width-q{q}-L{L}", q=q, L=L, R=R, K=K, beta_end=beta_t(q), theta=theta,
                                 seed=seed, stream=m))
            m += 1
    return runs


# Inverse-temperature schedules of the paper's width study (Table I caption):
# steps of 1/N_beta = 0.001 in a window [b, c] around the transition, 0.01
# next to it and 0.05 below a and above d (this schedule stops at d); in
# thousandths of beta: (a, b, c, d).
TABLE_I_WINDOWS = {6: (995, 1135, 1305, 1545), 8: (1110, 1250, 1420, 1660), 10: (1165, 1305, 1475, 1715),
                   20: (1595, 1735, 1905, 2145)}

# The paper's Table I (R = 1000, theta = 100, averages over 200 runs): for
# (q, L), (omega_max(e), T_max(e), omega_max(m), T_max(m)).
TABLE_I = {
    (6, 16): (0.71, 0.82, 0.51, 0.82), (6, 32): (0.39, 0.81, 0.41, 0.81), (6, 64): (0.23, 0.80, 0.40, 0.80),
    (6, 128): (0.07, 0.80, 0.16, 0.80), (6, 256): (0.03, 0.80, 0.055, 0.79),
    (8, 16): (0.64, 0.75, 0.46, 0.75), (8, 32): (0.34, 0.74, 0.36, 0.74), (8, 64): (0.22, 0.74, 0.31, 0.74),
    (8, 96): (0.11, 0.74, 0.12, 0.74), (8, 128): (0.074, 0.74, 0.09, 0.73), (8, 192): (0.045, 0.73, 0.052, 0.73),
    (8, 256): (0.032, 0.73, 0.037, 0.73),
    (10, 16): (0.74, 0.71, 0.50, 0.71), (10, 32): (0.38, 0.70, 0.43, 0.70), (10, 64): (0.20, 0.69, 0.27, 0.69),
    (10, 128): (0.074, 0.69, 0.088, 0.68), (10, 256): (0.032, 0.69, 0.026, 0.68),
    (20, 16): (0.84, 0.57, 0.64, 0.57), (20, 32): (0.57, 0.57, 0.48, 0.57), (20, 64): (0.18, 0.57, 0.17, 0.56),
    (20, 128): (0.07, 0.57, 0.06, 0.52), (20, 256): (0.029, 0.57, 0.018, 0.52),
}


def table1_betas(q: int, n_beta: int = 1000) -> np.ndarray:
    """beta_0 = 0, ..., d / 1000 for q's window (a, b, c, d): steps of 0.05
    up to a, 0.01 up to b, 1 / n_beta up to c, 0.01 up to d (each part ending
    exactly on its bound; n_beta divides 10000)."""
    a, b, c, d = (10 * x for x in TABLE_I_WINDOWS[q])
    k = [0]
    for bound, step in ((a, 500), (b, 100), (c, 10000 // n_beta), (d, 100)):
        while k[-1] < bound:
            k.append(min(k[-1] + step, bound))
    return np.array(k, dtype=np.float64) / 10000.0


# The paper's Tables II and III (q = 8, L = 64, R = 1000, the schedule of
# Table I): (omega_max(e), T_max(e), omega_max(m), T_max(m)) against theta
# (N_beta = 1000), and against N_beta (theta = 100).
TABLE_II = {10: (0.10, 0.73, 0.14, 0.72), 25: (0.13, 0.74, 0.20, 0.73), 50: (0.17, 0.74, 0.23, 0.74),
            100: (0.22, 0.74, 0.31, 0.74), 200: (0.28, 0.74, 0.39, 0.74), 500: (0.29, 0.74, 0.36, 0.74),
            1000: (0.34, 0.74, 0.42, 0.74)}
TABLE_III = {100: (0.11, 0.73, 0.15, 0.72), 200: (0.13, 0.74, 0.21, 0.72), 500: (0.17, 0.74, 0.27, 0.73),
             1000: (0.23, 0.74, 0.34, 0.74), 2000: (0.27, 0.74, 0.38, 0.74)}
