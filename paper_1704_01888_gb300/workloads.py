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
