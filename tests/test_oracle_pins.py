"""Pins for the CPU oracle against facts it does not compute itself.

The oracle (oracle/pa_oracle.c) is the reference every GPU parity test trusts,
so it is checked here against published known-answer vectors, closed forms
from the paper and from the exact Ising solution, exact enumeration, detailed
balance of the exact transition matrix, and invariants of the resampling step.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert [int(x) for x in oracle.philox(ctr, key)] == expect


_TRITON_SCRIPT = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
@triton.jit
def k(c_ptr, out_ptr, seed, BLOCK: tl.constexpr):
    i = tl.arange(0, BLOCK)
    c0 = tl.load(c_ptr + 4 * i + 0); c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2); c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a); tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c); tl.store(out_ptr + 4 * i + 3, d)
ctr = np.fromfile(sys.argv[1], dtype=np.uint32)
seed = int(sys.argv[2])
c = torch.from_numpy(ctr.view(np.int32).copy())
out = torch.zeros_like(c)
k[(1,)](c, out, seed, BLOCK=ctr.size // 4)
out.numpy().view(np.uint32).tofile(sys.argv[3])
"""


def test_philox_matches_triton_library(tmp_path):
    """An independent library implementation (triton.language.philox, run by
    its CPU interpreter) agrees on 256 random counters."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0x1234_5678_9ABC_DEF1
    cf, of = tmp_path / "c.bin", tmp_path / "o.bin"
    ctr.tofile(cf)
    script = tmp_path / "t.py"
    script.write_text(_TRITON_SCRIPT)
    res = subprocess.run([sys.executable, str(script), str(cf), str(seed), str(of)],
                         capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-200:])
    got = np.fromfile(of, dtype=np.uint32).reshape(256, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(256):
        assert list(oracle.philox(ctr[i], key)) == list(got[i])


# --------------------------------------------------------------------------
# Hamiltonian (Sec. 3, Eq. 3) and exact enumeration
# --------------------------------------------------------------------------
def _kaufman_lnZ(K, m, n):
    """ln Z of the Ising model sum exp(K sum_<ij> s_i s_j) on an m x n torus,
    B. Kaufman, Phys. Rev. 76, 1232 (1949)."""
    def gamma(l):
        if l == 0:
            return 2 * K + math.log(math.tanh(K))
        return math.acosh(math.cosh(2 * K) / math.tanh(2 * K) - math.cos(math.pi * l / n))
    z = [1.0, 1.0, 1.0, 1.0]
    for r in range(n):
        g1, g0 = gamma(2 * r + 1), gamma(2 * r)
        z[0] *= 2 * math.cosh(m * g1 / 2)
        z[1] *= 2 * math.sinh(m * g1 / 2)
        z[2] *= 2 * math.cosh(m * g0 / 2)
        z[3] *= 2 * math.sinh(m * g0 / 2)
    return math.log(0.5) + (m * n / 2) * math.log(2 * math.sinh(2 * K)) + math.log(sum(z))


def _lnZ_from_dos(g, N, beta):
    E = np.arange(-2 * N, 1, dtype=np.float64)
    gg = g.astype(np.float64)
    a = np.where(gg > 0, np.log(np.maximum(gg, 1)) - beta * E, -np.inf)
    mx = a.max()
    return mx + math.log(np.exp(a - mx).sum())


def _mean_E_from_dos(g, N, beta):
    E = np.arange(-2 * N, 1, dtype=np.float64)
    gg = g.astype(np.float64)
    a = np.where(gg > 0, np.log(np.maximum(gg, 1)) - beta * E, -np.inf)
    w = np.exp(a - a.max())
    return float((w * E).sum() / w.sum())


@pytest.mark.parametrize("L", [3, 4])
@pytest.mark.parametrize("beta", [0.3, 0.9, 1.7])
def test_q2_partition_function_matches_kaufman(L, beta):
    """q = 2 Potts is Ising with K = beta/2 shifted by e^{beta N}:
    delta(s,s') = (1 + sigma sigma')/2, so Z_Potts(beta) = e^{beta N} Z_Ising(beta/2)."""
    N = L * L
    g = oracle.density_of_states(2, L)
    assert _lnZ_from_dos(g, N, beta) == pytest.approx(beta * N + _kaufman_lnZ(beta / 2, L, L), rel=1e-12)


@pytest.mark.parametrize("q,L", [(5, 3), (3, 4), (4, 3), (2, 4)])
def test_density_of_states_closed_forms(q, L):
    N = L * L
    g = oracle.density_of_states(q, L)
    assert int(g.sum()) == q ** N
    # ground states: the q uniform configurations, E_0 = -2N (Sec. 6, Eqs. 7-8)
    assert int(g[0]) == q
    # nothing between E_0 and one flipped spin, which breaks its 4 bonds
    assert int(g[1:4].sum()) == 0
    assert int(g[4]) == q * N * (q - 1)
    # at beta = 0 every bond is satisfied with probability 1/q: <E> = -2N/q
    E = np.arange(-2 * N, 1)
    assert float((g.astype(np.float64) * E).sum()) == pytest.approx(-2 * N * q ** N / q, rel=1e-14)
    # relabelling a state leaves H unchanged: g is symmetric under nothing
    # simpler, but E is never positive and -2N is reached
    assert g[-1] >= 0


def test_energy_and_max_count_small_cases():
    s = np.zeros((4, 4), np.uint8)
    assert oracle.energy(s) == -32
    assert oracle.max_count(3, s) == 16
    s[1, 2] = 2
    assert oracle.energy(s) == -28
    s[1, 3] = 2  # a domino of equal flipped spins breaks 6 bonds
    assert oracle.energy(s) == -26
    s[1, 3] = 1  # unequal neighbours inside the domino break 7
    assert oracle.energy(s) == -25
    assert oracle.max_count(3, s) == 14
    chk = (np.add.outer(np.arange(4), np.arange(4)) % 2).astype(np.uint8)
    assert oracle.energy(chk) == 0  # checkerboard: no bond satisfied
    # L = 2: both horizontal bonds of a row join the same two sites
    assert oracle.energy(np.zeros((2, 2), np.uint8)) == -8


# --------------------------------------------------------------------------
# Metropolis update: exact detailed balance (Sec. 2 step 3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("q", [2, 3, 4, 6])
@pytest.mark.parametrize("beta", [0.4, 1.3])
def test_site_kernels_satisfy_detailed_balance(q, beta):
    L = 2
    N = L * L
    n = q ** N
    E = np.zeros(n)
    for a in range(n):
        s = np.array([(a // q ** i) % q for i in range(N)], np.uint8).reshape(L, L)
        E[a] = oracle.energy(s)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    order = [0, 3, 1, 2]  # colour 0 ((x+y) even) row-major, then colour 1
    sweep = np.eye(n)
    for site in order:
        P = oracle.site_matrix(q, L, site, beta)
        assert np.allclose(P.sum(axis=1), 1.0, atol=1e-14)
        flow = pi[:, None] * P
        # the proposal is exactly symmetric; the 32-bit thresholds bound the
        # remaining asymmetry by about 2^-32 relative to pi
        assert np.max(np.abs(flow - flow.T)) <= 1e-8 * pi.max()
        sweep = sweep @ P
    assert np.max(np.abs(pi @ sweep - pi)) < 1e-8
    # the chain moves: the sweep matrix is not the identity
    assert np.min(np.diag(sweep)) < 0.999


def test_thresholds_are_quantised_boltzmann_factors():
    for beta in (0.0, 0.37, 1.426, 3.0):
        t = oracle.thresholds(beta)
        assert int(t[0]) == 2**32
        for d in range(1, 5):
            exact = math.exp(-beta * d) * 2**32
            assert int(t[d]) == math.floor(exact)


@pytest.mark.parametrize("q", [2, 3, 4, 5, 6, 9, 10, 17, 20, 33, 128])
def test_proposal_is_symmetric_and_reaches_every_other_state(q):
    """Over the 2^B equally likely (sigma, u), the offset s' - s mod q never
    vanishes, covers 1..q-1, and has the same probability as its inverse
    (detailed balance needs no more); for q - 1 a power of two it is uniform."""
    B = oracle.state_bits(q)
    assert 2 ** (B - 1) < q <= 2**B
    for cur in sorted({0, q // 2, q - 1}):
        count = np.zeros(q, int)
        for sigma in (0, 1):
            for u in range(2 ** (B - 1) if B > 0 else 1):
                new = oracle.propose(q, cur, sigma, u)
                assert 0 <= new < q and new != cur
                count[(new - cur) % q] += 1
        assert count[0] == 0 and count[1:].min() > 0
        assert all(count[k] == count[q - k] for k in range(1, q))
        if (q - 1) & (q - 2) == 0:
            assert count[1:].min() == count[1:].max()


def test_bitwise_comparison_equals_integer_comparison():
    rng = np.random.default_rng(11)
    vs = [0, 1, 2**31 - 1, 2**31, 2**32 - 2, 2**32 - 1] + [int(x) for x in rng.integers(0, 2**32, 300)]
    Ts = [0, 1, 2**31, 2**32 - 1, 2**32] + [int(x) for x in rng.integers(0, 2**32, 60)]
    for v in vs:
        for T in Ts + [v, v + 1, max(v - 1, 0)]:
            assert oracle.below_value(v, T) == (v < T), (v, T)


@pytest.mark.parametrize("L", [2, 4, 6, 8, 16, 24, 32, 48, 64, 66, 80, 96, 128, 144])
def test_sweep_attempts_every_site_exactly_once(L):
    """At beta = 0 every move is accepted, and for q = 2 a move flips the spin,
    so one sweep flips a site an odd number of times exactly when it is
    attempted an odd number of times: every site flipped means the site words
    (packed rows for L = 8, 16, 32, banded 8-column segments for L = 48, 80,
    96, 144, padded rows otherwise) cover each site of each colour once.  With
    q = 3 every site must also have changed."""
    rng = np.random.default_rng(L)
    s = rng.integers(0, 2, size=(L, L)).astype(np.uint8)
    out = oracle.sweep_replica(2, s, 0.0, 1, step=1, slot=3, seed=5)
    assert np.all(out != s)
    s3 = rng.integers(0, 3, size=(L, L)).astype(np.uint8)
    out3 = oracle.sweep_replica(3, s3, 0.0, 1, step=1, slot=3, seed=5)
    assert np.all(out3 != s3)


def test_acceptance_is_a_threshold_on_v():
    """Moves that do not raise the energy are always taken; a move raising it
    by dE is taken exactly for v < T[dE] (a prefix of the 2^32 values)."""
    q = 10
    for beta in (0.3, 1.3):
        T = oracle.thresholds(beta)
        # a site in state 0: neighbours with k zeros and 4 - k in state 5
        for k in range(5):
            nb = [0] * k + [5] * (4 - k)
            for sigma, u in ((0, 4), (1, 3), (0, 0)):
                prop = oracle.propose(q, 0, sigma, u)
                dE = k - sum(1 for x in nb if x == prop)
                if dE <= 0:
                    assert oracle.metropolis_decide(q, 0, nb, sigma, u, 2**32 - 1, T) == prop
                    continue
                t = int(T[dE])
                assert oracle.metropolis_decide(q, 0, nb, sigma, u, t - 1, T) == prop
                assert oracle.metropolis_decide(q, 0, nb, sigma, u, t, T) == 0
                assert oracle.metropolis_decide(q, 0, nb, sigma, u, 0, T) == prop


# --------------------------------------------------------------------------
# Initial populations
# --------------------------------------------------------------------------
def test_random_init_is_uniform_and_at_beta_zero():
    q, L, R = 10, 16, 4000
    s = oracle.init_random(q, L, 0, R, seed=1)
    counts = np.bincount(s.ravel(), minlength=q)
    expect = s.size / q
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 40.0  # 9 degrees of freedom; p < 1e-5 beyond this
    N = L * L
    E = np.array([oracle.energy(x) for x in s])
    sigma = math.sqrt(2 * N * (1 / q) * (1 - 1 / q))  # bonds are pairwise independent
    assert abs(E.mean() + 2 * N / q) < 5 * sigma / math.sqrt(R)
    # slots are independent streams: a range call equals the full call
    assert np.array_equal(oracle.init_random(q, L, 1234, 7, seed=1), s[1234:1241])


def test_ground_init_uniform_over_ground_states():
    q, L, R = 6, 8, 6000
    s = oracle.init_ground(q, L, 0, R, seed=5)
    assert all(oracle.energy(x) == -2 * L * L for x in s[:50])
    alpha = s[:, 0, 0]
    assert np.all(s == alpha[:, None, None])
    counts = np.bincount(alpha, minlength=q)
    chi2 = float(((counts - R / q) ** 2 / (R / q)).sum())
    assert chi2 < 30.0


# --------------------------------------------------------------------------
# Resampling (Sec. 2 step 2, Eq. 2)
# --------------------------------------------------------------------------
def test_equal_energies_give_exact_Q_and_single_copies():
    R, N = 500, 64
    E = np.full(R, -2 * N, np.int32)  # a ground-state population
    for dbeta in (0.01, 0.5, -0.2):
        r, lnQ, Rn, rho = oracle.copy_numbers(E, dbeta, R, oracle.NEAREST_INT, 3, 9)
        assert lnQ == -dbeta * (-2 * N)
        assert np.all(rho == 1.0) and np.all(r == 1) and Rn == R


def test_copy_numbers_properties():
    rng = np.random.default_rng(11)
    R = 4000
    E = rng.integers(-400, -100, size=R).astype(np.int32)
    dbeta = 0.02
    r, lnQ, Rn, rho = oracle.copy_numbers(E, dbeta, R, oracle.NEAREST_INT, 5, 1)
    assert rho.sum() == pytest.approx(R, rel=1e-12)
    # the two nearest integers only
    assert np.all((r == np.floor(rho)) | (r == np.floor(rho) + 1))
    # log-sum-exp through numpy's own reduction
    Emin = E.min()
    ref = -dbeta * Emin + math.log(np.exp(-dbeta * (E - Emin).astype(np.float64)).sum() / R)
    assert lnQ == pytest.approx(ref, rel=1e-13)
    # deterministic rounding: nearest integer with halves up
    r2, _, _, rho2 = oracle.copy_numbers(E, dbeta, R, oracle.ROUND, 5, 1)
    assert np.array_equal(r2, np.floor(rho2 + 0.5).astype(np.int32))
    # the parent map lists j exactly r_j times, in ascending order
    par = oracle.parents(r)
    assert par.size == Rn and np.array_equal(np.bincount(par, minlength=R), r)
    assert np.all(np.diff(par) >= 0)


def test_stochastic_rounding_is_unbiased():
    """E[r_j] = rho_j: average over many steps (fresh counters per step)."""
    rng = np.random.default_rng(2)
    R = 64
    E = rng.integers(-60, -20, size=R).astype(np.int32)
    acc = np.zeros(R)
    steps = 3000
    for step in range(1, steps + 1):
        r, _, _, rho = oracle.copy_numbers(E, 0.05, R, oracle.NEAREST_INT, step, 4)
        acc += r
    frac = rho - np.floor(rho)
    sd = np.sqrt(frac * (1 - frac) / steps) + 1e-12
    assert np.all(np.abs(acc / steps - rho) < 6 * sd + 1e-12)


def test_reweight_derivatives():
    rng = np.random.default_rng(5)
    # a population-like spread of energies (width ~ sqrt(N) for N = 256)
    E = np.rint(rng.normal(-300.0, 12.0, size=3000)).astype(np.int32)
    O = rng.normal(size=3000)
    d = 0.013
    lnQ, mE, mO, cov = oracle.reweight(E, d, O)
    h = 1e-4
    lp = oracle.reweight(E, d + h, O)
    lm = oracle.reweight(E, d - h, O)
    assert (lp[0] - lm[0]) / (2 * h) == pytest.approx(-mE, rel=1e-6)
    assert (lp[2] - lm[2]) / (2 * h) == pytest.approx(-cov, rel=1e-5, abs=1e-9)
    l0 = oracle.reweight(E, 0.0, O)
    assert l0[0] == 0.0
    assert l0[1] == pytest.approx(E.mean(), rel=1e-14)


# --------------------------------------------------------------------------
# PA as a whole against exact enumeration (Sec. 2 Eq. 2, Sec. 6)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("q,L", [(3, 4), (5, 3)])
def test_pa_free_energy_and_energy_match_exact_enumeration(q, L):
    """PA estimates of ln Z(beta) and <E>(beta) agree with exact values from
    the density of states within 5 standard errors (over seeds).  L = 3 is odd:
    the colour-ordered in-place sweep is still a sequence of single-site
    Metropolis updates and keeps the Boltzmann distribution stationary."""
    N = L * L
    g = oracle.density_of_states(q, L)
    K = 16
    betas = np.linspace(0.0, 1.6, K + 1)
    R = 6000
    lnz, me = [], []
    for seed in range(1, 7):
        out = oracle.run(q, L, R, seed, 5, betas, want_state=False)
        lnz.append(out["lnZ"])
        me.append(out["meanE"])
    lnz, me = np.array(lnz), np.array(me)
    for i in (0, 4, 8, 12, 16):
        ex = _lnZ_from_dos(g, N, betas[i])
        se = lnz[:, i].std(ddof=1) / math.sqrt(lnz.shape[0])
        if i == 0:
            assert lnz[0, 0] == pytest.approx(N * math.log(q), rel=1e-15)
            continue
        assert abs(lnz[:, i].mean() - ex) < 5 * se + 2e-3, (i, lnz[:, i].mean(), ex, se)
        exE = _mean_E_from_dos(g, N, betas[i])
        seE = me[:, i].std(ddof=1) / math.sqrt(me.shape[0])
        assert abs(me[:, i].mean() - exE) < 5 * seE + 2e-2, (i, me[:, i].mean(), exE, seE)


def test_heating_run_recovers_infinite_temperature_free_energy():
    """Ground-state start at beta = 3 with the zero-temperature normalisation
    ln Z = ln q - beta E_0 (Sec. 6, Eqs. 7-8), negative dbeta (Sec. 5),
    arrives at ln Z(0) = N ln q."""
    q, L = 3, 4
    N = L * L
    g = oracle.density_of_states(q, L)
    betas = np.linspace(3.0, 0.0, 31)
    ends = []
    for seed in range(1, 5):
        out = oracle.run(q, L, 4000, seed, 5, betas, init_mode=oracle.INIT_GROUND, want_state=False)
        assert out["lnZ"][0] == math.log(q) + 2 * N * 3.0
        ends.append(out["lnZ"][-1])
    # the normalisation itself is exact up to the excited states at beta = 3
    assert _lnZ_from_dos(g, N, 3.0) == pytest.approx(math.log(q) + 2 * N * 3.0, abs=1e-3)
    assert abs(np.mean(ends) - N * math.log(q)) < 0.05


def test_run_invariants_and_families():
    q, L, R = 10, 8, 800
    betas = np.linspace(0.0, 1.5, 21)
    out = oracle.run(q, L, R, 3, 4, betas, want_hist=True)
    N = L * L
    assert out["S_f"][0] == pytest.approx(math.log(R), rel=1e-14)
    assert out["n_families"][0] == R
    assert np.all(np.diff(out["n_families"]) <= 0)  # families never come back
    assert np.all(out["hist"].sum(axis=1) == out["R"])
    assert np.all(np.abs(out["R"] - R) < 60)
    # ln Z is the running sum of ln Q on top of N ln q (Eq. 2)
    assert np.allclose(out["lnZ"], N * math.log(q) + np.cumsum(out["lnQ"]), rtol=0, atol=1e-9)
    # final energies are the energies of the final spins
    for j in range(0, out["R_final"], 97):
        assert oracle.energy(out["spins"][j]) == out["E"][j]
    # past beta_t = ln(1 + sqrt 10) = 1.426 order grows (Eq. 5), even though a
    # fast cooling stays partly metastable (Sec. 4)
    assert out["meanM"][-1] > 3 * out["meanM"][0]


# --------------------------------------------------------------------------
# Differentiable reweighting and the adaptive step
# --------------------------------------------------------------------------
def _population_energies(seed=5, n=4000, mean=-300.0, sd=12.0):
    rng = np.random.default_rng(seed)
    return np.rint(rng.normal(mean, sd, size=n)).astype(np.int32)


def test_second_derivative_of_lnQ_is_the_reweighted_variance():
    E = _population_energies()
    for d in (0.0, 0.011, -0.007):
        r = oracle.reweight_all(E, d)
        h = 1e-4
        fd2 = (oracle.reweight_all(E, d + h)[0] - 2 * r[0] + oracle.reweight_all(E, d - h)[0]) / h**2
        assert fd2 == pytest.approx(r[2], rel=2e-4)
        fdE = -(oracle.reweight_all(E, d + h)[1] - oracle.reweight_all(E, d - h)[1]) / (2 * h)
        assert fdE == pytest.approx(r[2], rel=1e-6)
        fdV = -(oracle.reweight_all(E, d + h)[2] - oracle.reweight_all(E, d - h)[2]) / (2 * h)
        assert fdV == pytest.approx(r[7], rel=1e-3, abs=1e-3 * r[2] ** 1.5)
    # at dbeta = 0 the reweighted moments are the population's own
    r0 = oracle.reweight_all(E, 0.0)
    assert r0[2] == pytest.approx(E.astype(np.float64).var(), rel=1e-12)


def test_overlap_limits_and_derivative():
    E = _population_energies(n=6000, mean=-2500.0, sd=50.0)
    a0, da0 = oracle.overlap(E, 0.0)
    assert a0 == 1.0 and da0 == 0.0
    prev = 1.0
    for d in (0.002, 0.005, 0.01, 0.02, 0.05):
        a, da = oracle.overlap(E, d)
        assert a < prev  # the overlap falls as the step grows
        prev = a
        h = 1e-7
        fd = (oracle.overlap(E, d + h)[0] - oracle.overlap(E, d - h)[0]) / (2 * h)
        assert fd == pytest.approx(da, rel=1e-4)
    # equal energies: every weight is one, the overlap stays one
    assert oracle.overlap(np.full(100, -64, np.int32), 0.3)[0] == 1.0


def test_newton_step_meets_the_target_overlap():
    E = _population_energies(n=6000, mean=-2500.0, sd=50.0)
    for target in (0.6, 0.85, 0.95):
        d = oracle.newton_dbeta(E, target, 1.0)
        assert d * 2**24 == int(d * 2**24) and d > 0  # a multiple of 2^-24
        a, da = oracle.overlap(E, d)
        # rounding down by less than 2^-24 can only raise the overlap
        assert target <= a <= target + abs(da) * 2**-24 + 1e-9
    # a step that already meets the target is returned whole
    assert oracle.newton_dbeta(E, 0.001, 1e-4) == 1e-4


def test_adaptive_run_free_energy_matches_exact_enumeration():
    """Adaptive steps (overlap 0.85) from beta = 0 to 1.6 on 4x4, q = 3: ln Z at
    the end agrees with exact enumeration, and the last beta is exactly 1.6."""
    q, L = 3, 4
    N = L * L
    g = oracle.density_of_states(q, L)
    ends = []
    for seed in range(1, 6):
        out = oracle.run_adaptive(q, L, 5000, seed, 5, 1.6, target=0.85, dbeta_max=0.2)
        assert out["betas"][-1] == 1.6
        assert np.all(np.diff(out["betas"]) > 0)
        ends.append(out["lnZ"][-1])
    ex = _lnZ_from_dos(g, N, 1.6)
    se = np.std(ends, ddof=1) / math.sqrt(len(ends))
    assert abs(np.mean(ends) - ex) < 5 * se + 2e-3


def test_streams_give_independent_runs_under_one_key():
    """Stream numbers (top byte of the slot counter word) separate runs that
    share a key; stream 0 is the plain run."""
    q, L = 10, 8
    a = oracle.init_random(q, L, 0, 200, 1, stream=0)
    b = oracle.init_random(q, L, 0, 200, 1, stream=1)
    assert (a != b).mean() > 0.8
    betas = np.linspace(0.0, 1.0, 6)
    r0 = oracle.run(q, L, 300, 1, 2, betas)
    r0s = oracle.run(q, L, 300, 1, 2, betas, stream=0)
    r5 = oracle.run(q, L, 300, 1, 2, betas, stream=5)
    assert np.array_equal(r0["spins"], r0s["spins"])
    assert not np.array_equal(r0["sumE"], r5["sumE"])


def test_poisson_copy_numbers_follow_eq_1():
    """r_j ~ Pois(rho_j) (Sec. 2, Eq. 1): over many steps the counts of one
    replica have the Poisson mean and variance, and the total is Poisson(R)
    on average; a mean above the 64 piece size is handled."""
    rng = np.random.default_rng(9)
    R = 50
    E = rng.integers(-60, -40, size=R).astype(np.int32)
    draws, tot = [], []
    for step in range(1, 4001):
        r, _, Rn, rho = oracle.copy_numbers(E, 0.08, R, oracle.POISSON, step, 2)
        draws.append(r)
        tot.append(Rn)
    d = np.array(draws)
    mean, var = d.mean(axis=0), d.var(axis=0)
    se = np.sqrt(rho / 4000)
    assert np.all(np.abs(mean - rho) < 6 * se + 1e-9)
    big = np.argmax(rho)
    assert var[big] == pytest.approx(rho[big], rel=0.15)
    assert abs(np.mean(tot) - R) < 6 * math.sqrt(R / 4000)
    # one replica holding the whole population (mean R > 64)
    Ebig = np.array([-100] + [-10] * 9, np.int32)
    vals = [oracle.copy_numbers(Ebig, 1.0, 300, oracle.POISSON, s, 3)[0][0] for s in range(1, 1501)]
    assert abs(np.mean(vals) - 300) < 6 * math.sqrt(300 / 1500)
    assert np.var(vals) == pytest.approx(300, rel=0.15)


def test_resampling_off_keeps_every_replica():
    E = np.arange(-50, -10, dtype=np.int32)
    r, lnQ, Rn, _ = oracle.copy_numbers(E, 0.3, 40, oracle.OFF, 1, 1)
    assert np.all(r == 1) and Rn == 40
    out = oracle.run(6, 8, 300, 1, 2, np.linspace(0, 1.5, 11), mode=oracle.OFF)
    assert np.all(out["R"] == 300) and np.all(out["n_families"] == 300)  # no family is lost


# --------------------------------------------------------------------------
# The normaliser S: the exact sum of the weights, rounded once (Sec. 2 step 2)
# --------------------------------------------------------------------------
def _correctly_rounded_sum(xs):
    """Python's rational arithmetic: the exact sum, then one correctly rounded
    conversion (int / int true division rounds correctly)."""
    from fractions import Fraction

    return float(sum((Fraction(float(x)) for x in xs), Fraction(0)))


def test_exact_sum_is_the_correctly_rounded_sum():
    rng = np.random.default_rng(11)
    eps = 2.0 ** -52
    cases = [
        rng.random(2000),
        np.exp(-0.008 * rng.integers(0, 8193, size=5000)),      # PA weights at dbeta = 0.008
        np.exp(-0.7 * rng.integers(0, 300, size=3000)),         # down to 1e-91
        np.array([1.0] + [2.0 ** -60] * 5000),                  # naive summation drops every small term
        np.array([1.0, 2.0 ** -53]),                            # exactly halfway: ties to even (down)
        np.array([1.0, 2.0 ** -53, 2.0 ** -300]),               # just above halfway: up
        np.array([1.0 + eps, 2.0 ** -53]),                      # halfway from an odd mantissa: up
        np.array([5e-324, 5e-324, 3 * 5e-324, 2.0 ** -1022]),   # subnormals
        np.array([0.0, 0.0]),
        np.array([2.0 ** 52, 0.5, 0.5, 0.25]),
        np.array([1e300, 1e300, 1e-300]),
        rng.random(7) * 2.0 ** rng.integers(-1070, 1000, size=7),
    ]
    for xs in cases:
        want = _correctly_rounded_sum(xs)
        got = oracle.exact_sum(xs)
        assert got == want, (xs[:4], got, want)
        assert oracle.exact_sum(rng.permutation(xs)) == got  # no summation order
        assert got == math.fsum(xs)
    assert oracle.exact_sum(np.array([1.0, 2.0 ** -53])) == 1.0
    assert oracle.exact_sum(np.array([1.0 + eps, 2.0 ** -53])) == 1.0 + 2 * eps


def test_copy_number_normaliser_is_exact_and_order_free():
    """S enters ln Q and every rho_j; with the exact sum, the oracle's ln Q
    equals -dbeta E_ref + ln(S/R) for the correctly rounded S, and a permuted
    population gives bit-identical rho (as a multiset)."""
    rng = np.random.default_rng(3)
    E = rng.integers(-700, -400, size=3000).astype(np.int32)
    dbeta = 0.0123
    r, lnq, Rn, rho = oracle.copy_numbers(E, dbeta, 3000, oracle.NEAREST_INT, 4, 9)
    # the C library's exp, as the oracle uses (numpy's exp rounds differently)
    w = np.array([math.exp(-dbeta * float(e - E.min())) for e in E])
    S = _correctly_rounded_sum(w)
    assert lnq == -dbeta * float(E.min()) + math.log(S / E.size)
    assert np.array_equal(rho, (3000.0 * w) / S)
    perm = rng.permutation(E.size)
    _, lnq2, _, rho2 = oracle.copy_numbers(E[perm], dbeta, 3000, oracle.NEAREST_INT, 4, 9)
    assert lnq2 == lnq
    assert np.array_equal(np.sort(rho2), np.sort(rho))


# --------------------------------------------------------------------------
# Near-tie flags of the copy-number rules
# --------------------------------------------------------------------------
def _nudged(rho, k):
    x = rho
    for _ in range(abs(k)):
        x = np.nextafter(x, math.inf if k > 0 else -math.inf)
    return x


def test_near_tie_flag_marks_every_draw_a_last_place_change_could_flip():
    """Unflagged draws keep their copy number when rho moves by up to eight
    units in the last place; draws placed exactly on a boundary are flagged;
    the flag fires for a fraction of random draws close to 2 delta 2^32."""
    rng = np.random.default_rng(5)
    flagged = 0
    n = 20000
    for _ in range(n):
        rho = float(rng.exponential(1.5))
        u = int(rng.integers(0, 2**32))
        for mode in (oracle.NEAREST_INT, oracle.ROUND):
            r, tie = oracle.round_copies(mode, rho, u)
            assert r in (math.floor(rho), math.floor(rho) + 1)
            flagged += tie
            if not tie:
                for k in (-8, -3, -1, 1, 3, 8):
                    assert oracle.round_copies(mode, _nudged(rho, k), u)[0] == r, (mode, rho, u, k)
    assert flagged <= 3  # expected about 2 n 2^-48 2^32 ~ 6e-4
    # on the boundary: frac(rho) = u / 2^32, or 1/2 for ROUND
    for n0 in (0, 1, 3, 17):
        for u in (1, 12345, 2**31, 2**32 - 7):
            rho = n0 + u * 2.0 ** -32
            assert oracle.round_copies(oracle.NEAREST_INT, rho, u)[1]
            r_lo = oracle.round_copies(oracle.NEAREST_INT, _nudged(rho, -1), u)[0]
            r_hi = oracle.round_copies(oracle.NEAREST_INT, _nudged(rho, 1), u)[0]
            assert (r_lo, r_hi) == (n0, n0 + 1)
        assert oracle.round_copies(oracle.ROUND, n0 + 0.5)[1]
        assert oracle.round_copies(oracle.ROUND, _nudged(n0 + 0.5, -1))[0] == n0


def test_near_tie_count_of_a_run_matches_the_flags():
    q, L, R = 6, 8, 1500
    betas = np.linspace(0.0, 1.2, 9)
    out = oracle.run(q, L, R, 4, 2, betas, want_state=False)
    assert out["n_near_ties"][0] == 0
    assert np.all(out["n_near_ties"] >= 0) and out["n_near_ties"].sum() <= 2


# --------------------------------------------------------------------------
# Magnetisation and specific heat (Sec. 3, Eqs. 4-5; fluctuation formula)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("q,L", [(3, 4), (10, 6)])
def test_ground_state_population_has_full_magnetisation(q, L):
    """A replica in a ground state has m = 1 (Eq. 5, every site in one state),
    so a population of ground states has <M> = N exactly; a wrong (q - 1)
    normalisation would not give N."""
    N = L * L
    out = oracle.run(q, L, 500, 2, 3, np.array([2.5]), init_mode=oracle.INIT_GROUND, want_state=False)
    assert out["meanM"][0] == N
    assert out["sumMt"][0] == 500 * N


def test_infinite_temperature_magnetisation_matches_enumeration():
    """<M> at beta = 0 over q^N equally likely configurations (exact, by
    enumeration of the largest occupation) against the oracle's population of
    independent uniform replicas, within 5 standard errors."""
    import itertools

    q, L = 3, 2
    N = L * L
    Mt = np.array([max(np.bincount(c, minlength=q)) for c in itertools.product(range(q), repeat=N)], dtype=float)
    M = (q * Mt - N) / (q - 1)
    R = 40000
    out = oracle.run(q, L, R, 8, 1, np.array([0.0]), want_state=False)
    assert abs(out["meanM"][0] - M.mean()) < 5 * M.std() / math.sqrt(R)


def _var_E_from_dos(g, N, beta):
    E = np.arange(-2 * N, 1, dtype=np.float64)
    gg = g.astype(np.float64)
    a = np.where(gg > 0, np.log(np.maximum(gg, 1)) - beta * E, -np.inf)
    w = np.exp(a - a.max())
    m1 = (w * E).sum() / w.sum()
    return float((w * (E - m1) ** 2).sum() / w.sum())


def test_specific_heat_matches_exact_enumeration():
    """The oracle's C = beta^2 (<E^2> - <E>^2) / N from PA populations against
    beta^2 var(E) / N from the exact density of states (4 x 4, q = 3), within
    5 standard errors over seeds."""
    q, L = 3, 4
    N = L * L
    g = oracle.density_of_states(q, L)
    betas = np.linspace(0.0, 1.6, 17)
    C = np.array([oracle.run(q, L, 6000, s, 5, betas, want_state=False)["C"] for s in range(1, 7)])
    for i in (4, 8, 10, 12, 16):
        ex = betas[i] ** 2 * _var_E_from_dos(g, N, betas[i]) / N
        se = C[:, i].std(ddof=1) / math.sqrt(C.shape[0])
        assert abs(C[:, i].mean() - ex) < 5 * se + 5e-3 * ex, (i, C[:, i].mean(), ex, se)


# --------------------------------------------------------------------------
# The sweep's random-number rule: site words of each colour (Sec. 2 step 3 reading)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 16, 24, 32, 48, 64, 66, 80, 96, 112, 128, 130, 144, 160, 192, 256])
def test_site_words_are_a_bijection_onto_each_colour(L):
    """For each colour the valid (word, bit) pairs map one to one onto that
    colour's L^2/2 sites; with packed rows (L = 8, 16, 32, 64) and banded rows
    (L = 48, 80, 96, ...) every bit of every word holds a site."""
    words = oracle.colour_words(L)
    full = (L >= 8 and 64 % L == 0) or (L > 32 and L % 16 == 0 and L % 64 != 0)
    for c in (0, 1):
        seen = {}
        for w in range(words):
            for b in range(32):
                xy = oracle.word_site(L, c, w, b)
                if xy is None:
                    assert not full, (L, c, w, b)
                    continue
                x, y = xy
                assert 0 <= x < L and 0 <= y < L and (x + y) % 2 == c
                assert (x, y) not in seen, (L, c, w, b, seen.get((x, y)))
                seen[(x, y)] = (w, b)
        assert len(seen) == L * L // 2
    if full:
        assert words == L * L // 64
