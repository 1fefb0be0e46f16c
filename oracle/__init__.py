"""CPU oracle for population annealing of the 2D q-state Potts model.

TEST INFRASTRUCTURE, not part of the product.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  It wraps ``pa_oracle.c`` (plain,
single-threaded C; see that file for the paper passages each function
follows) with ctypes and numpy.  It never imports the CUDA package and the
CUDA package never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_LIB = os.path.join(_HERE, "libpa_oracle.so")

NEAREST_INT = 0
ROUND = 1
POISSON = 2
OFF = 3
INIT_RANDOM = 0
INIT_GROUND = 1


def build(force: bool = False) -> str:
    """Compile pa_oracle.c into libpa_oracle.so (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-Wall", "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


class Obs(ctypes.Structure):
    _fields_ = [
        ("beta", ctypes.c_double), ("lnQ", ctypes.c_double), ("lnZ", ctypes.c_double),
        ("meanE", ctypes.c_double), ("meanE2", ctypes.c_double), ("C", ctypes.c_double),
        ("meanM", ctypes.c_double), ("S_f", ctypes.c_double),
        ("R", ctypes.c_int64), ("n_families", ctypes.c_int64), ("sumE", ctypes.c_int64),
        ("sumE2", ctypes.c_int64), ("sumMt", ctypes.c_int64), ("n_near_ties", ctypes.c_int64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        P = ctypes.c_void_p
        i32, i64, u32, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_energy.argtypes = [ctypes.c_int, P]
        L.orc_energy.restype = i64
        L.orc_max_count.argtypes = [ctypes.c_int, ctypes.c_int, P]
        L.orc_max_count.restype = i64
        L.orc_state_bits.argtypes = [ctypes.c_int]
        L.orc_state_bits.restype = ctypes.c_int
        L.orc_thresholds.argtypes = [f64, P]
        L.orc_propose.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32]
        L.orc_propose.restype = ctypes.c_int
        L.orc_metropolis_decide.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, u32, u32, P]
        L.orc_metropolis_decide.restype = ctypes.c_int
        L.orc_below_value.argtypes = [u32, u64]
        L.orc_below_value.restype = ctypes.c_int
        L.orc_sweep_replica.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, u32, u32, u64, u32]
        L.orc_sweep_replica.restype = i64
        L.orc_init_random.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, u64, u32, P]
        L.orc_init_ground.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, u64, u32, P]
        L.orc_copy_numbers.argtypes = [i64, P, f64, i64, ctypes.c_int, u32, u64, u32, P, P, P, P, P]
        L.orc_copy_numbers.restype = i64
        L.orc_round_copies.argtypes = [ctypes.c_int, f64, u32, P]
        L.orc_round_copies.restype = i32
        L.orc_exact_sum.argtypes = [i64, P]
        L.orc_exact_sum.restype = f64
        L.orc_colour_words.argtypes = [ctypes.c_int]
        L.orc_colour_words.restype = ctypes.c_int
        L.orc_word_site.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
        L.orc_word_site.restype = ctypes.c_int
        L.orc_parents.argtypes = [i64, P, P]
        L.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, u64, u32, ctypes.c_int, ctypes.c_int, P,
                              ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        L.orc_run.restype = i64
        L.orc_obs_size.restype = ctypes.c_int
        L.orc_density_of_states.argtypes = [ctypes.c_int, ctypes.c_int, P]
        L.orc_density_of_states.restype = ctypes.c_int
        L.orc_site_matrix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, f64, P]
        L.orc_site_matrix.restype = ctypes.c_int
        L.orc_reweight.argtypes = [i64, P, P, f64, P]
        L.orc_overlap.argtypes = [i64, P, f64, P]
        L.orc_newton_dbeta.argtypes = [i64, P, f64, f64, ctypes.c_int]
        L.orc_newton_dbeta.restype = f64
        L.orc_run_adaptive.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, u64, u32, ctypes.c_int, f64, f64, f64,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P]
        L.orc_run_adaptive.restype = ctypes.c_int
        assert L.orc_obs_size() == ctypes.sizeof(Obs)
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def energy(spins: np.ndarray) -> int:
    s = np.ascontiguousarray(spins, dtype=np.uint8)
    return int(lib().orc_energy(s.shape[-1], _p(s)))


def max_count(q: int, spins: np.ndarray) -> int:
    s = np.ascontiguousarray(spins, dtype=np.uint8)
    return int(lib().orc_max_count(q, s.shape[-1], _p(s)))


def state_bits(q: int) -> int:
    return int(lib().orc_state_bits(q))


def thresholds(beta: float) -> np.ndarray:
    """T[d] = floor(exp(-beta d) 2^32) for d = 1..4 (T[0] = 2^32)."""
    t = np.zeros(5, dtype=np.uint64)
    lib().orc_thresholds(float(beta), _p(t))
    return t


def propose(q: int, cur: int, sigma: int, u: int) -> int:
    return int(lib().orc_propose(q, cur, sigma, int(u)))


def below_value(v: int, T: int) -> bool:
    """The sweep's most-significant-bit-first comparison v < T."""
    return bool(lib().orc_below_value(int(v), int(T)))


def metropolis_decide(q, cur, nb, sigma, u, v, T) -> int:
    n = np.ascontiguousarray(nb, dtype=np.int32)
    t = np.ascontiguousarray(T, dtype=np.uint64)
    return int(lib().orc_metropolis_decide(q, cur, _p(n), int(sigma), int(u), int(v), _p(t)))


def sweep_replica(q: int, spins: np.ndarray, beta: float, theta: int, step: int, slot: int, seed: int,
                  stream: int = 0, with_calls: bool = False):
    """theta sweeps of one L x L replica; returns a new array (and, with
    with_calls, the number of Philox calls its site words drew)."""
    s = np.array(spins, dtype=np.uint8, copy=True, order="C")
    thr = thresholds(beta)
    calls = lib().orc_sweep_replica(q, s.shape[-1], _p(s), _p(thr), theta, step, slot, seed, stream)
    return (s, int(calls)) if with_calls else s


def init_random(q: int, L: int, slot_begin: int, count: int, seed: int, stream: int = 0) -> np.ndarray:
    out = np.zeros((count, L, L), dtype=np.uint8)
    lib().orc_init_random(q, L, slot_begin, count, seed, stream, _p(out))
    return out


def init_ground(q: int, L: int, slot_begin: int, count: int, seed: int, stream: int = 0) -> np.ndarray:
    out = np.zeros((count, L, L), dtype=np.uint8)
    lib().orc_init_ground(q, L, slot_begin, count, seed, stream, _p(out))
    return out


def copy_numbers(E: np.ndarray, dbeta: float, R_target: int, mode: int, step: int, seed: int, stream: int = 0,
                 with_ties: bool = False):
    """Returns (r, lnQ, R_new, rho), with the per-replica near-tie flags
    appended when with_ties."""
    e = np.ascontiguousarray(E, dtype=np.int32)
    r = np.zeros(e.size, dtype=np.int32)
    rho = np.zeros(e.size, dtype=np.float64)
    ties = np.zeros(e.size, dtype=np.int32)
    n_ties = ctypes.c_int64()
    lnq = ctypes.c_double()
    Rn = lib().orc_copy_numbers(e.size, _p(e), float(dbeta), R_target, mode, step, seed, stream, _p(r),
                                ctypes.byref(lnq), _p(rho), _p(ties), ctypes.byref(n_ties))
    if with_ties:
        return r, lnq.value, int(Rn), rho, ties
    return r, lnq.value, int(Rn), rho


def round_copies(mode: int, rho: float, u: int = 0):
    """(r, near_tie) of the nearest-integer (uniform word u) or ROUND rule."""
    tie = ctypes.c_int()
    r = lib().orc_round_copies(mode, float(rho), int(u), ctypes.byref(tie))
    return int(r), bool(tie.value)


def exact_sum(x) -> float:
    """The exact sum of non-negative finite doubles, rounded once to the
    nearest double (ties to even)."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().orc_exact_sum(a.size, _p(a)))


def colour_words(L: int) -> int:
    """Site words of one colour per replica (the sweep's random-number rule)."""
    return int(lib().orc_colour_words(L))


def word_site(L: int, colour: int, w: int, b: int):
    """(x, y) of the site at bit b of site word w of colour `colour`, or None."""
    x, y = ctypes.c_int(), ctypes.c_int()
    ok = lib().orc_word_site(L, colour, w, b, ctypes.byref(x), ctypes.byref(y))
    return (x.value, y.value) if ok else None


def parents(r: np.ndarray) -> np.ndarray:
    rr = np.ascontiguousarray(r, dtype=np.int32)
    out = np.zeros(int(rr.sum()), dtype=np.int32)
    lib().orc_parents(rr.size, _p(rr), _p(out))
    return out


def run(q, L, R, seed, theta, betas, mode=NEAREST_INT, init_mode=INIT_RANDOM, R_cap=None,
        want_hist=False, want_state=True, stream=0):
    """Full PA run over betas[0..K].  Returns a dict of numpy arrays."""
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    K = betas.size - 1
    N = L * L
    if R_cap is None:
        R_cap = R + R // 4 + 64
    obs = (Obs * (K + 1))()
    hist = np.zeros((K + 1, 2 * N + 1), dtype=np.int32) if want_hist else None
    spins = np.zeros((R_cap, L, L), dtype=np.uint8) if want_state else None
    E = np.zeros(R_cap, dtype=np.int32) if want_state else None
    anc = np.zeros(R_cap, dtype=np.int32) if want_state else None
    Rf = lib().orc_run(q, L, R, R_cap, seed, stream, theta, K, _p(betas), mode, init_mode,
                       ctypes.cast(obs, ctypes.c_void_p),
                       _p(hist) if hist is not None else None,
                       _p(spins) if spins is not None else None,
                       _p(E) if E is not None else None,
                       _p(anc) if anc is not None else None)
    out = {name: np.array([getattr(o, name) for o in obs]) for name, _ in Obs._fields_}
    out["R_final"] = int(Rf)
    if want_hist:
        out["hist"] = hist
    if want_state and Rf > 0:
        out["spins"] = spins[:Rf]
        out["E"] = E[:Rf]
        out["anc"] = anc[:Rf]
    return out


def density_of_states(q: int, L: int) -> np.ndarray:
    g = np.zeros(2 * L * L + 1, dtype=np.uint64)
    rc = lib().orc_density_of_states(q, L, _p(g))
    if rc != 0:
        raise ValueError("lattice too large for enumeration")
    return g


def site_matrix(q: int, L: int, site: int, beta: float) -> np.ndarray:
    n = q ** (L * L)
    P = np.zeros((n, n), dtype=np.float64)
    rc = lib().orc_site_matrix(q, L, site, float(beta), _p(P))
    if rc != 0:
        raise ValueError("state space too large")
    return P


def reweight(E: np.ndarray, dbeta: float, O: np.ndarray | None = None):
    """Returns (lnQ, <E>_tau, <O>_tau, cov_tau(O, E))."""
    r = reweight_all(E, dbeta, O)
    return r[0], r[1], (r[3] if O is not None else None), (r[4] if O is not None else None)


def reweight_all(E: np.ndarray, dbeta: float, O: np.ndarray | None = None) -> np.ndarray:
    """[lnQ, <E>_tau, var_tau(E), <O>_tau, cov_tau(O, E), E_ref, S, k3_tau(E)]."""
    e = np.ascontiguousarray(E, dtype=np.int32)
    o = np.ascontiguousarray(O, dtype=np.float64) if O is not None else None
    out = np.zeros(8, dtype=np.float64)
    lib().orc_reweight(e.size, _p(e), _p(o) if o is not None else None, float(dbeta), _p(out))
    return out


def overlap(E: np.ndarray, dbeta: float):
    """(alpha, alpha') of the weight overlap."""
    e = np.ascontiguousarray(E, dtype=np.int32)
    out = np.zeros(2, dtype=np.float64)
    lib().orc_overlap(e.size, _p(e), float(dbeta), _p(out))
    return float(out[0]), float(out[1])


def newton_dbeta(E: np.ndarray, target: float, dbeta_max: float, iters: int = 12) -> float:
    e = np.ascontiguousarray(E, dtype=np.int32)
    return float(lib().orc_newton_dbeta(e.size, _p(e), float(target), float(dbeta_max), int(iters)))


def run_adaptive(q, L, R, seed, theta, beta_end, target=0.85, dbeta_max=0.05, iters=12, max_steps=10000,
                 mode=NEAREST_INT, R_cap=None, stream=0):
    """PA with the Newton step on the weight overlap; returns a dict with the
    per-step estimators, the betas taken and the final population."""
    N = L * L
    if R_cap is None:
        R_cap = R + R // 4 + 64
    obs = (Obs * (max_steps + 1))()
    betas = np.zeros(max_steps + 1, dtype=np.float64)
    spins = np.zeros((R_cap, L, L), dtype=np.uint8)
    E = np.zeros(R_cap, dtype=np.int32)
    K = lib().orc_run_adaptive(q, L, R, R_cap, seed, stream, theta, float(beta_end), float(target), float(dbeta_max),
                               iters, max_steps, mode, ctypes.cast(obs, ctypes.c_void_p), _p(betas), _p(spins), _p(E))
    out = {name: np.array([getattr(o, name) for o in obs[: max(K, 0) + 1]]) for name, _ in Obs._fields_}
    out["K"] = K
    out["betas"] = betas[: max(K, 0) + 1]
    if K >= 0:
        Rf = int(out["R"][-1])
        out["spins"] = spins[:Rf]
        out["E"] = E[:Rf]
    return out
