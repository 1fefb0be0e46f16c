"""GB300 population annealing for the 2D q-state Potts model.

A thin ctypes binding over the C ABI in ``include/pa.h`` (library
``libpa_gb300.so``, built by :mod:`paper_1704_01888_gb300.build`).  The
binding only marshals arguments: every step of the method runs in the
library's CUDA kernels.  PyTorch supplies the CUDA stream
(``torch.cuda.current_stream()``).  If the library is missing the binding
raises; there is no CPU fallback.

The method is population annealing as in Barash, Weigel, Shchur & Janke,
"Exploring first-order phase transitions with population annealing"
(arXiv:1704.01888), Sec. 2 (algorithm, Eq. 2), Sec. 3 (model, Eqs. 3-5),
Sec. 5 (heating, Eq. 6) and Sec. 6 (free-energy normalisations, Eqs. 7-8).
"""
from __future__ import annotations

import ctypes
import os
import time
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpa_gb300.so")

(PA_OK, PA_ERR_INVALID, PA_ERR_CAPACITY, PA_ERR_CUDA, PA_ERR_TIMEOUT, PA_ERR_STATE, PA_ERR_NOMEM,
 PA_ERR_TOO_LARGE) = range(8)
RESAMPLE_NEAREST_INT = 0
RESAMPLE_ROUND = 1
RESAMPLE_POISSON = 2
RESAMPLE_OFF = 3
INIT_RANDOM = 0
INIT_GROUND = 1

# Every extern "C" symbol declared in include/pa.h.
EXPORTED = (
    "pa_init", "pa_resample", "pa_sweep", "pa_energy", "pa_observables", "pa_population_size",
    "pa_get_spins", "pa_get_ancestors", "pa_run", "pa_destroy", "pa_status_str", "pa_last_cuda_error",
    "pa_set_launch", "pa_kernel_launch_count", "pa_profile", "pa_profile_read", "pa_observables_history",
    "pa_get_launch", "pa_resample_noalloc", "pa_reweight_forward", "pa_reweight_scale", "pa_reweight_grad_O",
    "pa_overlap", "pa_next_dbeta", "pa_run_adaptive", "pa_batch_create", "pa_batch_autotune", "pa_batch_set_launch",
    "pa_batch_get_launch", "pa_batch_run", "pa_batch_observables", "pa_batch_get_spins", "pa_batch_destroy",
    "pa_batch_population_size", "pa_save", "pa_load", "pa_occupations", "pa_batch_measurements",
    "pa_get_parents", "pa_shard_plan", "pa_shard_init", "pa_shard_get_buffers", "pa_shard_counts", "pa_shard_pack",
    "pa_shard_accept", "pa_shard_finalize", "pa_shard_range",
)


class PAError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(what)


class Config(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int32), ("L", ctypes.c_int32), ("R", ctypes.c_int32), ("R_cap", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("resample_mode", ctypes.c_int32), ("init_mode", ctypes.c_int32),
        ("beta0", ctypes.c_double), ("track_families", ctypes.c_int32), ("stream", ctypes.c_int32),
    ]


class RunDesc(ctypes.Structure):
    _fields_ = [("cfg", Config), ("betas", ctypes.c_void_p), ("K", ctypes.c_int32), ("theta", ctypes.c_int32)]


class ShardBuffers(ctypes.Structure):
    _fields_ = [
        ("hist", ctypes.c_void_p), ("sums", ctypes.c_void_p), ("fam", ctypes.c_void_p), ("send", ctypes.c_void_p),
        ("send_anc", ctypes.c_void_p), ("send_cnt", ctypes.c_void_p), ("recv", ctypes.c_void_p),
        ("recv_anc", ctypes.c_void_p), ("recv_cnt", ctypes.c_void_p),
        ("replica_words", ctypes.c_int64), ("capacity", ctypes.c_int64), ("n_bins", ctypes.c_int64),
    ]


class Obs(ctypes.Structure):
    _fields_ = [
        ("beta", ctypes.c_double), ("lnQ", ctypes.c_double), ("lnZ", ctypes.c_double),
        ("meanE", ctypes.c_double), ("meanE2", ctypes.c_double), ("C", ctypes.c_double),
        ("meanM", ctypes.c_double), ("S_f", ctypes.c_double),
        ("R", ctypes.c_int64), ("n_families", ctypes.c_int64), ("sumE", ctypes.c_int64),
        ("sumE2", ctypes.c_int64), ("sumMt", ctypes.c_int64), ("n_near_ties", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def load_library(path: str | None = None):
    """Loads libpa_gb300.so, or the library the PA_LIBRARY environment
    variable names (e.g. the checked build); raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or os.environ.get("PA_LIBRARY") or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: run paper_1704_01888_gb300.build.build() first")
    lib = ctypes.CDLL(p)
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "pa_init": ([ctypes.POINTER(Config), P, ctypes.POINTER(P)], st),
        "pa_resample": ([P, f64, i32, P, P], st),
        "pa_sweep": ([P, f64, i32, i32], st),
        "pa_energy": ([P, P, i32], st),
        "pa_observables": ([P, ctypes.POINTER(Obs), P, i32], st),
        "pa_population_size": ([P, P], st),
        "pa_get_spins": ([P, i64, i64, P], st),
        "pa_get_ancestors": ([P, P], st),
        "pa_get_parents": ([P, P, i32], st),
        "pa_shard_plan": ([P, i32, i32, P, P, P, P, P], st),
        "pa_shard_init": ([ctypes.POINTER(Config), i32, i32, P, ctypes.POINTER(P)], st),
        "pa_shard_get_buffers": ([P, ctypes.POINTER(ShardBuffers)], st),
        "pa_shard_counts": ([P, f64, i32, P], st),
        "pa_shard_pack": ([P, P, P], st),
        "pa_shard_accept": ([P, P], st),
        "pa_shard_finalize": ([P, f64], st),
        "pa_shard_range": ([P, P, P, P], st),
        "pa_run": ([P, P, i32, i32, P, P, i32, P, i32], st),
        "pa_destroy": ([P], None),
        "pa_status_str": ([st], ctypes.c_char_p),
        "pa_last_cuda_error": ([], ctypes.c_char_p),
        "pa_set_launch": ([P, i32, i32], st),
        "pa_kernel_launch_count": ([], i64),
        "pa_profile": ([P, i32], st),
        "pa_profile_read": ([P, P, P], st),
        "pa_observables_history": ([P, i32, P], st),
        "pa_get_launch": ([P, P, P, P], st),
        "pa_resample_noalloc": ([P, i32, i32, f64, i32, i32, i32, ctypes.c_uint64, i32, P, i32, P, P, P], st),
        "pa_reweight_forward": ([P, P, i32, P, P, P], st),
        "pa_reweight_scale": ([P, i32, f64, P, P, P], st),
        "pa_reweight_grad_O": ([P, i32, P, P, P, P, P], st),
        "pa_overlap": ([P, i32, P, P, P], st),
        "pa_next_dbeta": ([P, f64, f64, i32, P], st),
        "pa_run_adaptive": ([P, f64, f64, f64, i32, i32, i32, P, P, P], st),
        "pa_batch_create": ([P, i32, P, ctypes.POINTER(P)], st),
        "pa_batch_autotune": ([P, P, P], st),
        "pa_batch_set_launch": ([P, i32, i32], st),
        "pa_batch_get_launch": ([P, P, P, P], st),
        "pa_batch_run": ([P, i32], st),
        "pa_batch_observables": ([P, i32, P], st),
        "pa_batch_get_spins": ([P, i32, i64, i64, P], st),
        "pa_batch_destroy": ([P], None),
        "pa_batch_population_size": ([P, i32, P], st),
        "pa_occupations": ([P, P, i32], st),
        "pa_batch_measurements": ([P, i32, P, P], st),
        "pa_save": ([P, ctypes.c_char_p], st),
        "pa_load": ([ctypes.c_char_p, P, ctypes.POINTER(P)], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def _check(status: int, what: str):
    if status != PA_OK:
        lib = load_library()
        msg = lib.pa_status_str(status).decode()
        cuda = lib.pa_last_cuda_error().decode()
        raise PAError(status, f"{what}: {msg}" + (f" ({cuda})" if cuda and status == PA_ERR_CUDA else ""))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _current_stream() -> int:
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("population annealing runs on a CUDA GPU; none is available")
    return torch.cuda.current_stream().cuda_stream


def resample_noalloc(E_ptr: int, R_prev: int, L: int, dbeta: float, R_target: int, mode: int, step: int,
                     seed: int, parent_ptr: int, parent_cap: int, lnQ_ptr: int, R_ptr: int, stream: int,
                     rng_stream: int = 0) -> None:
    """pa_resample_noalloc on device pointers (see include/pa.h): resampling
    for callers that may not allocate device memory.  Raises PAError on a
    rejected call; the results land in the device outputs."""
    _check(load_library().pa_resample_noalloc(
        ctypes.c_void_p(E_ptr), R_prev, L, float(dbeta), R_target, mode, step, seed, int(rng_stream),
        ctypes.c_void_p(parent_ptr), parent_cap, ctypes.c_void_p(lnQ_ptr), ctypes.c_void_p(R_ptr),
        ctypes.c_void_p(stream)), "pa_resample_noalloc")


def shard_plan(totals, world: int, rank: int):
    """The exchange plan of one step of a population spread over `world`
    ranks (pa_shard_plan; host only): (R_new, lo, hi, send_counts,
    recv_counts)."""
    t = np.ascontiguousarray(totals, dtype=np.int64)
    if t.size != world:
        raise ValueError("one total per rank")
    send = np.zeros(world, dtype=np.int64)
    recv = np.zeros(world, dtype=np.int64)
    R_new, lo, hi = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().pa_shard_plan(_ptr(t), world, rank, ctypes.byref(R_new), ctypes.byref(lo), ctypes.byref(hi),
                                        _ptr(send), _ptr(recv)), "pa_shard_plan")
    return R_new.value, lo.value, hi.value, send, recv


def kernel_launch_count() -> int:
    return int(load_library().pa_kernel_launch_count())


@dataclass
class PAParams:
    q: int
    L: int
    R: int
    seed: int = 1
    R_cap: int = 0
    resample_mode: int = RESAMPLE_NEAREST_INT
    init_mode: int = INIT_RANDOM
    beta0: float = 0.0
    track_families: bool = False
    stream: int = 0


class Population:
    """One PA run on the GPU: a population of R_i replicas of the L x L Potts
    lattice at the current inverse temperature (Sec. 2)."""

    def __init__(self, params: PAParams, stream: int | None = None, _ctx=None, _step=0, _beta=None):
        self.params = params
        self.lib = load_library()
        self._stream = _current_stream() if stream is None else stream
        if _ctx is not None:
            self._ctx = _ctx
            self.N = params.L * params.L
            self.step = _step
            self.beta = _beta
            return
        cfg = Config(params.q, params.L, params.R, params.R_cap, params.seed, params.resample_mode,
                     params.init_mode, params.beta0, int(params.track_families), int(params.stream))
        self._ctx = ctypes.c_void_p()
        _check(self.lib.pa_init(ctypes.byref(cfg), ctypes.c_void_p(self._stream), ctypes.byref(self._ctx)),
               "pa_init")
        self.N = params.L * params.L
        self.step = 0
        self.beta = params.beta0

    # -- lifecycle -------------------------------------------------------
    def close(self):
        if self._ctx:
            self.lib.pa_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the PA step (Sec. 2 steps 2-4) -----------------------------------
    def resample(self, dbeta: float, step: int | None = None, sync: bool = False):
        """Sec. 2 step 2.  With sync=True returns (ln Q_i, R_i)."""
        step = self.step + 1 if step is None else step
        if sync:
            lnq = ctypes.c_double()
            rr = ctypes.c_int32()
            _check(self.lib.pa_resample(self._ctx, float(dbeta), step, ctypes.byref(lnq), ctypes.byref(rr)),
                   "pa_resample")
            self._pending = step
            return lnq.value, rr.value
        _check(self.lib.pa_resample(self._ctx, float(dbeta), step, None, None), "pa_resample")
        self._pending = step
        return None

    def sweep(self, beta: float, theta: int, step: int | None = None):
        """Sec. 2 step 3: theta checkerboard Metropolis sweeps at beta."""
        if step is None:
            step = getattr(self, "_pending", None) or self.step
        _check(self.lib.pa_sweep(self._ctx, float(beta), int(theta), int(step)), "pa_sweep")
        self._pending = None
        self.step = step
        self.beta = beta

    def observables(self, with_hist: bool = False):
        obs = Obs()
        hist = np.zeros(2 * self.N + 1, dtype=np.int32) if with_hist else None
        _check(self.lib.pa_observables(self._ctx, ctypes.byref(obs), _ptr(hist) if with_hist else None,
                                       hist.size if with_hist else 0), "pa_observables")
        return (obs.as_dict(), hist) if with_hist else obs.as_dict()

    def save(self, path: str):
        """Checkpoint (include/pa.h, pa_save)."""
        _check(self.lib.pa_save(self._ctx, os.fsencode(path)), "pa_save")

    @classmethod
    def load(cls, path: str, stream: int | None = None) -> "Population":
        """Resume from a checkpoint written by save()."""
        lib = load_library()
        s = _current_stream() if stream is None else stream
        ctx = ctypes.c_void_p()
        _check(lib.pa_load(os.fsencode(path), ctypes.c_void_p(s), ctypes.byref(ctx)), "pa_load")
        obs = Obs()
        _check(lib.pa_observables(ctx, ctypes.byref(obs), None, 0), "pa_observables")
        # the configuration travels in the file; rebuild the parameters from it
        with open(path, "rb") as f:
            head = f.read(16 + ctypes.sizeof(Config) + 8 + 8)
        cfg = Config.from_buffer_copy(head[16:16 + ctypes.sizeof(Config)])
        step = int.from_bytes(head[16 + ctypes.sizeof(Config):20 + ctypes.sizeof(Config)], "little", signed=True)
        p = PAParams(q=cfg.q, L=cfg.L, R=cfg.R, seed=cfg.seed, R_cap=cfg.R_cap, resample_mode=cfg.resample_mode,
                     init_mode=cfg.init_mode, beta0=cfg.beta0, track_families=bool(cfg.track_families),
                     stream=cfg.stream)
        return cls(p, stream=s, _ctx=ctx, _step=step, _beta=obs.beta)

    def history(self, count: int) -> list:
        """Estimators of the last `count` completed steps, oldest first."""
        recs = (Obs * count)()
        _check(self.lib.pa_observables_history(self._ctx, int(count), ctypes.cast(recs, ctypes.c_void_p)),
               "pa_observables_history")
        return [r.as_dict() for r in recs]

    def size(self) -> int:
        r = ctypes.c_int32()
        _check(self.lib.pa_population_size(self._ctx, ctypes.byref(r)), "pa_population_size")
        return r.value

    def energies(self) -> np.ndarray:
        cap = self.params.R_cap or (self.params.R + self.params.R // 4 + 1024)
        out = np.zeros(cap, dtype=np.int32)
        _check(self.lib.pa_energy(self._ctx, _ptr(out), 0), "pa_energy")
        return out[: self.size()]

    def energies_to_device(self, dev_ptr: int):
        _check(self.lib.pa_energy(self._ctx, ctypes.c_void_p(dev_ptr), 1), "pa_energy")

    def occupations(self) -> np.ndarray:
        """Per-replica occupation of the most common state (Eq. 5)."""
        out = np.zeros(self.size(), dtype=np.int32)
        _check(self.lib.pa_occupations(self._ctx, _ptr(out), 0), "pa_occupations")
        return out

    def spins(self, begin: int = 0, count: int | None = None) -> np.ndarray:
        if count is None:
            count = self.size() - begin
        out = np.zeros((count, self.params.L, self.params.L), dtype=np.uint8)
        _check(self.lib.pa_get_spins(self._ctx, begin, count, _ptr(out)), "pa_get_spins")
        return out

    def ancestors(self) -> np.ndarray:
        out = np.zeros(self.size(), dtype=np.int32)
        _check(self.lib.pa_get_ancestors(self._ctx, _ptr(out)), "pa_get_ancestors")
        return out

    def parents(self, count: int | None = None) -> np.ndarray:
        """Parent map of the latest resampling step (Sec. 2 step 2): entry k is
        the previous-population slot that new slot k copies.  `count` is the
        new size R_i (the current size once the step has been swept)."""
        n = self.size() if count is None else int(count)
        out = np.zeros(n, dtype=np.int32)
        _check(self.lib.pa_get_parents(self._ctx, _ptr(out), 0), "pa_get_parents")
        return out

    def set_launch(self, replicas_per_block: int = 0, threads_per_block: int = 0):
        _check(self.lib.pa_set_launch(self._ctx, replicas_per_block, threads_per_block), "pa_set_launch")

    def launch_shape(self):
        """(replicas per block, threads per block, blocks) of the sweep kernel."""
        v = [ctypes.c_int32() for _ in range(3)]
        _check(self.lib.pa_get_launch(self._ctx, *[ctypes.byref(x) for x in v]), "pa_get_launch")
        return tuple(x.value for x in v)

    def profile(self, enable: bool = True):
        _check(self.lib.pa_profile(self._ctx, int(enable)), "pa_profile")

    def profile_read(self):
        """Returns {"sweep": (ms, launches), "resample": (ms, launches)}."""
        ms = np.zeros(2, dtype=np.float64)
        n = np.zeros(2, dtype=np.int64)
        _check(self.lib.pa_profile_read(self._ctx, _ptr(ms), _ptr(n)), "pa_profile_read")
        return {"sweep": (float(ms[0]), int(n[0])), "resample": (float(ms[1]), int(n[1]))}

    def next_dbeta(self, target: float, dbeta_cap: float, iters: int = 12) -> float:
        """Newton step holding the weight overlap at `target` (see include/pa.h)."""
        d = ctypes.c_double()
        _check(self.lib.pa_next_dbeta(self._ctx, float(target), float(dbeta_cap), int(iters), ctypes.byref(d)),
               "pa_next_dbeta")
        return d.value

    def run_adaptive(self, beta_end: float, theta: int, target: float = 0.85, dbeta_max: float = 0.05,
                     iters: int = 12, max_steps: int = 10000, log=None):
        """PA to beta_end with adaptive steps.  Returns (obs list, betas).
        log: a path or text file that receives one JSON line per step
        (paper_1704_01888_gb300.log)."""
        obs = (Obs * max_steps)()
        betas = np.zeros(max_steps, dtype=np.float64)
        K = ctypes.c_int32()
        beta0 = self.beta
        t0 = time.perf_counter()
        _check(self.lib.pa_run_adaptive(self._ctx, float(beta_end), float(target), float(dbeta_max), int(iters),
                                        int(theta), int(max_steps), ctypes.cast(obs, ctypes.c_void_p), _ptr(betas),
                                        ctypes.byref(K)), "pa_run_adaptive")
        dt = time.perf_counter() - t0
        self.step += K.value
        if K.value:
            self.beta = float(betas[K.value - 1])
        out = [o.as_dict() for o in obs[: K.value]]
        if log is not None and out:
            from . import log as _log

            _log.write_jsonl(log, _log.step_records(out, self.N, beta0, dt / len(out), overlap_target=target))
        return out, betas[: K.value].copy()

    def run(self, betas, theta: int, hist_steps=(), use_graph: bool = False, log=None):
        """Runs betas[1..K] (betas[0] = current beta).  Returns (obs list,
        hists).  log: a path or text file that receives one JSON line per
        step (paper_1704_01888_gb300.log)."""
        betas = np.ascontiguousarray(betas, dtype=np.float64)
        K = betas.size - 1
        obs = (Obs * K)()
        hs = np.ascontiguousarray(hist_steps, dtype=np.int32)
        hist = np.zeros((hs.size, 2 * self.N + 1), dtype=np.int32)
        t0 = time.perf_counter()
        _check(self.lib.pa_run(self._ctx, _ptr(betas), K, int(theta), ctypes.cast(obs, ctypes.c_void_p),
                               _ptr(hs) if hs.size else None, hs.size, _ptr(hist) if hs.size else None,
                               int(use_graph)), "pa_run")
        dt = time.perf_counter() - t0
        self.step += K
        self.beta = float(betas[-1])
        if log is not None and K > 0:
            from . import log as _log

            _log.write_jsonl(log, _log.step_records([o.as_dict() for o in obs], self.N, float(betas[0]), dt / K))
        return [o.as_dict() for o in obs], hist


class Batch:
    """M independent PA runs advanced together (include/pa.h, pa_batch_*).
    `runs` is a list of (PAParams, betas, theta); all runs share one seed and
    should differ in PAParams.stream."""

    def __init__(self, runs, stream: int | None = None, autotune: bool = False):
        self.lib = load_library()
        self.runs = [(p, np.ascontiguousarray(b, dtype=np.float64), int(t)) for p, b, t in runs]
        descs = (RunDesc * len(self.runs))()
        for d, (p, b, t) in zip(descs, self.runs):
            d.cfg = Config(p.q, p.L, p.R, p.R_cap, p.seed, p.resample_mode, p.init_mode, p.beta0,
                           int(p.track_families), int(p.stream))
            d.betas = b.ctypes.data
            d.K = b.size - 1
            d.theta = t
        self._stream = _current_stream() if stream is None else stream
        self._b = ctypes.c_void_p()
        _check(self.lib.pa_batch_create(ctypes.cast(descs, ctypes.c_void_p), len(self.runs),
                                        ctypes.c_void_p(self._stream), ctypes.byref(self._b)), "pa_batch_create")
        self.tuned = None
        if autotune:
            self.tuned = self.autotune()

    def close(self):
        if self._b:
            self.lib.pa_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def autotune(self):
        a, t = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.pa_batch_autotune(self._b, ctypes.byref(a), ctypes.byref(t)), "pa_batch_autotune")
        return a.value, t.value

    def set_launch(self, smem_budget: int, threads: int):
        _check(self.lib.pa_batch_set_launch(self._b, smem_budget, threads), "pa_batch_set_launch")

    def launch_shape(self):
        v = [ctypes.c_int32() for _ in range(3)]
        _check(self.lib.pa_batch_get_launch(self._b, *[ctypes.byref(x) for x in v]), "pa_batch_get_launch")
        return tuple(x.value for x in v)

    def run(self, use_graph: bool = True):
        _check(self.lib.pa_batch_run(self._b, int(use_graph)), "pa_batch_run")

    def observables(self, m: int):
        K = self.runs[m][1].size - 1
        recs = (Obs * (K + 1))()
        _check(self.lib.pa_batch_observables(self._b, m, ctypes.cast(recs, ctypes.c_void_p)), "pa_batch_observables")
        return [r.as_dict() for r in recs]

    def size(self, m: int) -> int:
        r = ctypes.c_int32()
        _check(self.lib.pa_batch_population_size(self._b, m, ctypes.byref(r)), "pa_batch_population_size")
        return r.value

    def status(self, m: int) -> int:
        r = ctypes.c_int32()
        return int(self.lib.pa_batch_population_size(self._b, m, ctypes.byref(r)))

    def spins(self, m: int, begin: int, count: int) -> np.ndarray:
        L = self.runs[m][0].L
        out = np.zeros((count, L, L), dtype=np.uint8)
        _check(self.lib.pa_batch_get_spins(self._b, m, begin, count, _ptr(out)), "pa_batch_get_spins")
        return out

    def measurements(self, m: int):
        """(E, Mt) of run m's current population: energies (Eq. 3) and
        occupations of the most common state (Eq. 5)."""
        n = self.size(m)
        E = np.zeros(n, dtype=np.int32)
        Mt = np.zeros(n, dtype=np.int32)
        _check(self.lib.pa_batch_measurements(self._b, m, _ptr(E), _ptr(Mt)), "pa_batch_measurements")
        return E, Mt
