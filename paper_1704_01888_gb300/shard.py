"""One population-annealing population spread over several GPUs.

Replicas are independent between resampling steps (Sec. 2 of
arXiv:1704.01888); a temperature step couples them only through the
normaliser Q_i (Eq. 2) and the offsets of the copy numbers.  Each rank holds a
contiguous range of global slots; per step it

  1. sums the energy histogram over the ranks (then every rank computes the
     same exact S, ln Q_i and copy numbers of its own replicas),
  2. gathers the ranks' child totals, from which pa_shard_plan places every
     child's new global slot,
  3. sends each rank the runs of its children placed there (a run: the
     consecutive children of one parent, sent as the parent replica and a
     child count) with one all-to-all exchange in new-slot order,
  4. sweeps its new replicas, gathered from the received runs (random numbers
     keyed by global slot), and sums the measurement sums, family counts and
     histogram over the ranks.

The library does the arithmetic (include/pa.h, pa_shard_*); this module only
moves buffers between ranks through a communicator:

  TorchComm   torch.distributed (NCCL between GPUs, one process per GPU);
  ThreadComm  the ranks as threads of one process sharing one GPU (each
              collective meets at a barrier; no kernel waits for another).

The result equals the single-GPU run (pa_init) bit for bit for any number
of ranks.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import Config, Obs, PAParams, ShardBuffers, _check, _current_stream, load_library


class _DeviceArray:
    """A device buffer owned by the library, seen by torch without a copy."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 2}


def _view(ptr, n, dtype):
    import torch

    typestr = {torch.int32: "<i4", torch.int64: "<i8"}[dtype]
    if n == 0:
        return torch.zeros(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda")


class TorchComm:
    """Collectives of a torch.distributed process group (NCCL for GPU tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allreduce_(self, t):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)

    def allgather_int(self, value: int) -> list:
        import torch

        t = torch.tensor([int(value)], dtype=torch.int64, device="cuda")
        out = [torch.zeros_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=self.group)
        return [int(x.item()) for x in out]

    def all_to_all(self, out, inp, out_splits, in_splits):
        self.dist.all_to_all_single(out, inp, [int(x) for x in out_splits], [int(x) for x in in_splits],
                                    group=self.group)

    def all_to_all_counts(self, counts) -> list:
        """counts[d] goes to rank d; returns what each rank sent here."""
        import torch

        t = torch.tensor([int(x) for x in counts], dtype=torch.int64, device="cuda")
        out = torch.empty_like(t)
        self.dist.all_to_all_single(out, t, group=self.group)
        return [int(x) for x in out.tolist()]


class ThreadComm:
    """`world` ranks as threads of one process on one GPU.  All ranks enqueue
    on one CUDA stream; each collective waits at a barrier until every rank
    has enqueued its part, so stream order matches the exchange order.  A rank
    that fails breaks the barrier and the others raise instead of waiting."""

    class Shared:
        def __init__(self, world: int, timeout: float = 600.0):
            self.world = world
            self.barrier = threading.Barrier(world, timeout=timeout)
            self.slots = [None] * world

    def __init__(self, shared: "ThreadComm.Shared", rank: int):
        self.shared = shared
        self.rank = rank
        self.world = shared.world

    def _meet(self, value):
        sh = self.shared
        sh.slots[self.rank] = value
        sh.barrier.wait()
        got = list(sh.slots)
        sh.barrier.wait()
        return got

    def allreduce_(self, t):
        sh = self.shared
        sh.slots[self.rank] = t
        sh.barrier.wait()
        if self.rank == 0:
            total = sh.slots[0].clone()
            for x in sh.slots[1:]:
                total += x
            for x in sh.slots:
                x.copy_(total)
        sh.barrier.wait()

    def allgather_int(self, value: int) -> list:
        return [int(v) for v in self._meet(int(value))]

    def all_to_all_counts(self, counts) -> list:
        got = self._meet([int(x) for x in counts])
        return [row[self.rank] for row in got]

    def all_to_all(self, out, inp, out_splits, in_splits):
        import torch

        sh = self.shared
        sh.slots[self.rank] = (inp, [int(x) for x in in_splits])
        sh.barrier.wait()
        pieces = []
        for src, splits in sh.slots:
            off = sum(splits[: self.rank])
            pieces.append(src[off: off + splits[self.rank]])
        if out.numel():
            out.copy_(torch.cat(pieces))
        sh.barrier.wait()


class ShardedPopulation:
    """This rank's part of one PA population spread over comm.world GPUs."""

    def __init__(self, params: PAParams, comm, stream: int | None = None):
        self.params = params
        self.comm = comm
        self.lib = load_library()
        self._stream = _current_stream() if stream is None else stream
        cfg = Config(params.q, params.L, params.R, params.R_cap, params.seed, params.resample_mode,
                     params.init_mode, params.beta0, int(params.track_families), int(params.stream))
        self._ctx = ctypes.c_void_p()
        _check(self.lib.pa_shard_init(ctypes.byref(cfg), comm.rank, comm.world, ctypes.c_void_p(self._stream),
                                      ctypes.byref(self._ctx)), "pa_shard_init")
        self.N = params.L * params.L
        self.step_index = 0
        self.beta = params.beta0
        self._finish(params.beta0)

    def close(self):
        if self._ctx:
            self.lib.pa_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _buffers(self) -> ShardBuffers:
        b = ShardBuffers()
        _check(self.lib.pa_shard_get_buffers(self._ctx, ctypes.byref(b)), "pa_shard_get_buffers")
        return b

    def _finish(self, beta: float):
        """Sums this step's histogram, measurement sums and family counts over
        the ranks, then the estimators (identical on every rank)."""
        import torch

        b = self._buffers()
        self.comm.allreduce_(_view(b.hist, b.n_bins, torch.int32))
        self.comm.allreduce_(_view(b.sums, 4, torch.int64))
        if self.params.track_families:
            self.comm.allreduce_(_view(b.fam, self.params.R, torch.int32))
        _check(self.lib.pa_shard_finalize(self._ctx, float(beta)), "pa_shard_finalize")

    def step(self, beta: float, theta: int, step: int | None = None):
        """One temperature step to beta (Sec. 2 steps 2-4) on every rank."""
        import torch

        step = self.step_index + 1 if step is None else int(step)
        dbeta = float(beta) - float(self.beta)
        T = ctypes.c_int64()
        _check(self.lib.pa_shard_counts(self._ctx, dbeta, step, ctypes.byref(T)), "pa_shard_counts")
        totals = np.ascontiguousarray(self.comm.allgather_int(T.value), dtype=np.int64)
        send = np.zeros(self.comm.world, dtype=np.int64)
        _check(self.lib.pa_shard_pack(self._ctx, totals.ctypes.data_as(ctypes.c_void_p),
                                      send.ctypes.data_as(ctypes.c_void_p)), "pa_shard_pack")
        recv = np.ascontiguousarray(self.comm.all_to_all_counts(send), dtype=np.int64)
        b = self._buffers()
        RW = int(b.replica_words)
        ns, nr = int(send.sum()), int(recv.sum())
        self.comm.all_to_all(_view(b.recv, nr * RW, torch.int32), _view(b.send, ns * RW, torch.int32), recv * RW,
                             send * RW)
        self.comm.all_to_all(_view(b.recv_cnt, nr, torch.int32), _view(b.send_cnt, ns, torch.int32), recv, send)
        if self.params.track_families:
            self.comm.all_to_all(_view(b.recv_anc, nr, torch.int32), _view(b.send_anc, ns, torch.int32), recv, send)
        _check(self.lib.pa_shard_accept(self._ctx, recv.ctypes.data_as(ctypes.c_void_p)), "pa_shard_accept")
        _check(self.lib.pa_sweep(self._ctx, float(beta), int(theta), step), "pa_sweep")
        self._finish(beta)
        self.step_index = step
        self.beta = float(beta)

    def observables(self, with_hist: bool = False):
        """The step's estimators (the whole population's, on every rank), and
        with_hist the whole population's energy histogram."""
        obs = Obs()
        hist = np.zeros(2 * self.N + 1, dtype=np.int32) if with_hist else None
        _check(self.lib.pa_observables(self._ctx, ctypes.byref(obs),
                                       hist.ctypes.data_as(ctypes.c_void_p) if with_hist else None,
                                       hist.size if with_hist else 0), "pa_observables")
        return (obs.as_dict(), hist) if with_hist else obs.as_dict()

    def profile(self, enable: bool = True):
        _check(self.lib.pa_profile(self._ctx, int(enable)), "pa_profile")

    def profile_read(self):
        """{"sweep": (ms, launches), ...}: event-timed sweep launches on this rank."""
        ms = np.zeros(2, dtype=np.float64)
        n = np.zeros(2, dtype=np.int64)
        _check(self.lib.pa_profile_read(self._ctx, ms.ctypes.data_as(ctypes.c_void_p),
                                        n.ctypes.data_as(ctypes.c_void_p)), "pa_profile_read")
        return {"sweep": (float(ms[0]), int(n[0])), "resample": (float(ms[1]), int(n[1]))}

    def launch_shape(self):
        v = [ctypes.c_int32() for _ in range(3)]
        _check(self.lib.pa_get_launch(self._ctx, *[ctypes.byref(x) for x in v]), "pa_get_launch")
        return tuple(x.value for x in v)

    def history(self, count: int) -> list:
        recs = (Obs * count)()
        _check(self.lib.pa_observables_history(self._ctx, int(count), ctypes.cast(recs, ctypes.c_void_p)),
               "pa_observables_history")
        return [r.as_dict() for r in recs]

    def range(self):
        """(global slot of the first local replica, local count, whole population size)."""
        a, n, R = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.pa_shard_range(self._ctx, ctypes.byref(a), ctypes.byref(n), ctypes.byref(R)),
               "pa_shard_range")
        return a.value, n.value, R.value

    def spins(self) -> np.ndarray:
        _, n, _ = self.range()
        out = np.zeros((n, self.params.L, self.params.L), dtype=np.uint8)
        _check(self.lib.pa_get_spins(self._ctx, 0, n, out.ctypes.data_as(ctypes.c_void_p)), "pa_get_spins")
        return out

    def energies(self) -> np.ndarray:
        _, n, _ = self.range()
        out = np.zeros(max(n, 1), dtype=np.int32)
        _check(self.lib.pa_energy(self._ctx, out.ctypes.data_as(ctypes.c_void_p), 0), "pa_energy")
        return out[:n]

    def ancestors(self) -> np.ndarray:
        _, n, _ = self.range()
        out = np.zeros(max(n, 1), dtype=np.int32)
        _check(self.lib.pa_get_ancestors(self._ctx, out.ctypes.data_as(ctypes.c_void_p)), "pa_get_ancestors")
        return out[:n]
