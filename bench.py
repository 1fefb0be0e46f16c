#!/usr/bin/env python
"""Benchmark: population annealing of the 2D q-state Potts model on GB300.

One benchmark step is one PA temperature step over the whole population
(resampling with the replica gather, theta checkerboard Metropolis sweeps,
measurements), the hot path of Sec. 2 of arXiv:1704.01888.  The workload is
plain PA with q = 10, L = 64, R = 100000, theta = 10, beta from 0 to 1.6 in
200 equal steps; warm-up steps are the first steps of that schedule and the
timed steps follow (past step 200 the same spacing continues).

Prints one JSON line.  --impl reference times the CPU oracle instead (the
only reference this method has), on a bounded sample of the same workload.
Under torchrun the N ranks hold one population of N x R replicas (each GPU
R of them: weak scaling), coupled at every step by a histogram all-reduce and
the exchange of the resampled replicas (paper_1704_01888_gb300.shard);
value = the population's attempts / max over ranks of the timed span.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1704_01888_gb300 import workloads as wl  # noqa: E402

METRIC = "spin-flip attempts/ns & PA steps/s, q=10 L=64 R=1e5; batched vs plain, %roofline"
UNIT = "attempts/ns"
# Algorithmic ALU-pipe operations of the multi-spin-coded Metropolis update, per
# site word (32 same-colour sites, one attempt each) for B = ceil(log2 q) bit
# planes.  The update is integer logic; its binding unit is the ALU pipe (it
# executes every three-input logic operation); the 32 x 32 -> 64 bit products of
# Philox run on the FMA-heavy pipe, which is not binding and is not counted:
#   Philox4x32-10 words: B for the proposal, A for the acceptance, a quarter
#     call each (10 rounds x 2 three-input xors = 20 per call): 5 (B + A);
#     and the counter word of each acceptance call: A / 4;
#   the fourth neighbour (the same-row word shifted by one column): B shifts;
#   proposal s +- (1 + u) mod q: two ripple-carry adders over B and B + 1
#     planes (3 per plane), the choice of result and its select: 7B + 4;
#   dE class: eight B-plane equality tests, a carry-save count of the eight
#     indicator bits (14) and the class bits (3): 8B + 17;
#   acceptance: per plane of v, the choice between the two threshold-bit
#     selections by the class bit dE >= 3 (1; the selections themselves are
#     multiply-adds on the FMA-heavy pipe) and the outcome and undecided
#     updates (2): 3A;  merge of the accepted proposals: the mask of decided
#     acceptances and B selects, B + 1;
#   the step's measurements (Eqs. 3, 5), shared by the 2 theta site-word
#     updates of each word of a replica: four B-plane equality tests per
#     colour-0 word for E (8B - 4 per pair of words) and one B-plane test per
#     word and state for the largest occupation (2 q B per pair):
#     (8B - 4 + 2qB) / (2 theta).
# A = acceptance planes a word needs: a site's comparison of v with T ends at
# its first differing bit, and the word draws whole Philox calls (four planes)
# until its deepest site is decided.  Counted by the oracle on the at-scale
# schedule (oracle/acceptance_planes.py -> profiles/acceptance_planes_q10-L64.txt):
# 5.9 at steps 6-25, 7.5 at beta_t, 6.7 over the whole schedule; 6 where no
# count exists.
ACC_PLANES = 6.0


def ops_per_word(q: int, A: float = ACC_PLANES, theta: int = 10) -> float:
    B = max(1, (q - 1).bit_length())
    return (5 * (B + A) + A / 4 + B + (7 * B + 4) + (8 * B + 17) + 3 * A + B + 1
            + (8 * B - 4 + 2 * q * B) / (2 * theta))


def ops_per_attempt(q: int, A: float = ACC_PLANES, theta: int = 10) -> float:
    return ops_per_word(q, A, theta) / 32.0


def acceptance_planes(w, first: int, last: int):
    """Mean counted acceptance planes per site word over steps first..last
    of the workload's schedule (profiles/acceptance_planes_<case>.txt), or
    (ACC_PLANES, None) where no count exists."""
    path = os.path.join(ROOT, "profiles", f"acceptance_planes_q{w.q}-L{w.L}.txt")
    try:
        vals, schedule = [], None
        for line in open(path):
            if line.startswith("#"):
                m = re.search(r"theta=(\d+), beta 0 -> ([\d.]+) in (\d+) steps", line)
                if m:
                    schedule = (int(m.group(1)), float(m.group(2)), int(m.group(3)))
                continue
            if not line.strip():
                continue
            i, _, a = line.split()[:3]
            if first <= int(i) <= last:
                vals.append(float(a))
        # the count holds for the schedule it was taken on
        if vals and schedule and schedule[0] == w.theta and abs(schedule[1] - w.beta_end) < 1e-9 and schedule[2] == w.K:
            return sum(vals) / len(vals), os.path.relpath(path, ROOT)
    except OSError:
        pass
    return ACC_PLANES, None


def replica_bytes(q: int, L: int) -> int:
    """Device bytes of one replica: 2 colours x site words per colour x P planes
    x 4 bytes, P = ceil(log2 q) rounded up to 1, 2 or 4 when at most 4; a colour has
    L^2 / 64 site words when L/2 divides 32 (rows packed) or when L is a
    multiple of 16 but not of 64 and L > 32 (banded segments), else
    L ceil(L/64)."""
    B = max(1, (q - 1).bit_length())
    P = 1 if B <= 1 else 2 if B <= 2 else 4 if B <= 4 else B
    full = (L >= 8 and 64 % L == 0) or (L > 32 and L % 16 == 0 and L % 64 != 0)
    words = L * L // 64 if full else L * ((L + 63) // 64)
    return (2 * words * P + 3) // 4 * 4 * 4


# ALU pipe: 4 schedulers x 16 lanes per SM and clock (ncu counts its peak as half a
# warp instruction per scheduler and cycle)
LANES_PER_SM_PER_CLK = 64
PA_OBS_BYTES = 112
DEVSTATE_BYTES = 48


def reduce_over_ranks(elapsed, attempts, device):
    """Whole-job figures over the ranks: the slowest rank's time (max) and
    the sum of the ranks' attempts."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    a = torch.tensor([float(attempts)], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return float(t.item()), float(a.item())


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=197)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2",
                    choices=["c1", "c2", "c3", "c5", "widths", "table1", "table2", "table3", "hysteresis"],
                    help="c3 runs the batch of 64 runs alone (its first --steps steps); widths runs the "
                         "histogram-width study (20 runs, one batch); table1-3 the width studies of the "
                         "paper's Tables I-III (--runs runs per row); hysteresis the cooling and heating "
                         "branches of its Figs. 2-3")
    ap.add_argument("--runs", type=int, default=8, help="runs per row of the table1-3 workloads")
    ap.add_argument("--batch-launch", default="", help="smem_budget,threads for the batched sweep kernel (c3)")
    ap.add_argument("--no-graph", action="store_true", help="c3 without graph capture")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--R", type=int, default=0, help="override the population size (profiling runs)")
    ap.add_argument("--launch", default="", help="replicas_per_block,threads_per_block for the sweep kernel")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, adaptive and strong first-order measurements")
    return ap.parse_args()


def _workload(name, R=0):
    w = {"c1": wl.C1, "c2": wl.C2, "c5": wl.C5, "c3": wl.C2}[name]
    return wl.scaled(w, R=R, name=f"{w.name}-R{R}") if R else w


def _betas(w, n):
    """beta_i = beta_end * i / K for i = 0..n (continues past K at the same spacing)."""
    return np.array([w.beta_end * i / w.K for i in range(n + 1)], dtype=np.float64)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _sweep_sources() -> bytes:
    csrc = os.path.join(ROOT, "paper_1704_01888_gb300", "csrc")
    return b"".join(open(os.path.join(csrc, f), "rb").read()
                    for f in ("pa_sweep.cu", "pa_sweep_body.cuh", "pa_internal.cuh"))


def _sweep_record(w):
    """The sweep kernel's ncu record (profiles/sweep_traffic.txt): DRAM bytes
    per replica per launch and the issue activity, valid only for the
    workload's (q, L) it was taken on and while the sweep kernel's sources
    hash to the recorded value."""
    rec = {}
    try:
        for line in open(os.path.join(ROOT, "profiles", "sweep_traffic.txt")):
            if line.startswith("#") or ":" not in line:
                continue
            key, val = line.split(":", 1)
            rec[key.strip()] = val.strip().split()[0]
    except OSError:
        return None
    if rec.get("source_sha256") != hashlib.sha256(_sweep_sources()).hexdigest():
        return None
    if rec.get("case") != f"q{w.q}-L{w.L}":
        return None
    out = {"dram_bytes_per_replica": float(rec["dram_bytes_per_replica"])}
    if "issue_active" in rec:
        out["issue_active"] = float(rec["issue_active"])
    return out


def _cpu_baseline(w, R_sample=1000, steps=3):
    """The oracle as it stands, single-threaded, on R_sample replicas for the
    first `steps` temperature steps of the same workload."""
    import oracle

    oracle.build()
    b = _betas(w, steps)
    t0 = time.perf_counter()
    out = oracle.run(w.q, w.L, R_sample, w.seed, w.theta, b, want_state=False)
    dt = time.perf_counter() - t0
    attempts = int(sum(out["R"][1:]) * w.N * w.theta)
    value = attempts / (dt * 1e9)
    n = os.cpu_count() or 1
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{w.name} with R={R_sample} replicas, init + {steps} steps, single thread, {dt:.1f} s",
            "host_cores": n, "all_cores_ideal": value * n,
            "all_cores_note": "the single-thread rate times the host's cores (replicas sweep independently); "
                              "a projection, not a measurement"}


def run_reference(args):
    """The oracle as the reference arm: a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    w = _workload(args.workload, args.R)
    R_sample = 64 if w.N >= 16384 else 256
    W, K = args.warmup, args.steps
    bw = _betas(w, W)
    ball = _betas(w, W + K)
    t0 = time.perf_counter()
    oracle.run(w.q, w.L, R_sample, w.seed, w.theta, bw, want_state=False)
    t1 = time.perf_counter()
    out = oracle.run(w.q, w.L, R_sample, w.seed, w.theta, ball, want_state=False)
    t2 = time.perf_counter()
    timed = (t2 - t1) - (t1 - t0)
    attempts = int(sum(out["R"][W + 1:]) * w.N * w.theta)
    value = attempts / (timed * 1e9)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": timed * 1e3 / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w.name, "q": w.q, "L": w.L, "R": w.R, "theta": w.theta, "sample_R": R_sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{w.name} with R={R_sample} replicas per step, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


class _PlainSteps:
    """A single-GPU population driven step by step through the C ABI."""

    def __init__(self, pa, params, betas, theta, launch=None):
        self.pop = pa.Population(params)
        if launch:
            self.pop.set_launch(*launch)
        self.betas, self.theta = betas, theta

    def step(self, i):
        self.pop.resample(self.betas[i] - self.betas[i - 1], i)
        self.pop.sweep(self.betas[i], self.theta, i)


class _ShardedSteps:
    """This rank's part of one population spread over the job's GPUs."""

    def __init__(self, pa, params, betas, theta, launch=None):
        from paper_1704_01888_gb300.shard import ShardedPopulation, TorchComm

        self.pop = ShardedPopulation(params, TorchComm())
        self.betas, self.theta = betas, theta

    def step(self, i):
        self.pop.step(self.betas[i], self.theta, i)


def run_ours(args):
    import torch

    import paper_1704_01888_gb300 as pa
    from paper_1704_01888_gb300 import build as pabuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0 or not os.path.exists(pa.LIB_PATH):
        pabuild.build()
    if world > 1:
        torch.distributed.barrier()

    w = _workload(args.workload, args.R)
    W, K = args.warmup, args.steps
    betas = _betas(w, W + K)
    launch = tuple(int(x) for x in args.launch.split(",")) if args.launch else None
    # N GPUs hold one population of N x R replicas (weak scaling: R per GPU)
    R_total = w.R * world
    params = pa.PAParams(q=w.q, L=w.L, R=R_total, seed=w.seed, track_families=w.track_families)
    Steps = _ShardedSteps if world > 1 else _PlainSteps
    stream = torch.cuda.current_stream()

    run = Steps(pa, params, betas, w.theta, launch)
    pop = run.pop
    for i in range(1, W + 1):
        run.step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launch_used = pop.launch_shape()

    pop.profile(True)
    launches0 = pa.kernel_launch_count()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        start.record(stream)
        for i in range(W + 1, W + K + 1):
            run.step(i)
        stop.record(stream)
        stop.synchronize()
    launches = pa.kernel_launch_count() - launches0
    elapsed_ms = start.elapsed_time(stop)
    prof = pop.profile_read()
    hist = pop.history(K)
    # every rank holds the whole population's estimators
    attempts = int(sum(h["R"] for h in hist)) * w.N * w.theta
    final_obs = hist[-1]
    pop.close()

    if world > 1:
        elapsed_ms, _ = reduce_over_ranks(elapsed_ms, 0.0, "cuda")
    value = attempts / (elapsed_ms * 1e6)
    ms_per_step = elapsed_ms / K
    clocks = clk.summary()

    # roofline of the dominant kernel (the fused gather + sweeps + measurement)
    # on this rank: its launches cover this rank's share of the replicas
    sweep_ms, sweep_n = prof["sweep"]
    sweep_avg_s = sweep_ms / sweep_n / 1e3
    per_launch_attempts = attempts / world / sweep_n
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = _peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    A, A_src = acceptance_planes(w, W + 1, min(W + K, w.K))
    opa = ops_per_attempt(w.q, A, w.theta)
    achieved = opa * per_launch_attempts / sweep_avg_s / 1e12
    peak = sms * LANES_PER_SM_PER_CLK * f_max / 1e12
    rec = _sweep_record(w)
    per_launch_replicas = per_launch_attempts / (w.N * w.theta)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": (rec["dram_bytes_per_replica"] * per_launch_replicas) if rec else None,
                "traffic_unit": "bytes per launch (ncu dram read + write, scaled by replicas)",
                "algorithmic_bytes_per_launch": 2 * replica_bytes(w.q, w.L) * per_launch_replicas,
                "kernel": "k_sweep", "ops_per_attempt": opa, "acceptance_planes": A,
                "acceptance_planes_source": A_src or "model value (no count for this workload)",
                "kernel_ms_avg": sweep_avg_s * 1e3, "kernel_share": sweep_ms / elapsed_ms,
                "peak_basis": f"ALU pipe: {sms} SMs x {LANES_PER_SM_PER_CLK} lanes x {f_max / 1e6:.0f} MHz "
                              f"(max SM clock), of measured clock"}
    if rec and "issue_active" in rec:
        roofline["issue_active_ncu"] = rec["issue_active"]
    if clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (sms * LANES_PER_SM_PER_CLK * clocks["sm_mhz"] * 1e6 / 1e12)

    e2e = None
    if not args.no_e2e:
        e2e = _e2e(pa, w, params, betas, W, K, world, launch, Steps)

    cpu = None
    if world == 1 and not args.no_cpu:
        # the oracle on the host cores: one GPU only (a multi-GPU run reports the GPUs alone)
        cpu = _cpu_baseline(w)

    extras = {}
    if world == 1 and not args.no_extras and not args.R:
        # measured after the timed region; one that fails is reported as such
        # and does not take the headline line with it
        def extra(name, fn, *a):
            try:
                extras[name] = fn(*a)
            except Exception as exc:  # noqa: BLE001
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}
            return extras[name]

        extra("batched", _batched, pa)
        cool = extra("observables_c2", _observables_c2, pa)
        if "_lnZ" in cool:
            extra("cooling_heating_crossing", _crossing, pa, cool.pop("_lnZ"))
        extra("strong_first_order", _observables_c5, pa)
        extra("adaptive", _adaptive, pa)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "q": w.q, "L": w.L, "R": R_total, "R_per_gpu": w.R, "theta": w.theta,
                   "beta": f"0 -> {w.beta_end} in {w.K} equal steps (timed steps {W + 1}..{W + K})",
                   "parallelism": ("one population over %d GPUs (histogram all-reduce, run exchange)" % world
                                   if world > 1 else "one population, one GPU"),
                   "l2": f"inputs larger than L2: 2 x {w.R * replica_bytes(w.q, w.L) / 1e6:.0f} MB spin buffers "
                         "per GPU",
                   "launch": {"replicas_per_block": launch_used[0], "threads_per_block": launch_used[1],
                              "blocks": launch_used[2]}},
        "pa_steps_per_s": K / (elapsed_ms / 1e3),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "final": {"beta": final_obs["beta"], "lnZ": final_obs["lnZ"], "meanE_per_site": final_obs["meanE"] / w.N,
                  "R": final_obs["R"], "n_near_ties": final_obs["n_near_ties"]},
    }
    line.update(extras)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def _e2e(pa, w, params, betas, W, K, world, launch, Steps):
    """The same metric through the public API as a user drives it: each step
    resamples, sweeps, and reads the step's estimators (ln Q_i and R_i among
    them) and its energy histogram into host memory: one host round trip per
    step."""
    import torch

    run = Steps(pa, params, betas, w.theta, launch)
    for i in range(1, W + 1):
        run.step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    attempts = 0
    t0 = time.perf_counter()
    for i in range(W + 1, W + K + 1):
        run.step(i)
        obs, hist = run.pop.observables(with_hist=True)
        attempts += obs["R"] * w.N * w.theta
    dt = time.perf_counter() - t0
    run.pop.close()
    if world > 1:
        dt, _ = reduce_over_ranks(dt, 0.0, "cuda")
    d2h = DEVSTATE_BYTES + PA_OBS_BYTES + 4 * (2 * w.N + 1)
    return {"value": attempts / (dt * 1e9), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
            "note": "no per-step host input exists: the population is generated on the device from the seed and "
                    "never leaves it, and a step's only inputs, beta_i and dbeta_i (16 bytes), travel as kernel "
                    "arguments; per step the host reads ln Q_i, R_i, the estimators and the energy histogram"}


def _batched(pa):
    """64 independent runs (q in {5,6,8,10}, L in {16,32,48,64}, R in [1e4, 5e4],
    150 steps, theta = 10): one persistent launch per kernel and a graph per
    temperature step, against the same runs launched one after another."""
    import torch

    ws = wl.batched_runs()
    runs = [(pa.PAParams(q=w.q, L=w.L, R=w.R, seed=w.seed, stream=w.stream), w.betas(), w.theta) for w in ws]
    attempts = sum(w.R * w.N * w.theta * w.K for w in ws)  # expected; exact counts below
    steps = sum(w.K for w in ws)
    b = pa.Batch(runs)
    tuned = b.autotune()
    launches0 = pa.kernel_launch_count()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(use_graph=True)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    launches_batch = pa.kernel_launch_count() - launches0
    exact = sum(sum(o["R"] for o in b.observables(m)[1:]) * ws[m].N * ws[m].theta for m in range(len(ws)))
    last_b = [b.observables(m)[-1]["sumE"] for m in range(len(ws))]
    b.close()
    t_plain, last_p = 0.0, []
    for p, betas, theta in runs:
        with pa.Population(p) as pop:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            obs, _ = pop.run(betas, theta)
            torch.cuda.synchronize()
            t_plain += time.perf_counter() - t0
            last_p.append(obs[-1]["sumE"])
    return {"workload": "batch of 64 runs, q 5-10, L 16-64, R 1e4-5e4, 150 steps, theta 10",
            "pa_steps_per_s": steps / t_batch, "attempts_per_ns": exact / t_batch / 1e9,
            "plain_pa_steps_per_s": steps / t_plain, "plain_attempts_per_ns": exact / t_plain / 1e9,
            "speedup_vs_plain": t_plain / t_batch, "graph": True, "launches": launches_batch,
            "autotuned": {"smem_budget": tuned[0], "threads": tuned[1]},
            "identical_to_plain": last_b == last_p, "expected_attempts": attempts}


def _hist_report(hist, N, width=4):
    """Energy histogram per site in bins of `width` units: its occupied range,
    counts, modes (analysis.modes) and whether it has two."""
    from paper_1704_01888_gb300 import analysis

    centres, counts = analysis.rebin_energy_histogram(hist, N, width)
    nz = np.flatnonzero(counts)
    lo, hi = int(nz[0]), int(nz[-1]) + 1
    md = analysis.modes(counts)
    return {"bin_width": width, "e_first_bin": float(centres[lo]), "counts": [int(x) for x in counts[lo:hi]],
            "modes_e": [round(float(centres[k]), 5) for k in md], "two_peaks": len(md) >= 2,
            "fwhm_e": round(analysis.fwhm(centres[lo:hi], counts[lo:hi]), 6)}


def _observables_c2(pa):
    """Plain PA at scale (q = 10, L = 64, R = 1e5), all 200 steps as one
    graph: the energy histogram in bins of 4 at the grid point nearest
    beta_t (step 178) and ln Z per site along the cooling branch.  Whether
    the histogram has two peaks is recorded, not required: cooling at
    theta = 10 stays in one phase at beta_t (Sec. 4)."""
    import torch

    w = wl.C2
    b = w.betas()
    s = w.hist_steps[0]
    with pa.Population(pa.PAParams(q=w.q, L=w.L, R=w.R, seed=w.seed)) as pop:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        obs, hists = pop.run(b, w.theta, hist_steps=(s,), use_graph=True)
        dt = time.perf_counter() - t0
    att = sum(o["R"] for o in obs) * w.N * w.theta
    out = {"workload": f"{w.name}, {w.K} steps, one graph", "seconds": dt, "attempts_per_ns": att / dt / 1e9,
           "pa_steps_per_s": w.K / dt, "hist_step": s, "hist_beta": float(b[s]), "beta_t": wl.beta_t(w.q),
           "hist": _hist_report(hists[0], w.N), "lnZ_per_site_final": obs[-1]["lnZ"] / w.N,
           "near_ties_total": int(sum(o["n_near_ties"] for o in obs))}
    out["_lnZ"] = (b[1:], np.array([o["lnZ"] for o in obs]))
    return out


def _crossing(pa, cooling):
    """Cooling and heating branches of ln Z (Sec. 5-6, Eqs. 6-8): the heating
    run starts from ground states at beta = 4 with ln Z = ln q + 2 N beta and
    steps down on the cooling run's grid (0.008); the beta where the two
    branches of -beta F cross locates the transition, against
    beta_t = ln(1 + sqrt q)."""
    from paper_1704_01888_gb300 import analysis

    w = wl.C2
    b_cool, lnZ_cool = cooling
    n = 500
    b_heat = np.array([4.0 * (n - k) / n for k in range(n + 1)])
    with pa.Population(pa.PAParams(q=w.q, L=w.L, R=w.R, seed=w.seed + 1, init_mode=pa.INIT_GROUND,
                                   beta0=4.0)) as pop:
        obs, _ = pop.run(b_heat, w.theta, use_graph=True)
    lnZ_heat = {round(float(o["beta"]) / 0.008): o["lnZ"] for o in obs}
    idx = [k for k in range(1, b_cool.size + 1) if k in lnZ_heat]
    beta = np.array([b_cool[k - 1] for k in idx])
    fc = np.array([lnZ_cool[k - 1] for k in idx]) / w.N
    fh = np.array([lnZ_heat[k] for k in idx]) / w.N
    # the crossing between separated branches (where both populations are in
    # one phase the branches coincide up to noise)
    cs = analysis.crossings(beta, fc, fh)
    x = max(cs, key=lambda c: c[1])[0] if cs else None
    bt = wl.beta_t(w.q)
    return {"workload": f"q={w.q} L={w.L} R={w.R} theta={w.theta}: cooling 0 -> 1.6 and heating 4 -> 0 "
                        "(ground-state start), steps of 0.008",
            "beta_cross": x, "beta_t": bt, "relative_deviation": (x - bt) / bt if x is not None else None,
            "lnZ_per_site_at_1.6": {"cooling": float(fc[-1]), "heating": float(fh[-1])},
            "heating_lnZ_per_site_at_0": obs[-1]["lnZ"] / w.N, "ln_q": float(np.log(w.q))}


def _observables_c5(pa):
    """Strong first order (q = 20, L = 256, R = 1e5, theta = 20), all 300
    steps with families: S_f at every step, the energy histograms (bins of 4)
    at steps 268 and 269 around beta_t = 1.6997, and the sweep kernel's
    event-timed rate."""
    import torch

    w = wl.C5
    b = w.betas()
    with pa.Population(pa.PAParams(q=w.q, L=w.L, R=w.R, seed=w.seed, track_families=True)) as pop:
        pop.profile(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        obs, hists = pop.run(b, w.theta, hist_steps=w.hist_steps)
        dt = time.perf_counter() - t0
        prof = pop.profile_read()
        shape = pop.launch_shape()
    att = sum(o["R"] for o in obs) * w.N * w.theta
    return {"workload": f"{w.name}, {w.K} steps, families", "seconds": dt, "attempts_per_ns": att / dt / 1e9,
            "sweep_kernel_attempts_per_ns": att / prof["sweep"][0] / 1e6, "launch": list(shape),
            "S_f": [round(o["S_f"], 6) for o in obs], "n_families_final": obs[-1]["n_families"],
            "hists": {str(s): dict(beta=float(b[s]), **_hist_report(hists[k], w.N))
                      for k, s in enumerate(w.hist_steps)},
            "beta_t": wl.beta_t(w.q), "near_ties_total": int(sum(o["n_near_ties"] for o in obs))}


def _adaptive(pa, R=200000):
    """q = 8, L = 128, R = 2e5, theta = 10, beta 0 -> 1.1 beta_t: free-energy
    accuracy of the adaptive schedule (Newton on the weight overlap, target
    0.85) against constant steps.  Reference: a heating run from ground
    states at beta = 3 (ln Z = ln q + 2 N beta, Eqs. 7-8) down to beta_end,
    where the ordered phase is the stable one; floor: ln Z / N >= 2 beta_end +
    ln q / N (the q ground states alone).  bias = ln Z / N - reference."""
    import torch

    w = wl.C4
    N, be = w.N, w.beta_end
    bh = np.linspace(3.0, be, 301)
    with pa.Population(pa.PAParams(q=w.q, L=w.L, R=R, seed=11, init_mode=pa.INIT_GROUND, beta0=3.0)) as pop:
        obs, _ = pop.run(bh, w.theta, use_graph=True)
    ref = obs[-1]["lnZ"] / N
    out = {"workload": f"q={w.q} L={w.L} R={R} theta={w.theta}, beta 0 -> {be:.5f}, overlap 0.85",
           "reference_lnZ_per_site": ref, "reference": "heating from ground states at beta 3 in 300 steps",
           "floor_lnZ_per_site": 2 * be + np.log(w.q) / N}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    with pa.Population(pa.PAParams(q=w.q, L=w.L, R=R, seed=1)) as pop:
        (obs, betas), dt = timed(lambda: pop.run_adaptive(be, w.theta, target=0.85, dbeta_max=0.05))
    K = len(betas)
    out["adaptive"] = {"steps": K, "lnZ_per_site": obs[-1]["lnZ"] / N, "bias": obs[-1]["lnZ"] / N - ref,
                       "pa_steps_per_s": K / dt, "seconds": dt}
    const = []
    for name, Kc in (("constant", K), ("constant_2x", 2 * K), ("constant_3x", 3 * K)):
        bc = np.array([be * i / Kc for i in range(Kc + 1)])
        with pa.Population(pa.PAParams(q=w.q, L=w.L, R=R, seed=1)) as pop:
            (res, _), dt = timed(lambda: pop.run(bc, w.theta))
        out[name] = {"steps": Kc, "lnZ_per_site": res[-1]["lnZ"] / N, "bias": res[-1]["lnZ"] / N - ref,
                     "pa_steps_per_s": Kc / dt, "seconds": dt}
        const.append(out[name])
    a, c = abs(out["adaptive"]["bias"]), abs(out["constant"]["bias"])
    out["adaptive_more_accurate_at_equal_steps"] = bool(a < c)
    # constant steps at the adaptive schedule's accuracy: |bias| interpolated
    # linearly in the step count between the constant runs that bracket it
    for lo, hi in zip(const, const[1:]):
        blo, bhi = abs(lo["bias"]), abs(hi["bias"])
        if bhi <= a <= blo and blo > bhi:
            Ke = lo["steps"] + (blo - a) / (blo - bhi) * (hi["steps"] - lo["steps"])
            out["constant_steps_at_equal_accuracy"] = Ke
            out["time_ratio_at_equal_accuracy"] = (Ke / hi["pa_steps_per_s"]) / out["adaptive"]["seconds"]
            break
    return out


def run_batch_only(args):
    """The batched configuration on its own: the first --steps temperature
    steps of all 64 runs, one JSON line (PA steps/s and attempts/ns)."""
    import torch

    import paper_1704_01888_gb300 as pa
    from paper_1704_01888_gb300 import build as pabuild

    torch.cuda.set_device(0)
    pabuild.build()
    ws = wl.batched_runs()
    K = max(1, min(args.steps, 150))
    runs = [(pa.PAParams(q=w.q, L=w.L, R=w.R, seed=w.seed, stream=w.stream), w.betas()[:K + 1], w.theta) for w in ws]
    b = pa.Batch(runs)
    if args.batch_launch:
        b.set_launch(*[int(x) for x in args.batch_launch.split(",")])
    else:
        b.autotune()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(use_graph=not args.no_graph)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    att = sum(sum(o["R"] for o in b.observables(m)[1:]) * ws[m].N * ws[m].theta for m in range(len(ws)))
    shape = b.launch_shape()
    b.close()
    print(json.dumps({"metric": METRIC, "value": att / dt / 1e9, "unit": UNIT, "n_gpus": 1, "steps": K,
                      "pa_steps_per_s": len(ws) * K / dt, "config": {"workload": "batch of 64 runs", "launch": shape,
                                                                     "graph": not args.no_graph}}))
    return 0


def run_width_study(args):
    """Histogram widths in the style of the paper's Table I: q in {6, 8, 10,
    20} x L in {16, ..., 256}, R = 1000, theta = 100, 100 steps to beta_t(q),
    all 20 runs as one batch; FWHM of the energy-per-site and magnetisation
    histograms of each final population.  One JSON line."""
    import torch

    import paper_1704_01888_gb300 as pa
    from paper_1704_01888_gb300 import analysis
    from paper_1704_01888_gb300 import build as pabuild

    torch.cuda.set_device(0)
    pabuild.build()
    ws = wl.width_study_runs()
    runs = [(pa.PAParams(q=w.q, L=w.L, R=w.R, seed=w.seed, stream=w.stream), w.betas(), w.theta) for w in ws]
    b = pa.Batch(runs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(use_graph=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    att = sum(sum(o["R"] for o in b.observables(m)[1:]) * ws[m].N * ws[m].theta for m in range(len(ws)))
    table = []
    for m, w in enumerate(ws):
        E, Mt = b.measurements(m)
        we, wm = analysis.widths(w.q, w.L, E, Mt)
        table.append({"q": w.q, "L": w.L, "omega_e": round(we, 5), "omega_m": round(wm, 5),
                      "meanE_per_site": round(float(E.mean()) / w.N, 5)})
    shape = b.launch_shape()
    b.close()
    print(json.dumps({"metric": "histogram widths (FWHM) at beta_t; PA steps/s", "value": len(ws) * ws[0].K / dt,
                      "unit": "PA steps/s", "n_gpus": 1, "attempts_per_ns": att / dt / 1e9, "seconds": dt,
                      "config": {"workload": "width study: q 6, 8, 10, 20 x L 16-256, R=1000, theta=100, "
                                             "100 steps to beta_t(q), one batch", "launch": shape},
                      "widths": table}))
    return 0


def _width_row(pa, analysis, q, L, theta, n_beta, n, R=1000):
    """One row of the paper's width tables: n runs (streams 0..n-1) of q, L,
    R replicas, theta sweeps, the Table I schedule with fine steps 1/n_beta;
    after every step the FWHM of the energy and magnetisation histograms
    (outermost crossings and main peak), averaged over the runs and maximised
    over the schedule; T_max = 1 / beta there."""
    b = wl.table1_betas(q, n_beta)
    # [run, step, (e, m), (outermost crossings, main peak)]
    w = np.zeros((n, b.size, 2, 2))
    attempts = 0
    for r in range(n):
        with pa.Population(pa.PAParams(q=q, L=L, R=R, seed=1, stream=r)) as pop:
            for i in range(1, b.size):
                pop.resample(b[i] - b[i - 1], i)
                pop.sweep(b[i], theta, i)
                E, Mt = pop.energies(), pop.occupations()
                w[r, i, :, 0] = analysis.ranged_widths(q, L, E, Mt)
                w[r, i, :, 1] = analysis.ranged_widths(q, L, E, Mt, main_peak=True)
                attempts += E.size * L * L * theta
    mean = w.mean(axis=0)
    row = {"q": q, "L": L, "theta": theta, "N_beta": n_beta}
    for k, sfx in enumerate(("", "_main_peak")):
        ie, im = int(np.argmax(mean[1:, 0, k])) + 1, int(np.argmax(mean[1:, 1, k])) + 1
        row.update({"omega_e_max" + sfx: round(float(mean[ie, 0, k]), 4), "T_e" + sfx: round(1.0 / b[ie], 4),
                    "omega_m_max" + sfx: round(float(mean[im, 1, k]), 4), "T_m" + sfx: round(1.0 / b[im], 4)})
    row["omega_e_max_sd_runs"] = round(float(w[:, :, 0, 0].max(axis=1).std()), 4)
    return row, attempts, n * (b.size - 1)


def run_width_tables(args):
    """The width studies of the paper's Tables I-III (Sec. 4): table1, q in
    {6, 8, 10, 20} and the table's L values at theta = 100, N_beta = 1000;
    table2, q = 8, L = 64 against theta; table3, q = 8, L = 64 against
    N_beta.  R = 1000, the table caption's piecewise schedule, --runs runs per
    row (the paper: 200).  One JSON line, the paper's values beside each row."""
    import torch

    import paper_1704_01888_gb300 as pa
    from paper_1704_01888_gb300 import analysis
    from paper_1704_01888_gb300 import build as pabuild

    torch.cuda.set_device(0)
    pabuild.build()
    n = max(1, args.runs)
    if args.workload == "table1":
        specs = [((q, L, 100, 1000), wl.TABLE_I[(q, L)]) for q, L in sorted(wl.TABLE_I)]
    elif args.workload == "table2":
        specs = [((8, 64, th, 1000), wl.TABLE_II[th]) for th in sorted(wl.TABLE_II)]
    else:
        specs = [((8, 64, 100, nb), wl.TABLE_III[nb]) for nb in sorted(wl.TABLE_III)]
    rows, attempts, steps = [], 0, 0
    t0 = time.perf_counter()
    for (q, L, theta, n_beta), (pe, te, pm, tm) in specs:
        row, att, st = _width_row(pa, analysis, q, L, theta, n_beta, n)
        row["paper"] = {"omega_e_max": pe, "T_e": te, "omega_m_max": pm, "T_m": tm}
        rows.append(row)
        attempts += att
        steps += st
    dt = time.perf_counter() - t0
    print(json.dumps({"metric": "histogram widths (FWHM) at their maxima over the schedule; PA steps/s",
                      "value": steps / dt, "unit": "PA steps/s", "n_gpus": 1, "attempts_per_ns": attempts / dt / 1e9,
                      "seconds": dt,
                      "config": {"workload": f"{args.workload} of the paper (Sec. 4), R=1000, {n} runs per row, one "
                                             "population at a time, host reads E and Mt after every step"},
                      "widths": rows}))
    return 0


def run_hysteresis(args):
    """The protocol of the paper's Figs. 1-3 (Secs. 4-6): q = 3, 6, 10,
    L = 32, R = 10000, theta = 10, steps of 0.01 between beta = 0 and 3;
    cooling from random states at beta = 0 (ln Z_0 = N ln q) and heating from
    ground states at beta = 3 (ln Z = ln q + 2 N beta, Eqs. 7-8).  Per q: the
    area between the cooling and heating energy curves (hysteresis), the
    same with resampling off (q = 10), and the beta where the ln Z branches
    cross against beta_t = ln(1 + sqrt q); for q = 6 the cooling run's energy
    histograms at beta = 0.8, 1.24 and 1.4 (FWHM, number of modes).  One JSON
    line."""
    import torch

    import paper_1704_01888_gb300 as pa
    from paper_1704_01888_gb300 import analysis
    from paper_1704_01888_gb300 import build as pabuild

    torch.cuda.set_device(0)
    pabuild.build()
    L, R, theta, n = 32, 10000, 10, 300
    N = L * L
    up = np.array([k / 100.0 for k in range(n + 1)])
    down = up[::-1].copy()
    t0 = time.perf_counter()

    fig1 = {}

    def branches(q, mode):
        with pa.Population(pa.PAParams(q=q, L=L, R=R, seed=1, resample_mode=mode)) as pop:
            c0 = pop.observables()
            # Fig. 1 (left): the q = 6 cooling run's energy histograms at beta 0.8, 1.24 (beta_t), 1.4
            steps = (80, 124, 140) if q == 6 and mode == pa.RESAMPLE_NEAREST_INT else ()
            cool, hists = pop.run(up, theta, hist_steps=steps, use_graph=True)
            for k, st in enumerate(steps):
                x, h = analysis.rebin_energy_histogram(hists[k], N, 4)
                fig1[f"{up[st]:.2f}"] = {"fwhm": analysis.fwhm(x, h), "modes": len(analysis.modes(h)),
                                         "mean_e": float(cool[st - 1]["meanE"]) / N}
        with pa.Population(pa.PAParams(q=q, L=L, R=R, seed=2, resample_mode=mode, init_mode=pa.INIT_GROUND,
                                       beta0=3.0)) as pop:
            h0 = pop.observables()
            heat, _ = pop.run(down, theta, use_graph=True)
        cool, heat = [c0] + cool, ([h0] + heat)[::-1]  # both on up's grid
        e_c = np.array([o["meanE"] for o in cool]) / N
        e_h = np.array([o["meanE"] for o in heat]) / N
        f_c = np.array([o["lnZ"] for o in cool]) / N
        f_h = np.array([o["lnZ"] for o in heat]) / N
        return e_c, e_h, f_c, f_h

    rows = []
    for q in (3, 6, 10):
        e_c, e_h, f_c, f_h = branches(q, pa.RESAMPLE_NEAREST_INT)
        cs = analysis.crossings(up, f_c, f_h)
        x = max(cs, key=lambda c: c[1]) if cs else None
        row = {"q": q, "beta_t": wl.beta_t(q), "hysteresis_area": float(np.abs(e_c - e_h).sum() * 0.01),
               "max_energy_gap": float(np.abs(e_c - e_h).max()),
               "max_lnZ_gap_per_site": float(np.abs(f_c - f_h).max()),
               "beta_cross": x[0] if x else None, "cross_score": x[1] if x else None}
        if q == 10:
            e_c0, e_h0, _, _ = branches(q, pa.RESAMPLE_OFF)
            row["hysteresis_area_resampling_off"] = float(np.abs(e_c0 - e_h0).sum() * 0.01)
            row["max_energy_gap_resampling_off"] = float(np.abs(e_c0 - e_h0).max())
        if q == 6:
            row["energy_histograms"] = fig1
        rows.append(row)
    dt = time.perf_counter() - t0
    print(json.dumps({"metric": "hysteresis and free-energy branches (Figs. 2-3 protocol)", "value": dt,
                      "unit": "s", "n_gpus": 1, "higher_is_better": False,
                      "config": {"workload": f"q 3, 6, 10, L={L}, R={R}, theta={theta}, beta 0 <-> 3 in steps of 0.01, "
                                             "cooling from beta 0, heating from ground states at beta 3"},
                      "branches": rows}))
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c3":
        return run_batch_only(args)
    if args.workload == "widths":
        return run_width_study(args)
    if args.workload in ("table1", "table2", "table3"):
        return run_width_tables(args)
    if args.workload == "hysteresis":
        return run_hysteresis(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
