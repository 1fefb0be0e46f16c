"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
the same seeded inputs.

Bar: spins, energies, largest-state occupations, histograms, population sizes,
near-tie counts and family ids bit-exact; <E>, <E^2>, C and <M> bit-exact
(they come from exact integer sums through the same IEEE operations); ln Q and ln Z within
1e-10 relative (the device evaluates exp/log with CUDA's libm, the oracle
with the C library's); family entropy within 1e-12 relative.
"""
import math
import multiprocessing as mp

import numpy as np
import pytest

import oracle
import paper_1704_01888_gb300 as pa
from paper_1704_01888_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

LNZ_RTOL = 1e-10
SF_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_01888_gb300 import build

    build.build()
    oracle.build()


def _gpu_run(q, L, R, seed, theta, betas, mode=pa.RESAMPLE_NEAREST_INT, init=pa.INIT_RANDOM, fam=False,
             R_cap=0, launch=None, graph=False, stepwise=False, hist_steps=()):
    p = pa.PAParams(q=q, L=L, R=R, seed=seed, R_cap=R_cap, resample_mode=mode, init_mode=init,
                    beta0=float(betas[0]), track_families=fam)
    with pa.Population(p) as pop:
        if launch:
            pop.set_launch(*launch)
        obs0 = pop.observables()
        hists = {}
        if stepwise:
            obs = []
            for i in range(1, len(betas)):
                pop.resample(betas[i] - betas[i - 1], i)
                pop.sweep(betas[i], theta, i)
                o, h = pop.observables(with_hist=True)
                obs.append(o)
                hists[i] = h
        else:
            obs, hs = pop.run(betas, theta, hist_steps=hist_steps, use_graph=graph)
            hists = {s: hs[k] for k, s in enumerate(hist_steps)}
        out = {"obs": [obs0] + list(obs), "spins": pop.spins(), "E": pop.energies(), "hists": hists,
               "Mt": pop.occupations(), "q": q}
        _, out["hist_final"] = pop.observables(with_hist=True)
        if fam:
            out["anc"] = pop.ancestors()
    return out


def _oracle_run(q, L, R, seed, theta, betas, mode=0, init=0, R_cap=None):
    return oracle.run(q, L, R, seed, theta, betas, mode=mode, init_mode=init, R_cap=R_cap, want_hist=True)


def _compare(g, o, fam=False, check_hists=True):
    K = len(g["obs"]) - 1
    for i in range(K + 1):
        go = g["obs"][i]
        assert go["R"] == o["R"][i], ("R", i)
        for key in ("sumE", "sumE2", "sumMt"):
            assert go[key] == o[key][i], (key, i)
        for key in ("meanE", "meanE2", "C", "meanM", "beta"):
            assert go[key] == o[key][i], (key, i, go[key], o[key][i])
        assert go["lnZ"] == pytest.approx(o["lnZ"][i], rel=LNZ_RTOL, abs=1e-12), ("lnZ", i)
        if i > 0:
            assert go["lnQ"] == pytest.approx(o["lnQ"][i], rel=LNZ_RTOL, abs=1e-12), ("lnQ", i)
        assert go["n_near_ties"] == o["n_near_ties"][i], ("n_near_ties", i)
        if fam:
            assert go["n_families"] == o["n_families"][i], ("n_families", i)
            assert go["S_f"] == pytest.approx(o["S_f"][i], rel=SF_RTOL, abs=1e-14), ("S_f", i)
    Rf = o["R_final"]
    assert g["spins"].shape[0] == Rf
    assert np.array_equal(g["spins"], o["spins"])
    assert np.array_equal(g["E"], o["E"])
    # occupations of the most common state (Eq. 5) against the oracle's count on its own spins
    assert np.array_equal(g["Mt"], [oracle.max_count(g["q"], s) for s in o["spins"]])
    assert np.array_equal(g["hist_final"], o["hist"][K])
    if check_hists:
        for s, h in g["hists"].items():
            assert np.array_equal(h, o["hist"][s]), ("hist", s)
    if fam:
        assert np.array_equal(g["anc"], o["anc"])


# ---------------------------------------------------------------------------
# Plain PA, q = 10, L = 16, R = 1000, 100 steps, theta = 10: the whole run.
# ---------------------------------------------------------------------------
def test_plain_small_full_run_bit_exact():
    w = wl.C1
    b = w.betas()
    g = _gpu_run(w.q, w.L, w.R, w.seed, w.theta, b, hist_steps=(1, 50, 100))
    o = _oracle_run(w.q, w.L, w.R, w.seed, w.theta, b)
    _compare(g, o)


def test_step_api_graph_and_launch_shapes_agree():
    """The step-by-step calls, the enqueued run, the graph-captured run and
    other block shapes all give the same bits (reduced K)."""
    w = wl.C1
    b = w.betas()[:21]
    ref = _gpu_run(w.q, w.L, w.R, w.seed, w.theta, b)
    for kw in (dict(stepwise=True), dict(graph=True), dict(launch=(7, 64)), dict(launch=(40, 256)),
               dict(launch=(1, 32), graph=True)):
        g = _gpu_run(w.q, w.L, w.R, w.seed, w.theta, b, **kw)
        assert np.array_equal(g["spins"], ref["spins"]), kw
        assert [x["lnZ"] for x in g["obs"]] == [x["lnZ"] for x in ref["obs"]], kw
        assert [x["sumE"] for x in g["obs"]] == [x["sumE"] for x in ref["obs"]], kw


def test_run_writes_one_log_line_per_step(tmp_path):
    """pa_run through Population.run(log=...): one JSON line per temperature
    step carrying that step's observables."""
    import json

    w = wl.C1
    b = w.betas()[:11]
    path = tmp_path / "steps.jsonl"
    with pa.Population(pa.PAParams(q=w.q, L=w.L, R=w.R, seed=w.seed)) as pop:
        obs, _ = pop.run(b, w.theta, log=str(path))
    recs = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(recs) == 10
    assert [r["lnZ"] for r in recs] == [o["lnZ"] for o in obs] and [r["R"] for r in recs] == [o["R"] for o in obs]
    assert recs[0]["dbeta"] == pytest.approx(b[1]) and recs[-1]["e"] == pytest.approx(obs[-1]["meanE"] / w.N)


@pytest.mark.parametrize("q,L,R,other", [(8, 128, 3000, (8, 512)), (20, 256, 2500, (2, 512)), (3, 256, 2500, (1, 256))])
def test_large_lattice_launch_shapes_agree(q, L, R, other):
    """At L = 128 and 256 the automatic shape is one 1024-thread block per SM
    holding whole passes of lattices (measurements split over its warps when
    it holds few); it gives the bits of 512- and 256-thread blocks, and the
    first steps match the oracle."""
    betas = np.array([0.0, 0.3, 0.9, 1.3, 1.6, 1.9])[: 4 if L == 256 else 6]
    B = max(1, (q - 1).bit_length())
    words = L * ((L + 63) // 64)  # site words per colour (L a multiple of 64)
    lattice = 2 * words * (B if B > 4 else 4 if B > 2 else B) * 4
    with pa.Population(pa.PAParams(q=q, L=L, R=R, seed=3)) as pop:
        rpb, threads, _ = pop.launch_shape()
    assert threads == 1024 and rpb * lattice <= 204800 < (rpb + 1024 // words) * lattice
    assert (rpb * words) % 1024 == 0  # whole passes of the block's threads
    ref = _gpu_run(q, L, R, 3, 3, betas)
    g = _gpu_run(q, L, R, 3, 3, betas, launch=other)
    assert np.array_equal(g["spins"], ref["spins"]) and np.array_equal(g["Mt"], ref["Mt"])
    assert [x["lnZ"] for x in g["obs"]] == [x["lnZ"] for x in ref["obs"]]
    if L == 128:
        _compare(_gpu_run(q, L, R, 3, 3, betas[:3]), _oracle_run(q, L, R, 3, 3, betas[:3]))


# ---------------------------------------------------------------------------
# Edge cases: every row geometry of the multi-spin-coded kernel (L = 64; rows
# of whole words; rows packed several to a word at L = 8, 16, 32; four bands
# of 8-column segments at L = 48, 80, 96, 112; rows padded to whole words, one
# or several words per row),
# bit-plane counts B = 1..7 (q = 2 .. 128), R = 1, theta = 0, rounding modes.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("q,L,R,theta,K,extra", [
    (3, 2, 64, 3, 8, {}),               # smallest lattice: 1 column per row and colour
    (5, 4, 200, 4, 10, {}),             # q - 1 = 4: uniform proposal, B = 3
    (10, 6, 150, 2, 10, {}),
    (10, 8, 300, 3, 10, {}),            # packed rows: the whole colour in one word
    (2, 8, 100, 3, 6, {}),              # q = 2 at L = 8: a replica of 2 words, padded to 4
    (10, 32, 200, 3, 6, {}),            # packed rows: two rows per word
    (2, 16, 257, 5, 12, {}),            # Ising-like q = 2 (B = 1), ragged R
    (128, 16, 100, 2, 6, {}),           # largest q (B = 7)
    (40, 16, 120, 2, 6, {}),            # B = 6
    (10, 24, 90, 2, 6, {}),             # 12 columns in a 32-bit word
    (10, 48, 150, 3, 6, {}),            # banded rows: 3 segments of 8 columns, bands of 12 rows
    (2, 48, 120, 3, 6, {}),             # banded rows, q = 2 (one plane)
    (20, 80, 30, 2, 4, {}),             # banded rows: 5 segments, B = 5
    (3, 112, 12, 2, 3, {}),             # banded rows: 7 segments, B = 2
    (9, 64, 200, 3, 6, {}),             # one full word per row; q - 1 = 8 uniform
    (10, 128, 30, 2, 4, {}),            # rows of two full words
    (20, 66, 40, 2, 4, {}),             # 33 columns: a full word and one column (B = 5)
    (17, 96, 30, 2, 4, {}),             # banded rows: 6 segments; q - 1 = 16 uniform
    (2, 130, 8, 2, 3, {}),              # 65 columns: three words per row, q = 2
    (10, 16, 1, 3, 10, {}),             # one replica
    (6, 16, 500, 0, 8, {}),             # resampling only
    (8, 16, 400, 3, 10, {"mode": pa.RESAMPLE_ROUND}),
    (8, 16, 400, 3, 10, {"mode": pa.RESAMPLE_POISSON}),  # the paper's Eq. 1
    (10, 16, 300, 2, 8, {"mode": pa.RESAMPLE_OFF}),
])
def test_edge_cases_bit_exact(q, L, R, theta, K, extra):
    b = np.array([1.5 * i / K for i in range(K + 1)])
    g = _gpu_run(q, L, R, 11, theta, b, **extra)
    o = _oracle_run(q, L, R, 11, theta, b, **extra)
    _compare(g, o)


@pytest.mark.parametrize("q,L,R,betas", [
    (3, 40, 200, [0.0, 0.467, 0.933, 1.4]),   # steps large enough that exp overflows off E_ref
    (2, 64, 150, [0.0, 0.7, 1.4]),
    (4, 16, 300, [2.5, 1.2, 0.0]),           # heating with large negative steps
    (5, 16, 100, [0.0, 1.0, 2.0]),           # Poisson with means far above 64
])
def test_large_temperature_steps(q, L, R, betas):
    b = np.array(betas)
    init = pa.INIT_GROUND if b[0] > 0 else pa.INIT_RANDOM
    mode = pa.RESAMPLE_POISSON if q == 5 else pa.RESAMPLE_NEAREST_INT
    g = _gpu_run(q, L, R, 21, 2, b, init=init, mode=mode)
    o = _oracle_run(q, L, R, 21, 2, b, init=1 if init == pa.INIT_GROUND else 0, mode=mode)
    _compare(g, o)


def test_heating_from_ground_state_with_families():
    q, L, R, K = 6, 16, 600, 15
    b = np.array([3.0 - 3.0 * i / K for i in range(K + 1)])
    g = _gpu_run(q, L, R, 5, 3, b, init=pa.INIT_GROUND, fam=True)
    o = _oracle_run(q, L, R, 5, 3, b, init=1)
    _compare(g, o, fam=True)
    assert g["obs"][0]["lnZ"] == math.log(q) + 2 * L * L * 3.0


def test_families_cooling():
    w = wl.C1
    b = w.betas()[:31]
    g = _gpu_run(w.q, w.L, w.R, 2, w.theta, b, fam=True)
    o = _oracle_run(w.q, w.L, w.R, 2, w.theta, b)
    _compare(g, o, fam=True)


@pytest.mark.parametrize("mode", [pa.RESAMPLE_NEAREST_INT, pa.RESAMPLE_ROUND, pa.RESAMPLE_POISSON,
                                  pa.RESAMPLE_OFF])
def test_single_and_multi_block_resampling_bit_exact(mode):
    """Capacities up to 4096 replicas resample in one block that runs the
    weight, copy-number and scatter stages in turn; larger capacities use one
    kernel per stage over many blocks.  Both against the oracle."""
    q, L, R, K = 8, 16, 700, 10
    b = np.array([1.5 * i / K for i in range(K + 1)])
    for cap in (0, 5000):
        g = _gpu_run(q, L, R, 13, 3, b, mode=mode, R_cap=cap)
        o = _oracle_run(q, L, R, 13, 3, b, mode=mode, R_cap=cap or None)
        _compare(g, o)


@pytest.mark.parametrize("R", [1000, 5000])
def test_capacity_overflow_keeps_previous_population(R):
    q, L = 10, 16
    p = pa.PAParams(q=q, L=L, R=R, seed=3, R_cap=R)
    with pa.Population(p) as pop:
        beta = 0.0
        hit = False
        for i in range(1, 40):
            before = pop.spins()
            try:
                pop.resample(0.05, i, sync=True)
            except pa.PAError as e:
                assert e.status == pa.PA_ERR_CAPACITY
                assert np.array_equal(pop.spins(), before)
                hit = True
                break
            beta += 0.05
            pop.sweep(beta, 2, i)
        assert hit, "population never exceeded a capacity equal to R"
        # the context is usable again at the previous step (a resample with
        # dbeta = 0 could itself overflow: rho_j = R / R_{i-1} > 1 when the
        # population has shrunk below R)
        pop.sweep(beta, 1, i - 1)
        assert pop.energies().shape[0] == before.shape[0]


def test_call_order_is_enforced():
    p = pa.PAParams(q=4, L=8, R=50, seed=1)
    with pa.Population(p) as pop:
        with pytest.raises(pa.PAError) as e:
            pop.sweep(0.1, 1, 3)  # no resample pending for step 3
        assert e.value.status == pa.PA_ERR_STATE
        pop.resample(0.1, 1)
        with pytest.raises(pa.PAError):
            pop.resample(0.1, 2)  # one already pending
        pop.sweep(0.1, 1, 1)
        with pytest.raises(pa.PAError):
            pop.resample(0.1, 1)  # step must increase


# ---------------------------------------------------------------------------
# Plain PA at scale (q = 10, L = 64, R = 100000, theta = 10) in the launch
# shape the benchmark uses: step 1 on sampled slots, which the oracle can
# recompute one by one from the initial state, plus every initial energy.
# ---------------------------------------------------------------------------
def _init_energies(args):
    q, L, begin, count, seed = args
    import oracle as orc

    s = orc.init_random(q, L, begin, count, seed)
    return np.array([orc.energy(x) for x in s], dtype=np.int32)


@pytest.mark.parametrize("w", [wl.C2, wl.C4, wl.C5], ids=["q10-L64-R1e5", "q8-L128-R2e5", "q20-L256-R1e5"])
def test_full_size_step_one_sampled(w):
    """Full population, first temperature step: every initial energy, ln Q and
    the new size against the oracle, and sampled slots recomputed one by one
    from their parents' initial states (theta sweeps at beta_1)."""
    b = w.betas()
    p = pa.PAParams(q=w.q, L=w.L, R=w.R, seed=w.seed, track_families=w.track_families)
    rng = np.random.default_rng(2024)
    n_sample = 24 if w.L <= 64 else 8
    with pa.Population(p) as pop:
        E0 = pop.energies()
        lnq, R1 = pop.resample(b[1] - b[0], 1, sync=True)
        pop.sweep(b[1], w.theta, 1)
        E1 = pop.energies()
        assert E1.size == R1
        sample = np.unique(np.concatenate([rng.integers(0, R1, n_sample), [0, R1 - 1]]))
        spins = {int(s): pop.spins(int(s), 1)[0] for s in sample}
        o1, h1 = pop.observables(with_hist=True)

    per = 6250 if w.L <= 64 else 2000
    chunks = [(w.q, w.L, k, min(per, w.R - k), w.seed) for k in range(0, w.R, per)]
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as poolp:
        E0_ref = np.concatenate(poolp.map(_init_energies, chunks))
    assert np.array_equal(E0, E0_ref)
    r, lnq_ref, R1_ref, rho = oracle.copy_numbers(E0_ref, b[1] - b[0], w.R, oracle.NEAREST_INT, 1, w.seed)
    assert R1 == R1_ref
    assert lnq == pytest.approx(lnq_ref, rel=LNZ_RTOL)
    parents = oracle.parents(r)
    for s, got in spins.items():
        init = oracle.init_random(w.q, w.L, int(parents[s]), 1, w.seed)[0]
        ref = oracle.sweep_replica(w.q, init, b[1], w.theta, 1, s, w.seed)
        assert np.array_equal(got, ref), s
        assert E1[s] == oracle.energy(ref)
    # properties that hold at any size
    assert h1.sum() == R1 and np.array_equal(np.bincount(E1 + 2 * w.N, minlength=2 * w.N + 1), h1)
    assert o1["sumE"] == int(E1.astype(np.int64).sum())
    if w.track_families:
        assert o1["n_families"] == int(np.count_nonzero(r))


def test_plain_at_scale_launch_shape_reduced_population():
    """Three full steps at L = 64, q = 10, theta = 10 with R = 3000 in the
    block shape the default launch picks for R = 100000 (48 replicas x 512
    threads, six site words per thread and half sweep)."""
    w = wl.C2
    b = w.betas()[:4]
    R = 3000
    g = _gpu_run(w.q, w.L, R, w.seed, w.theta, b, launch=(48, 512))
    o = _oracle_run(w.q, w.L, R, w.seed, w.theta, b)
    _compare(g, o)


def test_checkpoint_resume_is_bit_identical(tmp_path):
    """Save after 6 steps, resume from the file, run 6 more: identical to the
    uninterrupted 12-step run (counter-based random numbers); a corrupted
    file is refused."""
    q, L, R = 10, 16, 800
    b = np.array([1.2 * i / 12 for i in range(13)])
    p = pa.PAParams(q=q, L=L, R=R, seed=17, track_families=True)
    path = str(tmp_path / "pa.ckpt")
    with pa.Population(p) as pop:
        pop.run(b[:7], 4)
        pop.save(path)
        obs_ref, _ = pop.run(b[6:], 4)
        spins_ref, anc_ref = pop.spins(), pop.ancestors()
    # spins are stored in the canonical layout right after the header
    raw0 = open(path, "rb").read()
    header_bytes = int.from_bytes(raw0[12:16], "little")
    assert int.from_bytes(raw0[8:12], "little") == 4
    with pa.Population(p) as pop3:
        pop3.run(b[:7], 4)
        canon = pop3.spins()
    assert raw0[header_bytes: header_bytes + canon.size] == canon.tobytes()
    with pa.Population.load(path) as pop2:
        assert pop2.step == 6 and pop2.beta == b[6]
        obs, _ = pop2.run(b[6:], 4)
        assert [o["lnZ"] for o in obs] == [o["lnZ"] for o in obs_ref]
        assert [o["S_f"] for o in obs] == [o["S_f"] for o in obs_ref]
        assert np.array_equal(pop2.spins(), spins_ref) and np.array_equal(pop2.ancestors(), anc_ref)
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(pa.PAError) as e:
        pa.Population.load(bad)
    assert e.value.status == pa.PA_ERR_INVALID
