"""Full-schedule parity at the configured sizes, step by step.

Every temperature step of a run is driven through the C ABI (pa_resample,
pa_get_parents, pa_sweep) and checked against the oracle as it goes:

* resampling (Sec. 2 step 2, Eq. 2): from the GPU's own energies of step i-1
  the oracle recomputes ln Q_i (within 1e-10 relative), every copy number and
  hence the parent map (bit for bit) and the near-tie count;
* sweeps (Sec. 2 step 3): sampled slots of the new population are replayed by
  the oracle from their parents' spins of step i-1 (theta sweeps at beta_i,
  keyed by the slot) and must equal the GPU's spins and energies bit for bit;
  at three steps of the plain case every slot is replayed;
* measurements (Sec. 2 step 4, Eqs. 3-5): the histogram, the integer sums and
  (with families) the family ids and S_f against their definitions.

The plain case at scale (q = 10, L = 64, R = 1e5, 200 steps, theta = 10)
replays 64 slots at every step and the whole population at steps 1, 100 and
178 (beta_178 = 1.424, next to beta_t); the strong first-order case (q = 20, L = 256,
R = 1e5, 300 steps, theta = 20) checks resampling and families at every step
and replays slots at steps 1, 2 and around beta_t (267-269); the adaptive
case (q = 8, L = 128, R = 2e5) checks the Newton step of each of its first 20
steps against the oracle's on the same energies and replays the whole
population of step 20.
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


@pytest.fixture(scope="module")
def pool():
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as p:
        yield p


def _replay_one(args):
    q, parent_spins, beta, theta, step, slot, seed, child, E_child = args
    import oracle as orc

    ref = orc.sweep_replica(q, parent_spins, beta, theta, step, slot, seed)
    return bool(np.array_equal(ref, child)) and orc.energy(ref) == E_child, slot


def _replay_chunk(args):
    q, par, beta, theta, step, slots, seed, child, E_child = args
    import oracle as orc

    bad = []
    for k, s in enumerate(slots):
        ref = orc.sweep_replica(q, par[k], beta, theta, step, int(s), seed)
        if not (np.array_equal(ref, child[k]) and orc.energy(ref) == E_child[k]):
            bad.append(int(s))
    return bad


class Replay:
    """Drives one run step by step and checks each step against the oracle."""

    def __init__(self, w, pool, R=None, n_slots=64, seed_rng=2024):
        self.w = w
        self.R = w.R if R is None else R
        self.pool = pool
        self.n_slots = n_slots
        self.rng = np.random.default_rng(seed_rng)
        self.jobs = []
        self.ties = 0
        self.steps = 0
        self.full_replayed = 0
        self.pop = pa.Population(pa.PAParams(q=w.q, L=w.L, R=self.R, seed=w.seed,
                                             track_families=w.track_families))
        self.E = self.pop.energies()
        self.anc = self.pop.ancestors() if w.track_families else None

    def close(self):
        self.pop.close()

    def step(self, i, beta_prev, beta, replay_slots, replay_all=False):
        w, pop = self.w, self.pop
        dbeta = beta - beta_prev
        lnq, R_i = pop.resample(dbeta, i, sync=True)
        parents = pop.parents(R_i)
        r, lnq_ref, R_ref, _, ties = oracle.copy_numbers(self.E, dbeta, self.R, oracle.NEAREST_INT, i, w.seed,
                                                         with_ties=True)
        assert R_i == R_ref, (i, R_i, R_ref)
        assert lnq == pytest.approx(lnq_ref, rel=LNZ_RTOL, abs=1e-12), (i, lnq, lnq_ref)
        assert np.array_equal(parents, oracle.parents(r)), i
        sample = []
        if replay_slots:
            sample = np.unique(np.concatenate([self.rng.integers(0, R_i, self.n_slots), [0, R_i - 1]]))
            par_spins = {int(p): pop.spins(int(p), 1)[0] for p in np.unique(parents[sample])}
        par_all = pop.spins(0, self.E.size) if replay_all else None
        pop.sweep(beta, w.theta, i)
        obs, hist = pop.observables(with_hist=True)
        E = pop.energies()
        assert E.size == R_i and obs["R"] == R_i
        assert obs["n_near_ties"] == int(ties.sum()), i
        assert obs["sumE"] == int(E.astype(np.int64).sum()) and obs["sumE2"] == int((E.astype(np.int64) ** 2).sum())
        assert np.array_equal(np.bincount(E + 2 * w.N, minlength=2 * w.N + 1), hist)
        if self.anc is not None:
            anc = pop.ancestors()
            assert np.array_equal(anc, self.anc[parents]), i
            counts = np.bincount(anc, minlength=self.R)
            nu = counts[counts > 0] / R_i
            assert obs["n_families"] == nu.size
            assert obs["S_f"] == pytest.approx(float(-(nu * np.log(nu)).sum()), rel=SF_RTOL)
            self.anc = anc
        for s in sample:
            s = int(s)
            self.jobs.append((w.q, par_spins[int(parents[s])], beta, w.theta, i, s, w.seed, pop.spins(s, 1)[0],
                              int(E[s])))
        if replay_all:
            child_all = pop.spins(0, R_i)
            chunk = 500
            jobs = ((w.q, par_all[parents[a:a + chunk]], beta, w.theta, i, np.arange(a, min(a + chunk, R_i)), w.seed,
                     child_all[a:a + chunk], E[a:a + chunk]) for a in range(0, R_i, chunk))
            bad = [s for b in self.pool.imap_unordered(_replay_chunk, jobs) for s in b]
            assert not bad, (i, bad[:10])
            self.full_replayed += R_i
        self.ties += int(ties.sum())
        self.steps += 1
        self.E = E
        return obs, hist

    def check_sweeps(self):
        bad = [s for ok, s in self.pool.map(_replay_one, self.jobs, chunksize=4) if not ok]
        n = len(self.jobs)
        self.jobs = []
        assert not bad, bad[:10]
        return n


def test_plain_at_scale_every_step(pool):
    """q = 10, L = 64, R = 1e5, all 200 steps of the schedule, theta = 10,
    in the benchmark's launch shape."""
    w = wl.C2
    b = w.betas()
    rp = Replay(w, pool)
    full_steps = (1, 100, w.hist_steps[0])
    try:
        replayed = 0
        for i in range(1, w.K + 1):
            obs, hist = rp.step(i, b[i - 1], b[i], replay_slots=True, replay_all=i in full_steps)
            if i % 20 == 0:
                replayed += rp.check_sweeps()
            if i == w.hist_steps[0]:
                h4 = np.add.reduceat(hist, np.arange(0, hist.size, 4))
                assert h4.sum() == obs["R"]
        replayed += rp.check_sweeps()
    finally:
        rp.close()
    assert rp.steps == w.K and replayed >= 64 * w.K and rp.full_replayed > 0.99 * len(full_steps) * w.R
    print(f"c2: {rp.steps} steps, {replayed} sampled and {rp.full_replayed} whole-population replayed slots, "
          f"{rp.ties} flagged near ties")


def test_strong_first_order_every_resample_and_steps_near_beta_t(pool):
    """q = 20, L = 256, R = 1e5, theta = 20, 300 steps with families: every
    step's resampling, families and S_f; slots replayed at steps 1, 2 and
    267-269 (beta_t = 1.6997 lies between steps 268 and 269)."""
    w = wl.C5
    b = w.betas()
    replay = {1, 2, 267, 268, 269}
    rp = Replay(w, pool, n_slots=24)
    try:
        for i in range(1, w.K + 1):
            rp.step(i, b[i - 1], b[i], replay_slots=i in replay)
            if i in (2, 269):
                rp.check_sweeps()
    finally:
        rp.close()
    assert rp.steps == w.K
    print(f"c5: {rp.steps} steps, {rp.ties} flagged near ties")


def test_adaptive_first_steps_at_full_size(pool):
    """q = 8, L = 128, R = 2e5, theta = 10, overlap 0.85: the Newton step of
    each of the first 20 steps equals the oracle's on the GPU's energies, and
    each step is checked as above (every slot at step 20)."""
    w = wl.C4
    rp = Replay(w, pool, n_slots=16)
    try:
        beta = 0.0
        for i in range(1, 21):
            cap = min(0.05, w.beta_end - beta)
            dbeta = rp.pop.next_dbeta(0.85, cap, 12)
            dref = oracle.newton_dbeta(rp.E, 0.85, cap, 12)
            assert dbeta == dref, (i, dbeta, dref)
            a, _ = oracle.overlap(rp.E, dbeta)
            assert abs(a - 0.85) < 1e-4 or dbeta == cap
            rp.step(i, beta, beta + dbeta, replay_slots=i in (1, 10, 20), replay_all=i == 20)
            beta += dbeta
        rp.check_sweeps()
    finally:
        rp.close()
    assert rp.full_replayed > 0.99 * w.R
    print(f"c4: 20 adaptive steps to beta = {beta:.6f}, {rp.full_replayed} slots replayed at step 20, "
          f"{rp.ties} flagged near ties")
