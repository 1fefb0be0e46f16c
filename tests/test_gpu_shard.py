"""One population spread over several ranks (pa_shard_*, shard.py) against
the same population on one context (pa_init), bit for bit.

The ranks run as threads of this process on one GPU (ThreadComm): each
collective waits at a barrier until every rank has enqueued its part on the
shared stream, and no kernel waits for another.  The single-context run is
itself checked against the oracle by the other parity tests."""
import threading

import numpy as np
import pytest

import paper_1704_01888_gb300 as pa
from paper_1704_01888_gb300.shard import ShardedPopulation, ThreadComm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_01888_gb300 import build

    build.build()


def _sharded(params, G, betas, theta):
    import torch

    stream = torch.cuda.Stream()
    shared = ThreadComm.Shared(G, timeout=300.0)
    out = [None] * G
    errors = []

    def rank(g):
        try:
            with torch.cuda.stream(stream):
                sp = ShardedPopulation(params, ThreadComm(shared, g), stream=stream.cuda_stream)
                obs = [sp.observables()]
                for i in range(1, len(betas)):
                    sp.step(betas[i], theta, i)
                    obs.append(sp.observables())
                res = {"obs": obs, "spins": sp.spins(), "E": sp.energies(), "range": sp.range()}
                if params.track_families:
                    res["anc"] = sp.ancestors()
                sp.close()
                out[g] = res
        except BaseException as e:  # noqa: BLE001 - reported below
            errors.append(e)
            shared.barrier.abort()

    threads = [threading.Thread(target=rank, args=(g,)) for g in range(G)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    torch.cuda.synchronize()
    return out


def _single(params, betas, theta):
    with pa.Population(params) as pop:
        obs0 = pop.observables()
        obs, _ = pop.run(betas, theta)
        res = {"obs": [obs0] + obs, "spins": pop.spins(), "E": pop.energies()}
        if params.track_families:
            res["anc"] = pop.ancestors()
    return res


@pytest.mark.parametrize("q,L,R,G,theta,K,fam", [
    (10, 16, 1000, 2, 4, 12, False),
    (8, 32, 3001, 3, 3, 8, True),      # ragged shares, families
    (10, 64, 5000, 4, 5, 6, False),    # the benchmark geometry, many-block resampling
    (20, 80, 300, 2, 2, 5, True),      # banded rows, five bit planes
])
def test_sharded_population_equals_single_context(q, L, R, G, theta, K, fam):
    params = pa.PAParams(q=q, L=L, R=R, seed=3, track_families=fam)
    betas = np.linspace(0.0, 1.5, K + 1)
    ref = _single(params, betas, theta)
    got = _sharded(params, G, betas, theta)
    # the ranks' slot ranges tile the population in order
    starts = [g["range"][0] for g in got]
    counts = [g["range"][1] for g in got]
    assert starts[0] == 0 and all(starts[g] + counts[g] == starts[g + 1] for g in range(G - 1))
    assert sum(counts) == ref["spins"].shape[0] and max(counts) - min(counts) <= 1
    assert np.array_equal(np.concatenate([g["spins"] for g in got]), ref["spins"])
    assert np.array_equal(np.concatenate([g["E"] for g in got]), ref["E"])
    if fam:
        assert np.array_equal(np.concatenate([g["anc"] for g in got]), ref["anc"])
    for g in got:  # every rank holds the whole population's estimators
        for a, b in zip(g["obs"], ref["obs"]):
            for key in ("R", "sumE", "sumE2", "sumMt", "meanE", "C", "meanM", "lnQ", "lnZ", "n_near_ties",
                        "n_families", "beta"):
                assert a[key] == b[key], (key, a[key], b[key])
            assert a["S_f"] == pytest.approx(b["S_f"], rel=1e-12, abs=1e-14)


def test_sharded_benchmark_workload_first_steps():
    """q = 10, L = 64, R = 1e5 over four ranks: five steps equal the single run."""
    params = pa.PAParams(q=10, L=64, R=100000, seed=1)
    betas = np.array([1.6 * i / 200 for i in range(6)])
    ref = _single(params, betas, 10)
    got = _sharded(params, 4, betas, 10)
    assert np.array_equal(np.concatenate([g["E"] for g in got]), ref["E"])
    for a, b in zip(got[0]["obs"], ref["obs"]):
        assert (a["R"], a["sumE"], a["lnZ"]) == (b["R"], b["sumE"], b["lnZ"])
