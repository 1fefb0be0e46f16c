"""pa_resample_noalloc, the resampling entry point for callers that may not
allocate device memory (for example a plug-in whose host framework owns all
device memory, or a runtime that must not touch the allocator after set-up).
It must give what pa_resample gives on the same population: the same new
size, ln Q within the tolerance of the other parity tests, and a parent map
that reproduces the population pa_resample builds.  Checked on two calls in a
row (the fixed working memory is reused and must be cleared), for a run with a
nonzero random-number stream, for the one-block and many-block resampling
paths in every copy-number rule, and for a capacity overflow.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import paper_1704_01888_gb300 as pa

pytestmark = pytest.mark.gpu

LNZ_RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_01888_gb300 import build

    build.build()


def _noalloc(torch, E_dev, R_prev, L, dbeta, R_target, step, seed, cap, mode=pa.RESAMPLE_NEAREST_INT,
             rng_stream=0):
    stream = torch.cuda.current_stream().cuda_stream
    parent = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    lnq = torch.zeros(1, dtype=torch.float64, device="cuda")
    rn = torch.zeros(1, dtype=torch.int32, device="cuda")
    pa.resample_noalloc(E_dev.data_ptr(), R_prev, L, dbeta, R_target, mode, step, seed, parent.data_ptr(), cap,
                        lnq.data_ptr(), rn.data_ptr(), stream, rng_stream=rng_stream)
    torch.cuda.synchronize()
    return parent.cpu().numpy(), float(lnq.item()), int(rn.item())


def _against_pa_resample(q, L, R, seed, theta, R_cap, mode, rng_stream, noalloc_cap):
    import torch

    cap = R_cap or R + R // 4 + 1024
    betas = np.array([0.05 * i for i in range(6)])
    p = pa.PAParams(q=q, L=L, R=R, seed=seed, R_cap=R_cap, resample_mode=mode, stream=rng_stream)
    with pa.Population(p) as pop:
        pop.run(betas[:3], theta)  # steps 1, 2: a population with spread energies
        for step in (3, 4):  # two calls in a row
            dbeta = betas[step] - betas[step - 1]
            R_prev = pop.size()
            E_dev = torch.zeros(cap, dtype=torch.int32, device="cuda")
            pop.energies_to_device(E_dev.data_ptr())
            torch.cuda.synchronize()
            before = pop.spins()
            parent, lnq_na, R_na = _noalloc(torch, E_dev, R_prev, L, dbeta, R, step, seed, noalloc_cap(R_prev),
                                            mode, rng_stream)
            lnq, R_i = pop.resample(dbeta, step, sync=True)
            assert np.array_equal(parent[:R_i], pop.parents(R_i))
            pop.sweep(betas[step], 0, step)  # the gather alone
            after = pop.spins()
            assert R_na == R_i
            assert lnq_na == pytest.approx(lnq, rel=LNZ_RTOL, abs=1e-12)
            assert parent[:R_na].min() >= 0 and parent[:R_na].max() < R_prev
            assert np.array_equal(after, before[parent[:R_na]])
            assert np.all(np.diff(parent[:R_na]) >= 0)


def test_noalloc_resample_matches_pa_resample_two_calls():
    # many-block path (capacity above 4096 replicas)
    _against_pa_resample(10, 16, 3000, 7, 4, 0, pa.RESAMPLE_NEAREST_INT, 0, lambda R_prev: 3000 + 750 + 1024)


def test_noalloc_uses_the_run_stream():
    """A run with random-number stream 3 (as in a batch): the copy numbers of
    both calls are keyed by that stream."""
    _against_pa_resample(8, 16, 2500, 5, 3, 0, pa.RESAMPLE_NEAREST_INT, 3, lambda R_prev: 5000)


@pytest.mark.parametrize("mode", [pa.RESAMPLE_ROUND, pa.RESAMPLE_POISSON, pa.RESAMPLE_OFF])
def test_noalloc_single_block_path_every_rule(mode):
    """Capacities of at most 4096 replicas take the one-block resampling
    kernel; every other copy-number rule."""
    _against_pa_resample(6, 16, 1500, 9, 3, 0, mode, 1, lambda R_prev: 4000)


def test_noalloc_reports_capacity_overflow():
    """A new population larger than parent_cap is reported as -PA_ERR_CAPACITY
    in the device size output (and a following call works again)."""
    import torch

    L, R = 16, 2000
    rng = np.random.default_rng(4)
    E = torch.from_numpy(rng.integers(-300, -200, size=R).astype(np.int32)).cuda()
    # R_target = 3 R: about 3 R children into a capacity of R
    _, _, rn = _noalloc(torch, E, R, L, 0.01, 3 * R, 1, 1, R)
    assert rn == -pa.PA_ERR_CAPACITY
    parent, _, rn = _noalloc(torch, E, R, L, 0.01, R, 1, 1, 2 * R)
    assert 0 < rn <= 2 * R and parent[:rn].max() < R


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch

    E = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(pa.PAError) as e:
        pa.resample_noalloc(E.data_ptr(), 16, 258, 0.1, 16, 0, 1, 1, out.data_ptr(), 16, d.data_ptr(), r.data_ptr(), s)
    assert e.value.status == pa.PA_ERR_TOO_LARGE
    with pytest.raises(pa.PAError) as e:
        pa.resample_noalloc(E.data_ptr(), 300000, 16, 0.1, 16, 0, 1, 1, out.data_ptr(), 300000, d.data_ptr(),
                            r.data_ptr(), s)
    assert e.value.status == pa.PA_ERR_TOO_LARGE
    with pytest.raises(pa.PAError) as e:
        pa.resample_noalloc(E.data_ptr(), 16, 4, 0.1, 16, 0, 1, 1, out.data_ptr(), 16, d.data_ptr(), r.data_ptr(), s,
                            rng_stream=256)
    assert e.value.status == pa.PA_ERR_INVALID
    # an energy outside [-2N, 0] is reported through the device size output
    E[3] = 5
    pa.resample_noalloc(E.data_ptr(), 16, 4, 0.1, 16, 0, 1, 1, out.data_ptr(), 16, d.data_ptr(), r.data_ptr(), s)
    torch.cuda.synchronize()
    assert int(r.item()) == -pa.PA_ERR_INVALID
