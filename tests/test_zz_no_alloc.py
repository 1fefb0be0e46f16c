"""pa_resample_noalloc, the resampling entry point for callers that may not
allocate device memory (for example a plug-in whose host framework owns all
device memory, or a runtime that must not touch the allocator after set-up).  It must give what pa_resample gives on the same population: the
same new size, ln Q within the tolerance of the other parity tests, and a
parent map that reproduces the population pa_resample builds.  Checked on two
calls in a row (the fixed working memory is reused and must be cleared).

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


def _noalloc(torch, E_dev, R_prev, L, dbeta, R_target, step, seed, cap):
    stream = torch.cuda.current_stream().cuda_stream
    parent = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    lnq = torch.zeros(1, dtype=torch.float64, device="cuda")
    rn = torch.zeros(1, dtype=torch.int32, device="cuda")
    pa.resample_noalloc(E_dev.data_ptr(), R_prev, L, dbeta, R_target, pa.RESAMPLE_NEAREST_INT, step, seed,
                        parent.data_ptr(), cap, lnq.data_ptr(), rn.data_ptr(), stream)
    torch.cuda.synchronize()
    return parent.cpu().numpy(), float(lnq.item()), int(rn.item())


def test_noalloc_resample_matches_pa_resample_two_calls():
    import torch

    q, L, R, seed, theta = 10, 16, 3000, 7, 4
    N = L * L
    cap = R + R // 4 + 1024
    betas = np.array([0.05 * i for i in range(6)])
    with pa.Population(pa.PAParams(q=q, L=L, R=R, seed=seed)) as pop:
        pop.run(betas[:3], theta)  # steps 1, 2: a population with spread energies
        for step in (3, 4):  # two calls in a row
            dbeta = betas[step] - betas[step - 1]
            R_prev = pop.size()
            E_dev = torch.zeros(cap, dtype=torch.int32, device="cuda")
            pop.energies_to_device(E_dev.data_ptr())
            torch.cuda.synchronize()
            before = pop.spins()
            parent, lnq_na, R_na = _noalloc(torch, E_dev, R_prev, L, dbeta, R, step, seed, cap)
            lnq, R_i = pop.resample(dbeta, step, sync=True)
            pop.sweep(betas[step], 0, step)  # the gather alone
            after = pop.spins()
            assert R_na == R_i
            assert lnq_na == pytest.approx(lnq, rel=LNZ_RTOL, abs=1e-12)
            assert parent[:R_na].min() >= 0 and parent[:R_na].max() < R_prev
            assert np.array_equal(after, before[parent[:R_na]])
            assert np.all(np.diff(parent[:R_na]) >= 0)
            assert N == L * L


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
    # an energy outside [-2N, 0] is reported through the device size output
    E[3] = 5
    pa.resample_noalloc(E.data_ptr(), 16, 4, 0.1, 16, 0, 1, 1, out.data_ptr(), 16, d.data_ptr(), r.data_ptr(), s)
    torch.cuda.synchronize()
    assert int(r.item()) == -pa.PA_ERR_INVALID
