"""GPU parity of the differentiable reweighting and of the adaptive schedule.

Reweighting moments come from one block with a fixed summation order and
CUDA's exp/log; the oracle sums sequentially with the C library's: ln Q and
<E>_tau agree to 1e-12 relative, the central moments (var, cov, k3) to 1e-9
relative.  The adaptive run's steps are rounded to multiples of 2^-24 on both
sides, so its betas, spins and estimators are compared bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1704_01888_gb300 as pa

pytestmark = pytest.mark.gpu


def _five_point(f, x0, h=1e-4):
    """Derivative of f at x0 by the five-point stencil (truncation error
    O(h^4)); the plain central difference's O(h^2) term, set by the third
    derivative (higher cumulants of E), reaches 1e-5 relative on these
    populations."""
    return (-f(x0 + 2 * h) + 8 * f(x0 + h) - 8 * f(x0 - h) + f(x0 - 2 * h)) / (12 * h)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_01888_gb300 import build

    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def population():
    """Energies and estimators of a q = 8, L = 32, R = 20000 population after
    cooling to beta = 0.9 (20 steps, theta = 5)."""
    import torch

    q, L, R = 8, 32, 20000
    p = pa.PAParams(q=q, L=L, R=R, seed=3)
    betas = np.array([0.9 * i / 20 for i in range(21)])
    with pa.Population(p) as pop:
        obs, _ = pop.run(betas, 5)
        E_dev = torch.zeros(R + R // 4 + 1024, dtype=torch.int32, device="cuda")
        pop.energies_to_device(E_dev.data_ptr())
        n = pop.size()
        torch.cuda.synchronize()
    return {"E": E_dev[:n].clone(), "E_host": E_dev[:n].cpu().numpy(), "obs": obs[-1], "beta": betas[-1], "N": L * L}


def test_reweight_forward_matches_oracle(population):
    import torch
    from paper_1704_01888_gb300 import autograd as ag

    E, Eh = population["E"], population["E_host"]
    rng = np.random.default_rng(0)
    O = rng.normal(size=Eh.size)
    O_dev = torch.tensor(O, dtype=torch.float64, device="cuda")
    for d in (0.0, 0.004, 0.02, -0.01):
        out = ag.reweight_forward(E, torch.tensor(d, dtype=torch.float64, device="cuda"), O_dev).cpu().numpy()
        ref = oracle.reweight_all(Eh, d, O)
        assert out[0] == pytest.approx(ref[0], rel=1e-12)
        assert out[1] == pytest.approx(ref[1], rel=1e-12)
        assert out[2] == pytest.approx(ref[2], rel=1e-9)
        assert out[3] == pytest.approx(ref[3], rel=1e-9, abs=1e-12)
        assert out[4] == pytest.approx(ref[4], rel=1e-9, abs=1e-9)
        assert out[5] == ref[5]
        assert out[6] == pytest.approx(ref[6], rel=1e-12)
        assert out[7] == pytest.approx(ref[7], rel=1e-6, abs=1e-6 * ref[2] ** 1.5)


def test_lnQ_gradients_backward_kernels_and_finite_differences(population):
    import torch
    from paper_1704_01888_gb300 import autograd as ag

    E, Eh = population["E"], population["E_host"]
    for d0 in (0.0, 0.006):
        d = torch.tensor(d0, dtype=torch.float64, device="cuda", requires_grad=True)
        y = ag.lnQ(d, E)
        (g1,) = torch.autograd.grad(y, d, create_graph=True)
        (g2,) = torch.autograd.grad(g1, d)
        ref = oracle.reweight_all(Eh, d0)
        # d lnQ / d dbeta = -<E>_tau ; d^2 lnQ / d dbeta^2 = var_tau(E)
        assert g1.item() == pytest.approx(-ref[1], rel=1e-12)
        assert g2.item() == pytest.approx(ref[2], rel=1e-9)
        # the first-order backward without create_graph runs the scale kernel
        d2 = torch.tensor(d0, dtype=torch.float64, device="cuda", requires_grad=True)
        (g1b,) = torch.autograd.grad(ag.lnQ(d2, E), d2)
        assert g1b.item() == g1.item()
        fd = _five_point(lambda x: ag.lnQ(torch.tensor(x, dtype=torch.float64, device="cuda"), E).item(), d0)
        assert fd == pytest.approx(g1.item(), rel=1e-6)


def test_specific_heat_three_ways(population):
    """C = beta^2 var(E) / N from (a) the run's exact integer sums (fluctuation
    formula), (b) autograd of <E>_tau at dbeta = 0 (d<E>/d beta = -var), and
    (c) finite differences of <E>_tau (five-point stencil, h = 1e-4)."""
    import torch
    from paper_1704_01888_gb300 import autograd as ag

    E, beta, N = population["E"], population["beta"], population["N"]
    C_fluct = population["obs"]["C"]
    d = torch.tensor(0.0, dtype=torch.float64, device="cuda", requires_grad=True)
    mE = ag.mean_energy(d, E)
    (dmE,) = torch.autograd.grad(mE, d)
    C_auto = -beta * beta * dmE.item() / N
    dmE_fd = _five_point(lambda x: ag.mean_energy(torch.tensor(x, dtype=torch.float64, device="cuda"), E).item(), 0.0)
    C_fd = -beta * beta * dmE_fd / N
    assert C_auto == pytest.approx(C_fluct, rel=1e-10)
    assert C_fd == pytest.approx(C_fluct, rel=1e-6)


def test_reweighted_observable_gradients(population):
    import torch
    from paper_1704_01888_gb300 import autograd as ag

    E, Eh = population["E"], population["E_host"]
    rng = np.random.default_rng(1)
    O = rng.normal(size=Eh.size)
    d0 = 0.01
    O_dev = torch.tensor(O, dtype=torch.float64, device="cuda", requires_grad=True)
    d = torch.tensor(d0, dtype=torch.float64, device="cuda", requires_grad=True)
    y = ag.reweighted_mean(O_dev, d, E)
    gO, gd = torch.autograd.grad(y, (O_dev, d))
    ref = oracle.reweight_all(Eh, d0, O)
    assert y.item() == pytest.approx(ref[3], rel=1e-9)
    assert gd.item() == pytest.approx(-ref[4], rel=1e-9)
    tau_over_R = np.exp(-d0 * (Eh - ref[5]).astype(np.float64)) / ref[6]
    assert np.allclose(gO.cpu().numpy(), tau_over_R, rtol=1e-12, atol=0)
    fd = _five_point(
        lambda x: ag.reweighted_mean(O_dev.detach(), torch.tensor(x, dtype=torch.float64, device="cuda"), E).item(), d0)
    assert fd == pytest.approx(gd.item(), rel=1e-6)


def test_overlap_matches_oracle(population):
    from paper_1704_01888_gb300 import autograd as ag

    E, Eh = population["E"], population["E_host"]
    for d in (0.0, 0.002, 0.01, 0.05):
        a, da = ag.overlap(d, E).cpu().numpy()
        ra, rda = oracle.overlap(Eh, d)
        assert a == pytest.approx(ra, rel=1e-12)
        assert da == pytest.approx(rda, rel=1e-9, abs=1e-12)


def test_newton_step_matches_oracle():
    q, L, R = 8, 32, 5000
    with pa.Population(pa.PAParams(q=q, L=L, R=R, seed=4)) as pop:
        pop.run(np.array([0.05 * i for i in range(9)]), 3)
        E = pop.energies()
        for target, cap in ((0.85, 0.05), (0.85, 1.0), (0.5, 1.0), (0.99, 0.2)):
            d = pop.next_dbeta(target, cap)
            assert d == oracle.newton_dbeta(E, target, cap)


@pytest.mark.parametrize("q,L,R,beta_end,theta,cap", [
    (8, 16, 2000, 1.1 * math.log(1 + math.sqrt(8)), 5, 0.05),
    (5, 8, 700, 1.5, 3, 0.2),
])
def test_adaptive_run_bit_exact(q, L, R, beta_end, theta, cap):
    with pa.Population(pa.PAParams(q=q, L=L, R=R, seed=2)) as pop:
        obs, betas = pop.run_adaptive(beta_end, theta, target=0.85, dbeta_max=cap)
        spins = pop.spins()
        E = pop.energies()
    ref = oracle.run_adaptive(q, L, R, 2, theta, beta_end, target=0.85, dbeta_max=cap)
    K = ref["K"]
    assert len(betas) == K and np.array_equal(betas, ref["betas"][1:])
    assert betas[-1] == beta_end
    for i, o in enumerate(obs, start=1):
        assert o["R"] == ref["R"][i] and o["sumE"] == ref["sumE"][i] and o["meanE"] == ref["meanE"][i]
        assert o["lnZ"] == pytest.approx(ref["lnZ"][i], rel=1e-10)
    assert np.array_equal(spins, ref["spins"]) and np.array_equal(E, ref["E"])


def test_adaptive_large_lattice_first_steps():
    """The adaptive configuration's lattice (q = 8, L = 128) at R = 1500 for
    the first 4 adaptive steps, bit for bit."""
    q, L, R = 8, 128, 1500
    beta_end = 1.1 * math.log(1 + math.sqrt(8))
    with pa.Population(pa.PAParams(q=q, L=L, R=R, seed=1)) as pop:
        obs, betas = pop.run_adaptive(beta_end, 10, target=0.85, dbeta_max=0.05, max_steps=4)
        spins = pop.spins(0, 64)
    ref = oracle.run_adaptive(q, L, R, 1, 10, beta_end, target=0.85, dbeta_max=0.05, max_steps=4)
    assert np.array_equal(betas, ref["betas"][1:])
    assert [o["sumE"] for o in obs] == list(ref["sumE"][1:])
    assert np.array_equal(spins, ref["spins"][:64])
