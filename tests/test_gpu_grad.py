"""GPU nuclear gradient (eri_jk_grad) and the autograd wrapper.

- against the oracle's gradient, which differentiates all four centres of
  every quartet (the GPU uses the bra-only form of SI Eq. si_dE_J / si_dE_K);
- against central finite differences (h = 1e-4 bohr) of the GPU FP64 energy
  with the lists frozen at the reference geometry;
- zero net force (translational invariance);
- J and K parts separately;
- torch.autograd: dE/dR equals eri_jk_grad, dE/dD equals J - K/2.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14920_gb300.build import build
    build()
    import paper_2406_14920_gb300 as m
    return m


@pytest.mark.parametrize("comp,want", [(["1s1p1d", "2s1p1f"], (True, True)), (["1s1p1d", "2s1p1f"], (True, False)),
                                       (["1s1p1d", "2s1p1f"], (False, True)), (["1d1f", "1p1f", "1s"], (True, True)),
                                       (["1f", "1f"], (True, True))])
def test_grad_vs_oracle(eri, comp, want):
    import torch
    basis, D = W.small_system(comp, seed=21, side=2.5)
    plan = eri.Plan(basis, thresh=1e-14)
    Dt = torch.from_numpy(D).cuda()
    g = plan.grad(Dt, want_j=want[0], want_k=want[1]).cpu().numpy()
    o = oracle.Oracle(basis)
    gr = o.grad(D, 1e-14, o.schwarz(), *want)
    scale = max(1.0, np.abs(gr).max())
    assert np.abs(g - gr).max() < 1e-9 * scale, (g, gr)
    assert np.abs(g.sum(axis=0)).max() < 1e-10 * scale


def test_grad_vs_finite_difference_w0(eri):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=1e-12)
    Dt = torch.from_numpy(D).cuda()
    g = plan.grad(Dt).cpu().numpy()
    assert np.abs(g.sum(axis=0)).max() < 1e-10 * np.abs(g).max()
    h = 1e-4
    c0 = torch.from_numpy(basis.coords).cuda()

    def energy(c):
        plan.set_coords(c, freeze_lists=True)
        J, K = plan.build_jk(Dt)
        return float(plan.energy(Dt, J, K).sum())

    fd = np.zeros_like(g)
    for a in range(basis.natom):
        for t in range(3):
            cp = c0.clone(); cp[a, t] += h
            cm = c0.clone(); cm[a, t] -= h
            fd[a, t] = (energy(cp) - energy(cm)) / (2 * h)
    plan.set_coords(c0, freeze_lists=True)
    assert np.abs(g - fd).max() < 2e-7 * max(1.0, np.abs(g).max()), (g, fd)


def test_autograd_function(eri):
    import torch
    basis, D = W.small_system(["2s1p1d", "1s1p1f", "1s1p"], seed=9)
    plan = eri.Plan(basis, thresh=1e-12)
    R = torch.from_numpy(basis.coords).cuda().requires_grad_(True)
    Dt = torch.from_numpy(D).cuda().requires_grad_(True)
    E = eri.jk_energy(R, Dt, plan)
    gR, gD = torch.autograd.grad(E, (R, Dt))
    g_ref = plan.grad(Dt.detach())
    assert torch.allclose(gR, g_ref, atol=1e-12, rtol=0)
    J, K = plan.build_jk(Dt.detach())
    assert torch.allclose(gD, J - 0.5 * K, atol=1e-12, rtol=0)
    # E is quadratic in D: a central difference along a symmetric direction is exact up to rounding
    X = torch.randn_like(Dt.detach()); X = X + X.T
    eps = 1e-3
    with torch.no_grad():
        ep = eri.jk_energy(R.detach(), Dt.detach() + eps * X, plan)
        em = eri.jk_energy(R.detach(), Dt.detach() - eps * X, plan)
    assert abs(float((ep - em) / (2 * eps)) - float((gD * X).sum())) < 1e-9 * max(1.0, abs(float((gD * X).sum())))


def test_autograd_two_geometries_one_plan(eri):
    """Two forwards at different geometries on one shared plan, then one
    backward through their sum: each gradient is taken at its own forward's
    geometry (the plan is moved back as needed) and matches the oracle's
    four-centre gradient there."""
    import torch
    basis, D = W.small_system(["1s1p1d", "2s1p1f"], seed=21, side=2.5)
    plan = eri.Plan(basis, thresh=1e-14)
    c1 = basis.coords.copy()
    c2 = c1.copy()
    c2[1] += np.array([0.31, -0.17, 0.23])
    R1 = torch.from_numpy(c1).cuda().requires_grad_(True)
    R2 = torch.from_numpy(c2).cuda().requires_grad_(True)
    Dt = torch.from_numpy(D).cuda()
    E1 = eri.jk_energy(R1, Dt, plan)
    E2 = eri.jk_energy(R2, Dt, plan)
    (E1 + E2).backward()
    for R, c in ((R1, c1), (R2, c2)):
        o = oracle.Oracle(basis.with_coords(c))
        gr = o.grad(D, 1e-14, o.schwarz())
        scale = max(1.0, np.abs(gr).max())
        assert np.abs(R.grad.cpu().numpy() - gr).max() < 1e-9 * scale
    assert np.abs(R1.grad.cpu().numpy() - R2.grad.cpu().numpy()).max() > 1e-4


@pytest.mark.parametrize("which", ["w0", "small"])
def test_mixed_gradient(eri, which):
    """ERI_MIXED gradient: items whose density-weighted bound is below tau run in
    FP32 (FP64 accumulation).  Within 1e-6 of the oracle's four-centre gradient
    and of the FP64 gradient, not bit-identical to the latter (the FP32 tier ran),
    zero net force to 1e-8."""
    import torch
    if which == "w0":
        basis, D = W.workload(0)
    else:
        basis, D = W.small_system(["2s1p1d1f", "1s1p1d", "2s1p"], seed=5, side=6.0, dmin=2.5)
    plan = eri.Plan(basis, thresh=1e-12, precision=eri.ERI_MIXED, mixed_tau=1e-3)
    Dt = torch.from_numpy(D).cuda()
    g64 = plan.grad(Dt).cpu().numpy()
    gm = plan.grad(Dt, precision=eri.ERI_MIXED).cpu().numpy()
    o = oracle.Oracle(basis)
    gr = o.grad(D, 1e-12, o.schwarz())
    assert np.abs(gm - gr).max() < 1e-6 and np.abs(gm - g64).max() < 1e-6, np.abs(gm - g64).max()
    assert np.abs(gm - g64).max() > 0.0
    assert np.abs(gm.sum(axis=0)).max() < 1e-8
