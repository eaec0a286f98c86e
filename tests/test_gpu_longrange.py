"""GPU parity of the long-range operator erf(omega r)/r (paper Sec. 2.5,
Eq. eri_longrange_definition, Eq. eri_longrange_formula) against the oracle
(Obara-Saika with the attenuated auxiliary integrals, pinned in
tests/test_oracle_longrange.py), every call through the C ABI:

- FP64 J and K within 1e-10 on workload 0 and on small systems that isolate
  class families, at two omegas;
- the J-engine (J alone) with the attenuated operator;
- the mixed-precision path within 1e-6 Eh of the oracle's energies;
- the nuclear gradient within 1e-9 of the oracle's four-centre gradient;
- omega = 0 restores the Coulomb result (to rounding).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14920_gb300.build import build
    build()
    import paper_2406_14920_gb300 as m
    return m


def _oracle_jk(basis, D, omega, thresh=1e-12):
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    o.set_omega(omega)
    J, K = o.jk(D, thresh, Q)
    return o, Q, J, K, o.energy(D, J, K)


@pytest.mark.parametrize("omega", [0.25, 1.1])
def test_longrange_jk_fp64_w0(eri, omega):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=1e-12)
    Dt = torch.from_numpy(D).cuda()
    J0, K0 = plan.build_jk(Dt)
    J0, K0 = J0.cpu().numpy(), K0.cpu().numpy()
    plan.set_omega(omega)
    J, K = plan.build_jk(Dt)
    E = plan.energy(Dt, J, K).cpu().numpy()
    J, K = J.cpu().numpy(), K.cpu().numpy()
    _, _, Jr, Kr, (ej, ek) = _oracle_jk(basis, D, omega)
    assert np.abs(J - Jr).max() < TOL, np.abs(J - Jr).max()
    assert np.abs(K - Kr).max() < TOL, np.abs(K - Kr).max()
    assert abs(E[0] - ej) < TOL and abs(E[1] - ek) < TOL
    assert np.abs(J - J0).max() > 1e-3  # the operator changed the result
    # J alone takes the J-engine (Eq. j_formula) with the same attenuated R
    Jo, _ = plan.build_jk(Dt, want_k=False)
    assert np.abs(Jo.cpu().numpy() - Jr).max() < TOL
    # back to the Coulomb operator (equal to rounding: FP64 atomics add in any order)
    plan.set_omega(0.0)
    J2, K2 = plan.build_jk(Dt)
    assert np.abs(J2.cpu().numpy() - J0).max() < 1e-12 and np.abs(K2.cpu().numpy() - K0).max() < 1e-12


@pytest.mark.parametrize("comp", [["1s", "1p"], ["1d", "1s1p"], ["1f", "1p"], ["1f", "1f"], ["2s1p1d1f", "1s1p"]])
def test_longrange_jk_fp64_small(eri, comp):
    import torch
    basis, D = W.small_system(comp, seed=len(comp) * 11 + len(comp[-1]))
    plan = eri.Plan(basis, thresh=1e-12)
    plan.set_omega(0.6)
    Dt = torch.from_numpy(D).cuda()
    J, K = plan.build_jk(Dt)
    _, _, Jr, Kr, _ = _oracle_jk(basis, D, 0.6)
    assert np.abs(J.cpu().numpy() - Jr).max() < TOL
    assert np.abs(K.cpu().numpy() - Kr).max() < TOL


def test_longrange_mixed_w0(eri):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=1e-12, precision=eri.ERI_MIXED, mixed_tau=1e-3)
    plan.set_omega(0.4)
    Dt = torch.from_numpy(D).cuda()
    J, K = plan.build_jk(Dt)
    E = plan.energy(Dt, J, K).cpu().numpy()
    st = plan.stats()
    _, _, _, _, (ej, ek) = _oracle_jk(basis, D, 0.4)
    assert st["quartets_k_fp32"] > 0
    assert abs(E[0] - ej) < 1e-6 and abs(E[1] - ek) < 1e-6, (E[0] - ej, E[1] - ek)


def test_longrange_gradient_vs_oracle(eri):
    import torch
    basis, D = W.small_system(["1s1p1d", "2s1p1f"], seed=21, side=2.5)
    plan = eri.Plan(basis, thresh=1e-14)
    plan.set_omega(0.5)
    Dt = torch.from_numpy(D).cuda()
    g = plan.grad(Dt).cpu().numpy()
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    o.set_omega(0.5)
    gr = o.grad(D, 1e-14, Q)
    scale = max(1.0, np.abs(gr).max())
    assert np.abs(g - gr).max() < 1e-9 * scale, (g, gr)
    assert np.abs(g.sum(axis=0)).max() < 1e-10 * scale
