"""GPU parity of the point-charge attraction matrix V and of the gradient of
E_V = sum D_mn V_mn (paper Sec. 2.4, Eq. v1e_definition, Eq. v1e_formula;
SI Sec. 1.3) against the oracle (Obara-Saika three-centre integrals,
pinned in tests/test_oracle_nuclear.py), through the C ABI:

- V within 1e-10 on workload 0 with its nuclei as charges and with a cloud of
  seeded point charges, and on small systems that isolate f and d shells;
- dE/dR (basis centres) and dE/dC (charge positions) within 1e-9 of the
  oracle; forces on atoms and charges sum to zero;
- a batched plan: every molecule's block equals its own plan's V;
- no charges: V = 0.
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


def _cloud(basis, n, seed, spread=4.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, n), basis.coords.mean(axis=0) + rng.normal(0.0, spread, (n, 3))


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


@pytest.mark.parametrize("which", ["nuclei", "cloud"])
def test_v_w0(eri, which):
    basis, D = W.workload(0)
    if which == "nuclei":
        q, C = -np.full(basis.natom, 6.0), basis.coords.copy()
    else:
        q, C = _cloud(basis, 300, seed=3)
    plan = eri.Plan(basis, thresh=1e-12)
    V = plan.nuclear(_t(q), _t(C)).cpu().numpy()
    Vr = oracle.Oracle(basis).nuclear(q, C)
    assert np.abs(V - Vr).max() < TOL * max(1.0, np.abs(Vr).max()), np.abs(V - Vr).max()


@pytest.mark.parametrize("comp", [["1s", "1p"], ["1d", "1s1p"], ["1f", "1p1d"], ["1f", "1f"], ["2s1p1d1f"]])
def test_v_small(eri, comp):
    basis, _ = W.small_system(comp, seed=17)
    q, C = _cloud(basis, 37, seed=5)
    plan = eri.Plan(basis, thresh=1e-12)
    V = plan.nuclear(_t(q), _t(C)).cpu().numpy()
    Vr = oracle.Oracle(basis).nuclear(q, C)
    assert np.abs(V - Vr).max() < TOL * max(1.0, np.abs(Vr).max())


@pytest.mark.parametrize("comp", [["1s1p1d", "2s1p", "1p1f"], ["1f", "1f"], ["2s1p1d1f"]])
def test_v_gradient(eri, comp):
    basis, D = W.small_system(comp, seed=21, side=3.0)
    q, C = _cloud(basis, 41, seed=9, spread=2.0)
    plan = eri.Plan(basis, thresh=1e-12)
    gR, gC = plan.nuclear_grad(_t(D), _t(q), _t(C))
    gR, gC = gR.cpu().numpy(), gC.cpu().numpy()
    rR, rC = oracle.Oracle(basis).nuclear_grad(D, q, C)
    scale = max(1.0, np.abs(rR).max(), np.abs(rC).max())
    assert np.abs(gR - rR).max() < 1e-9 * scale, np.abs(gR - rR).max()
    assert np.abs(gC - rC).max() < 1e-9 * scale, np.abs(gC - rC).max()
    assert np.abs(gR.sum(axis=0) + gC.sum(axis=0)).max() < 1e-10 * scale


def test_v_batched_and_empty(eri):
    mols = [W.small_system(["1s1p1d", "2s1p"], seed=s) for s in (1, 2, 3)]
    q, C = _cloud(mols[0][0], 25, seed=11)
    pb = eri.Plan([b for b, _ in mols], thresh=1e-12)
    Vb = pb.unpack(pb.nuclear(_t(q), _t(C)))
    for (b, _), Vm in zip(mols, Vb):
        p1 = eri.Plan(b, thresh=1e-12)
        assert np.abs(Vm.cpu().numpy() - p1.nuclear(_t(q), _t(C)).cpu().numpy()).max() < 1e-13
    import torch
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    V0 = pb.nuclear(z, torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert float(V0.abs().max()) == 0.0
