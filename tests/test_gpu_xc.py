"""GPU parity of the exchange-correlation quadrature (paper Sec. 2.6:
Eq. xc_density_0, Eq. xc_density_1, Eq. xc_grid_sum_0, Eq. xc_grid_sum_1)
against the oracle (pinned in tests/test_oracle_xc.py), through the C ABI:

- the grid: every point and weight of the device grid against the oracle's
  grid of the same definition (relative 1e-12);
- density and gradient at every point within 1e-10 (relative to max(1, |rho|));
- the XC matrix for seeded synthetic point potentials within 1e-10 of the
  oracle's double sum, for a plan that keeps the basis values resident and one
  that recomputes them in small chunks;
- E_xc and V_xc of the built-in Slater and Becke-88 exchange within 1e-10;
- the closed-form Slater energy of one normalised s Gaussian;
- after eri_plan_set_coords with every atom shifted the grid follows and
  E_xc is unchanged;
- at the bench size (workload 1, 60 atoms, 900 basis functions, 32 radial x
  16 x 32 angular points per atom): sampled points, weights and densities
  against the oracle, sampled matrix elements for synthetic potentials, and
  the integral of rho equal to tr(D S) within the grid's quadrature error.
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


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def _unpartitioned(natom, nrad, nt):
    """Radial x angular weight of every point (the grid of one atom, where the
    Becke factor is 1, repeated per atom): the scale of the Becke-weighted one."""
    one = W.Basis(np.zeros(1, np.int32), np.zeros(1, np.int32), np.ones(1, np.int32), np.zeros(1, np.int32),
                  np.array([1.0]), np.array([1.0]), np.zeros((1, 3)), "one")
    _, w1 = oracle.Oracle(one).xc_grid(nrad, nt)
    return np.tile(w1, natom)


def _grid_close(pg, wg, po, wo, wscale):
    """Points to 1e-12 of the coordinate scale; weights to 1e-12 of the point's
    radial x angular weight (the Becke factor lies in [0, 1] and is compared
    absolutely: where it is tiny its relative rounding is large)."""
    assert pg.shape == po.shape and wg.shape == wo.shape
    assert np.abs(pg - po).max() < 1e-12 * max(1.0, np.abs(po).max())
    assert np.all(np.abs(wg - wo) <= 1e-12 * wscale)


SYSTEMS = {
    "w0": lambda: W.workload(0),
    "fd": lambda: W.small_system(["2s1p1d1f", "1s1p1d"], seed=5),
    "sp3": lambda: W.small_system(["2s1p", "1s1p1d", "2s1p"], seed=11, side=4.0, dmin=1.8),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_grid_and_density(eri, name):
    basis, D = SYSTEMS[name]()
    nrad, nt = 24, 8
    plan = eri.Plan(basis, thresh=1e-12)
    G = plan.xc_grid(nrad, nt)
    pts, w = plan.xc_get_grid()
    o = oracle.Oracle(basis)
    po, wo = o.xc_grid(nrad, nt)
    assert G == po.shape[0]
    _grid_close(pts.cpu().numpy(), w.cpu().numpy(), po, wo, _unpartitioned(basis.natom, nrad, nt))
    rho, grad = plan.xc_density(_t(D))
    ro, go = o.xc_density(D, po)
    sc = np.maximum(1.0, np.abs(ro))
    assert np.all(np.abs(rho.cpu().numpy() - ro) <= TOL * sc)
    assert np.all(np.abs(grad.cpu().numpy() - go) <= TOL * sc[:, None])
    st = plan.xc_stats()
    assert st["npoints"] == G and st["resident"] == 1
    plan.close()


@pytest.mark.parametrize("cap", [0.0, 2e5])
def test_matrix_synthetic_potentials(eri, cap):
    basis, D = W.small_system(["2s1p1d1f", "1s1p1d", "2s1p"], seed=13, side=4.0, dmin=1.8)
    nrad, nt = 20, 8
    plan = eri.Plan(basis, thresh=1e-12)
    G = plan.xc_grid(nrad, nt, cap_bytes=cap)
    st = plan.xc_stats()
    assert (st["resident"] == 1) == (cap == 0.0)
    if cap:
        assert st["nchunk"] > 1
    rng = np.random.default_rng(21)
    vrho = rng.normal(0.0, 1.0, G)
    vgrad = rng.normal(0.0, 1.0, (G, 3))
    V = plan.xc_matrix(_t(vrho), _t(vgrad)).cpu().numpy()
    o = oracle.Oracle(basis)
    po, wo = o.xc_grid(nrad, nt)
    Vo = o.xc_matrix(po, wo, vrho, vgrad)
    assert np.abs(V - Vo).max() < TOL * max(1.0, np.abs(Vo).max())
    assert np.abs(V - V.T).max() < 1e-12 * max(1.0, np.abs(V).max())
    plan.close()


@pytest.mark.parametrize("kind", [1, 2])
def test_xc_energy_and_matrix(eri, kind):
    basis, D = W.small_system(["2s1p1d1f", "1s1p1d"], seed=5)
    nrad, nt = 30, 8
    plan = eri.Plan(basis, thresh=1e-12)
    plan.xc_grid(nrad, nt)
    E, V = plan.xc(_t(D), functional=kind)
    Eo, Vo = oracle.Oracle(basis).xc(D, nrad, nt, kind)
    assert abs(float(E.cpu()[0]) - Eo) < TOL * max(1.0, abs(Eo))
    assert np.abs(V.cpu().numpy() - Vo).max() < TOL * max(1.0, np.abs(Vo).max())
    plan.close()


def test_slater_single_gaussian_closed_form(eri):
    a = 0.8
    b = W.Basis(np.zeros(1, np.int32), np.zeros(1, np.int32), np.ones(1, np.int32), np.zeros(1, np.int32),
                np.array([a]), np.array([1.0]), np.zeros((1, 3)), "one")
    plan = eri.Plan(b, thresh=1e-12)
    plan.xc_grid(120, 8)
    E, V = plan.xc(_t(np.ones((1, 1))), functional=eri.ERI_XC_SLATER)
    cx = 0.75 * (3 / np.pi) ** (1 / 3)
    exact = -cx * (2 * a / np.pi) ** 2 * (3 * np.pi / (8 * a)) ** 1.5
    assert abs(float(E.cpu()[0]) - exact) < 1e-10 * abs(exact)
    assert abs(float(V.cpu()[0, 0]) - 4.0 / 3.0 * exact) < 1e-10 * abs(exact)
    plan.close()


def test_grid_follows_coordinates(eri):
    basis, D = W.small_system(["2s1p1d", "1s1p1d"], seed=3)
    plan = eri.Plan(basis, thresh=1e-12)
    plan.xc_grid(24, 8)
    E0, _ = plan.xc(_t(D), functional=eri.ERI_XC_B88)
    p0, _ = plan.xc_get_grid()
    shift = np.array([0.9, -1.7, 0.4])
    plan.set_coords(_t(basis.coords + shift))
    E1, _ = plan.xc(_t(D), functional=eri.ERI_XC_B88)
    p1, _ = plan.xc_get_grid()
    assert np.abs((p1 - p0).cpu().numpy() - shift).max() < 1e-12
    assert abs(float(E1.cpu()[0]) - float(E0.cpu()[0])) < 1e-11 * abs(float(E0.cpu()[0]))
    plan.close()


def test_errors(eri):
    basis, D = W.small_system(["1s1p"], seed=3)
    plan = eri.Plan(basis, thresh=1e-12)
    with pytest.raises(eri.EriError) as e:
        plan.xc_density(_t(D))  # no grid yet
    assert e.value.code == -1
    for bad in [(1, 8), (24, 7), (24, 0), (24, 66)]:
        with pytest.raises(eri.EriError):
            plan.xc_grid(*bad)
    plan.close()
    bases = [W.small_system(["1s1p"], seed=s)[0] for s in (1, 2)]
    pb = eri.Plan(bases, thresh=1e-12)
    with pytest.raises(eri.EriError) as e:
        pb.xc_grid(24, 8)
    assert e.value.code == -4
    pb.close()


@pytest.fixture(scope="module")
def w1xc(eri):
    basis, D = W.workload(1)
    plan = eri.Plan(basis, thresh=1e-12)
    G = plan.xc_grid(32, 16)
    o = oracle.Oracle(basis)
    po, wo = o.xc_grid(32, 16)
    yield basis, D, plan, G, o, po, wo
    plan.close()


def test_w1_grid_density_sampled(eri, w1xc):
    basis, D, plan, G, o, po, wo = w1xc
    pts, w = plan.xc_get_grid()
    _grid_close(pts.cpu().numpy(), w.cpu().numpy(), po, wo, _unpartitioned(basis.natom, 32, 16))
    rho, grad = plan.xc_density(_t(D))
    rho, grad = rho.cpu().numpy(), grad.cpu().numpy()
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.integers(0, G, 3000), np.argsort(-rho)[:200]])
    ro, go = o.xc_density(D, po[idx])
    sc = np.maximum(1.0, np.abs(ro))
    assert np.all(np.abs(rho[idx] - ro) <= TOL * sc)
    assert np.all(np.abs(grad[idx] - go) <= TOL * sc[:, None])
    # electron count: int rho = tr(D S) within the grid's quadrature error
    n = basis.nbf
    S = np.zeros((n, n))
    off = basis.ao_offsets()
    for a in range(basis.nshell):
        for b in range(basis.nshell):
            S[off[a]:off[a + 1], off[b]:off[b + 1]] = o.overlap_block(a, b)
    assert abs((wo * rho).sum() - (D * S).sum()) < 1e-3 * (D * S).sum()


def test_w1_matrix_sampled(eri, w1xc):
    basis, D, plan, G, o, po, wo = w1xc
    rng = np.random.default_rng(9)
    vrho = rng.normal(0.0, 1.0, G)
    vgrad = rng.normal(0.0, 1.0, (G, 3))
    V = plan.xc_matrix(_t(vrho), _t(vgrad)).cpu().numpy()
    mn = rng.integers(0, basis.nbf, (48, 2))
    ref = o.xc_matrix_elements(po, wo, vrho, vgrad, mn)
    assert np.abs(V[mn[:, 0], mn[:, 1]] - ref).max() < TOL * max(1.0, np.abs(ref).max())
    assert np.abs(V - V.T).max() < 1e-12 * max(1.0, np.abs(V).max())
