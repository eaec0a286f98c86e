"""Pins for the oracle's exchange-correlation quadrature (paper Sec. 2.6:
Eq. xc_density_0, Eq. xc_density_1, Eq. xc_grid_sum_0, Eq. xc_grid_sum_1).

Each pin rests on something other than the oracle's own formulas:

- the angular rule integrates monomials of the unit vector exactly
  (textbook moments 4 pi/(k+1) of u_x^k, 4 pi/15 of u_x^2 u_y^2), its theta
  nodes and weights are numpy's Gauss-Legendre ones, and the radial rule of a
  one-atom grid integrates a normalised Gaussian to 1 (closed form);
- the Becke cells are a partition of unity: a normalised Gaussian placed
  anywhere in a molecule integrates to 1 over the whole molecular grid;
- the grid integral of phi_m phi_n is the overlap S_mn of the oracle's
  Obara-Saika overlap (itself pinned by quadrature), so the basis-function
  values and norms are right, and the integral of rho is tr(D S) (number of
  electrons);
- grad phi and grad rho equal central differences of phi and rho in r;
- Slater exchange of a single normalised s Gaussian has the closed form
  -C_x (2a/pi)^2 (3 pi/(8a))^(3/2); Becke-88 reduces to Slater when
  grad rho = 0; v_rho and v_grad equal central differences of eps;
- V_xc = dE_xc/dD (central differences in D, both functionals), V is
  symmetric, and the sampled-element routine equals the full matrix.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _S(basis, o):
    off = basis.ao_offsets()
    n = basis.nbf
    S = np.zeros((n, n))
    for a in range(basis.nshell):
        for b in range(basis.nshell):
            S[off[a]:off[a + 1], off[b]:off[b + 1]] = o.overlap_block(a, b)
    return S


def _one_atom(l_list, exps, coefs=None):
    """One atom at the origin with one single-primitive shell per l."""
    n = len(l_list)
    coefs = np.ones(n) if coefs is None else np.asarray(coefs, float)
    return W.Basis(np.zeros(n, np.int32), np.asarray(l_list, np.int32), np.ones(n, np.int32),
                   np.arange(n, dtype=np.int32), np.asarray(exps, float), coefs, np.zeros((1, 3)), "one")


def test_angular_rule_moments():
    b = _one_atom([0], [1.0])
    o = oracle.Oracle(b)
    nrad, nt = 2, 8
    pts, w = o.xc_grid(nrad, nt)
    nang = nt * 2 * nt
    for i in range(nrad):  # one radial shell: weights = w_rad * w_ang, points = r u
        sl = slice(i * nang, (i + 1) * nang)
        r = np.linalg.norm(pts[sl], axis=1)
        assert np.allclose(r, r[0], rtol=1e-14)
        u = pts[sl] / r[:, None]
        wa = w[sl] / w[sl].sum() * 4 * np.pi
        assert abs(wa.sum() - 4 * np.pi) < 1e-12
        for k in (1, 2, 3, 4, 5, 6):
            exact = 4 * np.pi / (k + 1) if k % 2 == 0 else 0.0
            assert abs((wa * u[:, 0] ** k).sum() - exact) < 1e-12
            assert abs((wa * u[:, 2] ** k).sum() - exact) < 1e-12
        assert abs((wa * u[:, 0] ** 2 * u[:, 1] ** 2).sum() - 4 * np.pi / 15) < 1e-12
        assert abs((wa * u[:, 1] ** 2 * u[:, 2] ** 2).sum() - 4 * np.pi / 15) < 1e-12


@pytest.mark.parametrize("a", [0.2, 1.0, 7.0])
def test_radial_rule_gaussian(a):
    b = _one_atom([0], [1.0])
    pts, w = oracle.Oracle(b).xc_grid(120, 4)
    r2 = (pts ** 2).sum(axis=1)
    val = (w * (a / np.pi) ** 1.5 * np.exp(-a * r2)).sum()
    assert abs(val - 1.0) < 1e-10


def test_becke_partition_of_unity():
    basis, _ = W.small_system(["2s1p", "1s1p1d", "2s1p"], seed=11, side=4.0, dmin=1.8)
    pts, w = oracle.Oracle(basis).xc_grid(100, 24)
    rng = np.random.default_rng(3)
    for _ in range(4):
        c = basis.coords.mean(axis=0) + rng.normal(0, 1.0, 3)
        a = rng.uniform(0.3, 2.0)
        r2 = ((pts - c) ** 2).sum(axis=1)
        assert abs((w * (a / np.pi) ** 1.5 * np.exp(-a * r2)).sum() - 1.0) < 2e-6


def test_overlap_and_electron_count():
    basis, D = W.small_system(["2s1p1d1f", "1s1p1d"], seed=5)
    o = oracle.Oracle(basis)
    S = _S(basis, o)
    pts, w = o.xc_grid(150, 24)
    # int phi_m phi_n = S_mn on a subset of points chunks (memory)
    n = basis.nbf
    Sg = np.zeros((n, n))
    idx = np.nonzero(w)[0]
    for k in range(0, idx.shape[0], 4000):
        sel = idx[k:k + 4000]
        P = np.stack([o.xc_ao(pts[g])[0] for g in sel])
        Sg += (P * w[sel, None]).T @ P
    assert np.abs(Sg - S).max() < 5e-7
    rho, _ = o.xc_density(D, pts)
    assert abs((w * rho).sum() - (D * S).sum()) < 1e-7


def test_gradients_are_derivatives():
    basis, D = W.small_system(["2s1p1d1f", "1p1d"], seed=9)
    o = oracle.Oracle(basis)
    rng = np.random.default_rng(1)
    h = 1e-5
    for _ in range(5):
        r = basis.coords.mean(axis=0) + rng.normal(0, 1.0, 3)
        phi, dphi = o.xc_ao(r)
        rho, grad = o.xc_density(D, r[None])
        for x in range(3):
            e = np.zeros(3)
            e[x] = h
            fd = (o.xc_ao(r + e)[0] - o.xc_ao(r - e)[0]) / (2 * h)
            assert np.abs(fd - dphi[x]).max() < 1e-8 * max(1.0, np.abs(dphi).max())
            fr = (o.xc_density(D, (r + e)[None])[0] - o.xc_density(D, (r - e)[None])[0]) / (2 * h)
            assert abs(fr[0] - grad[0, x]) < 1e-8 * max(1.0, abs(grad).max())


@pytest.mark.parametrize("a", [0.5, 2.0])
def test_slater_closed_form_single_gaussian(a):
    b = _one_atom([0], [a])
    o = oracle.Oracle(b)
    D = np.ones((1, 1))
    E, V = o.xc(D, 120, 8, kind=1)
    cx = 0.75 * (3 / np.pi) ** (1 / 3)
    exact = -cx * (2 * a / np.pi) ** 2 * (3 * np.pi / (8 * a)) ** 1.5
    assert abs(E - exact) < 1e-10 * abs(exact)
    # V_11 = dE/dD_11; for rho = D phi^2, E(D) = D^(4/3) E(1) => V = 4/3 E
    assert abs(V[0, 0] - 4.0 / 3.0 * exact) < 1e-10 * abs(exact)


def test_b88_reduces_to_slater_and_derivatives():
    rng = np.random.default_rng(2)
    rho = 10 ** rng.uniform(-6, 1, 50)
    grad = rng.normal(0, 1, (50, 3)) * rho[:, None] ** (4 / 3) * rng.uniform(0, 5, (50, 1))
    e1, v1, g1 = oracle.xc_functional(1, rho, grad)
    e0, v0, _ = oracle.xc_functional(2, rho, np.zeros_like(grad))
    assert np.allclose(e0, e1, rtol=1e-14) and np.allclose(v0, v1, rtol=1e-14)
    assert np.all(g1 == 0)
    for kind in (1, 2):
        e, v, g = oracle.xc_functional(kind, rho, grad)
        h = 1e-6 * rho
        fd = (oracle.xc_functional(kind, rho + h, grad)[0] - oracle.xc_functional(kind, rho - h, grad)[0]) / (2 * h)
        assert np.allclose(fd, v, rtol=1e-6, atol=1e-12)
        for x in range(3):
            hg = 1e-6 * np.maximum(np.abs(grad[:, x]), rho ** (4 / 3))
            gp, gm = grad.copy(), grad.copy()
            gp[:, x] += hg
            gm[:, x] -= hg
            fd = (oracle.xc_functional(kind, rho, gp)[0] - oracle.xc_functional(kind, rho, gm)[0]) / (2 * hg)
            assert np.allclose(fd, g[:, x], rtol=1e-5, atol=1e-12)
    # B88 lowers the exchange energy when the density varies
    e2, _, _ = oracle.xc_functional(2, rho, grad)
    assert np.all(e2 <= e1 + 1e-300)
    # below the density cutoff a point contributes nothing
    e, v, g = oracle.xc_functional(2, np.array([1e-15]), np.array([[1e-3, 0, 0]]))
    assert e[0] == 0 and v[0] == 0 and np.all(g == 0)


@pytest.mark.parametrize("kind", [1, 2])
def test_matrix_is_energy_derivative(kind):
    basis, D = W.small_system(["2s1p1d", "1s1p"], seed=4)
    o = oracle.Oracle(basis)
    nrad, nt = 40, 8
    E, V = o.xc(D, nrad, nt, kind)
    assert np.abs(V - V.T).max() < 1e-13 * np.abs(V).max()
    rng = np.random.default_rng(6)
    n = basis.nbf
    h = 1e-5
    for _ in range(6):
        m, v = rng.integers(0, n, 2)
        dD = np.zeros((n, n))
        dD[m, v] += h
        dD[v, m] += h if m != v else 0.0
        Ep, _ = o.xc(D + dD, nrad, nt, kind)
        Em, _ = o.xc(D - dD, nrad, nt, kind)
        fd = (Ep - Em) / 2
        pred = (V * dD).sum()
        assert abs(fd - pred) < 1e-9 * max(1.0, abs(pred)) + 1e-12


def test_matrix_elements_match_full_matrix():
    basis, D = W.small_system(["2s1p1d1f", "1s1p1d"], seed=5)
    o = oracle.Oracle(basis)
    pts, w = o.xc_grid(20, 8)
    rng = np.random.default_rng(8)
    vrho = rng.normal(0, 1, w.shape[0])
    vgrad = rng.normal(0, 1, (w.shape[0], 3))
    V = o.xc_matrix(pts, w, vrho, vgrad)
    mn = rng.integers(0, basis.nbf, (20, 2))
    el = o.xc_matrix_elements(pts, w, vrho, vgrad, mn)
    assert np.allclose(el, V[mn[:, 0], mn[:, 1]], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("nt", [4, 8, 16, 24])
def test_angular_nodes_are_gauss_legendre(nt):
    """cos(theta) of the grid points are numpy's Gauss-Legendre nodes and the
    theta weights (summed over azimuths, normalised) its weights."""
    b = _one_atom([0], [1.0])
    pts, w = oracle.Oracle(b).xc_grid(2, nt)
    nang = nt * 2 * nt
    sl = slice(0, nang)
    r = np.linalg.norm(pts[sl], axis=1)
    ct = (pts[sl, 2] / r).reshape(nt, 2 * nt)
    wt = w[sl].reshape(nt, 2 * nt).sum(axis=1)
    x, wx = np.polynomial.legendre.leggauss(nt)
    assert np.allclose(ct, ct[:, :1], atol=1e-15)
    assert np.abs(ct[:, 0] - x).max() < 1e-14
    assert np.abs(wt / wt.sum() * 2.0 - wx).max() < 1e-14
