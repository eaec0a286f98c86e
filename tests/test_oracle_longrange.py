"""Pins for the oracle's long-range ERIs, (mu nu| erf(omega r)/r |lambda sigma)
(paper Sec. 2.5, Eq. eri_longrange_definition and Eq. eri_longrange_formula).

- primitive ERIs of erf(omega r)/r against brute-force quadrature: the
  operator is (2/sqrt(pi)) int_0^omega exp(-t^2 r^2) dt, so the quadrature of
  tests/quadrature.py stops its t-integral at omega (no recurrence, no Boys
  function);
- four identical normalised s Gaussians (exponent a) on one centre: the two
  charge clouds are Gaussians of exponent 2a, their separation a Gaussian of
  exponent a, and its erf-attenuated interaction is
  2 sqrt(a/pi) omega / sqrt(a + omega^2) (closed form, independent of the
  recurrences);
- omega -> infinity recovers the Coulomb ERI;
- omega -> 0: erf(omega r)/r = (2 omega/sqrt(pi)) (1 - omega^2 r^2/3 + ...),
  so (ab|erf|cd) / omega -> (2/sqrt(pi)) S_ab S_cd with an O(omega^2) error;
- contracted J and K with the attenuated operator: the 8-fold canonical build
  equals the no-symmetry definition, and the nuclear gradient equals central
  finite differences, with zero net force;
- the Schwarz bounds stay the Coulomb ones and bound every attenuated quartet
  (erfc(omega r)/r is positive definite, so (ab|erf|ab) <= (ab|ab)).
"""
import numpy as np
import pytest

import oracle
import quadrature as quad
import workloads as W

RNG = np.random.default_rng(1406)


def _centres(n, scale=0.9):
    return [RNG.normal(0.0, scale, 3) for _ in range(n)]


@pytest.mark.parametrize("ls,omega", [((0, 0, 0, 0), 0.4), ((1, 0, 0, 0), 1.3), ((1, 1, 1, 0), 0.25),
                                      ((2, 1, 1, 0), 0.8), ((1, 1, 1, 1), 2.5), ((3, 1, 2, 0), 0.6),
                                      ((2, 2, 1, 1), 1.1)])
def test_prim_eri_erf_vs_quadrature(ls, omega):
    la, lb, lc, ld = ls
    A, B, Cc, D = _centres(4)
    ex = (0.8, 1.6, 0.55, 2.3)
    got = oracle.prim_eri_erf(la, lb, lc, ld, *ex, A, B, Cc, D, omega)
    ref = quad.prim_eri(la, lb, lc, ld, *ex, A, B, Cc, D, t_max=omega)
    scale = np.abs(ref).max()
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-12 * scale), np.abs(got - ref).max() / scale


def _single_shell_basis(l, exps, coefs, centre=(0.0, 0.0, 0.0)):
    n = len(exps)
    return W.Basis(np.array([0], np.int32), np.array([l], np.int32), np.array([n], np.int32),
                   np.array([0], np.int32), np.array(exps, float), np.array(coefs, float),
                   np.array([centre], float))


@pytest.mark.parametrize("alpha,omega", [(0.13, 0.2), (1.0, 0.33), (7.5, 2.0), (2.0e4, 0.4), (0.5, 50.0)])
def test_ssss_same_centre_closed_form(alpha, omega):
    o = oracle.Oracle(_single_shell_basis(0, [alpha], [0.37]))
    o.set_omega(omega)
    v = o.eri_block(0, 0, 0, 0)[0, 0, 0, 0]
    assert v == pytest.approx(2.0 * np.sqrt(alpha / np.pi) * omega / np.sqrt(alpha + omega * omega), rel=1e-13)


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (2, 1, 1, 0), (3, 3, 2, 1)])
def test_large_omega_recovers_coulomb(ls):
    A, B, Cc, D = _centres(4)
    ex = (0.8, 1.6, 0.55, 2.3)
    full = oracle.prim_eri(*ls, *ex, A, B, Cc, D)
    lr = oracle.prim_eri_erf(*ls, *ex, A, B, Cc, D, 1.0e6)
    assert np.allclose(lr, full, rtol=1e-10, atol=1e-12 * np.abs(full).max())


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 1, 0, 0), (2, 0, 1, 1), (2, 2, 2, 0)])
def test_small_omega_overlap_limit(ls):
    """(ab|erf|cd)/omega -> (2/sqrt(pi)) S_ab S_cd, error O(omega^2): checked at
    two omegas, the second-order error shrinking by the square of their ratio."""
    la, lb, lc, ld = ls
    A, B, Cc, D = _centres(4, 0.6)
    ex = (0.8, 1.6, 0.55, 2.3)
    Sab = oracle.prim_overlap(la, lb, ex[0], ex[1], A, B)
    Scd = oracle.prim_overlap(lc, ld, ex[2], ex[3], Cc, D)
    lim = 2.0 / np.sqrt(np.pi) * np.einsum("ab,cd->abcd", Sab, Scd)
    scale = np.abs(lim).max()
    errs = []
    for w in (1e-2, 5e-3):
        v = oracle.prim_eri_erf(la, lb, lc, ld, *ex, A, B, Cc, D, w) / w
        errs.append(np.abs(v - lim).max() / scale)
    assert errs[0] < 1e-3
    assert errs[1] == pytest.approx(errs[0] / 4.0, rel=0.02)


def test_contracted_jk_eight_fold_equals_definition():
    basis, D = W.small_system(["2s1p1d", "1s1p1f", "1s1p"], seed=9)
    o = oracle.Oracle(basis)
    o.set_omega(0.4)
    Q = o.schwarz()
    J0, K0 = o.jk(D, 1e-14, Q, mode=0)
    J1, K1 = o.jk(D, 1e-14, Q, mode=1)
    assert np.abs(J1 - J0).max() < 1e-13 * max(1.0, np.abs(J0).max())
    assert np.abs(K1 - K0).max() < 1e-13 * max(1.0, np.abs(K0).max())
    o.set_omega(0.0)
    Jc, Kc = o.jk(D, 1e-14, Q, mode=1)
    assert np.abs(J1 - Jc).max() > 1e-3  # the operator did change


def test_schwarz_bounds_attenuated_quartets():
    basis, _ = W.small_system(["2s1p1d", "1p1f"], seed=3)
    o = oracle.Oracle(basis)
    Q = o.schwarz().astype(np.float64)
    o.set_omega(0.7)
    assert np.array_equal(o.schwarz(), Q.astype(np.float32))
    ns = basis.nshell
    pi = lambda a, b: a * (a + 1) // 2 + b if a >= b else b * (b + 1) // 2 + a
    for a in range(ns):
        for b in range(ns):
            for c in range(ns):
                for d in range(ns):
                    v = np.abs(o.eri_block(a, b, c, d)).max()
                    assert v <= Q[pi(a, b)] * Q[pi(c, d)] * (1 + 1e-12)


def test_gradient_vs_finite_difference_and_net_force():
    basis, D = W.small_system(["1s1p1d", "2s1p"], seed=21, side=2.5)
    o = oracle.Oracle(basis)
    o.set_omega(0.6)
    Q = o.schwarz()
    g = o.grad(D, 1e-14, Q)
    assert np.abs(g.sum(axis=0)).max() < 1e-10 * max(1.0, np.abs(g).max())
    h = 1e-4
    fd = np.zeros_like(g)
    for a in range(basis.natom):
        for t in range(3):
            e = []
            for sgn in (1, -1):
                c = basis.coords.copy()
                c[a, t] += sgn * h
                o.set_coords(c)
                J, K = o.jk(D, 1e-14, Q)
                e.append(sum(o.energy(D, J, K)))
            fd[a, t] = (e[0] - e[1]) / (2 * h)
    o.set_coords(basis.coords)
    assert np.abs(g - fd).max() < 2e-7 * max(1.0, np.abs(g).max()), (g, fd)
