"""Pins for the oracle's integrals.

- primitive overlap / point-charge attraction / ERIs against brute-force
  quadrature (tests/quadrature.py: no recurrence, no Boys function);
- (ss|ss) of four identical normalised s Gaussians on one centre equals
  2 sqrt(alpha/pi) (from the base case, paper Eq. eri_base_case, with F_0(0)=1);
- unit self-overlap of every normalised function (Eq. overlap_formula);
- point-charge limit: a charge-normalised ket Gaussian of exponent c -> inf
  turns the ERI into the attraction integral V (Eq. v1e_definition2);
- far-field limit: R (mu nu|lambda sigma) -> S_mu_nu S_lambda_sigma;
- 8-fold permutational symmetry (Eq. 8_fold_symmetry);
- translation invariance and signed axis permutations.
"""
import itertools

import numpy as np
import pytest

import oracle
import quadrature as quad
import workloads as W

RNG = np.random.default_rng(20240614)


def _centres(n, scale=1.3):
    return [RNG.normal(0.0, scale, 3) for _ in range(n)]


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (2, 1), (3, 3), (4, 2)])
def test_prim_overlap_vs_quadrature(la, lb):
    A, B = _centres(2)
    a, b = 0.7, 1.9
    got = oracle.prim_overlap(la, lb, a, b, A, B)
    ref = quad.prim_overlap(la, lb, a, b, A, B)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (1, 1), (2, 1), (3, 2)])
def test_prim_nuclear_vs_quadrature(la, lb):
    A, B, Cc = _centres(3)
    a, b = 0.9, 0.45
    got = oracle.prim_nuclear(la, lb, a, b, A, B, Cc)
    ref = quad.prim_nuclear(la, lb, a, b, A, B, Cc)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("ls", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (1, 1, 1, 1),
                                (0, 1, 1, 0), (2, 1, 1, 0), (2, 2, 1, 1), (3, 1, 2, 0), (3, 3, 1, 0),
                                (2, 0, 3, 2), (4, 1, 2, 1)])
def test_prim_eri_vs_quadrature(ls):
    la, lb, lc, ld = ls
    A, B, Cc, D = _centres(4, 0.9)
    ex = (0.8, 1.6, 0.55, 2.3)
    got = oracle.prim_eri(la, lb, lc, ld, *ex, A, B, Cc, D)
    ref = quad.prim_eri(la, lb, lc, ld, *ex, A, B, Cc, D)
    scale = np.abs(ref).max()
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-12 * scale), np.abs(got - ref).max() / scale


def _single_shell_basis(l, exps, coefs, centre=(0.0, 0.0, 0.0)):
    n = len(exps)
    return W.Basis(np.array([0], np.int32), np.array([l], np.int32), np.array([n], np.int32),
                   np.array([0], np.int32), np.array(exps, float), np.array(coefs, float),
                   np.array([centre], float))


@pytest.mark.parametrize("alpha", [0.13, 1.0, 7.5, 2.0e4])
def test_ssss_same_centre_closed_form(alpha):
    o = oracle.Oracle(_single_shell_basis(0, [alpha], [0.37]))
    v = o.eri_block(0, 0, 0, 0)[0, 0, 0, 0]
    assert v == pytest.approx(2.0 * np.sqrt(alpha / np.pi), rel=1e-14)


def test_unit_self_overlap_all_functions():
    for i in (0, 2):
        basis, _ = W.workload(i)
        o = oracle.Oracle(basis)
        for s in range(basis.nshell):
            S = o.overlap_block(s, s)
            assert np.allclose(np.diag(S), 1.0, rtol=0, atol=2e-14), (s, np.diag(S))


def test_contracted_overlap_vs_quadrature():
    basis, _ = W.workload(0)
    o = oracle.Oracle(basis)
    cn = o.norm_coefs()
    from math import prod

    def fac(c):
        df = lambda n: prod(range(n, 0, -2)) if n > 0 else 1
        l = sum(c)
        return np.sqrt(df(2 * l - 1) / (df(2 * c[0] - 1) * df(2 * c[1] - 1) * df(2 * c[2] - 1)))

    for sa, sb in [(0, 3), (3, 5), (6, 13), (7, 20)]:
        la, lb = int(basis.shell_l[sa]), int(basis.shell_l[sb])
        A, B = basis.coords[basis.shell_atom[sa]], basis.coords[basis.shell_atom[sb]]
        ref = np.zeros((len(quad.cart_list(la)), len(quad.cart_list(lb))))
        for ka in range(basis.shell_nprim[sa]):
            for kb in range(basis.shell_nprim[sb]):
                pa, pb = basis.shell_prim_offset[sa] + ka, basis.shell_prim_offset[sb] + kb
                ref += cn[pa] * cn[pb] * quad.prim_overlap(la, lb, basis.exps[pa], basis.exps[pb], A, B)
        fa = np.array([fac(c) for c in quad.cart_list(la)])
        fb = np.array([fac(c) for c in quad.cart_list(lb)])
        ref *= np.outer(fa, fb)
        assert np.allclose(o.overlap_block(sa, sb), ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 0), (2, 1), (3, 0), (3, 3)])
def test_point_charge_limit(la, lb):
    """(mu nu| (c/pi)^(3/2) exp(-c|r-C|^2)) -> V_mu_nu(C) as c -> inf, error O(1/c)."""
    A, B, Cc = np.array([0.1, -0.3, 0.2]), np.array([0.9, 0.4, -0.5]), np.array([-0.6, 1.1, 0.8])
    a, b = 0.8, 1.3
    V = oracle.prim_nuclear(la, lb, a, b, A, B, Cc)
    vals = {}
    for c in (1e4, 1e5, 1e6):
        e = oracle.prim_eri(la, lb, 0, 0, a, b, c / 2, c / 2, A, B, Cc, Cc)[:, :, 0, 0]
        vals[c] = e * (c / np.pi) ** 1.5
    scale = np.abs(V).max()
    errs = [np.abs(vals[c] - V).max() / scale for c in (1e4, 1e5, 1e6)]
    assert errs[2] < 2e-5
    assert errs[1] < errs[0] * 0.2 and errs[2] < errs[1] * 0.2  # O(1/c)
    rich = (1e6 * vals[1e6] - 1e5 * vals[1e5]) / (1e6 - 1e5)  # first-order Richardson
    assert np.abs(rich - V).max() / scale < 1e-8


def test_far_field_limit():
    """R * (mu nu|lambda sigma) -> S_mu_nu S_lambda_sigma for |bra - ket| = R -> inf."""
    basis, _ = W.workload(0)
    o = oracle.Oracle(basis)
    shells = {l: [s for s in range(basis.nshell) if basis.shell_l[s] == l] for l in range(4)}
    a, b = shells[3][0], shells[2][1]   # f on atom 0, d on atom 1
    c, d = shells[1][4], shells[3][2]   # p on atom 2, f on atom 2
    direction = np.array([0.36, -0.48, 0.8])
    devs = []
    for R in (100.0, 200.0, 400.0):
        coords = basis.coords.copy()
        coords[2] = coords[0] + R * direction
        o.set_coords(coords)
        eri = o.eri_block(a, b, c, d)
        Sab = o.overlap_block(a, b)
        Scd = o.overlap_block(c, d)
        mono = np.einsum("ij,kl->ijkl", Sab, Scd)
        # the distance that matters is between the charge centres; use the
        # atom-atom distance and allow O(1/R) corrections from the offset
        devs.append(np.abs(R * eri - mono).max() / np.abs(mono).max())
    assert devs[2] < 0.05
    assert devs[1] < 0.6 * devs[0] and devs[2] < 0.6 * devs[1]


def test_eight_fold_symmetry():
    basis, _ = W.workload(0)
    o = oracle.Oracle(basis)
    # f(atom0) p(atom1) | d(atom2) s(atom1): mixed centres and classes
    sh = {l: [s for s in range(basis.nshell) if basis.shell_l[s] == l] for l in range(4)}
    a, b, c, d = sh[3][0], sh[1][2], sh[2][2], sh[0][4]
    X = o.eri_block(a, b, c, d)
    perms = {
        (b, a, c, d): X.transpose(1, 0, 2, 3),
        (a, b, d, c): X.transpose(0, 1, 3, 2),
        (b, a, d, c): X.transpose(1, 0, 3, 2),
        (c, d, a, b): X.transpose(2, 3, 0, 1),
        (d, c, a, b): X.transpose(3, 2, 0, 1),
        (c, d, b, a): X.transpose(2, 3, 1, 0),
        (d, c, b, a): X.transpose(3, 2, 1, 0),
    }
    for key, ref in perms.items():
        Y = o.eri_block(*key)
        assert np.allclose(Y, ref, rtol=1e-12, atol=1e-13 * np.abs(X).max()), key


def test_translation_invariance():
    basis, D = W.small_system(["2s1p1d", "1s1p1f"], seed=3)
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    J, K = o.jk(D, 1e-12, Q)
    o.set_coords(basis.coords + np.array([3.7, -12.1, 0.45]))
    Q2 = o.schwarz()
    J2, K2 = o.jk(D, 1e-12, Q2)
    assert np.allclose(J, J2, rtol=1e-12, atol=1e-13 * np.abs(J).max())
    assert np.allclose(K, K2, rtol=1e-12, atol=1e-13 * np.abs(K).max())


def test_signed_axis_permutation():
    """r' = P r with P a signed permutation: every Cartesian function maps to one
    function with permuted exponents and a sign, so J' = S J S^T, K' = S K S^T."""
    basis, D = W.small_system(["1s1p1d", "1s1p1f"], seed=5)
    perm, sign = (2, 0, 1), np.array([-1.0, 1.0, -1.0])   # x' = -z, y' = x, z' = -y
    P = np.zeros((3, 3))
    for k in range(3):
        P[k, perm[k]] = sign[k]
    n = basis.nbf
    S = np.zeros((n, n))
    off = basis.ao_offsets()
    for s in range(basis.nshell):
        l = int(basis.shell_l[s])
        comps = quad.cart_list(l)
        for i, e in enumerate(comps):
            # new function x'^e0 y'^e1 z'^e2 = prod_k (sign_k r_perm[k])^e_k
            old = [0, 0, 0]
            sgn = 1.0
            for k in range(3):
                old[perm[k]] += e[k]
                sgn *= sign[k] ** e[k]
            S[off[s] + i, off[s] + comps.index(tuple(old))] = sgn
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    J, K = o.jk(D, 1e-14, Q)
    Dn = S @ D @ S.T
    o.set_coords(basis.coords @ P.T)
    Q2 = o.schwarz()
    assert np.array_equal(Q, Q2) or np.allclose(Q, Q2, rtol=1e-6)
    J2, K2 = o.jk(Dn, 1e-14, Q2)
    assert np.allclose(J2, S @ J @ S.T, rtol=1e-12, atol=1e-13 * np.abs(J).max())
    assert np.allclose(K2, S @ K @ S.T, rtol=1e-12, atol=1e-13 * np.abs(K).max())
    e1, e2 = o.energy(D, J, K), o.energy(Dn, J2, K2)
    assert e1[0] == pytest.approx(e2[0], rel=1e-13) and e1[1] == pytest.approx(e2[1], rel=1e-13)
