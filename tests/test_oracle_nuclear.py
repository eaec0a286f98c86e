"""Pins for the oracle's point-charge attraction matrix and its gradient
(paper Sec. 2.4, Eq. v1e_definition, Eq. v1e_summation_over_C; the
derivatives of SI Sec. 1.3).

- V equals the sum over charges of the separately written one-charge blocks
  (or_nuclear_block, pinned at primitive level by quadrature and by the
  point-charge limit of the ERIs in test_oracle_integrals.py), and is
  symmetric;
- V is unchanged when the molecule and the charges move together;
- the gradient of E_V = sum D V with respect to the basis centres and to the
  charge positions equals central finite differences (h = 1e-4 bohr), and the
  forces on atoms and charges sum to zero (translational invariance);
- a unit charge at the position of a distant point: V -> S / R (monopole).
"""
import numpy as np

import oracle
import workloads as W


def _charges(rng, n, centre, spread=3.0):
    return rng.uniform(-1.0, 1.0, n), centre + rng.normal(0.0, spread, (n, 3))


def test_matrix_equals_sum_of_one_charge_blocks():
    basis, _ = W.small_system(["2s1p1d1f", "1s1p1d"], seed=5)
    rng = np.random.default_rng(4)
    q, Cc = _charges(rng, 5, basis.coords.mean(axis=0))
    o = oracle.Oracle(basis)
    V = o.nuclear(q, Cc)
    off = basis.ao_offsets()
    for a in range(basis.nshell):
        for b in range(basis.nshell):
            ref = sum(qk * o.nuclear_block(a, b, ck) for qk, ck in zip(q, Cc))
            assert np.allclose(V[off[a]:off[a + 1], off[b]:off[b + 1]], ref, rtol=1e-13, atol=1e-14)
    assert np.abs(V - V.T).max() < 1e-13 * np.abs(V).max()


def test_translation_invariance():
    basis, _ = W.small_system(["1s1p1d", "1p1f"], seed=6)
    rng = np.random.default_rng(7)
    q, Cc = _charges(rng, 4, basis.coords.mean(axis=0))
    V0 = oracle.Oracle(basis).nuclear(q, Cc)
    shift = np.array([0.7, -1.3, 2.1])
    V1 = oracle.Oracle(basis.with_coords(basis.coords + shift)).nuclear(q, Cc + shift)
    assert np.abs(V1 - V0).max() < 1e-12 * np.abs(V0).max()


def test_far_charge_monopole_limit():
    basis, _ = W.small_system(["1s1p", "1d"], seed=8)
    o = oracle.Oracle(basis)
    n = basis.nbf
    S = np.zeros((n, n))
    off = basis.ao_offsets()
    for a in range(basis.nshell):
        for b in range(basis.nshell):
            S[off[a]:off[a + 1], off[b]:off[b + 1]] = o.overlap_block(a, b)
    errs = []
    for R in (200.0, 400.0):
        Cc = basis.coords.mean(axis=0) + np.array([[R, 0.0, 0.0]])
        V = o.nuclear(np.array([1.0]), Cc)
        errs.append(np.abs(V * R - S).max())
    assert errs[0] < 5e-2 and errs[1] < errs[0] / 1.8  # O(1/R) dipole correction


def test_gradient_vs_finite_difference_and_net_force():
    basis, D = W.small_system(["1s1p1d", "2s1p", "1p1f"], seed=21, side=3.0)
    rng = np.random.default_rng(9)
    q, Cc = _charges(rng, 3, basis.coords.mean(axis=0), spread=2.0)
    o = oracle.Oracle(basis)
    gA, gC = o.nuclear_grad(D, q, Cc)
    assert np.abs(gA.sum(axis=0) + gC.sum(axis=0)).max() < 1e-11 * max(1.0, np.abs(gA).max())
    h = 1e-4

    def ev(coords, charges):
        o.set_coords(coords)
        return float((D * o.nuclear(q, charges)).sum())

    for a in range(basis.natom):
        for t in range(3):
            cp = basis.coords.copy(); cp[a, t] += h
            cm = basis.coords.copy(); cm[a, t] -= h
            fd = (ev(cp, Cc) - ev(cm, Cc)) / (2 * h)
            assert abs(fd - gA[a, t]) < 1e-7 * max(1.0, abs(fd)), (a, t, fd, gA[a, t])
    for k in range(len(q)):
        for t in range(3):
            cp = Cc.copy(); cp[k, t] += h
            cm = Cc.copy(); cm[k, t] -= h
            fd = (ev(basis.coords, cp) - ev(basis.coords, cm)) / (2 * h)
            assert abs(fd - gC[k, t]) < 1e-7 * max(1.0, abs(fd)), (k, t, fd, gC[k, t])
    o.set_coords(basis.coords)
