"""Pins for the oracle's screening, J/K assembly and energies.

- the Cauchy-Schwarz bound (paper Eq. cauchy_schwarz_bound) holds for every
  shell quartet of workload 0, and Q is sqrt(max diagonal ERI) rounded up to
  float32;
- lists: the significance counts follow the quartet test on Q;
- J and K over canonical quartets with 8-fold weights equal the plain
  definitions Eq. j_definition / Eq. k_definition summed over every ordered
  quartet (the classic place for factor-of-two slips);
- E(D) = 1/2 tr(D J) - 1/4 tr(D K) is quadratic in D with gradient J - K/2
  (SI Eq. si_E_J_K), so a central difference in D is exact;
- J and K are symmetric for symmetric D.
"""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def w0():
    basis, D = W.workload(0)
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    return basis, D, o, Q


def test_schwarz_bound_and_rounding(w0):
    basis, D, o, Q = w0
    ns = basis.nshell
    pidx = lambda a, b: a * (a + 1) // 2 + b if a >= b else b * (b + 1) // 2 + a
    for a in range(ns):
        for b in range(a + 1):
            X = o.eri_block(a, b, a, b)
            na, nb = X.shape[0], X.shape[1]
            diag = max(abs(X[i, j, i, j]) for i in range(na) for j in range(nb))
            q = float(Q[pidx(a, b)])
            ex = np.sqrt(diag)
            assert q >= ex and float(np.nextafter(np.float32(q), np.float32(0))) < ex
    rng = np.random.default_rng(1)
    for _ in range(400):
        a, b, c, d = rng.integers(0, ns, 4)
        X = o.eri_block(a, b, c, d)
        assert np.abs(X).max() <= float(Q[pidx(a, b)]) * float(Q[pidx(c, d)]) * (1 + 1e-12)


def test_lists_counts(w0):
    basis, D, o, Q = w0
    thresh = 1e-7  # large enough that some quartets drop out
    sig, counts = o.lists(thresh, Q)
    ns = basis.nshell
    cls = {}
    for a in range(ns):
        for b in range(a + 1):
            hi, lo = max(basis.shell_l[a], basis.shell_l[b]), min(basis.shell_l[a], basis.shell_l[b])
            cls[a * (a + 1) // 2 + b] = hi * (hi + 1) // 2 + lo
    qmax = float(Q.max())
    dropped = 0
    for i in range(Q.shape[0]):
        assert sig[i] == (float(Q[i]) * qmax >= thresh)
        ref = np.zeros(10, int)
        for j in range(Q.shape[0]):
            if sig[i] and sig[j] and float(Q[i]) * float(Q[j]) >= thresh:
                ref[cls[j]] += 1
            elif sig[i] and sig[j]:
                dropped += 1
        assert np.array_equal(counts[i], ref)
    assert dropped > 0


def test_jk_eightfold_equals_definition(w0):
    basis, D, o, Q = w0
    J1, K1 = o.jk(D, 1e-12, Q, mode=1)
    J0, K0 = o.jk(D, 1e-12, Q, mode=0)
    assert np.allclose(J1, J0, rtol=0, atol=1e-13 * np.abs(J0).max())
    assert np.allclose(K1, K0, rtol=0, atol=1e-13 * np.abs(K0).max())
    assert np.allclose(J1, J1.T, atol=1e-14 * np.abs(J1).max())
    assert np.allclose(K1, K1.T, atol=1e-14 * np.abs(K1).max())


def test_jk_eightfold_equals_definition_thresholded():
    basis, D = W.small_system(["2s2p1d1f", "1s1p1d"], seed=11)
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    for thresh in (1e-6, 1e-3):
        J1, K1 = o.jk(D, thresh, Q, mode=1)
        J0, K0 = o.jk(D, thresh, Q, mode=0)
        assert np.allclose(J1, J0, rtol=0, atol=1e-13 * np.abs(J0).max())
        assert np.allclose(K1, K0, rtol=0, atol=1e-13 * np.abs(K0).max())


def test_energy_gradient_in_density():
    basis, D = W.small_system(["2s1p1d", "1s1p1f"], seed=2)
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    rng = np.random.default_rng(3)
    X = rng.standard_normal(D.shape)
    X = X + X.T

    def E(Dm):
        J, K = o.jk(Dm, 1e-14, Q)
        ej, ek = o.energy(Dm, J, K)
        return ej + ek

    J, K = o.jk(D, 1e-14, Q)
    h = 1e-3
    fd = (E(D + h * X) - E(D - h * X)) / (2 * h)
    assert fd == pytest.approx(np.sum(X * (J - 0.5 * K)), rel=1e-11)


def test_sampled_blocks_match_full(w0):
    basis, D, o, Q = w0
    J, K = o.jk(D, 1e-12, Q)
    off = basis.ao_offsets()
    for a, b in [(0, 0), (3, 10), (20, 6), (13, 13)]:
        jb = o.j_block(D, a, b, 1e-12, Q)
        assert np.allclose(jb, J[off[a]:off[a + 1], off[b]:off[b + 1]], atol=1e-13 * np.abs(J).max())
        kb = o.k_block(D, a, b, 1e-12, Q)
        assert np.allclose(kb, K[off[a]:off[a + 1], off[b]:off[b + 1]], atol=1e-13 * np.abs(K).max())
