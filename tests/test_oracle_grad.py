"""Pins for the oracle's nuclear gradient (SI Sec. 1.4, Eq. si_E_J_K).

The oracle differentiates all four centres of every ordered quartet.  It is
checked against central finite differences of its own energy with the lists
frozen (Schwarz Q held at the reference geometry), and for zero net force
(translational invariance).
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _energy(o, D, Q, thresh, want_j=True, want_k=True):
    J, K = o.jk(D, thresh, Q)
    ej, ek = o.energy(D, J, K)
    return (ej if want_j else 0.0) + (ek if want_k else 0.0)


@pytest.mark.parametrize("want", [(True, False), (False, True), (True, True)])
def test_gradient_vs_finite_difference(want):
    basis, D = W.small_system(["1s1p1d", "2s1p1f"], seed=21, side=2.5)
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    thresh = 1e-14
    g = o.grad(D, thresh, Q, *want)
    h = 1e-4
    fd = np.zeros_like(g)
    for a in range(basis.natom):
        for t in range(3):
            cp = basis.coords.copy(); cp[a, t] += h
            cm = basis.coords.copy(); cm[a, t] -= h
            o.set_coords(cp); ep = _energy(o, D, Q, thresh, *want)
            o.set_coords(cm); em = _energy(o, D, Q, thresh, *want)
            fd[a, t] = (ep - em) / (2 * h)
    o.set_coords(basis.coords)
    assert np.allclose(g, fd, rtol=0, atol=2e-8 * max(1.0, np.abs(g).max())), (g, fd)
    assert np.abs(g.sum(axis=0)).max() < 1e-10 * max(1.0, np.abs(g).max())


@pytest.mark.slow
def test_gradient_workload0_fd_spot():
    basis, D = W.workload(0)
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    g = o.grad(D, 1e-12, Q)
    assert np.abs(g.sum(axis=0)).max() < 1e-10 * np.abs(g).max()
    h = 1e-4
    for a, t in [(0, 0), (2, 1)]:
        cp = basis.coords.copy(); cp[a, t] += h
        cm = basis.coords.copy(); cm[a, t] -= h
        o.set_coords(cp); ep = _energy(o, D, Q, 1e-12)
        o.set_coords(cm); em = _energy(o, D, Q, 1e-12)
        assert g[a, t] == pytest.approx((ep - em) / (2 * h), abs=2e-8 * np.abs(g).max())
    o.set_coords(basis.coords)
