"""Test-only brute-force quadrature for Gaussian integrals.

Independent of both the oracle and the CUDA path: no recurrence and no Boys
function.  The Coulomb operator is written as
    1/r = (2/sqrt(pi)) int_0^inf exp(-t^2 r^2) dt
(and the long-range erf(omega r)/r as the same integral up to t = omega),
which makes every Cartesian direction separate for fixed t.  Each 1-D (or
coupled 2-D) Gaussian-times-polynomial integral is done exactly by
Gauss-Hermite quadrature after completing the square (a Cholesky map for the
2-D case), and the t-integral by adaptive quadrature (scipy quad_vec).
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad_vec

_GH_X, _GH_W = np.polynomial.hermite.hermgauss(16)  # exact to degree 31


def cart_list(l):
    return [(x, y, l - x - y) for x in range(l, -1, -1) for y in range(l - x, -1, -1)]


def _overlap_1d(i, j, a, b, A, B):
    p = a + b
    P = (a * A + b * B) / p
    x = P + _GH_X / np.sqrt(p)
    return np.exp(-a * b / p * (A - B) ** 2) / np.sqrt(p) * np.sum(_GH_W * (x - A) ** i * (x - B) ** j)


def prim_overlap(la, lb, a, b, A, B):
    out = np.zeros((len(cart_list(la)), len(cart_list(lb))))
    for ia, ca in enumerate(cart_list(la)):
        for ib, cb in enumerate(cart_list(lb)):
            out[ia, ib] = np.prod([_overlap_1d(ca[t], cb[t], a, b, A[t], B[t]) for t in range(3)])
    return out


def _na_1d_all(li, lj, a, b, A, B, Cc, t):
    """table[i][j] of int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2 - t^2 (x-C)^2) dx"""
    p = a + b
    P = (a * A + b * B) / p
    s = p + t * t
    m = (p * P + t * t * Cc) / s
    pref = np.exp(-a * b / p * (A - B) ** 2 - p * t * t / s * (P - Cc) ** 2) / np.sqrt(s)
    x = m + _GH_X / np.sqrt(s)
    return np.array([[pref * np.sum(_GH_W * (x - A) ** i * (x - B) ** j) for j in range(lj + 1)]
                     for i in range(li + 1)])


def prim_nuclear(la, lb, a, b, A, B, Cc):
    ca, cb = cart_list(la), cart_list(lb)

    def f(t):
        tabs = [_na_1d_all(la, lb, a, b, A[k], B[k], Cc[k], t) for k in range(3)]
        return np.array([[np.prod([tabs[k][u[k], v[k]] for k in range(3)]) for v in cb] for u in ca]).ravel()

    val, _ = quad_vec(f, 0.0, np.inf, epsabs=0.0, epsrel=1e-13, limit=400)
    return (2.0 / np.sqrt(np.pi) * val).reshape(len(ca), len(cb))


def _eri_1d_all(li, lj, lk, ll, a, b, c, d, A, B, Cc, D, t):
    """table[i][j][k][l] of the coupled 2-D integral for one direction."""
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * Cc + d * D) / q
    t2 = t * t
    M = np.array([[p + t2, -t2], [-t2, q + t2]])
    rhs = np.array([p * P, q * Q])
    m = np.linalg.solve(M, rhs)
    const = p * P * P + q * Q * Q - rhs @ m
    Lc = np.linalg.cholesky(M)                # M = L L^T
    Linv_T = np.linalg.inv(Lc.T)
    y1, y2 = np.meshgrid(_GH_X, _GH_X, indexing="ij")
    w = np.outer(_GH_W, _GH_W)
    Y = np.stack([y1.ravel(), y2.ravel()])
    X = m[:, None] + Linv_T @ Y
    x1, x2 = X[0], X[1]
    pref = np.exp(-a * b / p * (A - B) ** 2 - c * d / q * (Cc - D) ** 2 - const) / np.sqrt(np.linalg.det(M))
    w = w.ravel()
    out = np.zeros((li + 1, lj + 1, lk + 1, ll + 1))
    pa = [(x1 - A) ** i for i in range(li + 1)]
    pb = [(x1 - B) ** j for j in range(lj + 1)]
    pc = [(x2 - Cc) ** k for k in range(lk + 1)]
    pd = [(x2 - D) ** l for l in range(ll + 1)]
    for i in range(li + 1):
        for j in range(lj + 1):
            ab = w * pa[i] * pb[j]
            for k in range(lk + 1):
                abc = ab * pc[k]
                for l in range(ll + 1):
                    out[i, j, k, l] = pref * np.sum(abc * pd[l])
    return out


def prim_eri(la, lb, lc, ld, a, b, c, d, A, B, Cc, D, t_max=np.inf):
    """Primitive ERI of 1/r, or of erf(omega r)/r = (2/sqrt(pi)) int_0^omega
    exp(-t^2 r^2) dt with t_max = omega."""
    ca, cb, cc, cd = cart_list(la), cart_list(lb), cart_list(lc), cart_list(ld)
    A, B, Cc, D = (np.asarray(v, float) for v in (A, B, Cc, D))

    def f(t):
        tabs = [_eri_1d_all(la, lb, lc, ld, a, b, c, d, A[k], B[k], Cc[k], D[k], t) for k in range(3)]
        out = np.empty((len(ca), len(cb), len(cc), len(cd)))
        for i1, u in enumerate(ca):
            for i2, v in enumerate(cb):
                for i3, w_ in enumerate(cc):
                    for i4, z in enumerate(cd):
                        out[i1, i2, i3, i4] = (tabs[0][u[0], v[0], w_[0], z[0]] * tabs[1][u[1], v[1], w_[1], z[1]]
                                               * tabs[2][u[2], v[2], w_[2], z[2]])
        return out.ravel()

    val, _ = quad_vec(f, 0.0, t_max, epsabs=0.0, epsrel=1e-13, limit=400)
    return (2.0 / np.sqrt(np.pi) * val).reshape(len(ca), len(cb), len(cc), len(cd))
