"""Oracle: plain FP64 CPU reference for the J/K build (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's cpu_baseline /
``--impl reference`` legs may import this package.  The product path (the CUDA
library and its binding) never imports it.  The C source is oracle/oracle.c;
see its header for what each function follows in the paper.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle/oracle.c into oracle/liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", src,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        d, i, f = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_float)
        L.or_boys.argtypes = [C.c_int, C.c_double, d]
        L.or_prim_overlap.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, d, d, d]
        L.or_prim_nuclear.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, d, d, d, d]
        L.or_prim_eri.argtypes = [C.c_int] * 4 + [C.c_double] * 4 + [d] * 5
        L.or_prim_eri_erf.argtypes = [C.c_int] * 4 + [C.c_double] * 4 + [d] * 4 + [C.c_double, d]
        L.or_set_omega.argtypes = [C.c_void_p, C.c_double]
        L.or_nuclear.argtypes = [C.c_void_p, C.c_int, d, d, d]
        L.or_nuclear_grad.argtypes = [C.c_void_p, d, C.c_int, d, d, d, d]
        L.or_create.argtypes = [C.c_int, C.c_int, i, i, i, i, d, d, d]
        L.or_create.restype = C.c_void_p
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_set_coords.argtypes = [C.c_void_p, d]
        L.or_nbf.argtypes = [C.c_void_p]
        L.or_nbf.restype = C.c_int
        L.or_norm_coefs.argtypes = [C.c_void_p, d]
        L.or_overlap_block.argtypes = [C.c_void_p, C.c_int, C.c_int, d]
        L.or_nuclear_block.argtypes = [C.c_void_p, C.c_int, C.c_int, d, d]
        L.or_eri_block.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, d]
        L.or_schwarz.argtypes = [C.c_void_p, f]
        L.or_lists.argtypes = [C.c_void_p, C.c_double, f, i, i]
        L.or_jk.argtypes = [C.c_void_p, d, C.c_double, f, C.c_int, d, d]
        L.or_energy.argtypes = [C.c_int, d, d, d, d, d]
        L.or_jk_quartets.argtypes = [C.c_void_p, d, C.c_int, i, d, d]
        L.or_j_block.argtypes = [C.c_void_p, d, C.c_double, f, C.c_int, C.c_int, d]
        L.or_k_block.argtypes = [C.c_void_p, d, C.c_double, f, C.c_int, C.c_int, d]
        L.or_grad.argtypes = [C.c_void_p, d, C.c_double, f, C.c_int, C.c_int, d]
        L.or_max_threads.restype = C.c_int
        L.or_quartet_batch.argtypes = [C.c_void_p, C.c_int, i]
        L.or_quartet_batch.restype = C.c_double
        i64 = C.c_int64
        L.or_xc_grid_size.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.or_xc_grid_size.restype = i64
        L.or_xc_grid.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, d, d]
        L.or_xc_ao.argtypes = [C.c_void_p, d, d, d]
        L.or_xc_density.argtypes = [C.c_void_p, d, i64, d, d, d]
        L.or_xc_functional.argtypes = [C.c_int, i64, d, d, d, d, d]
        L.or_xc_functional.restype = C.c_int
        L.or_xc_energy.argtypes = [i64, d, d]
        L.or_xc_energy.restype = C.c_double
        L.or_xc_matrix.argtypes = [C.c_void_p, i64, d, d, d, d, d]
        L.or_xc_matrix_elements.argtypes = [C.c_void_p, i64, d, d, d, d, C.c_int, i, d]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def ncart(l):
    return (l + 1) * (l + 2) // 2


def boys(mmax: int, x: float) -> np.ndarray:
    out = np.zeros(mmax + 1)
    lib().or_boys(mmax, float(x), _d(out))
    return out


def _v3(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))


def prim_overlap(la, lb, a, b, A, B):
    out = np.zeros(ncart(la) * ncart(lb))
    lib().or_prim_overlap(la, lb, a, b, _d(_v3(A)), _d(_v3(B)), _d(out))
    return out.reshape(ncart(la), ncart(lb))


def prim_nuclear(la, lb, a, b, A, B, Cc):
    out = np.zeros(ncart(la) * ncart(lb))
    lib().or_prim_nuclear(la, lb, a, b, _d(_v3(A)), _d(_v3(B)), _d(_v3(Cc)), _d(out))
    return out.reshape(ncart(la), ncart(lb))


def prim_eri(la, lb, lc, ld, a, b, c, d, A, B, Cc, D):
    out = np.zeros(ncart(la) * ncart(lb) * ncart(lc) * ncart(ld))
    lib().or_prim_eri(la, lb, lc, ld, a, b, c, d, _d(_v3(A)), _d(_v3(B)), _d(_v3(Cc)), _d(_v3(D)), _d(out))
    return out.reshape(ncart(la), ncart(lb), ncart(lc), ncart(ld))


def prim_eri_erf(la, lb, lc, ld, a, b, c, d, A, B, Cc, D, omega):
    """Primitive long-range ERI [ab| erf(omega r)/r |cd] (Eq. eri_longrange_definition)."""
    out = np.zeros(ncart(la) * ncart(lb) * ncart(lc) * ncart(ld))
    lib().or_prim_eri_erf(la, lb, lc, ld, a, b, c, d, _d(_v3(A)), _d(_v3(B)), _d(_v3(Cc)), _d(_v3(D)),
                          float(omega), _d(out))
    return out.reshape(ncart(la), ncart(lb), ncart(lc), ncart(ld))


def xc_functional(kind, rho, grad):
    """(eps, v_rho, v_grad[G, 3]) of functional `kind` (1 Slater, 2 Becke-88 exchange) at every point."""
    rho = np.ascontiguousarray(rho, np.float64).reshape(-1)
    grad = np.ascontiguousarray(grad, np.float64).reshape(-1, 3)
    G = rho.shape[0]
    eps, vrho, vgrad = np.zeros(G), np.zeros(G), np.zeros((G, 3))
    if lib().or_xc_functional(int(kind), G, _d(rho), _d(grad), _d(eps), _d(vrho), _d(vgrad)) != 0:
        raise ValueError(f"unknown functional {kind}")
    return eps, vrho, vgrad


def xc_energy(w, eps):
    """E_xc = sum_g w_g eps_g (compensated sum)."""
    w = np.ascontiguousarray(w, np.float64).reshape(-1)
    eps = np.ascontiguousarray(eps, np.float64).reshape(-1)
    return float(lib().or_xc_energy(w.shape[0], _d(w), _d(eps)))


def max_threads() -> int:
    return int(lib().or_max_threads())


class Oracle:
    """Oracle over one basis (shells in user order, lexicographic Cartesians)."""

    def __init__(self, basis):
        self.basis = basis
        self._arrs = [np.ascontiguousarray(basis.shell_atom, np.int32),
                      np.ascontiguousarray(basis.shell_l, np.int32),
                      np.ascontiguousarray(basis.shell_nprim, np.int32),
                      np.ascontiguousarray(basis.shell_prim_offset, np.int32),
                      np.ascontiguousarray(basis.exps, np.float64),
                      np.ascontiguousarray(basis.coefs, np.float64),
                      np.ascontiguousarray(basis.coords, np.float64)]
        a = self._arrs
        self.h = lib().or_create(basis.nshell, basis.natom, _i(a[0]), _i(a[1]), _i(a[2]), _i(a[3]),
                                 _d(a[4]), _d(a[5]), _d(a[6]))
        self.nbf = lib().or_nbf(self.h)
        self.l = basis.shell_l.astype(int)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_destroy(self.h)
            self.h = None

    def set_omega(self, omega):
        """Two-electron operator of every later ERI / J / K / gradient call:
        0 = 1/r, omega > 0 = erf(omega r)/r.  Schwarz bounds stay Coulomb."""
        lib().or_set_omega(self.h, float(omega))

    def set_coords(self, coords):
        c = np.ascontiguousarray(coords, np.float64)
        self._arrs[6] = c
        lib().or_set_coords(self.h, _d(c))

    def norm_coefs(self):
        out = np.zeros(self.basis.exps.shape[0])
        lib().or_norm_coefs(self.h, _d(out))
        return out

    def overlap_block(self, a, b):
        out = np.zeros(ncart(self.l[a]) * ncart(self.l[b]))
        lib().or_overlap_block(self.h, a, b, _d(out))
        return out.reshape(ncart(self.l[a]), ncart(self.l[b]))

    def nuclear_block(self, a, b, Cc):
        out = np.zeros(ncart(self.l[a]) * ncart(self.l[b]))
        lib().or_nuclear_block(self.h, a, b, _d(_v3(Cc)), _d(out))
        return out.reshape(ncart(self.l[a]), ncart(self.l[b]))

    def nuclear(self, q, Cxyz):
        """V_mn = sum_C q_C (m|1/|r-C||n) over point charges q[nc] at Cxyz[nc, 3]."""
        q = np.ascontiguousarray(q, np.float64).reshape(-1)
        Cc = np.ascontiguousarray(Cxyz, np.float64).reshape(-1, 3)
        V = np.zeros((self.nbf, self.nbf))
        lib().or_nuclear(self.h, int(q.shape[0]), _d(q), _d(Cc), _d(V))
        return V

    def nuclear_grad(self, D, q, Cxyz):
        """(dE/dR [natom, 3], dE/dC [nc, 3]) of E_V = sum D_mn V_mn, D fixed."""
        q = np.ascontiguousarray(q, np.float64).reshape(-1)
        Cc = np.ascontiguousarray(Cxyz, np.float64).reshape(-1, 3)
        gA = np.zeros((self.basis.natom, 3))
        gC = np.zeros((q.shape[0], 3))
        lib().or_nuclear_grad(self.h, _d(np.ascontiguousarray(D, np.float64)), int(q.shape[0]), _d(q), _d(Cc),
                              _d(gA), _d(gC))
        return gA, gC

    def xc_grid(self, nrad, ntheta, radius=1.0):
        """(points [G, 3], weights [G]) of the molecular grid (Sec. 2.6 step 1; readings in oracle.c)."""
        G = int(lib().or_xc_grid_size(self.h, int(nrad), int(ntheta)))
        pts, w = np.zeros((G, 3)), np.zeros(G)
        lib().or_xc_grid(self.h, int(nrad), int(ntheta), float(radius), _d(pts), _d(w))
        return pts, w

    def xc_ao(self, r):
        """(phi [nbf], grad phi [3, nbf]) of every basis function at point r."""
        phi, dphi = np.zeros(self.nbf), np.zeros((3, self.nbf))
        lib().or_xc_ao(self.h, _d(_v3(r)), _d(phi), _d(dphi))
        return phi, dphi

    def xc_density(self, D, pts):
        """(rho [G], grad rho [G, 3]) at points (Eq. xc_density_0, Eq. xc_density_1)."""
        pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        G = pts.shape[0]
        rho, grad = np.zeros(G), np.zeros((G, 3))
        lib().or_xc_density(self.h, _d(np.ascontiguousarray(D, np.float64)), G, _d(pts), _d(rho), _d(grad))
        return rho, grad

    def xc_matrix(self, pts, w, vrho, vgrad):
        """V_mn of Eq. xc_grid_sum_0 + Eq. xc_grid_sum_1 for given point potentials."""
        pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, np.float64).reshape(-1)
        vrho = np.ascontiguousarray(vrho, np.float64).reshape(-1)
        vgrad = np.ascontiguousarray(vgrad, np.float64).reshape(-1, 3)
        V = np.zeros((self.nbf, self.nbf))
        lib().or_xc_matrix(self.h, pts.shape[0], _d(pts), _d(w), _d(vrho), _d(vgrad), _d(V))
        return V

    def xc_matrix_elements(self, pts, w, vrho, vgrad, mn):
        """Selected elements V[m, n] for index pairs mn [k, 2] (each a full sum over the points)."""
        pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, np.float64).reshape(-1)
        vrho = np.ascontiguousarray(vrho, np.float64).reshape(-1)
        vgrad = np.ascontiguousarray(vgrad, np.float64).reshape(-1, 3)
        mn = np.ascontiguousarray(mn, np.int32).reshape(-1, 2)
        out = np.zeros(mn.shape[0])
        lib().or_xc_matrix_elements(self.h, pts.shape[0], _d(pts), _d(w), _d(vrho), _d(vgrad), mn.shape[0],
                                    _i(mn), _d(out))
        return out

    def xc(self, D, nrad, ntheta, kind, radius=1.0):
        """(E_xc, V_xc) of functional `kind` on the molecular grid: steps (1)-(4) of Sec. 2.6."""
        pts, w = self.xc_grid(nrad, ntheta, radius)
        rho, grad = self.xc_density(D, pts)
        eps, vrho, vgrad = xc_functional(kind, rho, grad)
        return xc_energy(w, eps), self.xc_matrix(pts, w, vrho, vgrad)

    def eri_block(self, a, b, c, d):
        sh = [ncart(self.l[s]) for s in (a, b, c, d)]
        out = np.zeros(int(np.prod(sh)))
        lib().or_eri_block(self.h, a, b, c, d, _d(out))
        return out.reshape(sh)

    def schwarz(self) -> np.ndarray:
        ns = self.basis.nshell
        Q = np.zeros(ns * (ns + 1) // 2, np.float32)
        lib().or_schwarz(self.h, _f(Q))
        return Q

    def lists(self, thresh, Q):
        npair = Q.shape[0]
        sig = np.zeros(npair, np.int32)
        counts = np.zeros(npair * 10, np.int32)
        lib().or_lists(self.h, float(thresh), _f(np.ascontiguousarray(Q, np.float32)), _i(sig), _i(counts))
        return sig, counts.reshape(npair, 10)

    def jk(self, D, thresh=1e-12, Q=None, mode=1):
        Q = self.schwarz() if Q is None else np.ascontiguousarray(Q, np.float32)
        D = np.ascontiguousarray(D, np.float64)
        J = np.zeros((self.nbf, self.nbf))
        K = np.zeros((self.nbf, self.nbf))
        lib().or_jk(self.h, _d(D), float(thresh), _f(Q), int(mode), _d(J), _d(K))
        return J, K

    def jk_quartets(self, D, abcd, J=None, K=None):
        """Add the J / K contributions of explicit canonical quartets abcd[n, 4]."""
        J = np.zeros((self.nbf, self.nbf)) if J is None else J
        K = np.zeros((self.nbf, self.nbf)) if K is None else K
        a = np.ascontiguousarray(abcd, np.int32).reshape(-1, 4)
        lib().or_jk_quartets(self.h, _d(np.ascontiguousarray(D, np.float64)), int(a.shape[0]), _i(a), _d(J), _d(K))
        return J, K

    def energy(self, D, J, K):
        ej, ek = C.c_double(), C.c_double()
        lib().or_energy(self.nbf, _d(np.ascontiguousarray(D)), _d(np.ascontiguousarray(J)),
                        _d(np.ascontiguousarray(K)), C.byref(ej), C.byref(ek))
        return ej.value, ek.value

    def j_block(self, D, a, b, thresh=1e-12, Q=None):
        Q = self.schwarz() if Q is None else np.ascontiguousarray(Q, np.float32)
        out = np.zeros(ncart(self.l[a]) * ncart(self.l[b]))
        lib().or_j_block(self.h, _d(np.ascontiguousarray(D)), float(thresh), _f(Q), a, b, _d(out))
        return out.reshape(ncart(self.l[a]), ncart(self.l[b]))

    def k_block(self, D, a, c, thresh=1e-12, Q=None):
        Q = self.schwarz() if Q is None else np.ascontiguousarray(Q, np.float32)
        out = np.zeros(ncart(self.l[a]) * ncart(self.l[c]))
        lib().or_k_block(self.h, _d(np.ascontiguousarray(D)), float(thresh), _f(Q), a, c, _d(out))
        return out.reshape(ncart(self.l[a]), ncart(self.l[c]))

    def quartet_batch(self, abcd):
        """Evaluate contracted quartets abcd[n, 4] (sum of |ERI| returned)."""
        a = np.ascontiguousarray(abcd, np.int32)
        return lib().or_quartet_batch(self.h, int(a.shape[0]), _i(a))

    def grad(self, D, thresh=1e-12, Q=None, want_j=True, want_k=True):
        Q = self.schwarz() if Q is None else np.ascontiguousarray(Q, np.float32)
        g = np.zeros(self.basis.natom * 3)
        lib().or_grad(self.h, _d(np.ascontiguousarray(D)), float(thresh), _f(Q), int(want_j), int(want_k), _d(g))
        return g.reshape(self.basis.natom, 3)
