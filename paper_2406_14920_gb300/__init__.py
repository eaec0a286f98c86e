"""GB300-native integral-direct Coulomb (J) and exchange (K) library.

Thin Python binding over the C ABI of include/eri.h (libgb300eri.so, built
in-tree by ``paper_2406_14920_gb300.build.build()``).  This module only
marshals arguments: every step of the J/K build runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  There is no CPU
fallback: if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgb300eri.so")
_lib = None

ERI_FP64 = 0
ERI_MIXED = 1
ERI_XC_SLATER = 1
ERI_XC_B88 = 2


class EriError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what} failed: {strerror(code)} ({code})")
        self.code = code


class ShellT(C.Structure):
    _fields_ = [("atom", C.c_int32), ("l", C.c_int32), ("nprim", C.c_int32), ("prim_offset", C.c_int32)]


class BasisT(C.Structure):
    _fields_ = [("nshell", C.c_int32), ("natom", C.c_int32), ("shells", C.POINTER(ShellT)),
                ("exps", C.POINTER(C.c_double)), ("coefs", C.POINTER(C.c_double))]


class OptsT(C.Structure):
    _fields_ = [("thresh", C.c_double), ("precision", C.c_int32), ("mixed_tau", C.c_double),
                ("device", C.c_int32), ("j_engine", C.c_int32), ("profile", C.c_int32),
                ("tune_cache", C.c_char_p), ("deterministic", C.c_int32), ("density_screen", C.c_int32)]


class LaunchProfT(C.Structure):
    _fields_ = [("bra_class", C.c_int32), ("ket_class", C.c_int32), ("tier", C.c_int32), ("launches", C.c_int32),
                ("ms", C.c_double), ("quartets", C.c_int64), ("prim_quartets", C.c_int64), ("flops", C.c_double)]


class StatsT(C.Structure):
    _fields_ = [("nbf", C.c_int32), ("nshell", C.c_int32), ("npair", C.c_int32), ("nsig_pair", C.c_int32),
                ("quartets_k", C.c_int64), ("quartets_j", C.c_int64), ("prim_quartets_k", C.c_int64),
                ("quartets_k_fp32", C.c_int64), ("flops_k", C.c_double), ("flops_j", C.c_double),
                ("device_status", C.c_int32), ("quartets_k_guard", C.c_int64), ("quartets_k_screened", C.c_int64),
                ("graph_branches", C.c_int32), ("quartets_j_fp32", C.c_int64)]


class XcStatsT(C.Structure):
    _fields_ = [("npoints", C.c_int64), ("nblock", C.c_int32), ("block_points", C.c_int32),
                ("resident", C.c_int32), ("nchunk", C.c_int32), ("sum_block_functions", C.c_double),
                ("sum_block_functions_sq", C.c_double), ("workspace_bytes", C.c_double),
                ("flops_density", C.c_double), ("flops_matrix", C.c_double)]


def lib():
    """Load libgb300eri.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2406_14920_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        vp, d, i32 = C.c_void_p, C.POINTER(C.c_double), C.c_int32
        L.eri_default_opts.argtypes = [C.POINTER(OptsT)]
        L.eri_plan.argtypes = [C.POINTER(BasisT), d, C.POINTER(OptsT), C.POINTER(vp)]
        L.eri_plan_batch.argtypes = [i32, C.POINTER(C.POINTER(BasisT)), C.POINTER(d), C.POINTER(OptsT),
                                     C.POINTER(vp)]
        L.eri_plan_layout.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int32)]
        L.eri_plan_set_coords.argtypes = [vp, vp, i32, vp]
        L.eri_build_jk.argtypes = [vp, vp, vp, vp, C.c_double, i32, vp]
        L.eri_build_jk_graph.argtypes = [vp, vp, vp, vp, i32, vp]
        L.eri_autotune.argtypes = [vp, vp, i32, C.c_double, vp]
        L.eri_get_tiles.argtypes = [vp, C.POINTER(C.c_int32)]
        L.eri_plan_set_shard.argtypes = [vp, i32, i32]
        L.eri_plan_set_omega.argtypes = [vp, C.c_double]
        L.eri_plan_set_tau.argtypes = [vp, C.c_double]
        L.eri_set_tiles.argtypes = [vp, C.POINTER(C.c_int32)]
        L.eri_energy.argtypes = [vp, vp, vp, vp, vp, vp]
        L.eri_jk_grad.argtypes = [vp, vp, vp, i32, i32, vp]
        L.eri_jk_grad_prec.argtypes = [vp, vp, vp, i32, i32, i32, vp]
        L.eri_get_lists.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.eri_get_stats.argtypes = [vp, C.POINTER(StatsT)]
        L.eri_check.argtypes = [vp]
        L.eri_get_profile.argtypes = [vp, C.POINTER(LaunchProfT), i32, C.POINTER(C.c_int32)]
        L.eri_build_jk_noalloc.argtypes = [vp, vp, vp, vp, vp]
        L.eri_peak_probe.argtypes = [i32, i32, C.POINTER(C.c_double), vp]
        L.eri_nuclear.argtypes = [vp, i32, vp, vp, vp, vp]
        L.eri_nuclear_grad.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp]
        L.eri_xc_grid.argtypes = [vp, i32, i32, C.c_double, C.c_double, C.POINTER(C.c_int64), vp]
        L.eri_xc_get_grid.argtypes = [vp, vp, vp, vp]
        L.eri_xc_density.argtypes = [vp, vp, vp, vp, vp]
        L.eri_xc_matrix.argtypes = [vp, vp, vp, vp, vp]
        L.eri_xc.argtypes = [vp, vp, i32, vp, vp, vp]
        L.eri_xc_stats.argtypes = [vp, C.POINTER(XcStatsT)]
        L.eri_plan_destroy.argtypes = [vp]
        L.eri_strerror.argtypes = [C.c_int]
        L.eri_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().eri_strerror(int(code)).decode()


def _check(rc, what):
    if rc != 0:
        raise EriError(rc, what)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _require(t, numel, what, device=None):
    """A device argument must be a contiguous float64 CUDA tensor of `numel`
    elements (on `device` when given): the library reads and writes exactly that
    many doubles through the raw pointer.  None passes (optional outputs)."""
    import torch
    if t is None:
        return
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{what}: need a contiguous float64 CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{what}: {t.numel()} elements, need {numel}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{what}: on cuda:{t.device.index}, the plan is on cuda:{device}")


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _basis_t(basis):
    """eri_basis_t for one basis (returns the struct and the arrays it points into)."""
    shells = (ShellT * basis.nshell)()
    for s in range(basis.nshell):
        shells[s].atom = int(basis.shell_atom[s])
        shells[s].l = int(basis.shell_l[s])
        shells[s].nprim = int(basis.shell_nprim[s])
        shells[s].prim_offset = int(basis.shell_prim_offset[s])
    exps = np.ascontiguousarray(basis.exps, np.float64)
    coefs = np.ascontiguousarray(basis.coefs, np.float64)
    b = BasisT(basis.nshell, basis.natom, shells, exps.ctypes.data_as(C.POINTER(C.c_double)),
               coefs.ctypes.data_as(C.POINTER(C.c_double)))
    return b, (shells, exps, coefs)


class Plan:
    """An eri_plan over one basis and geometry, or (a list of bases) an
    eri_plan_batch over several independent molecules (see include/eri.h).

    Batched plans take and return packed matrices: a 1-D float64 tensor with
    molecule m's nbf_m x nbf_m block at ``mat_off[m]`` (``pack`` / ``unpack``).
    """

    def __init__(self, basis, coords=None, thresh=1e-12, precision=ERI_FP64, mixed_tau=1e-5, device=None,
                 j_engine=True, profile=False, tune_cache=None, deterministic=False, density_screen=False):
        L = lib()
        self.batched = isinstance(basis, (list, tuple))
        bases = list(basis) if self.batched else [basis]
        if coords is None:
            coords = [b.coords for b in bases]
        elif not self.batched:
            coords = [coords]
        self.basis = basis
        keep = []
        bts = (BasisT * len(bases))()
        for m, bs in enumerate(bases):
            bt, arrs = _basis_t(bs)
            bts[m] = bt
            keep.append(arrs)
        if len(coords) != len(bases):
            raise ValueError(f"{len(coords)} coordinate sets for {len(bases)} bases")
        crds = [np.ascontiguousarray(c, np.float64).reshape(-1) for c in coords]
        for bs, c in zip(bases, crds):
            if c.size != 3 * bs.natom:
                raise ValueError(f"coordinates hold {c.size} values, the basis has {bs.natom} atoms (need natom x 3)")
        self._keep = (keep, crds)
        o = OptsT()
        L.eri_default_opts(C.byref(o))
        o.thresh = float(thresh)
        o.precision = int(precision)
        o.mixed_tau = float(mixed_tau)
        o.device = -1 if device is None else int(device)
        o.j_engine = int(bool(j_engine))
        o.profile = int(bool(profile))
        o.tune_cache = os.fsencode(tune_cache) if tune_cache else None
        o.deterministic = int(bool(deterministic))
        o.density_screen = int(bool(density_screen))
        h = C.c_void_p()
        if self.batched:
            bp = (C.POINTER(BasisT) * len(bases))(*[C.pointer(bts[m]) for m in range(len(bases))])
            cp = (C.POINTER(C.c_double) * len(bases))(*[c.ctypes.data_as(C.POINTER(C.c_double)) for c in crds])
            _check(L.eri_plan_batch(len(bases), bp, cp, C.byref(o), C.byref(h)), "eri_plan_batch")
        else:
            _check(L.eri_plan(C.byref(bts[0]), crds[0].ctypes.data_as(C.POINTER(C.c_double)), C.byref(o),
                              C.byref(h)), "eri_plan")
        self.h = h
        self.precision = int(precision)
        import torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        nm = C.c_int32()
        _check(L.eri_plan_layout(h, C.byref(nm), None, None, None), "eri_plan_layout")
        self.nmol = nm.value
        self.mat_off = np.zeros(self.nmol + 1, np.int64)
        self.mat_n = np.zeros(self.nmol, np.int32)
        self.atom_off = np.zeros(self.nmol + 1, np.int32)
        _check(L.eri_plan_layout(h, None, self.mat_off.ctypes.data_as(C.POINTER(C.c_int64)),
                                 self.mat_n.ctypes.data_as(C.POINTER(C.c_int32)),
                                 self.atom_off.ctypes.data_as(C.POINTER(C.c_int32))), "eri_plan_layout")
        self.nbf = int(self.mat_n.sum())
        self.nmat = int(self.mat_off[-1])
        self.xc_npoints = 0
        self.natom = int(self.atom_off[-1])
        self.npair = sum(b.nshell * (b.nshell + 1) // 2 for b in bases)
        # geometry bookkeeping for JKEnergy: geom_version counts set_coords calls,
        # list_version counts the ones that rebuilt the lists (freeze_lists False)
        self.geom_version = 0
        self.list_version = 0

    def _mat_shape(self):
        return (self.nmat,) if self.batched else (self.nbf, self.nbf)

    def pack(self, mats):
        """Packed 1-D tensor from a list of per-molecule nbf_m x nbf_m tensors."""
        import torch
        return torch.cat([m.reshape(-1) for m in mats]).contiguous()

    def unpack(self, packed):
        """Per-molecule nbf_m x nbf_m views of a packed tensor."""
        v = packed.reshape(-1)
        return [v[int(self.mat_off[m]):int(self.mat_off[m + 1])].view(int(self.mat_n[m]), int(self.mat_n[m]))
                for m in range(self.nmol)]

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().eri_plan_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_jk(self, D, J=None, K=None, want_j=True, want_k=True, thresh=-1.0, precision=None, stream=None):
        """J, K (torch float64 CUDA tensors, nbf x nbf) for the density D."""
        import torch
        shp = self._mat_shape()
        if want_j and J is None:
            J = torch.empty(shp, dtype=torch.float64, device=D.device)
        if want_k and K is None:
            K = torch.empty(shp, dtype=torch.float64, device=D.device)
        prec = self.precision if precision is None else int(precision)
        _require(D, self.nmat, "D", self.device)
        _require(J if want_j else None, self.nmat, "J", self.device)
        _require(K if want_k else None, self.nmat, "K", self.device)
        _check(lib().eri_build_jk(self.h, _ptr(D), _ptr(J if want_j else None), _ptr(K if want_k else None),
                                  float(thresh), prec, _stream_ptr(stream)), "eri_build_jk")
        return (J if want_j else None), (K if want_k else None)

    def build_jk_graph(self, D, J, K, precision=None, stream=None):
        """As build_jk into preallocated J / K (either may be None), replayed
        from a CUDA graph captured on the first call with these tensors."""
        prec = self.precision if precision is None else int(precision)
        for t, w in ((D, "D"), (J, "J"), (K, "K")):
            _require(t, self.nmat, w, self.device)
        _check(lib().eri_build_jk_graph(self.h, _ptr(D), _ptr(J), _ptr(K), prec, _stream_ptr(stream)),
               "eri_build_jk_graph")
        return J, K

    def autotune(self, D, precision=None, trial_ms=5.0, cache=None, stream=None):
        """Pick work-tile lengths per class launch (eri_autotune).  With `cache`
        (a JSON path), a table stored there for this device and plan shape is
        loaded instead of tuning, and a fresh result is stored."""
        import json
        import torch
        prec = self.precision if precision is None else int(precision)
        dev = torch.cuda.get_device_name(D.device)
        key = f"{dev}|prec{prec}|nbf{self.nbf}|nmol{self.nmol}"
        db = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                db = json.load(f)
            if key in db:
                self.set_tiles(np.asarray(db[key], np.int32))
                return self.tiles()
        _require(D, self.nmat, "D", self.device)
        _check(lib().eri_autotune(self.h, _ptr(D), prec, float(trial_ms), _stream_ptr(stream)), "eri_autotune")
        t = self.tiles()
        if cache:
            db[key] = t.reshape(-1).tolist()
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(db, f)
            os.replace(tmp, cache)
        return t

    def set_shard(self, shard, nshard):
        """Compute only this GPU's share of every build / gradient (partial sums;
        all-reduce them over the GPUs).  (0, 1) = the whole build."""
        _check(lib().eri_plan_set_shard(self.h, int(shard), int(nshard)), "eri_plan_set_shard")

    def set_omega(self, omega):
        """Two-electron operator of later builds and gradients: 0 = 1/r,
        omega > 0 = erf(omega r)/r (eri_plan_set_omega)."""
        _check(lib().eri_plan_set_omega(self.h, float(omega)), "eri_plan_set_omega")

    def set_tau(self, mixed_tau):
        """Mixed-precision threshold of later ERI_MIXED builds and gradients
        (eri_plan_set_tau; dynamic precision: tighten it as SCF converges)."""
        _check(lib().eri_plan_set_tau(self.h, float(mixed_tau)), "eri_plan_set_tau")

    def tiles(self):
        t = np.zeros(200, np.int32)
        _check(lib().eri_get_tiles(self.h, t.ctypes.data_as(C.POINTER(C.c_int32))), "eri_get_tiles")
        return t.reshape(10, 10, 2)

    def set_tiles(self, tiles):
        t = np.ascontiguousarray(np.asarray(tiles, np.int32).reshape(-1))
        _check(lib().eri_set_tiles(self.h, t.ctypes.data_as(C.POINTER(C.c_int32))), "eri_set_tiles")

    def energy(self, D, J, K, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(2 * self.nmol if self.batched else 2, dtype=torch.float64, device=D.device)
        for t, w in ((D, "D"), (J, "J"), (K, "K")):
            _require(t, self.nmat, w, self.device)
        _require(out, 2 * self.nmol, "out", self.device)
        _check(lib().eri_energy(self.h, _ptr(D), _ptr(J), _ptr(K), _ptr(out), _stream_ptr(stream)), "eri_energy")
        return out

    def set_coords(self, coords_dev, freeze_lists=False, stream=None):
        _require(coords_dev, 3 * self.natom, "coords", self.device)
        _check(lib().eri_plan_set_coords(self.h, _ptr(coords_dev), int(bool(freeze_lists)), _stream_ptr(stream)),
               "eri_plan_set_coords")
        self.geom_version += 1
        if not freeze_lists:
            self.list_version += 1

    def grad(self, D, out=None, want_j=True, want_k=True, precision=ERI_FP64, stream=None):
        """dE/dR (natom x 3): eri_jk_grad, or eri_jk_grad_prec for ERI_MIXED."""
        import torch
        if out is None:
            out = torch.empty((self.natom, 3), dtype=torch.float64, device=D.device)
        _require(D, self.nmat, "D", self.device)
        _require(out, 3 * self.natom, "out", self.device)
        _check(lib().eri_jk_grad_prec(self.h, _ptr(D), _ptr(out), int(want_j), int(want_k), int(precision),
                                      _stream_ptr(stream)), "eri_jk_grad_prec")
        return out

    def nuclear(self, q, xyz, V=None, stream=None):
        """V_mn = sum_C q_C (m|1/|r-C||n) for charges q [nc] at xyz [nc, 3]
        (float64 CUDA tensors); eri_nuclear."""
        import torch
        nc = int(q.numel())
        if V is None:
            V = torch.empty(self._mat_shape(), dtype=torch.float64, device=xyz.device)
        _require(q, nc, "q", self.device)
        _require(xyz, 3 * nc, "xyz", self.device)
        _require(V, self.nmat, "V", self.device)
        _check(lib().eri_nuclear(self.h, nc, _ptr(q), _ptr(xyz), _ptr(V), _stream_ptr(stream)), "eri_nuclear")
        return V

    def nuclear_grad(self, D, q, xyz, want_charges=True, stream=None):
        """(dE/dR [natom, 3], dE/dC [nc, 3] or None) of E_V = sum D V; eri_nuclear_grad."""
        import torch
        nc = int(q.numel())
        gR = torch.empty((self.natom, 3), dtype=torch.float64, device=D.device)
        gC = torch.empty((nc, 3), dtype=torch.float64, device=D.device) if want_charges else None
        _require(D, self.nmat, "D", self.device)
        _require(q, nc, "q", self.device)
        _require(xyz, 3 * nc, "xyz", self.device)
        _check(lib().eri_nuclear_grad(self.h, _ptr(D), nc, _ptr(q), _ptr(xyz), _ptr(gR), _ptr(gC),
                                      _stream_ptr(stream)), "eri_nuclear_grad")
        return gR, gC

    def xc_grid(self, nrad, ntheta, radius=1.0, cap_bytes=0.0, stream=None):
        """Build the plan's exchange-correlation grid on the device (eri_xc_grid);
        returns the number of points."""
        n = C.c_int64()
        _check(lib().eri_xc_grid(self.h, int(nrad), int(ntheta), float(radius), float(cap_bytes), C.byref(n),
                                 _stream_ptr(stream)), "eri_xc_grid")
        self.xc_npoints = int(n.value)
        return self.xc_npoints

    def xc_get_grid(self, stream=None):
        """(points [G, 3], weights [G]) of the grid, on the plan's device."""
        import torch
        dev = torch.device("cuda", self.device)
        pts = torch.empty((self.xc_npoints, 3), dtype=torch.float64, device=dev)
        w = torch.empty(self.xc_npoints, dtype=torch.float64, device=dev)
        _check(lib().eri_xc_get_grid(self.h, _ptr(pts), _ptr(w), _stream_ptr(stream)), "eri_xc_get_grid")
        return pts, w

    def xc_density(self, D, want_grad=True, stream=None):
        """(rho [G], grad rho [G, 3] or None) on the grid (eri_xc_density)."""
        import torch
        _require(D, self.nmat, "D", self.device)
        rho = torch.empty(self.xc_npoints, dtype=torch.float64, device=D.device)
        grad = torch.empty((self.xc_npoints, 3), dtype=torch.float64, device=D.device) if want_grad else None
        _check(lib().eri_xc_density(self.h, _ptr(D), _ptr(rho), _ptr(grad), _stream_ptr(stream)), "eri_xc_density")
        return rho, grad

    def xc_matrix(self, vrho, vgrad, V=None, stream=None):
        """V_mn for given point potentials vrho [G], vgrad [G, 3] (eri_xc_matrix)."""
        import torch
        if V is None:
            V = torch.empty(self._mat_shape(), dtype=torch.float64, device=vrho.device)
        _require(vrho, self.xc_npoints, "vrho", self.device)
        _require(vgrad, 3 * self.xc_npoints, "vgrad", self.device)
        _require(V, self.nmat, "V", self.device)
        _check(lib().eri_xc_matrix(self.h, _ptr(vrho), _ptr(vgrad), _ptr(V), _stream_ptr(stream)), "eri_xc_matrix")
        return V

    def xc(self, D, functional=ERI_XC_B88, V=None, stream=None):
        """(E_xc [1] device tensor, V_xc) with a built-in functional (eri_xc)."""
        import torch
        _require(D, self.nmat, "D", self.device)
        if V is None:
            V = torch.empty(self._mat_shape(), dtype=torch.float64, device=D.device)
        _require(V, self.nmat, "V", self.device)
        E = torch.empty(1, dtype=torch.float64, device=D.device)
        _check(lib().eri_xc(self.h, _ptr(D), int(functional), _ptr(V), _ptr(E), _stream_ptr(stream)), "eri_xc")
        return E, V

    def xc_stats(self):
        s = XcStatsT()
        _check(lib().eri_xc_stats(self.h, C.byref(s)), "eri_xc_stats")
        return {k: getattr(s, k) for k, _ in XcStatsT._fields_}

    def lists(self):
        Q = np.zeros(self.npair, np.float32)
        sig = np.zeros(self.npair, np.int32)
        counts = np.zeros(self.npair * 10, np.int32)
        srt = np.zeros(self.npair, np.int32)
        cc = np.zeros(10, np.int32)
        P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
        _check(lib().eri_get_lists(self.h, P(Q, C.c_float), P(sig, C.c_int32), P(counts, C.c_int32),
                                   P(srt, C.c_int32), P(cc, C.c_int32)), "eri_get_lists")
        return {"Q": Q, "sig": sig, "counts": counts.reshape(self.npair, 10), "sorted": srt[:int(cc.sum())],
                "class_count": cc}

    def profile(self):
        """Per (class pair, tier) device times of the builds since the last call."""
        buf = (LaunchProfT * 256)()
        n = C.c_int32()
        _check(lib().eri_get_profile(self.h, buf, 256, C.byref(n)), "eri_get_profile")
        return [{k: getattr(buf[i], k) for k, _ in LaunchProfT._fields_} for i in range(min(n.value, 256))]

    def check(self):
        """Raise EriError(ERI_EDEVICE) if a kernel of this plan reported a problem (eri_check)."""
        _check(lib().eri_check(self.h), "eri_check")

    def stats(self):
        s = StatsT()
        _check(lib().eri_get_stats(self.h, C.byref(s)), "eri_get_stats")
        return {k: getattr(s, k) for k, _ in StatsT._fields_}


def peak_probe(precision, iters, stream=None):
    """Measured FMA rate (TFLOP/s) of the current device: FP64 for ERI_FP64,
    FP32 for ERI_MIXED (eri_peak_probe)."""
    t = C.c_double()
    _check(lib().eri_peak_probe(int(precision), int(iters), C.byref(t), _stream_ptr(stream)), "eri_peak_probe")
    return t.value


def _autograd_function():
    import torch

    class JKEnergy(torch.autograd.Function):
        """E = 1/2 tr(D J) - 1/4 tr(D K) (SI Eq. si_E_J_K) as a differentiable function
        of the nuclear coordinates (natom x 3, float64, CUDA) and the density D.

        forward: moves the plan's atoms (eri_plan_set_coords), builds J and K, and
        returns E.  backward: dE/dR from eri_jk_grad (derivative ERIs contracted with
        D, D held fixed) and dE/dD = J - K/2.

        The plan is shared, mutable state.  backward differentiates at the
        geometry its own forward saw: if the plan has moved since (another
        forward on the same plan, a finite-difference step), backward moves it
        back first (rebuilding the lists, or with freeze_lists keeping the
        plan's frozen ones).  A frozen-list forward whose lists were rebuilt by
        a later unfrozen set_coords cannot be differentiated any more and
        raises RuntimeError.
        """

        @staticmethod
        def forward(ctx, coords, D, plan, freeze_lists=False):
            c = coords.detach().contiguous()
            plan.set_coords(c, freeze_lists=freeze_lists)
            J, K = plan.build_jk(D.detach().contiguous())
            E = plan.energy(D.detach(), J, K).sum()
            ctx.save_for_backward(D, J, K)
            ctx.plan = plan
            ctx.coords = c.clone()
            ctx.freeze = bool(freeze_lists)
            ctx.geom_version = plan.geom_version
            ctx.list_version = plan.list_version
            return E

        @staticmethod
        def backward(ctx, gE):
            D, J, K = ctx.saved_tensors
            gR = gD = None
            if ctx.needs_input_grad[0]:
                plan = ctx.plan
                if plan.geom_version != ctx.geom_version:
                    if ctx.freeze and plan.list_version != ctx.list_version:
                        raise RuntimeError("JKEnergy.backward: the plan's frozen lists were rebuilt after this "
                                           "forward; its gradient can no longer be taken on the same lists")
                    plan.set_coords(ctx.coords, freeze_lists=ctx.freeze)
                    ctx.geom_version = plan.geom_version
                    ctx.list_version = plan.list_version
                gR = plan.grad(D.detach().contiguous()) * gE
            if ctx.needs_input_grad[1]:
                gD = (J - 0.5 * K) * gE
            return gR, gD, None, None

    return JKEnergy


_JKENERGY = None


def __getattr__(name):
    """``JKEnergy`` (the autograd Function) is created on first access, so that
    importing this module does not import torch."""
    global _JKENERGY
    if name == "JKEnergy":
        if _JKENERGY is None:
            _JKENERGY = _autograd_function()
        return _JKENERGY
    raise AttributeError(name)


def jk_energy(coords, D, plan, freeze_lists=False):
    """Differentiable E_J + E_K; see JKEnergy."""
    return __getattr__("JKEnergy").apply(coords, D, plan, freeze_lists)


def build_jk(plan, D, **kw):
    """(J, K) of density D on `plan` (Plan.build_jk; keyword arguments as there)."""
    return plan.build_jk(D, **kw)
