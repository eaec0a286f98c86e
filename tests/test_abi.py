"""The C-ABI library loads, exports every symbol include/eri.h declares, and
rejects invalid plans on the host before touching a GPU (no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def eri():
    from paper_2406_14920_gb300.build import build
    build()
    import paper_2406_14920_gb300 as m
    return m


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(eri_\w+)\s*\(", txt, re.M))
    return names


def test_exports_every_declared_symbol(eri):
    L = eri.lib()
    names = _declared()
    assert {"eri_plan", "eri_build_jk", "eri_jk_grad"} <= names
    for n in names:
        assert hasattr(L, n), n


def test_strerror(eri):
    assert eri.strerror(0) == "success"
    assert "invalid" in eri.strerror(-1)


def _basis_struct(eri, shells, exps, coefs, natom):
    arr = (eri.ShellT * len(shells))()
    for i, (a, l, n, o) in enumerate(shells):
        arr[i].atom, arr[i].l, arr[i].nprim, arr[i].prim_offset = a, l, n, o
    ex = np.asarray(exps, np.float64)
    co = np.asarray(coefs, np.float64)
    b = eri.BasisT(len(shells), natom, arr, ex.ctypes.data_as(C.POINTER(C.c_double)),
                   co.ctypes.data_as(C.POINTER(C.c_double)))
    return b, (arr, ex, co)


@pytest.mark.parametrize("case,code", [
    ("l4", -4), ("nprim0", -1), ("negexp", -1), ("badatom", -1), ("nancoord", -1)])
def test_plan_rejects_bad_input(eri, case, code):
    shells = [(0, 0, 1, 0), (1, 1, 1, 1)]
    exps, coefs = [1.0, 0.5], [1.0, 1.0]
    coords = np.zeros((2, 3))
    coords[1, 0] = 1.5
    if case == "l4":
        shells[1] = (1, 4, 1, 1)
    if case == "nprim0":
        shells[0] = (0, 0, 0, 0)
    if case == "negexp":
        exps[1] = -0.5
    if case == "badatom":
        shells[1] = (5, 1, 1, 1)
    if case == "nancoord":
        coords[0, 1] = np.nan
    b, keep = _basis_struct(eri, shells, exps, coefs, 2)
    h = C.c_void_p()
    rc = eri.lib().eri_plan(C.byref(b), coords.ctypes.data_as(C.POINTER(C.c_double)), None, C.byref(h))
    assert rc == code
    assert not h.value


def test_null_arguments(eri):
    L = eri.lib()
    assert L.eri_plan(None, None, None, None) == -1
    assert L.eri_build_jk(None, None, None, None, -1.0, 0, None) == -1
    assert L.eri_plan_destroy(None) == 0


def test_plan_batch_rejects_bad_input(eri):
    """eri_plan_batch validates every molecule (and nmol) on the host."""
    L = eri.lib()
    good, k1 = _basis_struct(eri, [(0, 0, 1, 0), (1, 1, 1, 1)], [1.0, 0.5], [1.0, 1.0], 2)
    bad, k2 = _basis_struct(eri, [(0, 0, 1, 0), (1, 4, 1, 1)], [1.0, 0.5], [1.0, 1.0], 2)
    c = np.zeros((2, 3))
    c[1, 0] = 1.5
    cp = c.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    for nmol in (0, -3, 70000):
        bp = (C.POINTER(eri.BasisT) * 1)(C.pointer(good))
        cc = (C.POINTER(C.c_double) * 1)(cp)
        assert L.eri_plan_batch(nmol, bp, cc, None, C.byref(h)) == -1
    bp = (C.POINTER(eri.BasisT) * 2)(C.pointer(good), C.pointer(bad))
    cc = (C.POINTER(C.c_double) * 2)(cp, cp)
    assert L.eri_plan_batch(2, bp, cc, None, C.byref(h)) == -4
    assert L.eri_plan_batch(2, None, cc, None, C.byref(h)) == -1
    assert not h.value
    assert L.eri_plan_layout(None, None, None, None, None) == -1


def test_tuner_and_graph_null_arguments(eri):
    L = eri.lib()
    assert L.eri_autotune(None, None, 0, 1.0, None) == -1
    assert L.eri_get_tiles(None, None) == -1
    assert L.eri_set_tiles(None, None) == -1
    assert L.eri_build_jk_graph(None, None, None, None, 0, None) == -1


def test_shard_and_layout_null_arguments(eri):
    L = eri.lib()
    assert L.eri_plan_set_shard(None, 0, 1) == -1
    assert L.eri_build_jk_noalloc(None, None, None, None, None) == -1
    assert L.eri_peak_probe(0, 0, None, None) == -1
    assert L.eri_plan_set_omega(None, C.c_double(0.5)) == -1
    assert L.eri_plan_set_tau(None, C.c_double(1e-5)) == -1
    assert L.eri_nuclear(None, 0, None, None, None, None) == -1
    assert L.eri_check(None) == -1
    assert L.eri_jk_grad_prec(None, None, None, 1, 1, 0, None) == -1
    assert L.eri_nuclear_grad(None, None, 0, None, None, None, None, None) == -1
    assert L.eri_peak_probe(2, 100, None, None) == -1
    assert L.eri_get_profile(None, None, 0, None) == -1
    assert L.eri_get_stats(None, None) == -1


def test_xc_null_arguments(eri):
    L = eri.lib()
    assert L.eri_xc_grid(None, 24, 8, C.c_double(1.0), C.c_double(0.0), None, None) == -1
    assert L.eri_xc_get_grid(None, None, None, None) == -1
    assert L.eri_xc_density(None, None, None, None, None) == -1
    assert L.eri_xc_matrix(None, None, None, None, None) == -1
    assert L.eri_xc(None, None, 1, None, None, None) == -1
    assert L.eri_xc_stats(None, None) == -1


def test_binding_checks_coordinate_shapes(eri):
    """The binding refuses coordinates that do not match the basis before any
    call into the library (which would read natom x 3 doubles)."""
    import workloads as W
    b, _ = W.workload(0)
    with pytest.raises(ValueError):
        eri.Plan(b, coords=np.zeros((2, 3)))
    with pytest.raises(ValueError):
        eri.Plan([b, b], coords=[b.coords])


def test_binding_requires_device_float64_tensors(eri):
    """Device arguments are checked before their pointers reach the library."""
    import torch
    with pytest.raises(ValueError):
        eri._require(torch.zeros(4, dtype=torch.float64), 4, "D")      # host tensor
    with pytest.raises(ValueError):
        eri._require(np.zeros(4), 4, "D")                               # not a tensor
    eri._require(None, 4, "K")                                          # optional output


def test_module_level_api(eri):
    """eri.JKEnergy (the autograd Function, created on first access and then
    reused) and eri.build_jk(plan, D) exist; unknown names still raise."""
    import torch
    assert issubclass(eri.JKEnergy, torch.autograd.Function)
    assert eri.JKEnergy is eri.JKEnergy
    assert callable(eri.build_jk) and callable(eri.jk_energy)
    with pytest.raises(AttributeError):
        eri.no_such_name
