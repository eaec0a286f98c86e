"""eri_build_jk_noalloc: the J/K build for callers that cannot allocate device
memory while they run (graph capture, allocators, allocation-free hosts).

It is called here through the C ABI, twice in a row on the same plan, and must
match eri_build_jk within the parity tolerance each time (its scratch array
keeps the previous call's contents, so the second call checks that it clears
what must start at zero).  This file is collected last on purpose; it must
pass alone in a fresh process as well as after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14920_gb300.build import build
    build()
    import paper_2406_14920_gb300 as m
    return m


def _noalloc(eri, plan, D, J, K):
    import torch
    ptr = lambda t: C.c_void_p(t.data_ptr() if t is not None else 0)
    rc = eri.lib().eri_build_jk_noalloc(plan.h, ptr(D), ptr(J), ptr(K),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_noalloc_matches_build_jk_twice(eri):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=1e-12)
    Dt = torch.from_numpy(D).cuda()
    Jr, Kr = plan.build_jk(Dt)
    Jr, Kr = Jr.cpu().numpy(), Kr.cpu().numpy()
    for call in range(2):
        J = torch.full_like(Dt, np.nan)
        K = torch.full_like(Dt, np.nan)
        assert _noalloc(eri, plan, Dt, J, K) == 0
        torch.cuda.synchronize()
        assert np.abs(J.cpu().numpy() - Jr).max() < TOL, call
        assert np.abs(K.cpu().numpy() - Kr).max() < TOL, call
    # a second plan of another size reuses the same scratch
    basis2, D2 = W.small_system(["2s1p1d1f", "1s1p1d"], seed=5)
    plan2 = eri.Plan(basis2, thresh=1e-12)
    D2t = torch.from_numpy(D2).cuda()
    J2r, K2r = plan2.build_jk(D2t)
    J2 = torch.empty_like(D2t)
    K2 = torch.empty_like(D2t)
    assert _noalloc(eri, plan2, D2t, J2, K2) == 0
    torch.cuda.synchronize()
    assert np.abs(J2.cpu().numpy() - J2r.cpu().numpy()).max() < TOL
    assert np.abs(K2.cpu().numpy() - K2r.cpu().numpy()).max() < TOL


def test_noalloc_rejects_plans_above_the_limit(eri):
    import torch
    basis, D = W.small_system(["4s3p2d1f"] * 8, seed=2, side=8.0, dmin=2.0)
    assert basis.nbf > 256
    plan = eri.Plan(basis, thresh=1e-10)
    Dt = torch.from_numpy(D).cuda()
    J = torch.empty_like(Dt)
    K = torch.empty_like(Dt)
    assert _noalloc(eri, plan, Dt, J, K) == -4  # ERI_EUNSUPPORTED


def test_noalloc_j_only_and_k_only(eri):
    """J alone (eri_build_jk takes the J-engine there, this call the Cartesian
    path: equal to rounding) and K alone, each twice in a row; the stats then
    describe the allocation-free call."""
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=1e-12)
    Dt = torch.from_numpy(D).cuda()
    Jr, _ = plan.build_jk(Dt, want_k=False)
    _, Kr = plan.build_jk(Dt, want_j=False)
    Jr, Kr = Jr.cpu().numpy(), Kr.cpu().numpy()
    for call in range(2):
        J = torch.full_like(Dt, np.nan)
        assert _noalloc(eri, plan, Dt, J, None) == 0
        torch.cuda.synchronize()
        assert np.abs(J.cpu().numpy() - Jr).max() < TOL, call
        K = torch.full_like(Dt, np.nan)
        assert _noalloc(eri, plan, Dt, None, K) == 0
        torch.cuda.synchronize()
        assert np.abs(K.cpu().numpy() - Kr).max() < TOL, call
    st = plan.stats()
    assert st["quartets_k_fp32"] == 0
