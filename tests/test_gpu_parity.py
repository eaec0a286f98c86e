"""GPU parity: the CUDA path through the C ABI against the oracle.

- lists (Schwarz Q as float32, significance, per-class counts, class-sorted
  order) bit-exact;
- FP64 J and K within 1e-10 max abs element (the hot-path tolerance);
- E_J, E_K within 1e-10.
Sizes: workload 0 (75 bf, 21 shells: every class of shell pair, several
warps' worth of quartets per class and ragged tails) and small systems that
isolate class families.
"""
import numpy as np
import pytest

import oracle
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


def _oracle_lists(basis, Q, thresh):
    o = oracle.Oracle(basis)
    sig, counts = o.lists(thresh, Q)
    ns = basis.nshell
    cls = np.zeros(Q.shape[0], int)
    for a in range(ns):
        for b in range(a + 1):
            hi, lo = max(basis.shell_l[a], basis.shell_l[b]), min(basis.shell_l[a], basis.shell_l[b])
            cls[a * (a + 1) // 2 + b] = hi * (hi + 1) // 2 + lo
    idx = [i for i in range(Q.shape[0]) if sig[i]]
    idx.sort(key=lambda i: (cls[i], -float(Q[i]), i))
    return sig, counts, np.asarray(idx, np.int32)


@pytest.mark.parametrize("thresh", [1e-12, 1e-8])
def test_lists_bit_exact_w0(eri, thresh):
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=thresh)
    L = plan.lists()
    o = oracle.Oracle(basis)
    Qo = o.schwarz()
    assert np.array_equal(L["Q"].view(np.uint32), Qo.view(np.uint32))
    sig, counts, srt = _oracle_lists(basis, Qo, thresh)
    assert np.array_equal(L["sig"], sig)
    assert np.array_equal(L["counts"], counts)
    assert np.array_equal(L["sorted"], srt)


def _jk_check(eri, basis, D, thresh=1e-12):
    import torch
    plan = eri.Plan(basis, thresh=thresh)
    Dt = torch.from_numpy(D).cuda()
    J, K = plan.build_jk(Dt)
    E = plan.energy(Dt, J, K).cpu().numpy()
    J, K = J.cpu().numpy(), K.cpu().numpy()
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    Jr, Kr = o.jk(D, thresh, Q)
    ej, ek = o.energy(D, Jr, Kr)
    dj, dk = np.abs(J - Jr).max(), np.abs(K - Kr).max()
    assert dj < TOL, f"max|dJ| = {dj:.3e}"
    assert dk < TOL, f"max|dK| = {dk:.3e}"
    assert abs(E[0] - ej) < TOL and abs(E[1] - ek) < TOL, (E, ej, ek)
    return plan


def test_jk_fp64_w0(eri):
    basis, D = W.workload(0)
    _jk_check(eri, basis, D)


@pytest.mark.parametrize("comp", [["1s", "1s"], ["1p", "1s1p"], ["1d", "1s1p"], ["1f", "1p"], ["1d1f", "1s"],
                                  ["1f", "1f"], ["2s1p1d1f"], ["1s1p1d1f", "1s1p1d1f", "1s1p"]])
def test_jk_fp64_small(eri, comp):
    basis, D = W.small_system(comp, seed=len(comp) * 7 + len(comp[0]))
    _jk_check(eri, basis, D)


def test_jk_threshold_and_only_one(eri):
    import torch
    basis, D = W.small_system(["2s1p1d", "1s1p1f", "1s1p"], seed=9)
    plan = eri.Plan(basis, thresh=1e-12)
    Dt = torch.from_numpy(D).cuda()
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    for thresh in (1e-6, 1e-3):
        J, K = plan.build_jk(Dt, thresh=thresh)
        Jr, Kr = o.jk(D, thresh, Q)
        assert np.abs(J.cpu().numpy() - Jr).max() < TOL
        assert np.abs(K.cpu().numpy() - Kr).max() < TOL
    Jo, Ko = plan.build_jk(Dt, want_k=False, thresh=1e-12)
    assert Ko is None
    Jr, Kr = o.jk(D, 1e-12, Q)
    assert np.abs(Jo.cpu().numpy() - Jr).max() < TOL
    Jn, Kn = plan.build_jk(Dt, want_j=False)
    assert Jn is None and np.abs(Kn.cpu().numpy() - Kr).max() < TOL


def test_j_only_cartesian_route(eri):
    import torch
    basis, D = W.small_system(["2s1p1d1f", "1s1p1d"], seed=13)
    plan = eri.Plan(basis, thresh=1e-12, j_engine=False)
    Dt = torch.from_numpy(D).cuda()
    J, _ = plan.build_jk(Dt, want_k=False)
    o = oracle.Oracle(basis)
    Jr, _ = o.jk(D, 1e-12, o.schwarz())
    assert np.abs(J.cpu().numpy() - Jr).max() < TOL


@pytest.mark.parametrize("tau,etol,mtol", [(1e-5, 1e-6, 1e-6), (1e30, 2e-5, 2e-4)])
def test_mixed_precision_w0(eri, tau, etol, mtol):
    """Mixed path: quartets with Q_ab Q_cd max|D| < tau in FP32 (tau = 1e30: all of them).
    Energy error against the oracle within etol (1e-6 Eh at the default tau)."""
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=1e-12, precision=eri.ERI_MIXED, mixed_tau=tau)
    Dt = torch.from_numpy(D).cuda()
    J, K = plan.build_jk(Dt)
    E = plan.energy(Dt, J, K).cpu().numpy()
    st = plan.stats()
    o = oracle.Oracle(basis)
    Jr, Kr = o.jk(D, 1e-12, o.schwarz())
    ej, ek = o.energy(D, Jr, Kr)
    assert abs(E[0] - ej) < etol and abs(E[1] - ek) < etol, (E[0] - ej, E[1] - ek)
    assert np.abs(J.cpu().numpy() - Jr).max() < mtol
    assert np.abs(K.cpu().numpy() - Kr).max() < mtol
    if tau > 1:
        assert st["quartets_k_fp32"] == st["quartets_k"]
    else:  # the paper's default bound still sends part of workload 0 to the FP32 tier
        assert 0 < st["quartets_k_fp32"] < st["quartets_k"], st


@pytest.mark.parametrize("tau,etol,mtol", [(1e-5, 1e-6, 1e-6), (1e-2, 1e-6, 1e-5), (1e30, 2e-5, 2e-4)])
def test_mixed_jengine_w0(eri, tau, etol, mtol):
    """J-only mixed build through the J-engine (Eq. j_formula): ordered items
    with Q_ab Q_cd max|D| < tau in FP32 (tau = 1e30: all of them), FP64 Hermite
    J.  E_J against the oracle within etol, J within mtol; the FP32 share as
    the tier bound implies; the same build in a CUDA graph agrees."""
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=1e-12, precision=eri.ERI_MIXED, mixed_tau=tau)
    Dt = torch.from_numpy(D).cuda()
    J, _ = plan.build_jk(Dt, want_k=False)
    st = plan.stats()
    o = oracle.Oracle(basis)
    Jr, Kr = o.jk(D, 1e-12, o.schwarz())
    ej, _ = o.energy(D, Jr, Kr)
    Jn = J.cpu().numpy()
    e = 0.5 * float((D * Jn).sum())
    assert abs(e - ej) < etol, e - ej
    assert np.abs(Jn - Jr).max() < mtol
    assert np.abs(Jn - Jn.T).max() < 1e-12
    if tau > 1:
        assert st["quartets_j_fp32"] == st["quartets_j"]
    else:
        assert 0 < st["quartets_j_fp32"] < st["quartets_j"], st
    # the graph replay runs the same tiers; the FP32 tier's sums depend on how
    # the items fall into warps (the compacted lists are appended with atomics),
    # so the two builds agree to FP32 rounding of that tier, not bit for bit
    Jg = torch.empty_like(J)
    plan.build_jk_graph(Dt, Jg, None)
    assert np.abs(Jg.cpu().numpy() - Jn).max() < 0.1 * mtol
    J64, _ = plan.build_jk(Dt, want_k=False, precision=eri.ERI_FP64)
    assert plan.stats()["quartets_j_fp32"] == 0
    assert np.abs(J64.cpu().numpy() - Jr).max() < TOL


def test_dynamic_precision_set_tau(eri):
    """eri_plan_set_tau between builds of one plan (the dynamic-precision scheme
    of Sec. 4.1's citation): the FP32 share falls as tau falls, tau = 0 is the
    FP64 build, and a captured graph build follows the new threshold."""
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=1e-12, precision=eri.ERI_MIXED, mixed_tau=1e-1)
    Dt = torch.from_numpy(D).cuda()
    o = oracle.Oracle(basis)
    Jr, Kr = o.jk(D, 1e-12, o.schwarz())
    ej, ek = o.energy(D, Jr, Kr)
    J, K = torch.empty_like(Dt), torch.empty_like(Dt)
    plan.build_jk_graph(Dt, J, K)
    n32, err = [], []
    for tau in (1e-1, 1e-3, 1e-5, 0.0):
        plan.set_tau(tau)
        plan.build_jk(Dt, J, K)
        E = plan.energy(Dt, J, K).cpu().numpy()
        n32.append(plan.stats()["quartets_k_fp32"])
        err.append(max(abs(E[0] - ej), abs(E[1] - ek)))
    assert n32[0] > n32[1] > n32[2] > n32[3] == 0, n32
    assert err[1] < 1e-6 and err[2] < 1e-6 and err[3] < 1e-10, err
    # the graph captured at tau = 0.1 is dropped; the replay now runs all-FP64
    plan.build_jk_graph(Dt, J, K)
    assert np.abs(J.cpu().numpy() - Jr).max() < 1e-10 and np.abs(K.cpu().numpy() - Kr).max() < 1e-10
    with pytest.raises(RuntimeError):
        plan.set_tau(-1.0)

