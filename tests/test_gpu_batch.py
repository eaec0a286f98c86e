"""Batched plans (eri_plan_batch): several molecules of uneven size in one plan,
so every class launch covers all of them.

Per molecule, the batched plan must give what a single-molecule plan of that
molecule gives: the same lists bit for bit (screening is per molecule), the
same quartet and tier counts, J / K / energies / gradients equal up to the
order of floating-point atomics (1e-12), and J / K within 1e-10 of the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14920_gb300.build import build
    build()
    import paper_2406_14920_gb300 as m
    return m


@pytest.fixture(scope="module")
def mols():
    out = [W.workload(0)]
    out.append(W.small_system(["2s1p", "4s3p2d1f", "2s1p", "2s1p"], seed=3, side=5.0, dmin=1.8))
    out.append(W.small_system(["3s2p1d1f", "2s1p"], seed=5))
    out.append(W.small_system(["2s1p"], seed=11))
    b1, D1 = W.workload(1)
    out.append(W.subset_atoms(b1, D1, list(range(8))))
    return out


def _pack(mols):
    import torch
    return torch.cat([torch.from_numpy(D).reshape(-1) for _, D in mols]).cuda()


def test_layout(eri, mols):
    plan = eri.Plan([b for b, _ in mols])
    assert plan.nmol == len(mols)
    n = [b.nbf for b, _ in mols]
    assert list(plan.mat_n) == n
    assert list(plan.mat_off) == list(np.concatenate([[0], np.cumsum(np.square(n))]))
    assert list(plan.atom_off) == list(np.concatenate([[0], np.cumsum([b.natom for b, _ in mols])]))


@pytest.mark.parametrize("thresh", [1e-12, 1e-7])
def test_lists_match_single(eri, mols, thresh):
    bp = eri.Plan([b for b, _ in mols], thresh=thresh)
    LB = bp.lists()
    pb = 0
    seg = np.zeros(10, int)  # running offset of each class inside the batched sorted list
    coff = np.concatenate([[0], np.cumsum(LB["class_count"])])
    for b, _ in mols:
        L = eri.Plan(b, thresh=thresh).lists()
        npair = b.nshell * (b.nshell + 1) // 2
        sl = slice(pb, pb + npair)
        assert np.array_equal(LB["Q"][sl].view(np.uint32), L["Q"].view(np.uint32))
        assert np.array_equal(LB["sig"][sl], L["sig"])
        assert np.array_equal(LB["counts"][sl], L["counts"])
        so = np.concatenate([[0], np.cumsum(L["class_count"])])
        for X in range(10):
            nx = L["class_count"][X]
            got = LB["sorted"][coff[X] + seg[X]: coff[X] + seg[X] + nx] - pb
            assert np.array_equal(got, L["sorted"][so[X]:so[X] + nx]), X
            seg[X] += nx
        pb += npair
    assert np.array_equal(seg, LB["class_count"])


def test_jk_fp64_matches_single_and_oracle(eri, mols):
    import torch
    bp = eri.Plan([b for b, _ in mols])
    Dp = _pack(mols)
    J, K = bp.build_jk(Dp)
    E = bp.energy(Dp, J, K).cpu().numpy().reshape(-1, 2)
    st = bp.stats()
    Js, Ks = bp.unpack(J), bp.unpack(K)
    qk = 0
    for m, (b, D) in enumerate(mols):
        p = eri.Plan(b)
        Dt = torch.from_numpy(D).cuda()
        J1, K1 = p.build_jk(Dt)
        E1 = p.energy(Dt, J1, K1).cpu().numpy()
        qk += p.stats()["quartets_k"]
        assert torch.abs(Js[m] - J1).max().item() < 1e-12
        assert torch.abs(Ks[m] - K1).max().item() < 1e-12
        assert np.abs(E[m] - E1).max() < 1e-11
        if b.nbf <= 120:
            o = oracle.Oracle(b)
            Jr, Kr = o.jk(D, 1e-12, o.schwarz())
            assert np.abs(Js[m].cpu().numpy() - Jr).max() < 1e-10
            assert np.abs(Ks[m].cpu().numpy() - Kr).max() < 1e-10
    assert st["quartets_k"] == qk


def test_mixed_matches_single(eri, mols):
    import torch
    tau = 1e-3
    bp = eri.Plan([b for b, _ in mols], precision=eri.ERI_MIXED, mixed_tau=tau)
    Dp = _pack(mols)
    J, K = bp.build_jk(Dp)
    E = bp.energy(Dp, J, K).cpu().numpy().reshape(-1, 2)
    J64, K64 = bp.build_jk(Dp, precision=eri.ERI_FP64)
    E64 = bp.energy(Dp, J64, K64).cpu().numpy().reshape(-1, 2)
    assert np.abs(E - E64).max() < 1e-6
    bp.build_jk(Dp)
    n32 = bp.stats()["quartets_k_fp32"]
    tot32 = 0
    for m, (b, D) in enumerate(mols):
        p = eri.Plan(b, precision=eri.ERI_MIXED, mixed_tau=tau)
        Dt = torch.from_numpy(D).cuda()
        p.build_jk(Dt)
        tot32 += p.stats()["quartets_k_fp32"]
    assert n32 == tot32 and n32 > 0


def test_j_engine_matches_single(eri, mols):
    import torch
    bp = eri.Plan([b for b, _ in mols])
    Dp = _pack(mols)
    J, _ = bp.build_jk(Dp, want_k=False)
    Js = bp.unpack(J)
    for m, (b, D) in enumerate(mols):
        J1, _ = eri.Plan(b).build_jk(torch.from_numpy(D).cuda(), want_k=False)
        assert torch.abs(Js[m] - J1).max().item() < 1e-12


def test_grad_matches_single(eri, mols):
    import torch
    bp = eri.Plan([b for b, _ in mols])
    G = bp.grad(_pack(mols)).cpu().numpy()
    for m, (b, D) in enumerate(mols):
        g1 = eri.Plan(b).grad(torch.from_numpy(D).cuda()).cpu().numpy()
        a0, a1 = bp.atom_off[m], bp.atom_off[m + 1]
        assert np.abs(G[a0:a1] - g1).max() < 1e-10
        assert np.abs(G[a0:a1].sum(axis=0)).max() < 1e-8
