"""Work split over GPUs (eri_plan_set_shard), exercised on one GPU.

The shares shard = 0..n-1 of a build are run one after another on the same
device (no rank waits on another) and summed on the host side, which is what
the sum all-reduce over GPUs would do: the sum must equal the whole build, for
J+K, the J-engine, mixed precision and the gradient.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def eri():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14920_gb300.build import build
    build()
    import paper_2406_14920_gb300 as m
    return m


@pytest.mark.parametrize("nshard", [2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_shards_sum_to_whole_build(eri, nshard, precision):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, precision=precision, mixed_tau=1e-3)
    Dt = torch.from_numpy(D).cuda()
    J0, K0 = plan.build_jk(Dt)
    q0 = plan.stats()
    Js, Ks = torch.zeros_like(J0), torch.zeros_like(K0)
    nq, n32 = 0, 0
    for r in range(nshard):
        plan.set_shard(r, nshard)
        J, K = plan.build_jk(Dt)
        st = plan.stats()
        nq += st["flops_k"]
        n32 += st["quartets_k_fp32"]
        Js += J
        Ks += K
    plan.set_shard(0, 1)
    assert (Js - J0).abs().max().item() < TOL
    assert (Ks - K0).abs().max().item() < TOL
    assert n32 == q0["quartets_k_fp32"]
    assert abs(nq - q0["flops_k"]) <= 1e-9 * q0["flops_k"]


def test_shards_j_engine_and_gradient(eri):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis)
    Dt = torch.from_numpy(D).cuda()
    J0, _ = plan.build_jk(Dt, want_k=False)
    g0 = plan.grad(Dt)
    Js, gs = torch.zeros_like(J0), torch.zeros_like(g0)
    for r in range(2):
        plan.set_shard(r, 2)
        J, _ = plan.build_jk(Dt, want_k=False)
        Js += J
        gs += plan.grad(Dt)
    assert (Js - J0).abs().max().item() < TOL
    assert (gs - g0).abs().max().item() < 1e-11


def test_shard_rejects_bad_arguments(eri):
    basis, _ = W.workload(0)
    plan = eri.Plan(basis)
    for r, n in [(0, 0), (2, 2), (-1, 3)]:
        with pytest.raises(eri.EriError):
            plan.set_shard(r, n)
