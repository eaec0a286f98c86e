"""CUDA-graph builds (eri_build_jk_graph) and the work-tile autotuner.

A graph replay must give the eager build's J and K (up to the order of
floating-point atomics: the graph runs class launches concurrently), follow
new contents of D, and survive a list rebuild.  Every work-tile length gives
the same J and K; the autotuner only picks among them.
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


def _mx(a, b):
    return (a - b).abs().max().item()


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_matches_eager(eri, precision):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, precision=precision, mixed_tau=1e-3)
    Dt = torch.from_numpy(D).cuda()
    J0, K0 = plan.build_jk(Dt)
    J, K = torch.empty_like(J0), torch.empty_like(K0)
    for _ in range(2):
        plan.build_jk_graph(Dt, J, K)
        torch.cuda.synchronize()
        assert _mx(J, J0) < TOL and _mx(K, K0) < TOL
    # same pointers, new contents: J and K are linear in D
    Dt.mul_(0.5)
    plan.build_jk_graph(Dt, J, K)
    torch.cuda.synchronize()
    if precision == 0:
        assert _mx(J, 0.5 * J0) < TOL and _mx(K, 0.5 * K0) < TOL
    else:  # the tier split follows D, so compare with an eager build of the new D
        J1, K1 = plan.build_jk(Dt)
        assert _mx(J, J1) < TOL and _mx(K, K1) < TOL


def test_graph_j_only_and_rebuild(eri):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis)
    Dt = torch.from_numpy(D).cuda()
    J0, _ = plan.build_jk(Dt, want_k=False)
    J = torch.empty_like(J0)
    plan.build_jk_graph(Dt, J, None)
    torch.cuda.synchronize()
    assert _mx(J, J0) < TOL
    # another threshold rebuilds the lists; the next graph call re-captures
    J8, K8 = plan.build_jk(Dt, thresh=1e-8)
    K = torch.empty_like(J)
    plan.build_jk_graph(Dt, J, K)
    torch.cuda.synchronize()
    assert _mx(J, J8) < TOL and _mx(K, K8) < TOL


def test_graph_batched(eri):
    import torch
    mols = [W.workload(0), W.small_system(["2s1p", "4s3p2d1f", "2s1p"], seed=3, side=5.0, dmin=1.8)]
    plan = eri.Plan([b for b, _ in mols], precision=1, mixed_tau=1e-3)
    Dp = plan.pack([torch.from_numpy(D) for _, D in mols]).cuda()
    J0, K0 = plan.build_jk(Dp)
    J, K = torch.empty_like(J0), torch.empty_like(K0)
    plan.build_jk_graph(Dp, J, K)
    torch.cuda.synchronize()
    assert _mx(J, J0) < TOL and _mx(K, K0) < TOL


@pytest.mark.parametrize("tile", [1, 3, 16])
def test_every_tile_gives_the_same_jk(eri, tile):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, precision=1, mixed_tau=1e-3)
    Dt = torch.from_numpy(D).cuda()
    J0, K0 = plan.build_jk(Dt)
    n0 = plan.stats()["quartets_k_fp32"]
    t = np.zeros((10, 10, 2), np.int32)
    for X in range(10):
        t[X, :X + 1, :] = tile
    plan.set_tiles(t)
    assert (plan.tiles()[t > 0] == tile).all()
    J, K = plan.build_jk(Dt)
    assert _mx(J, J0) < TOL and _mx(K, K0) < TOL
    assert plan.stats()["quartets_k_fp32"] == n0


def test_autotune_and_cache(eri, tmp_path):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, precision=1, mixed_tau=1e-3)
    Dt = torch.from_numpy(D).cuda()
    J0, K0 = plan.build_jk(Dt)
    cache = str(tmp_path / "tiles.json")
    t = plan.autotune(Dt, trial_ms=0.5, cache=cache)
    used = t[np.tril_indices(10)[0], np.tril_indices(10)[1]]
    assert set(np.unique(used)) <= {1, 2, 4, 8, 16, 32}
    J, K = plan.build_jk(Dt)
    assert _mx(J, J0) < TOL and _mx(K, K0) < TOL
    # a second plan of the same shape loads the cached table instead of tuning
    p2 = eri.Plan(basis, precision=1, mixed_tau=1e-3)
    assert np.array_equal(p2.autotune(Dt, cache=cache), t)


def test_c_level_tune_cache(eri, tmp_path):
    """opts.tune_cache: eri_autotune stores the tuned table under this device,
    plan shape and precision; a new plan with the same cache loads it; a plan of
    another shape does not."""
    import torch
    basis, D = W.workload(0)
    path = str(tmp_path / "tiles.txt")
    p1 = eri.Plan(basis, precision=1, mixed_tau=1e-3, tune_cache=path)
    Dt = torch.from_numpy(D).cuda()
    p1.set_tiles(np.full((10, 10, 2), 3, np.int32))  # a table the tuner would not pick by itself
    t1 = p1.autotune(Dt, precision=1, trial_ms=0.5)
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and "|prec=1" in lines[0] and f"|nbf={basis.nbf}|" in lines[0]
    p2 = eri.Plan(basis, precision=1, mixed_tau=1e-3, tune_cache=path)
    assert np.array_equal(p2.tiles(), t1)
    b2, _ = W.small_system(["1s1p1d", "2s1p"], seed=4)
    p3 = eri.Plan(b2, precision=1, tune_cache=path)
    assert np.array_equal(p3.tiles(), eri.Plan(b2, precision=1).tiles())
    # FP64 tuning adds its own entry next to the mixed one
    p1.autotune(Dt, precision=0, trial_ms=0.5)
    assert len(open(path).read().splitlines()) == 2
