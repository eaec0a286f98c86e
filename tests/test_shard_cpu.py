"""Work split over GPUs, host side, on CPU ranks (gloo, world size 2).

The library splits every class-pair work list into tiles of `span`
consecutive canonical quartets and gives tile t to GPU t % nshard
(eri_plan_set_shard); each GPU returns partial J and K, and one sum
all-reduce gives the whole.  Here each gloo rank takes its tiles of the same
lists (in the library's order: classes ss..ff, bras by Q descending, kets by
Q descending, canonical cut for equal classes), computes its partial J and K
with the oracle, and the all-reduced sum must equal the oracle's whole build.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W


def _class_of(l1, l2):
    hi, lo = max(l1, l2), min(l1, l2)
    return hi * (hi + 1) // 2 + lo


def canonical_items(basis, thresh):
    """Per class pair (X, Y <= X): list of (a, b, c, d) in the library's item order."""
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    sig, counts = o.lists(thresh, Q)
    ns = basis.nshell
    pairs = {}
    for a in range(ns):
        for b in range(a + 1):
            ip = a * (a + 1) // 2 + b
            if sig[ip]:
                pairs.setdefault(_class_of(basis.shell_l[a], basis.shell_l[b]), []).append((ip, a, b))
    for X in pairs:
        pairs[X].sort(key=lambda t: (-float(Q[t[0]]), t[0]))
    out = {}
    for X in range(10):
        for Y in range(X + 1):
            items = []
            for i, (ip, a, b) in enumerate(pairs.get(X, [])):
                c = counts[ip, Y]
                if X == Y:
                    c = min(c, i + 1)
                for (kp, cc, d) in pairs.get(Y, [])[:c]:
                    items.append((a, b, cc, d))
            out[(X, Y)] = items
    return out, Q


def shard_of(item, span, nshard):
    return (item // span) % nshard


def _rank_main(rank, world, port, span, res_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    basis, D = W.small_system(["3s2p1d1f", "2s1p"], seed=5)
    items, _ = canonical_items(basis, 1e-12)
    mine = [q for lst in items.values() for i, q in enumerate(lst) if shard_of(i, span, world) == rank]
    o = oracle.Oracle(basis)
    J, K = o.jk_quartets(D, np.asarray(mine, np.int32).reshape(-1, 4))
    Jt, Kt = torch.from_numpy(J), torch.from_numpy(K)
    dist.all_reduce(Jt)
    dist.all_reduce(Kt)
    n_mine = torch.tensor([len(mine)])
    dist.all_reduce(n_mine)
    if rank == 0:
        np.savez(res_path, J=Jt.numpy(), K=Kt.numpy(), n=n_mine.numpy())
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_quartet_once():
    basis, _ = W.small_system(["3s2p1d1f", "2s1p"], seed=5)
    items, _ = canonical_items(basis, 1e-12)
    for lst in items.values():
        for span in (1, 4, 32):
            for nshard in (1, 2, 3, 5):
                owners = [shard_of(i, span, nshard) for i in range(len(lst))]
                assert all(0 <= r < nshard for r in owners)
                assert len(owners) == len(lst)


@pytest.mark.parametrize("span", [1, 32])
def test_gloo_ranks_sum_partial_jk(tmp_path, span):
    import torch.multiprocessing as mp
    res = str(tmp_path / "res.npz")
    mp.spawn(_rank_main, args=(2, _free_port(), span, res), nprocs=2, join=True)
    r = np.load(res)
    basis, D = W.small_system(["3s2p1d1f", "2s1p"], seed=5)
    items, Q = canonical_items(basis, 1e-12)
    assert int(r["n"][0]) == sum(len(v) for v in items.values())
    o = oracle.Oracle(basis)
    Jr, Kr = o.jk(D, 1e-12, Q, mode=1)
    assert np.abs(r["J"] - Jr).max() < 1e-12
    assert np.abs(r["K"] - Kr).max() < 1e-12
