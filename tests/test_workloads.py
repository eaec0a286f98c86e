"""The seeded synthetic inputs follow their stated recipe (CPU only).

Shapes and counts of the five workloads, minimum interatomic distances,
exponent ranges, the primitive counts per shell type, and the density
D = C C^T with C orthonormal (symmetric, D^2 = D, trace = number of columns).
Every generator is deterministic in its seed.
"""
import numpy as np
import pytest

import workloads as W


def _min_dist(c):
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=-1)
    return d[np.triu_indices(len(c), 1)].min()


def _density_checks(D, nocc):
    assert np.allclose(D, D.T, atol=1e-14)
    assert np.allclose(D @ D, D, atol=1e-12)
    assert abs(np.trace(D) - nocc) < 1e-10


@pytest.mark.parametrize("i,natom,nbf,dmin,nocc", [(0, 3, 75, 1.8, 10), (1, 60, 900, 2.0, 120),
                                                    (3, 30, 750, 2.0, 100)])
def test_single_workloads(i, natom, nbf, dmin, nocc):
    b, D = W.workload(i)
    assert b.natom == natom and b.nbf == nbf and D.shape == (nbf, nbf)
    assert _min_dist(b.coords) >= dmin - 1e-12
    _density_checks(D, nocc)
    b2, D2 = W.workload(i)
    assert np.array_equal(b.exps, b2.exps) and np.array_equal(D, D2)


def test_exponent_ranges_and_contractions():
    b, _ = W.workload(1)
    for s in range(b.nshell):
        o, n, l = int(b.shell_prim_offset[s]), int(b.shell_nprim[s]), int(b.shell_l[s])
        ex = b.exps[o:o + n]
        if l <= 1:
            assert n == 3 and ex.min() >= 0.1 and ex.max() <= 50.0
        else:
            assert n == 1 and 0.3 <= ex[0] <= 3.0


def test_metal_workload():
    b, D = W.workload(2)
    assert b.natom == 49
    metal = [s for s in range(b.nshell) if int(b.shell_atom[s]) == 0]
    ls = sorted(int(b.shell_l[s]) for s in metal)
    assert ls == [0] * 6 + [1] * 5 + [2] * 3 + [3] * 2
    s_prims = [int(b.shell_nprim[s]) for s in metal if int(b.shell_l[s]) == 0]
    assert all(n == 8 for n in s_prims)
    assert np.allclose(D, D.T, atol=1e-14)


def test_batched_workload():
    mols = W.workload(4)
    assert len(mols) == 64
    nbf = [b.nbf for b, _ in mols]
    assert min(nbf) >= 100 and max(nbf) <= 2000
    for b, D in mols[:4]:
        assert 10 <= b.natom <= 80
        assert _min_dist(b.coords) >= 2.0 - 1e-12
        assert D.shape == (b.nbf, b.nbf)
        assert np.allclose(D, D.T, atol=1e-14)
