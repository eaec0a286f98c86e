"""The stored oracle J/K of workload 1 (tests/golden/oracle_jk_w1.npz, written by
tests/golden/make_oracle_jk.py from the oracle alone) are for the inputs the
seeded generator produces today, and are self-consistent: the stored energies
equal 1/2 sum D J and -1/4 sum D K of the stored matrices, and J and K are
symmetric (upper triangles stored)."""
import os
import sys

import numpy as np

import workloads as W

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_oracle_jk as G  # noqa: E402


def test_w1_fixture_matches_generator_and_energies():
    basis, D = W.workload(1)
    assert G.matches(1, basis, D)
    J, K, ej, ek, Q = G.load(1)
    assert J.shape == (basis.nbf, basis.nbf) and Q.shape == (basis.nshell * (basis.nshell + 1) // 2,)
    assert abs(0.5 * (D * J).sum() - ej) < 1e-9 * abs(ej)
    assert abs(-0.25 * (D * K).sum() - ek) < 1e-9 * abs(ek)
    assert np.array_equal(J, J.T) and np.array_equal(K, K.T)
