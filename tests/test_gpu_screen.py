"""Density-weighted screening (opts.density_screen; Eq. kernel_upperbound with
the density factor): a quartet is dropped when Q_ab Q_cd max|D'| falls below
the threshold, max over the six blocks of D' = D f f (component norms folded
in) that the quartet touches, in float32 as the library evaluates it.

The rule is restated here on the library's own Q (integer work on given
floats); the oracle then builds J and K over exactly the kept canonical
quartets (or_jk_quartets), and the GPU build must match element by element
within 1e-10, drop the same number of quartets, and stay within the screening
error of the unscreened oracle build.
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


def _dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def _component_factors(basis):
    f = []
    for l in basis.shell_l.astype(int):
        for x in range(l, -1, -1):
            for y in range(l - x, -1, -1):
                z = l - x - y
                f.append(np.sqrt(_dfact(2 * l - 1) / (_dfact(2 * x - 1) * _dfact(2 * y - 1) * _dfact(2 * z - 1))))
    return np.asarray(f)


def _round_up_f32(x):
    y = np.float32(x)
    return np.nextafter(y, np.float32(np.inf)) if float(y) < x else y


def _kept_quartets(basis, D, Q, thresh):
    ns = basis.nshell
    off = basis.ao_offsets()
    f = _component_factors(basis)
    Dp = np.abs(D * f[:, None] * f[None, :])
    dm = np.empty((ns, ns), np.float32)
    for a in range(ns):
        for b in range(ns):
            blk = max(Dp[off[a]:off[a + 1], off[b]:off[b + 1]].max(), Dp[off[b]:off[b + 1], off[a]:off[a + 1]].max())
            dm[a, b] = _round_up_f32(blk)
    pi = lambda a, b: a * (a + 1) // 2 + b
    kept, dropped = [], 0
    t32 = np.float32(thresh)
    for a in range(ns):
        for b in range(a + 1):
            for c in range(a + 1):
                for d in range(c + 1):
                    if pi(c, d) > pi(a, b):
                        continue
                    qa, qc = Q[pi(a, b)], Q[pi(c, d)]
                    if float(qa) * float(qc) < thresh:
                        continue
                    d6 = max(dm[a, b], dm[c, d], dm[a, c], dm[a, d], dm[b, c], dm[b, d])
                    bound = np.float32(np.float32(qa) * np.float32(qc)) * np.float32(d6)
                    if bound < t32:
                        dropped += 1
                    else:
                        kept.append((a, b, c, d))
    return np.asarray(kept, np.int32), dropped


@pytest.mark.parametrize("thresh,precision", [(1e-8, 0), (1e-7, 0), (1e-8, 1)])
def test_density_screen_w0(eri, thresh, precision):
    import torch
    basis, D = W.workload(0)
    plan = eri.Plan(basis, thresh=thresh, precision=precision, mixed_tau=1e-3, density_screen=True)
    Dt = torch.from_numpy(D).cuda()
    J, K = plan.build_jk(Dt)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    st = plan.stats()
    Q = plan.lists()["Q"]
    kept, dropped = _kept_quartets(basis, D, Q, thresh)
    assert dropped > 0 and st["quartets_k_screened"] == dropped, (dropped, st["quartets_k_screened"])
    o = oracle.Oracle(basis)
    Jr, Kr = o.jk_quartets(D, kept)
    tol = 1e-10 if precision == 0 else 1e-6
    assert np.abs(J - Jr).max() < tol and np.abs(K - Kr).max() < tol
    # against the unscreened oracle build: each dropped quartet moves an element
    # by at most (bound) x (number of its components), far below the threshold scale
    Jf, Kf = o.jk(D, thresh, o.schwarz())
    assert np.abs(J - Jf).max() < 1e3 * thresh and np.abs(K - Kf).max() < 1e3 * thresh
