"""Parity at the full sizes the bench runs, on sampled outputs and properties.

Workload 1 (60 atoms, 900 basis functions, Schwarz 1e-12), built the way
bench.py builds it (autotuned tiles, eager build, mixed tier bound 1e-3):

- the screening: Q within one float32 ulp of the oracle's, and the lists
  (significance, per-class ket counts, class-sorted order) bit for bit against
  the oracle's list construction on the same Q;
- FP64 J and K blocks sampled over the shell-pair classes against the oracle's
  one-block sums, within 1e-10;
- the mixed path: energies within 1e-6 Eh of the FP64 build, J and K symmetric
  and finite, sampled blocks within 1e-6 of the oracle.

Workload 3 (30 atoms, 750 basis functions): the gradient has zero net force
and one Cartesian component matches central finite differences of the FP64
energy (lists frozen), the property checks that hold at any size.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

THRESH = 1e-12
TAU = 1e-3


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
def w1(eri):
    import torch
    basis, D = W.workload(1)
    plan = eri.Plan(basis, thresh=THRESH, precision=eri.ERI_MIXED, mixed_tau=TAU)
    Dt = torch.from_numpy(D).cuda()
    plan.autotune(Dt, trial_ms=2.0)
    J64, K64 = plan.build_jk(Dt, precision=eri.ERI_FP64)
    E64 = plan.energy(Dt, J64, K64).cpu().numpy()
    Jm, Km = plan.build_jk(Dt, precision=eri.ERI_MIXED)
    Em = plan.energy(Dt, Jm, Km).cpu().numpy()
    o = oracle.Oracle(basis)
    Q = o.schwarz()
    return dict(basis=basis, D=D, plan=plan, J64=J64.cpu().numpy(), K64=K64.cpu().numpy(), E64=E64,
                Jm=Jm.cpu().numpy(), Km=Km.cpu().numpy(), Em=Em, o=o, Q=Q)


def _class(l1, l2):
    hi, lo = max(l1, l2), min(l1, l2)
    return hi * (hi + 1) // 2 + lo


def _sample_pairs(basis, seed, per_class=1):
    rng = np.random.default_rng(seed)
    by = {}
    for a in range(basis.nshell):
        for b in range(basis.nshell):
            by.setdefault(_class(basis.shell_l[a], basis.shell_l[b]), []).append((a, b))
    out = []
    for c in sorted(by):
        for i in rng.choice(len(by[c]), size=min(per_class, len(by[c])), replace=False):
            out.append(by[c][i])
    return out


def test_w1_lists_bit_exact(eri, w1):
    """Q is a float32 rounded up from each side's own FP64 (ab|ab): the two
    algorithms (McMurchie-Davidson on the GPU, Obara-Saika/HGP in the oracle)
    agree to rounding, so a value that falls within rounding of a float32
    boundary may land one ulp apart; Q agrees to <= 1 ulp.  The lists are
    integer work on Q: given the GPU's Q, the oracle's list construction must
    reproduce the GPU's lists bit for bit."""
    basis, Q, o = w1["basis"], w1["Q"], w1["o"]
    L = w1["plan"].lists()
    ulps = np.abs(L["Q"].view(np.int32).astype(np.int64) - Q.view(np.int32).astype(np.int64))
    print(f"Q: {int((ulps > 0).sum())} of {ulps.size} pairs differ, max {int(ulps.max())} ulp")
    assert ulps.max() <= 1
    assert (ulps > 0).mean() < 1e-3
    Q = L["Q"]
    sig, counts = o.lists(THRESH, Q)
    assert np.array_equal(L["sig"], sig)
    assert np.array_equal(L["counts"], counts)
    ns = basis.nshell
    cls = np.zeros(Q.shape[0], int)
    for a in range(ns):
        for b in range(a + 1):
            cls[a * (a + 1) // 2 + b] = _class(basis.shell_l[a], basis.shell_l[b])
    idx = sorted(np.nonzero(sig)[0].tolist(), key=lambda i: (cls[i], -float(Q[i]), i))
    assert np.array_equal(L["sorted"], np.asarray(idx, np.int32))


def _blocks(w, J, K, tol, seed):
    basis, D, o, Q = w["basis"], w["D"], w["o"], w["Q"]
    off = basis.ao_offsets()
    worst = 0.0
    for a, b in _sample_pairs(basis, seed):
        sa, sb = slice(off[a], off[a + 1]), slice(off[b], off[b + 1])
        jr = o.j_block(D, a, b, THRESH, Q)
        kr = o.k_block(D, a, b, THRESH, Q)
        worst = max(worst, np.abs(J[sa, sb] - jr).max(), np.abs(K[sa, sb] - kr).max())
    assert worst < tol, worst


def test_w1_fp64_sampled_blocks(eri, w1):
    _blocks(w1, w1["J64"], w1["K64"], 1e-10, seed=11)


def test_w1_mixed_energy_symmetry_blocks(eri, w1):
    dE = np.abs(w1["Em"] - w1["E64"])
    assert dE.max() < 1e-6, dE
    for M in (w1["Jm"], w1["Km"]):
        assert np.isfinite(M).all()
        assert np.abs(M - M.T).max() < 1e-12
    _blocks(w1, w1["Jm"], w1["Km"], 1e-6, seed=12)


def test_w3_gradient_net_force_and_fd(eri):
    import torch
    basis, D = W.workload(3)
    plan = eri.Plan(basis, thresh=THRESH)
    Dt = torch.from_numpy(D).cuda()
    g = plan.grad(Dt).cpu().numpy()
    assert np.abs(g.sum(axis=0)).max() < 1e-8
    atom, comp, h = 7, 1, 1e-4
    c0 = torch.from_numpy(np.ascontiguousarray(basis.coords)).cuda()

    def energy(shift):
        c = c0.clone()
        c[atom, comp] += shift
        plan.set_coords(c, freeze_lists=True)
        J, K = plan.build_jk(Dt)
        return float(plan.energy(Dt, J, K).sum())

    fd = (energy(h) - energy(-h)) / (2 * h)
    plan.set_coords(c0, freeze_lists=True)
    assert abs(fd - g[atom, comp]) < 1e-6 * max(1.0, abs(fd)), (fd, g[atom, comp])
