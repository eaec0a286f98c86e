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

Workload 1 also against the oracle's full J and K, every element (stored by
tests/golden/make_oracle_jk.py, which calls only the oracle), and the lists
against the ones the oracle builds from its own Q (near-boundary items only).
Workload 2 (metal complex, exponents to 2e4): sampled metal blocks in FP64
against the oracle, and the mixed build with its FP32 range guard.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

THRESH = 1e-12
TAU = 1e-2  # the bench tier bound (bench.py)


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


def test_w1_lists_vs_oracle_own_q(eri, w1):
    """The GPU's lists against the lists the oracle builds from its OWN Q.
    Every difference (a pair's significance, a (bra, ket) membership behind
    the per-class counts, the relative order of two pairs) must involve a pair
    whose two Q values differ by one float32 ulp, and for significance and
    membership the bound products of the two sides must fall on opposite sides
    of thresh: those are the only items two correct implementations may split
    on.  The number of such items is printed."""
    basis, Qo, o = w1["basis"], w1["Q"], w1["o"]
    L = w1["plan"].lists()
    Qg = L["Q"]
    ulps = np.abs(Qg.view(np.int32).astype(np.int64) - Qo.view(np.int32).astype(np.int64))
    assert ulps.max() <= 1
    moved = ulps > 0
    sig_o, counts_o = o.lists(THRESH, Qo)
    qg, qo = Qg.astype(np.float64), Qo.astype(np.float64)
    qmax_g, qmax_o = qg.max(), qo.max()
    # significance
    dsig = np.nonzero(L["sig"] != sig_o)[0]
    for i in dsig:
        assert moved[i] or moved[int(np.argmax(qg))] or moved[int(np.argmax(qo))], i
        assert (qg[i] * qmax_g >= THRESH) != (qo[i] * qmax_o >= THRESH)
    # per-class counts: enumerate the (bra, ket) memberships behind every differing count
    ns = basis.nshell
    cls = np.zeros(Qg.shape[0], int)
    for a in range(ns):
        for b in range(a + 1):
            cls[a * (a + 1) // 2 + b] = _class(basis.shell_l[a], basis.shell_l[b])
    sg, so = L["sig"].astype(bool), sig_o.astype(bool)
    dmem = 0
    for i in np.unique(np.nonzero(L["counts"] != counts_o)[0]):
        in_g = sg[i] & sg & (qg[i] * qg >= THRESH)
        in_o = so[i] & so & (qo[i] * qo >= THRESH)
        for j in np.nonzero(in_g != in_o)[0]:
            dmem += 1
            assert moved[i] or moved[j] or i in dsig or j in dsig, (i, j)
            if sg[i] and so[i] and sg[j] and so[j]:
                assert (qg[i] * qg[j] >= THRESH) != (qo[i] * qo[j] >= THRESH), (i, j)
    # order: with the moved pairs removed, the class-sorted lists must agree exactly
    idx_o = sorted(np.nonzero(so)[0].tolist(), key=lambda i: (cls[i], -float(Qo[i]), i))
    flipped = set(dsig.tolist())
    keep = lambda seq: [int(i) for i in seq if not moved[i] and i not in flipped]
    assert keep(L["sorted"].tolist()) == keep(idx_o)
    nord = int(sum(1 for a_, b_ in zip(L["sorted"].tolist(), idx_o) if a_ != b_))
    print(f"near-boundary items: {int(moved.sum())} pairs with Q one ulp apart, {len(dsig)} significance "
          f"flips, {dmem} (bra, ket) memberships, {nord} list positions shifted")


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


def _golden(wl):
    import sys, os
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_oracle_jk as G
    r = G.load(wl)
    if r is None:
        pytest.fail(f"tests/golden/oracle_jk_w{wl}.npz is missing: run tests/golden/make_oracle_jk.py {wl}")
    return G, r


def test_w1_fp64_every_element_vs_oracle(eri, w1):
    """Every element of the FP64 J and K of workload 1 against the oracle's full
    build (stored by tests/golden/make_oracle_jk.py, oracle only), within 1e-10;
    the mixed build's E_J and E_K within 1e-6 Eh of the oracle's energies."""
    G, (Jo, Ko, ejo, eko, Qo) = _golden(1)
    assert G.matches(1, w1["basis"], w1["D"]), "stored oracle J/K are for other inputs"
    dj = np.abs(w1["J64"] - Jo).max()
    dk = np.abs(w1["K64"] - Ko).max()
    print(f"workload 1 FP64: max|dJ| {dj:.2e}, max|dK| {dk:.2e} over {Jo.size} elements each")
    assert dj < 1e-10 and dk < 1e-10, (dj, dk)
    e64, em = w1["E64"], w1["Em"]
    assert abs(e64[0] - ejo) < 1e-10 and abs(e64[1] - eko) < 1e-10, (e64, ejo, eko)
    print(f"workload 1 mixed: dE_J {em[0] - ejo:.2e}, dE_K {em[1] - eko:.2e} against the oracle")
    assert abs(em[0] - ejo) < 1e-6 and abs(em[1] - eko) < 1e-6


@pytest.fixture(scope="module")
def w2(eri):
    """Workload 2: metal 6s5p3d2f (exponents up to 2e4, 8-primitive s) with 48
    3s2p1d1f ligands, 1259 basis functions."""
    import torch
    basis, D = W.workload(2)
    plan = eri.Plan(basis, thresh=THRESH, precision=eri.ERI_MIXED, mixed_tau=TAU)
    Dt = torch.from_numpy(D).cuda()
    J64, K64 = plan.build_jk(Dt, precision=eri.ERI_FP64)
    E64 = plan.energy(Dt, J64, K64).cpu().numpy()
    Jm, Km = plan.build_jk(Dt, precision=eri.ERI_MIXED)
    Em = plan.energy(Dt, Jm, Km).cpu().numpy()
    st = plan.stats()
    o = oracle.Oracle(basis)
    return dict(basis=basis, D=D, plan=plan, J64=J64.cpu().numpy(), K64=K64.cpu().numpy(), E64=E64,
                Jm=Jm.cpu().numpy(), Km=Km.cpu().numpy(), Em=Em, st=st, o=o, Q=o.schwarz())


def _w2_blocks(basis):
    """Shell pairs of workload 2 that stress the wide-exponent metal: its f-f,
    f-d and 8-primitive s-s pairs, a metal f with a ligand f, and a seeded
    ligand-ligand pair."""
    sh = lambda atom, l: [s for s in range(basis.nshell)
                          if int(basis.shell_atom[s]) == atom and int(basis.shell_l[s]) == l]
    mf, md, ms = sh(0, 3), sh(0, 2), sh(0, 0)
    lf = sh(5, 3)
    rng = np.random.default_rng(22)
    lig = [s for s in range(basis.nshell) if int(basis.shell_atom[s]) > 0]
    a, b = (int(x) for x in rng.choice(lig, 2, replace=False))
    return [(mf[1], mf[0]), (mf[0], md[2]), (ms[0], ms[1]), (mf[1], lf[0]), (ms[5], lf[0]), (a, b)]


def test_w2_fp64_metal_blocks_vs_oracle(eri, w2):
    """FP64 J and K blocks of the metal complex against the oracle's one-block
    sums within 1e-10; among them the blocks of the (fd|ff)- and (ff|ff)-class
    quartets on the metal and the 8-primitive s contractions."""
    basis, D, o, Q = w2["basis"], w2["D"], w2["o"], w2["Q"]
    off = basis.ao_offsets()
    assert int(basis.shell_nprim[0]) == 8 and float(basis.exps[:8].max()) > 1e3
    worst = 0.0
    for a, b in _w2_blocks(basis):
        sa, sb = slice(off[a], off[a + 1]), slice(off[b], off[b + 1])
        jr = o.j_block(D, a, b, THRESH, Q)
        kr = o.k_block(D, a, b, THRESH, Q)
        worst = max(worst, np.abs(w2["J64"][sa, sb] - jr).max(), np.abs(w2["K64"][sa, sb] - kr).max())
    print(f"workload 2 FP64 metal blocks: max abs difference {worst:.2e}")
    assert worst < 1e-10, worst


def test_w2_mixed_range_guard(eri, w2):
    """The mixed build of the metal complex at the bench tier bound: finite,
    symmetric, E_J and E_K within 1e-6 Eh of FP64, some quartets in FP32, and
    the FP32 range guard (exponent sum above 1e3 or prefactor product above
    1e18 keeps a quartet in FP64) did trip: without it the tight metal
    exponents overflow FP32."""
    st = w2["st"]
    print(f"workload 2 mixed: {st['quartets_k_fp32']} of {st['quartets_k']} quartets in FP32, "
          f"{st['quartets_k_guard']} kept in FP64 by the range guard; dE {w2['Em'] - w2['E64']}")
    assert st["quartets_k_fp32"] > 0
    assert st["quartets_k_guard"] > 0
    for M in (w2["Jm"], w2["Km"]):
        assert np.isfinite(M).all()
        assert np.abs(M - M.T).max() < 1e-12
    assert np.abs(w2["Em"] - w2["E64"]).max() < 1e-6


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
