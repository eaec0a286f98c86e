"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no normalisation, no integrals, no screening).  Both the
oracle (``oracle/``) and the product library consume its output.

A basis is a list of shells in user order.  Each shell has an atom index, an
angular momentum l (0..3, Cartesian), and a contiguous run of primitives with
exponents and *raw* contraction coefficients.  Normalising those coefficients
is each implementation's own job (paper Sec. 2.1, Eq. contracted_basis and
Eq. primtive_basis; the reading of the normalisation is documented there).

Workloads follow the five synthetic systems of the hot-path specification:
  0  3 atoms, 3s2p1d1f each (75 bf)                       -- parity-size case
  1  60 atoms: 40 light 2s1p + 20 heavy 4s3p2d1f (900 bf)  -- organic-like
  2  metal 6s5p3d2f + 48 ligands 3s2p1d1f (1259 bf)        -- metal complex
  3  30 atoms 3s2p1d1f (750 bf)                            -- gradient case
  4  64 molecules of 10-80 atoms, mixed light/heavy        -- batched case
Seeds are 1000 + workload index.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

L_CHAR = {"s": 0, "p": 1, "d": 2, "f": 3}


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


@dataclass
class Basis:
    shell_atom: np.ndarray      # int32 [nshell]
    shell_l: np.ndarray         # int32 [nshell]
    shell_nprim: np.ndarray     # int32 [nshell]
    shell_prim_offset: np.ndarray  # int32 [nshell]
    exps: np.ndarray            # float64 [nprim_total]
    coefs: np.ndarray           # float64 [nprim_total], raw (unnormalised)
    coords: np.ndarray          # float64 [natom, 3], bohr
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def natom(self) -> int:
        return int(self.coords.shape[0])

    @property
    def nbf(self) -> int:
        return int(sum(ncart(int(l)) for l in self.shell_l))

    def ao_offsets(self) -> np.ndarray:
        off = np.zeros(self.nshell + 1, dtype=np.int64)
        off[1:] = np.cumsum([ncart(int(l)) for l in self.shell_l])
        return off

    def with_coords(self, coords: np.ndarray) -> "Basis":
        return Basis(self.shell_atom, self.shell_l, self.shell_nprim, self.shell_prim_offset,
                     self.exps, self.coefs, np.ascontiguousarray(coords, dtype=np.float64),
                     self.name, dict(self.meta))


@dataclass
class ShellSpec:
    l: int
    nprim: int
    exp_lo: float
    exp_hi: float


def _draw_shell(rng, spec: ShellSpec):
    e = np.exp(rng.uniform(np.log(spec.exp_lo), np.log(spec.exp_hi), size=spec.nprim))
    c = rng.uniform(0.1, 1.0, size=spec.nprim)
    return e, c


def atom_shells(composition: str, sp_prims=3, sp_range=(0.1, 50.0), df_range=(0.3, 3.0),
                s_prims=None, all_range=None) -> list[ShellSpec]:
    """Shell specs for a composition string like '3s2p1d1f' (s/p contracted,
    d/f single primitives unless all_range is given)."""
    specs = []
    i = 0
    while i < len(composition):
        j = i
        while composition[j].isdigit():
            j += 1
        count, l = int(composition[i:j]), L_CHAR[composition[j]]
        for _ in range(count):
            if all_range is not None:
                np_ = (s_prims if (l == 0 and s_prims) else (3 if l == 1 else 1))
                specs.append(ShellSpec(l, np_, *all_range))
            elif l <= 1:
                specs.append(ShellSpec(l, sp_prims, *sp_range))
            else:
                specs.append(ShellSpec(l, 1, *df_range))
        i = j + 1
    return specs


def build_basis(rng, coords: np.ndarray, atom_specs: list[list[ShellSpec]], name="") -> Basis:
    sa, sl, sn, so, ex, co = [], [], [], [], [], []
    off = 0
    for a, specs in enumerate(atom_specs):
        for s in sorted(specs, key=lambda s: s.l):
            e, c = _draw_shell(rng, s)
            sa.append(a); sl.append(s.l); sn.append(s.nprim); so.append(off)
            ex.extend(e.tolist()); co.extend(c.tolist())
            off += s.nprim
    return Basis(np.asarray(sa, np.int32), np.asarray(sl, np.int32), np.asarray(sn, np.int32),
                 np.asarray(so, np.int32), np.asarray(ex, np.float64), np.asarray(co, np.float64),
                 np.ascontiguousarray(coords, dtype=np.float64), name)


def random_packing(rng, natom: int, side: float, dmin: float, max_tries=200000) -> np.ndarray:
    """Sequential rejection: atoms uniform in a cube, each kept only if it is at
    least dmin from every atom already placed."""
    pts = []
    tries = 0
    while len(pts) < natom:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("packing failed")
        x = rng.uniform(0.0, side, size=3)
        if all(np.linalg.norm(x - p) >= dmin for p in pts):
            pts.append(x)
    return np.asarray(pts)


def density_from_orbitals(rng, nbf: int, nocc: int) -> np.ndarray:
    """D = C C^T with C an nbf x nocc matrix with orthonormal columns."""
    q, _ = np.linalg.qr(rng.standard_normal((nbf, nocc)))
    d = q @ q.T
    return np.ascontiguousarray(0.5 * (d + d.T))


def workload(i: int, seed: int | None = None):
    """Return (basis, D) for workload i (or a list of them for workload 4)."""
    seed = 1000 + i if seed is None else seed
    rng = np.random.default_rng(seed)
    if i == 0:
        while True:
            c = rng.uniform(0.0, 4.0, size=(3, 3))
            d = [np.linalg.norm(c[a] - c[b]) for a in range(3) for b in range(a)]
            if min(d) >= 1.8:
                break
        basis = build_basis(rng, c, [atom_shells("3s2p1d1f") for _ in range(3)], "w0_3atoms_75bf")
        return basis, density_from_orbitals(rng, basis.nbf, 10)
    if i == 1:
        n = 60
        coords = random_packing(rng, n, (n * 70.0) ** (1 / 3), 2.0)
        heavy = np.zeros(n, bool)
        heavy[rng.permutation(n)[:20]] = True
        specs = [atom_shells("4s3p2d1f") if h else atom_shells("2s1p") for h in heavy]
        basis = build_basis(rng, coords, specs, "w1_60atoms_900bf")
        return basis, density_from_orbitals(rng, basis.nbf, 120)
    if i == 2:
        coords = [np.zeros(3)]
        while len(coords) < 49:
            r = rng.uniform(2.5, 9.0)
            v = rng.standard_normal(3)
            x = r * v / np.linalg.norm(v)
            if all(np.linalg.norm(x - p) >= 2.0 for p in coords):
                coords.append(x)
        coords = np.asarray(coords)
        metal = atom_shells("6s5p3d2f", s_prims=8, all_range=(0.05, 2.0e4))
        specs = [metal] + [atom_shells("3s2p1d1f") for _ in range(48)]
        basis = build_basis(rng, coords, specs, "w2_metal_1259bf")
        return basis, density_from_orbitals(rng, basis.nbf, 150)
    if i == 3:
        n = 30
        coords = random_packing(rng, n, (n * 70.0) ** (1 / 3), 2.0)
        basis = build_basis(rng, coords, [atom_shells("3s2p1d1f") for _ in range(n)], "w3_30atoms_750bf")
        return basis, density_from_orbitals(rng, basis.nbf, 100)
    if i == 4:
        out = []
        for m in range(64):
            while True:
                n = int(rng.integers(10, 81))
                frac = rng.uniform(0.2, 0.6)
                heavy = rng.uniform(size=n) < frac
                nbf = int(heavy.sum()) * 35 + int((~heavy).sum()) * 5
                if 100 <= nbf <= 2000:
                    break
            coords = random_packing(rng, n, (n * 70.0) ** (1 / 3), 2.0)
            specs = [atom_shells("4s3p2d1f") if h else atom_shells("2s1p") for h in heavy]
            basis = build_basis(rng, coords, specs, f"w4_mol{m}_{nbf}bf")
            out.append((basis, density_from_orbitals(rng, basis.nbf, -(-basis.nbf // 7))))
        return out
    raise ValueError(i)


def small_system(compositions: list[str], seed: int = 7, side: float = 3.0, dmin: float = 1.2,
                 nocc: int | None = None):
    """A small seeded molecule for unit tests: one atom per composition string."""
    rng = np.random.default_rng(seed)
    coords = random_packing(rng, len(compositions), side, dmin)
    basis = build_basis(rng, coords, [atom_shells(c) for c in compositions], "small")
    nocc = nocc or max(1, basis.nbf // 3)
    return basis, density_from_orbitals(rng, basis.nbf, nocc)


def subset_atoms(basis: Basis, D: np.ndarray, atoms: list[int]):
    """Restrict a basis (and its density) to the given atoms, keeping order."""
    keep = [s for s in range(basis.nshell) if int(basis.shell_atom[s]) in atoms]
    amap = {a: i for i, a in enumerate(atoms)}
    off = basis.ao_offsets()
    ao = np.concatenate([np.arange(off[s], off[s + 1]) for s in keep])
    sa, sl, sn, so, ex, co = [], [], [], [], [], []
    p = 0
    for s in keep:
        o, n = int(basis.shell_prim_offset[s]), int(basis.shell_nprim[s])
        sa.append(amap[int(basis.shell_atom[s])]); sl.append(int(basis.shell_l[s])); sn.append(n); so.append(p)
        ex.extend(basis.exps[o:o + n]); co.extend(basis.coefs[o:o + n]); p += n
    b = Basis(np.asarray(sa, np.int32), np.asarray(sl, np.int32), np.asarray(sn, np.int32),
              np.asarray(so, np.int32), np.asarray(ex), np.asarray(co),
              np.ascontiguousarray(basis.coords[atoms]), basis.name + "_sub")
    return b, np.ascontiguousarray(D[np.ix_(ao, ao)])
