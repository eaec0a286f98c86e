"""Write the oracle's full FP64 J and K of a seeded workload to tests/golden/.

The stored matrices are the reference for the element-by-element full-size
parity test of the GPU build (tests/test_gpu_fullsize.py).  They come from the
oracle alone: J_mn = sum_ls (mn|ls) D_ls and K_ml = sum_ns (mn|ls) D_ns
(Eq. j_definition, Eq. k_definition) over the canonical quartets whose Schwarz
bound Q_ab Q_cd >= thresh (Eq. kernel_upperbound), every contracted ERI by
Obara-Saika / Head-Gordon-Pople, energies E_J = 1/2 tr(DJ), E_K = -1/4 tr(DK)
(SI Eq. si_E_J_K) in long double.  Nothing here touches the CUDA library.

J and K are symmetric for a symmetric D; the file holds the upper triangles of
(J + J^T)/2 and (K + K^T)/2 (symmetrising moves an element by rounding only)
plus the oracle's own energies and Schwarz bounds, keyed by the basis (shell
table exactly; exponents, raw coefficients and coordinates to 1e-13 relative:
the exponents come through exp(), whose last bit differs between libm
builds), thresh, and 4096 entries of D at seeded positions (D comes from a QR
factorisation, whose last bits depend on the BLAS library and its thread
count, so they are compared to 1e-12).  A test uses the key to tell when the
workload generator has changed and the file is stale.

Usage:  python tests/golden/make_oracle_jk.py 1          (about 2 h on 6 cores)
        python tests/golden/make_oracle_jk.py 1 --rekey  (rewrite the keys of an existing file)
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

THRESH = 1e-12


def golden_path(wl: int) -> str:
    return os.path.join(HERE, f"oracle_jk_w{wl}.npz")


def shell_hash(basis, thresh: float) -> str:
    """SHA-256 over the integer shell table and the threshold (exact on every platform)."""
    h = hashlib.sha256()
    for a in (basis.shell_atom, basis.shell_l, basis.shell_nprim, basis.shell_prim_offset):
        h.update(np.ascontiguousarray(a, np.int32).tobytes())
    h.update(np.float64(thresh).tobytes())
    return h.hexdigest()


def basis_floats(basis) -> np.ndarray:
    """Exponents, raw coefficients and coordinates, concatenated."""
    return np.concatenate([basis.exps, basis.coefs, basis.coords.reshape(-1)]).astype(np.float64)


def d_fingerprint(D) -> np.ndarray:
    """4096 entries of D at seeded positions (compared to 1e-12 absolute: the
    element-wise J/K tolerance is 1e-10, and BLAS rounding moves D by ~1e-15)."""
    rng = np.random.default_rng(99)
    i = rng.integers(0, D.shape[0], 4096)
    j = rng.integers(0, D.shape[1], 4096)
    return np.ascontiguousarray(D[i, j])


def upper(M: np.ndarray) -> np.ndarray:
    S = 0.5 * (M + M.T)
    return S[np.triu_indices(M.shape[0])]


def from_upper(u: np.ndarray, n: int) -> np.ndarray:
    M = np.zeros((n, n))
    iu = np.triu_indices(n)
    M[iu] = u
    M.T[iu] = u
    return M


def load(wl: int):
    """(J, K, E_J, E_K, Q) from the stored file, or None if absent."""
    p = golden_path(wl)
    if not os.path.exists(p):
        return None
    z = np.load(p)
    n = int(z["nbf"])
    return from_upper(z["J_upper"], n), from_upper(z["K_upper"], n), float(z["E_J"]), float(z["E_K"]), z["Q"]


def matches(wl: int, basis, D) -> bool:
    """True if the stored file was made for this basis and (to rounding) this D."""
    p = golden_path(wl)
    if not os.path.exists(p):
        return False
    z = np.load(p)
    if "shell_sha256" not in z or str(z["shell_sha256"]) != shell_hash(basis, THRESH):
        return False
    bf = basis_floats(basis)
    return (z["basis_floats"].shape == bf.shape and np.allclose(z["basis_floats"], bf, rtol=1e-13, atol=0.0)
            and float(np.abs(z["d_fingerprint"] - d_fingerprint(D)).max()) < 1e-12)


def keys(basis, D) -> dict:
    return {"shell_sha256": np.str_(shell_hash(basis, THRESH)), "basis_floats": basis_floats(basis),
            "d_fingerprint": d_fingerprint(D)}


def rekey(wl: int) -> None:
    """Rewrite the keys of an existing file (J, K, energies and Q are kept as the oracle wrote them)."""
    basis, D = workloads.workload(wl)
    z = {k: v for k, v in np.load(golden_path(wl)).items() if k != "input_sha256"}
    z.update(keys(basis, D))
    np.savez_compressed(golden_path(wl), **z)


def main(wl: int) -> None:
    basis, D = workloads.workload(wl)
    o = oracle.Oracle(basis)
    t0 = time.time()
    Q = o.schwarz()
    J, K = o.jk(D, thresh=THRESH, Q=Q, mode=1)
    ej, ek = o.energy(D, J, K)
    dt = time.time() - t0
    asym = max(float(np.abs(J - J.T).max()), float(np.abs(K - K.T).max()))
    np.savez_compressed(golden_path(wl), nbf=np.int64(basis.nbf), J_upper=upper(J), K_upper=upper(K),
                        E_J=np.float64(ej), E_K=np.float64(ek), Q=Q, thresh=np.float64(THRESH),
                        **keys(basis, D), oracle_seconds=np.float64(dt), oracle_threads=np.int64(oracle.max_threads()),
                        max_asymmetry=np.float64(asym))
    print(f"workload {wl}: nbf {basis.nbf}, E_J {ej:.15e}, E_K {ek:.15e}, {dt:.0f} s on "
          f"{oracle.max_threads()} threads, max |M - M^T| {asym:.2e} -> {golden_path(wl)}")


if __name__ == "__main__":
    wl_ = int(sys.argv[1]) if len(sys.argv) > 1 else 1
    if "--rekey" in sys.argv:
        rekey(wl_)
    else:
        main(wl_)
