"""Build the CUDA library libgb300eri.so in-tree (sm_103a only).

Each csrc/*.cu is compiled to an object in parallel (one nvcc per file), then
linked into paper_2406_14920_gb300/libgb300eri.so.  csrc/k_unit.cu and
csrc/g_unit.cu are compiled once per entry of csrc/units.h (bra class,
precision and, for J/K, the ket classes, passed as -D flags), so the class
kernels of one bra class compile in parallel.  Objects
go to _build/ (ignored by git).  Rebuilds only what changed (any header change
rebuilds all).
"""
from __future__ import annotations

import glob
import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(ROOT, "_build", "obj")
SO = os.path.join(HERE, "libgb300eri.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-diag-suppress", "177"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers_mtime() -> float:
    hs = (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
          glob.glob(os.path.join(ROOT, "include", "*.h")))
    return max([os.path.getmtime(h) for h in hs] + [0.0])


def jk_units() -> list[tuple[int, int, int, int]]:
    """(bra class, precision, first ket class, last ket class) of every J/K entry of csrc/units.h."""
    txt = open(os.path.join(CSRC, "units.h")).read()
    return [tuple(int(v) for v in m) for m in re.findall(r"U\((\d+), (\d+), (\d+), (\d+)\)", txt)]


def grad_units() -> list[tuple[int, int]]:
    """(bra class, precision) of every gradient entry of csrc/units.h."""
    txt = open(os.path.join(CSRC, "units.h")).read()
    return [tuple(int(v) for v in m) for m in re.findall(r"U\((\d+), (\d+)\)", txt)]


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    unit_src = os.path.join(CSRC, "k_unit.cu")
    gunit_src = os.path.join(CSRC, "g_unit.cu")
    jobs_list = [(s, os.path.join(OBJ, os.path.basename(s)[:-3] + ".o"), [])
                 for s in sorted(glob.glob(os.path.join(CSRC, "*.cu"))) if s not in (unit_src, gunit_src)]
    for x, p, ylo, yhi in jk_units():
        jobs_list.append((unit_src, os.path.join(OBJ, f"k_unit_{x}_{p}_{ylo}_{yhi}.o"),
                          [f"-DERI_UNIT_X={x}", f"-DERI_UNIT_P={p}", f"-DERI_UNIT_YLO={ylo}", f"-DERI_UNIT_YHI={yhi}"]))
    for x, p in grad_units():
        jobs_list.append((gunit_src, os.path.join(OBJ, f"g_unit_{x}_{p}.o"), [f"-DERI_UNIT_X={x}", f"-DERI_UNIT_P={p}"]))
    hdr = _headers_mtime()
    todo = []
    objs = []
    for s, o, defs in jobs_list:
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            todo.append((s, o, defs))
    stale = [f for f in glob.glob(os.path.join(OBJ, "*.o")) if f not in objs]
    for f in stale:  # objects of removed sources must not be linked
        os.remove(f)
    nvcc = _nvcc()

    def compile_one(so):
        s, o, defs = so
        cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {s}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        if verbose:
            print("compiled", os.path.basename(s), file=sys.stderr)

    if todo:
        jobs = jobs or min(len(todo), max(1, os.cpu_count() or 1))
        # heaviest translation units first: FP32 class units of high bra classes, then the rest by size
        def weight(so):
            name = os.path.basename(so[1])
            if name.startswith("k_unit_"):
                _, _, x, p, _, _ = name[:-2].split("_")
                return -1000 - 10 * int(x) - 100 * int(p)
            if name.startswith("g_unit_"):
                _, _, x, p = name[:-2].split("_")
                return -1000 - 12 * int(x)
            return -os.path.getsize(so[0])
        todo.sort(key=weight)
        with ThreadPoolExecutor(jobs) as ex:
            list(ex.map(compile_one, todo))
    if todo or not os.path.exists(SO):
        tmp = SO + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
