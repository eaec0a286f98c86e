"""The CUDA path and the oracle are independent: the product package imports
and loads its library with the oracle made unimportable, none of its sources
(Python, CUDA, headers) names the oracle, and the library does not link the
oracle's shared object.  Runs without a GPU (no compute calls)."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2406_14920_gb300")


def test_package_loads_without_the_oracle():
    code = (
        "import sys, importlib.abc\n"
        "class Block(importlib.abc.MetaPathFinder):\n"
        "    def find_spec(self, name, path, target=None):\n"
        "        if name == 'oracle' or name.startswith('oracle.'):\n"
        "            raise ImportError('oracle is test infrastructure')\n"
        "        return None\n"
        "sys.meta_path.insert(0, Block())\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_2406_14920_gb300.build import build\n"
        "build()\n"
        "import paper_2406_14920_gb300 as eri\n"
        "L = eri.lib()\n"
        "assert L.eri_plan(None, None, None, None) == -1\n"
        "assert 'oracle' not in sys.modules\n"
        "print('ok')\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().endswith("ok")


def test_sources_do_not_name_the_oracle():
    pat = re.compile(r"\boracle\b|liboracle|\bor_[a-z_]+\(")
    for d, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(d, f)).read()
                hits = [m.group(0) for m in pat.finditer(txt)]
                assert not hits, (f, hits[:5])
    for f in os.listdir(os.path.join(ROOT, "include")):
        assert not pat.search(open(os.path.join(ROOT, "include", f)).read()), f


def test_library_does_not_link_the_oracle():
    so = os.path.join(PKG, "libgb300eri.so")
    if not os.path.exists(so):
        from paper_2406_14920_gb300.build import build
        build()
    out = subprocess.run(["ldd", so], capture_output=True, text=True).stdout
    assert "oracle" not in out
