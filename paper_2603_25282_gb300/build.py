"""Build libsgp.so (the C-ABI CUDA library) in-tree for sm_103a.

Compiles the translation units in parallel with nvcc and links them into
``paper_2603_25282_gb300/libsgp.so``.  Object files go to
``paper_2603_25282_gb300/_build/``.  Rebuilds only when a source is newer
than the library (or when ``force`` is set).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsgp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]

# (object name, source, extra defines)
UNITS = [
    ("api", "sgp_api.cu", []),
    ("adjoint_flo", "sgp_adjoint.cu", ["-DSGP_REAL=float", "-DSGP_REDUCE_PARAMS=1"]),
    ("adjoint_dou", "sgp_adjoint.cu", ["-DSGP_REAL=double"]),
    ("lab", "sgp_lab.cu", []),
    ("persist_flo", "sgp_persist.cu", ["-DSGP_REAL=float", "-DSGP_PERSIST_DEFINE_SUPPORTED=1"]),
    ("persist_dou", "sgp_persist.cu", ["-DSGP_REAL=double"]),
] + [
    ("inst_%s_%s_v%d" % (r[0:3], "xl"[part], v), "sgp_inst.cu",
     ["-DSGP_REAL=%s" % r, "-DSGP_PART=%d" % part, "-DSGP_VAR=%d" % v]
     + (["-DSGP_LINE_TMA=1"] if (r, part, v) == ("float", 1, 1) else [])
     + (["-DSGP_XY_PLANE=1"] if (r, part, v) == ("float", 0, 1) else []))
    for r, nv in (("float", 4), ("double", 3)) for part in (0, 1) for v in range(nv)
]


def nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsgp.so")


def _sources():
    return glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(ROOT, "include", "*.h"))


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _compile(unit, verbose):
    name, src, defs = unit
    obj = os.path.join(BUILD, name + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, jobs=None):
    """Compile and link libsgp.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = jobs or min(len(UNITS), os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda u: _compile(u, verbose), UNITS))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
