"""In-tree build of libhpclust.so for sm_103a (nvcc, no CMake).

Each translation unit is compiled in parallel, then linked into a shared
library next to this file.  Objects go to ``_build/`` (git-ignored).
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
OUT = PKG / "libhpclust.so"
OBJ = PKG / "_build"
SOURCES = ["capi.cu", "lloyd.cu", "kmeanspp.cu", "sample.cu", "tc_objective.cu", "tc_split.cu", "noalloc.cu",
           "peaks.cu", "tc_wide.cu", "costmodel.cu", "tc_bf16.cu"]
HEADERS = ["common.cuh", "assign.cuh", "kernels.h", "tc.cuh", "round.cuh", "tc_rows.cuh", "costmodel.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _inputs():
    return ([CSRC / s for s in SOURCES] + [CSRC / h for h in HEADERS]
            + [PKG.parent / "include" / "hpclust.h", Path(__file__)])


def stale() -> bool:
    if not OUT.exists():
        return True
    t = OUT.stat().st_mtime
    return any(p.stat().st_mtime > t for p in _inputs())


def _nvcc(args):
    r = subprocess.run([NVCC] + args, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed: {' '.join(args)}\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> Path:
    if not force and not stale():
        return OUT
    OBJ.mkdir(exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", str(PKG.parent / "include"), "--expt-relaxed-constexpr"]
    if verbose:
        common += ["-Xptxas", "-v"]

    def one(src):
        o = OBJ / (Path(src).stem + ".o")
        log = _nvcc(common + ["-c", str(CSRC / src), "-o", str(o)])
        return o, log

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(one, SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    tmp = OUT.with_suffix(f".{os.getpid()}.tmp.so")
    _nvcc(ARCH + ["-shared", "-o", str(tmp)] + [str(o) for o, _ in results])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(OUT)
