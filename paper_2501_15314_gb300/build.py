"""Builds libibmschur.so in-tree for sm_103a with nvcc (no cmake, no torch
extension machinery: the C ABI takes plain pointers).  Translation units are
compiled in parallel, then linked with the static CUDA runtime."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
LIB_NAME = "libibmschur.so"
SOURCES = ["capi.cu", "krylov.cu", "krylov_df.cu", "multigrid.cu", "markers.cu", "stencil.cu",
           "noalloc.cu", "adjoint.cu", "cmode.cu", "fsi.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or Path(cand).exists()):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def lib_path() -> Path:
    return PKG / LIB_NAME


def build(verbose: bool = False, force: bool = False) -> Path:
    out = lib_path()
    deps = [CSRC / s for s in SOURCES] + [CSRC / "ibm_internal.cuh", CSRC / "ds.cuh", INCLUDE / "ibm_schur.h"]
    if (not force and out.exists()
            and out.stat().st_mtime > max(p.stat().st_mtime for p in deps)):
        return out
    bdir = PKG / "_build"
    bdir.mkdir(exist_ok=True)
    nv = nvcc()
    objs = [bdir / (Path(s).stem + ".o") for s in SOURCES]
    cmds = [[nv, *ARCH, *FLAGS, "-c", str(CSRC / s), "-o", str(o)]
            for s, o in zip(SOURCES, objs)]
    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        logs = list(ex.map(_run, cmds))
    tmp = out.with_suffix(".so.tmp")
    logs.append(_run([nv, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]))
    os.replace(tmp, out)
    if verbose:
        for line in logs:
            if line.strip():
                print(line, file=sys.stderr)
    return out


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
