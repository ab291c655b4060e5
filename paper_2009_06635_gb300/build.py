"""Build the C-ABI shared library libpdfgb300.so for sm_103a, and beside it
the measurement/test hooks of probe/ as libpdfgb300_probe.so.

Each .cu file is compiled by nvcc in parallel, then linked into its shared
library in _lib/ (git-ignored).  Usage:
    python -m paper_2009_06635_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
PROBE = PKG / "probe"
INCLUDE = ROOT / "include"
OUT_DIR = PKG / "_lib"
LIB = OUT_DIR / "libpdfgb300.so"
PROBE_LIB = OUT_DIR / "libpdfgb300_probe.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}", f"-I{PROBE}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (Path(cand).exists() or cand == "nvcc"):
            return cand
    return "nvcc"


def sources():
    return sorted(CSRC.glob("*.cu"))


def _stale(deps, target: Path) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> Path:
    """Build both libraries; returns the evaluation library's path."""
    OUT_DIR.mkdir(parents=True, exist_ok=True)
    headers = list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h")) + list(PROBE.glob("*.h"))
    flags = NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + list(extra_flags or [])
    libs = {LIB: sources(), PROBE_LIB: sorted(PROBE.glob("*.cu"))}
    objs, jobs = {}, []
    for lib, srcs in libs.items():
        objs[lib] = []
        for src in srcs:
            obj = OUT_DIR / (src.stem + ".o")
            objs[lib].append(obj)
            if force or _stale([src, *headers], obj):
                jobs.append([nvcc(), *ARCH, *flags, "-c", str(src), "-o", str(obj)])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    for lib, o in objs.items():
        if force or jobs or _stale(o, lib):
            tmp = lib.with_suffix(f".{os.getpid()}.tmp")
            cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", str(tmp), *map(str, o)]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError("link failed")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB, PROBE_LIB)
