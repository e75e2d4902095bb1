"""Build step for the CUDA library: nvcc for sm_103a, one object per translation unit in
parallel, linked into ``libcitron.so`` next to this file (in-tree, git-ignored)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
OUT_DIR = PKG / "_build"
LIB = PKG / "libcitron.so"
# longest first: the deep k compile longest and start first
SOURCES = ["count_k12.cu", "count_k11.cu", "count_k10.cu", "count_k9.cu", "count_k8.cu", "count_k7.cu",
           "count_k3_6.cu", "count.cu", "api.cu", "order.cu", "sort.cu", "relabel.cu", "core.cu", "list.cu",
           "noalloc.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcitron.so")


def _inputs() -> list[Path]:
    return [CSRC / s for s in SOURCES] + list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h"))


def stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    return any(p.stat().st_mtime > t for p in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_report: bool = False) -> Path:
    """Compile the CUDA sources for sm_103a and link libcitron.so (skipped when up to date)."""
    if not force and not stale():
        return LIB
    OUT_DIR.mkdir(exist_ok=True)
    exe = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_report else []

    def compile_one(src: str):
        obj = OUT_DIR / (Path(src).stem + ".o")
        cmd = [exe, *ARCH, *FLAGS, *extra, "-c", str(CSRC / src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    for src, _, r in results:
        if verbose or ptxas_report:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = [exe, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", str(tmp), *[str(o) for _, o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_report="--ptxas" in sys.argv)
    print(LIB)
