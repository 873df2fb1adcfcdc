"""Builds libfos.so in-tree for sm_103a with nvcc (translation units in parallel).

    python -m paper_2409_00165_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfos.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "--expt-relaxed-constexpr", "-I", INCLUDE]
# Per-file flags.  The photon walk is compiled without FMA contraction so that its
# FP32 operation order is exactly the one written (fmaf only where written).
EXTRA = {
    "mc_walk.cu": ["-fmad=false"],
}
SOURCES = ["runtime.cu", "mc_walk.cu", "mc_walk_fast.cu", "mie.cu", "mlp.cu", "solar.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps_mtime() -> float:
    t = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".h", ".cuh", ".cpp")):
                t = max(t, os.path.getmtime(os.path.join(d, f)))
    return max(t, os.path.getmtime(__file__))


# The checked build (`build(checked=True)`): in-kernel index checks in the walk that set a
# status word instead of accessing out of bounds (the stand-in for a memory checker).
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libfos.so")


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    return os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    out_dir = BUILD_CHECKED if checked else BUILD
    if not force and up_to_date(checked):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    defines = ["-DFOS_CHECKED"] if checked else []

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *COMMON, *defines, *EXTRA.get(src, []), "-c",
               os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                ptxas_info="--ptxas" in sys.argv))
