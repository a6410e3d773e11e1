"""Build libffmin.so (CUDA, sm_103a) in-tree with nvcc.

Translation units are compiled in parallel and linked into
paper_1810_03358_gb300/libffmin.so.  control/minimizer code is compiled with
-fmad=false (no implicit a*b+c contraction); the pair kernels keep FMA.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libffmin.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "pair.cu": ["-ftz=true"],
    "minimizer.cu": ["-fmad=false"],
    "parab.cu": ["-fmad=false"],
    "mlp.cu": [],
    "noalloc.cu": [],
    "peak.cu": [],
    "api.cu": [],
}


def nvcc():
    for p in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    raise RuntimeError("nvcc not found")


def _sources():
    return [u for u in UNITS if os.path.exists(os.path.join(CSRC, u))]


def _deps():
    out = [os.path.join(ROOT, "include", "ffmin.h"), __file__]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in _deps())
        if os.path.getmtime(LIB) >= newest:
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
              "-I", CSRC] + ARCH + os.environ.get("FFMIN_NVCC_FLAGS", "").split()
    if ptxas_v:
        common += ["-Xptxas", "-v"]

    def compile_one(u):
        obj = os.path.join(BUILD, u.replace(".cu", ".o"))
        cmd = [nv] + common + UNITS[u] + ["-c", os.path.join(CSRC, u), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose or ptxas_v:
        for obj, err in results:
            if err:
                print(err, file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nv, "-shared"] + ARCH + ["-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas" in sys.argv))
