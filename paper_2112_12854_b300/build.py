"""Build the CUDA library ``libep.so`` in-tree for sm_103a (B300).

    python -m paper_2112_12854_b300.build [--force] [--verbose]

Compiles ``csrc/*.cu`` and ``csrc/*.cpp`` with nvcc into
``paper_2112_12854_b300/libep.so``. nvcc cross-compiles, so this works on a
machine without a GPU.
"""
from __future__ import annotations

import argparse
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libep.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The kernels' FP32 arithmetic uses the hardware approximations (exp2/log2/rcp/rsqrt
# units, flush-to-zero); FP64 code is unaffected by these flags.
# kernels_tab.cu and kernels_f64.cu hold instances of the same step code and take the same flags.
FILE_FLAGS = {f: ["--use_fast_math"] for f in ("kernels.cu", "kernels_tab.cu", "kernels_f64.cu")}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _inputs():
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [__file__]
    return files


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and os.path.exists(LIB):
        if os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in _inputs()):
            return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    cmd_common = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp,-O3",
                  "-I", INCLUDE]
    if verbose:
        cmd_common += ["-Xptxas", "-v"]
    cmd_common += list(extra or [])
    jobs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = cmd_common + FILE_FLAGS.get(os.path.basename(src), []) + ["-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = cmd_common + ["-x", "cu", "-c", src, "-o", obj]
        jobs.append((src, obj, cmd))
    # the translation units compile independently: run them side by side
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda j: subprocess.run(j[2], capture_output=True, text=True), jobs))
    objs = []
    for (src, obj, _), r in zip(jobs, results):
        if r.returncode != 0 or verbose:
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}")
        objs.append(obj)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lgomp", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stderr)
        raise RuntimeError("nvcc link failed")
    os.replace(tmp, LIB)
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, verbose=a.verbose))


if __name__ == "__main__":
    main()
