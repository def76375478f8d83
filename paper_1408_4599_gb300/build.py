"""Builds libmdgpu.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit in ``csrc/`` (the force kernel's instantiation file
once per signature and stencil radius) is compiled in parallel with nvcc
into ``_build/``, then linked into ``paper_1408_4599_gb300/libmdgpu.so``.  The
compiled objects are not tracked by git.
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
LIB = os.path.join(HERE, "libmdgpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ftz=true: FP32 subnormals flush to zero (no FP32 quantity of the method
# comes near 1e-38); measured 1-7% faster force kernels
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-ftz=true", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I" + os.path.join(ROOT, "include"), "--extended-lambda"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


# Sources compiled once per variant (one object per set of defines): the
# force kernel's instantiations, one per compiled signature (the order of
# dispatch_sig) and stencil radius, so that they compile in parallel.
VARIANTS = {
    "md_force_inst.cu": [(f"s{sig}m{m}", [f"-DMD_FORCE_SIG={sig}", f"-DMD_FORCE_M={m}"])
                         for sig in range(6) for m in (1, 2)],
}


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def units():
    """(source, object, extra nvcc flags) of every object of the library."""
    out = []
    for src in sources():
        base = os.path.basename(src)[:-3]
        for tag, defs in VARIANTS.get(os.path.basename(src), [("", [])]):
            out.append((src, os.path.join(BUILD, base + ("_" + tag if tag else "") + ".o"), defs))
    return out


def _deps():
    return sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
        [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    todo = units()
    objs = [obj for _, obj, _ in todo]

    def compile_one(unit):
        src, obj, defs = unit
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, "-c", src, "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {' '.join(defs)}:\n{p.stderr}")
        return p.stderr

    # the slowest objects first, so that they do not start last
    order = sorted(todo, key=lambda u: 0 if u[2] else 1)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 8, len(order)))) as ex:
        logs = list(ex.map(compile_one, order))
    if verbose or ptxas_info:
        for (src, obj, defs), log in zip(order, logs):
            if log.strip():
                print(f"== {os.path.basename(obj)}\n{log}", file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    # no undefined symbols: a missing instantiation fails here, not at load
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-Xlinker", "--no-undefined"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
