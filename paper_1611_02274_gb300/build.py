"""Build ``libbatchode.so`` in-tree with nvcc for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled in parallel to an object
file, then linked into a shared library with the static CUDA runtime.  No
PyTorch headers or libraries are involved.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbatchode.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, "-I", BUILD]
# device headers compiled again at run time (NVRTC) for generated right-hand sides
JIT_HEADERS = [os.path.join(CSRC, h) for h in (
    "common.cuh", "f2.cuh", "team.cuh", "xmath.cuh", "rkc_coef.cuh", "integrators.cuh", "integrators_f2.cuh",
    "kernels.cuh", "rhs.cuh", "mlp.cuh", "mlp_warp.cuh")]


def write_jit_sources() -> None:
    """Embed the device headers as string literals for the run-time compiler."""
    delim = "BODEJIT"
    names, bodies = [], []
    for path in JIT_HEADERS:
        text = open(path).read()
        assert ")" + delim + "\"" not in text
        names.append(os.path.basename(path))
        bodies.append(text)
    # the public header's constants (its function declarations are host code)
    import re
    consts = ["#define %s %s" % m.groups() for m in
              re.finditer(r"^#define (ODE_\w+)\s+(\(?-?\w+\)?)", open(os.path.join(INCLUDE, "batchode.h")).read(), re.M)]
    names.insert(0, "batchode.h")
    bodies.insert(0, "#pragma once\n" + "\n".join(consts) + "\n")
    out = ["// generated by build.py: device headers for the run-time compiler"]
    out.append("static const char* const kJitHeaderNames[] = {" + ", ".join('"%s"' % n for n in names) + "};")
    out.append("static const char* const kJitHeaderSources[] = {")
    for b in bodies:
        out.append('R"%s(%s)%s",' % (delim, b, delim))
    out.append("};")
    out.append("static const int kJitHeaderCount = %d;" % len(names))
    text = "\n".join(out) + "\n"
    path = os.path.join(BUILD, "jit_sources.inc")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as fh:
            fh.write(text)


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found; the CUDA library cannot be built")
    return path


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stamp() -> str:
    h = hashlib.sha256()
    for p in _deps() + [os.path.abspath(__file__)]:
        with open(p, "rb") as fh:
            h.update(p.encode() + fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + ["fmad-split"]).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    stamp_file = os.path.join(BUILD, "stamp")
    stamp = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read() == stamp:
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    write_jit_sources()
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
        if src.endswith("_f64.cu"):
            # plain FP64 form: every operation rounded exactly as written
            cmd.insert(1, "--fmad=false")
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart=static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
