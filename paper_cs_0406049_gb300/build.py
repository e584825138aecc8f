"""Build ``libsincos_gb300.so`` in-tree with nvcc for sm_103a.

Each ``csrc/*.cu`` file compiles in parallel to an object under ``_build/``,
then nvcc links the shared library next to this file.  The library is rebuilt
only when a source, header or flag changes (a tag file holds their hash).

Numerics flags: ``-fmad=false`` (no contraction of separate multiplies and
adds), ``-ftz=false`` (keep binary32 subnormals), ``-prec-div=true`` and
``-prec-sqrt=true`` (IEEE division and square root); the kernels also use
explicitly rounded intrinsics, so every result is bit-reproducible.
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libsincos_gb300.so")
CONTEXT_SRC = os.path.join(HERE, "context", "cuda_libm.cu")
# The CUDA sincosf context kernels under three sets of nvcc floating-point
# flags: the defaults; -use_fast_math (which also maps sincosf to the
# __sincosf intrinsic); and the -prec-div / -prec-sqrt / -ftz switches of
# fast math alone, without the intrinsic mapping.
CONTEXT_VARIANTS = {
    "default": [],
    "use_fast_math": ["-use_fast_math"],
    "prec_off_ftz": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
}


def context_lib_path(variant: str = "default") -> str:
    return os.path.join(HERE, "context", f"libsincos_context_{variant}.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-lineinfo", "-O3", "-std=c++17",
    "-fmad=false", "-ftz=false", "-prec-div=true", "-prec-sqrt=true",
    "-Xcompiler", "-fPIC,-O2,-Wall",
    "-I", INCLUDE, "-I", CSRC,
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _tag(extra) -> str:
    h = hashlib.sha1()
    files = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(CSRC, "*.h"))) + sorted(glob.glob(os.path.join(INCLUDE, "*.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + list(extra)).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile and link the library if it is missing or stale; return its path."""
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    tag = _tag(extra)
    tag_file = LIB + ".srctag"
    if not force and os.path.exists(LIB) and os.path.exists(tag_file):
        with open(tag_file) as f:
            if f.read().strip() == tag:
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}{r.stderr}")
        return obj, r.stderr

    # longest translation units first, so the pool finishes evenly
    srcs = sorted(_sources(), key=lambda f: -os.path.getsize(f) -
                  (1 << 20 if os.path.basename(f).startswith(("batched_", "forward_")) else 0))
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose or ptxas_verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}{r.stderr}")
    os.replace(tmp, LIB)
    with open(tag_file, "w") as f:
        f.write(tag)
    return LIB


def build_context(force: bool = False, variant: str = "default") -> str:
    """The CUDA sincosf / __sincosf comparison kernels (benchmark context only),
    compiled with one of the CONTEXT_VARIANTS flag sets."""
    flags = CONTEXT_VARIANTS[variant]
    lib = context_lib_path(variant)
    tag_file = lib + ".srctag"
    with open(CONTEXT_SRC, "rb") as f:
        tag = hashlib.sha1(f.read() + " ".join(ARCH + flags).encode()).hexdigest()[:16]
    if not force and os.path.exists(lib) and os.path.exists(tag_file):
        with open(tag_file) as f:
            if f.read().strip() == tag:
                return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", *flags, "-Xcompiler", "-fPIC", "-shared", "-o", tmp, CONTEXT_SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on cuda_libm.cu ({variant}):\n{r.stdout}{r.stderr}")
    os.replace(tmp, lib)
    with open(tag_file, "w") as f:
        f.write(tag)
    return lib


def build_context_all(force: bool = False) -> dict:
    """Every context variant, compiled in parallel; {variant: library path}."""
    with ThreadPoolExecutor(max_workers=len(CONTEXT_VARIANTS)) as ex:
        paths = list(ex.map(lambda v: build_context(force, v), CONTEXT_VARIANTS))
    return dict(zip(CONTEXT_VARIANTS, paths))


if __name__ == "__main__":
    p = build(force="--force" in sys.argv, verbose=True,
              ptxas_verbose="--ptxas-verbose" in sys.argv)
    print(p)
    print(build_context_all(force="--force" in sys.argv))
