"""The Huygens term's distance and its reciprocal (core_rt.cuh: Markstein's
Newton schemes from rsqrt.approx and rcp.approx) against the correctly
rounded square root and reciprocal on every binary32 input, bit for bit, in
the scalar and the packed form.  Together with the oracle parity of the
Huygens sums (test_gpu_huygens.py) this shows the kernels compute each term
with IEEE sqrt and division, as the oracle does.  The checker kernel
(tests/root_recip_check.cu) is compiled with the library's own numerics
flags; the CPU test only compiles it."""
import ctypes
import os
import subprocess

import pytest

from paper_cs_0406049_gb300 import build as libbuild

HERE = os.path.dirname(os.path.abspath(__file__))


def compile_checker(out_dir: str) -> str:
    so = os.path.join(out_dir, "libroot_recip_check.so")
    cmd = [libbuild.nvcc(), *libbuild.NVCC_FLAGS, "-shared", "-o", so,
           os.path.join(HERE, "root_recip_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return so


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return compile_checker(str(tmp_path_factory.mktemp("root_recip")))


def test_checker_compiles(checker):
    assert os.path.getsize(checker) > 0


@pytest.mark.gpu
def test_root_and_reciprocal_on_every_input(cuda_lib, checker):
    lib = ctypes.CDLL(checker)
    lib.root_recip_check.argtypes = [ctypes.POINTER(ctypes.c_ulonglong),
                                     ctypes.POINTER(ctypes.c_uint)]
    mis = (ctypes.c_ulonglong * 2)()
    first = (ctypes.c_uint * 2)()
    rc = lib.root_recip_check(mis, first)
    assert rc == 0, f"CUDA error {rc}"
    assert mis[0] == 0, f"scalar: {mis[0]} mismatches, first input bits 0x{first[0]:08x}"
    assert mis[1] == 0, f"packed: {mis[1]} mismatches, first input bits 0x{first[1]:08x}"
