"""The packed pair (two angles per packed FP32 instruction, used by the
Huygens kernel and the binary32 bulk tiles) against the scalar pair on every
binary32 input, bit for bit, for both reductions and both coefficient sets.  The scalar pair is itself compared with the oracle on every input
(test_gpu_exhaustive.py), so together the packed pair equals the oracle on
every input.  The checker kernel (tests/pair_x2_check.cu) is compiled with
the library's own numerics flags; the CPU test only compiles it."""
import ctypes
import os
import subprocess

import pytest

from paper_cs_0406049_gb300 import build as libbuild

HERE = os.path.dirname(os.path.abspath(__file__))


def compile_checker(out_dir: str) -> str:
    so = os.path.join(out_dir, "libpair_x2_check.so")
    cmd = [libbuild.nvcc(), *libbuild.NVCC_FLAGS, "-shared", "-o", so,
           os.path.join(HERE, "pair_x2_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return so


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return compile_checker(str(tmp_path_factory.mktemp("pair_x2")))


def test_checker_compiles(checker):
    assert os.path.getsize(checker) > 0


@pytest.mark.gpu
@pytest.mark.parametrize("coef", [0, 1], ids=["normalized", "dagger"])
@pytest.mark.parametrize("red", [0, 1], ids=["plain", "compensated"])
def test_packed_pair_equals_scalar_pair_on_every_input(cuda_lib, checker, red, coef):
    lib = ctypes.CDLL(checker)
    lib.pair_x2_check.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong),
                                  ctypes.POINTER(ctypes.c_uint)]
    mis, first = ctypes.c_ulonglong(0), ctypes.c_uint(0)
    rc = lib.pair_x2_check(red, coef, ctypes.byref(mis), ctypes.byref(first))
    assert rc == 0, f"CUDA error {rc}"
    assert mis.value == 0, f"{mis.value} mismatching pairs, first input bits 0x{first.value:08x}"
