"""The C ABI from C: tests/c_abi_example.c is compiled with gcc against
include/sincos_pairs.h, linked with the library and the CUDA runtime (CPU
test), and run on the GPU with its results compared bit for bit with the
oracle (GPU test)."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from gpu_util import assert_f32_parity
from paper_cs_0406049_gb300 import build as libbuild

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def compile_example(out_dir: str) -> str:
    lib = libbuild.build()
    libdir = os.path.dirname(lib)
    exe = os.path.join(out_dir, "c_abi_example")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(HERE, "c_abi_example.c"), "-o", exe,
           "-L", libdir, "-l:" + os.path.basename(lib),
           "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_example_compiles_and_links(tmp_path):
    exe = compile_example(str(tmp_path))
    assert os.access(exe, os.X_OK)


@pytest.mark.gpu
def test_c_example_matches_the_oracle(tmp_path):
    exe = compile_example(str(tmp_path))
    n = (1 << 20) + 3
    out = str(tmp_path / "pairs.bin")
    r = subprocess.run([exe, str(n), out], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    raw = np.fromfile(out, dtype=np.float32)
    assert raw.size == 4 * n
    x = (np.arange(n, dtype=np.float64) * 0.001 - 500.0).astype(np.float32)
    want_s, want_c = oracle.sincos(x)
    assert_f32_parity(raw[:n], want_s, "C caller s")
    assert_f32_parity(raw[n:2 * n], want_c, "C caller c")
    z = raw[2 * n:].reshape(n, 2)
    assert_f32_parity(z[:, 0].copy(), want_c, "C caller exp(ix) real")
    assert_f32_parity(z[:, 1].copy(), want_s, "C caller exp(ix) imag")
