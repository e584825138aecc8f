"""The C-ABI library without a GPU: it loads, exports every declared symbol,
and rejects invalid arguments on the host before any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_cs_0406049_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sincos_pairs.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    with open(HEADER) as f:
        text = f.read()
    return re.findall(r"^[a-z_ 0-9]+\**\s*\*?(sincos_\w+)\(", text, flags=re.M)


def test_header_declares_the_entry_points():
    names = set(declared_functions())
    for n in ("sincos_pairs", "sincos_batched", "sincos_backward", "sincos_pairs_ex",
              "sincos_pairs_host", "sincos_strerror"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), f"{name} declared but not exported"
        assert name in _lib.SIGNATURES, f"{name} has no Python binding"


def test_binding_declares_nothing_extra():
    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_selftest_validation(lib):
    assert lib.sincos_selftest_wait_timeout(0, None) == _lib.EINVAL
    assert lib.sincos_selftest_wait_timeout(1000001, None) == _lib.EINVAL   # over 1 s


def test_status_strings(lib):
    for st in (0, -1, -2, -3, -4, -5):
        assert lib.sincos_strerror(st)
    assert lib.sincos_version() >= 10000


# Fake device addresses: validation rejects these calls before touching CUDA.
A = 0x7f0000000000


@pytest.mark.parametrize("args,status", [
    ((A, A + 4096, A + 8192, -1, 0, 0, 0, None), _lib.EINVAL),            # n < 0
    ((None, A + 4096, A + 8192, 16, 0, 0, 0, None), _lib.EINVAL),         # null x
    ((A, None, A + 8192, 16, 0, 0, 0, None), _lib.EINVAL),                # null s
    ((A, A + 4096, A + 8192, 16, 3, 0, 0, None), _lib.EINVAL),            # bad dtype
    ((A, A + 4096, A + 8192, 16, 0, 2, 0, None), _lib.EINVAL),            # bad reduction
    ((A, A + 4096, A + 8192, 16, 0, 0, 2, None), _lib.EINVAL),            # bad coefficients
    ((A, A + 4096, A + 4100, 16, 0, 0, 0, None), _lib.EOVERLAP),          # s, c overlap
    ((A, A + 4, A + 8192, 16, 0, 0, 0, None), _lib.EOVERLAP),             # x partly in s
    ((A, A, A + 8192, 16, 1, 0, 0, None), _lib.EOVERLAP),                 # in place, 16-bit out
    ((A, A + 4096, A + 8192, 0, 0, 0, 0, None), _lib.OK),                 # n == 0
    ((None, None, None, 0, 0, 0, 0, None), _lib.OK),                      # n == 0, nulls
])
def test_forward_validation(lib, args, status):
    assert lib.sincos_pairs_ex(*args) == status


def test_expi_validation(lib):
    assert lib.sincos_expi(A, A + 4096, -1, 0, 0, None) == _lib.EINVAL
    assert lib.sincos_expi(None, A + 4096, 8, 0, 0, None) == _lib.EINVAL
    assert lib.sincos_expi(A, A + 4096, 8, 5, 0, None) == _lib.EINVAL
    assert lib.sincos_expi(A, A + 16, 8, 0, 0, None) == _lib.EOVERLAP      # z overlaps x
    assert lib.sincos_expi(A, A, 8, 0, 0, None) == _lib.EOVERLAP           # no in-place
    assert lib.sincos_expi(None, None, 0, 0, 0, None) == _lib.OK


def test_plain_forward_validation(lib):
    assert lib.sincos_pairs(A, A + 4096, A + 8192, -5, None) == _lib.EINVAL
    assert lib.sincos_pairs(A, A + 4096, A + 4096, 8, None) == _lib.EOVERLAP
    assert lib.sincos_pairs(A, A + 4096, A + 8192, 0, None) == _lib.OK


def test_backward_validation(lib):
    assert lib.sincos_backward(A, A + 4096, A + 8192, A + 12288, A + 16384, -1, None) == _lib.EINVAL
    assert lib.sincos_backward(A, A + 4096, A + 8192, A + 12288, None, 8, None) == _lib.EINVAL
    assert lib.sincos_backward(A, A + 4096, None, A + 12288, A + 16384, 8, None) == _lib.EINVAL
    # gx partially overlapping an input
    assert lib.sincos_backward(A, A + 4096, A + 8192, A + 12288, A + 8, 8, None) == _lib.EOVERLAP
    assert lib.sincos_backward(None, None, None, None, A, 0, None) == _lib.OK


def test_batched_validation(lib):
    assert lib.sincos_batched(A, A + 4096, -1, None) == _lib.EINVAL
    assert lib.sincos_batched(None, A + 4096, 4, None) == _lib.EINVAL
    assert lib.sincos_batched(A, None, 4, None) == _lib.EINVAL
    assert lib.sincos_batched(None, None, 0, None) == _lib.OK
    assert lib.sincos_batched_ex(A, A + 4096, 4, 7, 0, 0, None) == _lib.EINVAL
    h = ctypes.c_void_p()
    assert lib.sincos_batched_graph_create(A, A + 8, 0, 0, 0, 0, ctypes.byref(h)) == _lib.EINVAL
    assert lib.sincos_batched_graph_launch(None, None) == _lib.EINVAL
    assert lib.sincos_batched_graph_destroy(None) == _lib.EINVAL


def test_host_path_validation(lib):
    ws = A
    assert lib.sincos_pairs_host(A, A + 4096, A + 8192, -1, 0, 0, 0, ws, 1 << 20, None) == _lib.EINVAL
    assert lib.sincos_pairs_host(A, A + 4096, A + 8192, 8, 0, 0, 0, ws + 4, 1 << 20, None) == _lib.EINVAL
    assert lib.sincos_pairs_host(A, A + 4096, A + 8192, 8, 0, 0, 0, ws, 64, None) == _lib.EINVAL
    assert lib.sincos_pairs_host(A, A + 4096, A + 4100, 8, 0, 0, 0, ws, 1 << 20, None) == _lib.EOVERLAP
    assert lib.sincos_host_last_path() == _lib.HOST_PATH_NONE     # refused calls took no route
    assert lib.sincos_host_route_set(2) == _lib.EINVAL
    assert lib.sincos_host_route_set(_lib.HOST_ROUTE_PIPELINE) == _lib.OK
    assert lib.sincos_host_route_set(_lib.HOST_ROUTE_AUTO) == _lib.OK
    assert lib.sincos_host_workspace_bytes(0, 64) == 3 * 64 * 12
    assert lib.sincos_host_workspace_bytes(1, 65) == 3 * 128 * 8
    assert lib.sincos_host_workspace_bytes(5, 64) == 0


def test_plan_validation(lib):
    bad = _lib.sincos_plan(100, 4, 8, 0)       # block not a multiple of 32
    assert lib.sincos_plan_set(0, 0, 1 << 20, ctypes.byref(bad)) == _lib.EINVAL
    bad = _lib.sincos_plan(256, 3, 8, 0)       # unroll not 1/2/4/8
    assert lib.sincos_plan_set(0, 0, 1 << 20, ctypes.byref(bad)) == _lib.EINVAL
    bad = _lib.sincos_plan(96, 2, 1, 0)        # bulk path needs 128/256/512/1024 threads
    assert lib.sincos_plan_set(0, 0, 1 << 20, ctypes.byref(bad)) == _lib.EINVAL
    bad = _lib.sincos_plan(256, 4, 8, 64)      # vector width not 0/16/32
    assert lib.sincos_plan_set(0, 0, 1 << 20, ctypes.byref(bad)) == _lib.EINVAL
    good = _lib.sincos_plan(256, 4, 8, 0)
    assert lib.sincos_plan_set(9, 0, 1 << 20, ctypes.byref(good)) == _lib.EINVAL
    assert lib.sincos_plan_get(0, 0, 1 << 20, None) == _lib.EINVAL
    assert lib.sincos_plan_cache_load(b"/nonexistent/path.json") == _lib.EINVAL


def test_huygens_validation(lib):
    f = lambda *a: lib.sincos_huygens(*a)
    P = (A, A + 4096, A + 8192)
    Q = (A + 12288, A + 16384, A + 20480, A + 24576, A + 28672)
    U = A + 65536
    assert f(*P, -1, *Q, 8, 6.28, 1, U, None) == _lib.EINVAL
    assert f(*P, 8, *Q, -1, 6.28, 1, U, None) == _lib.EINVAL
    assert f(*P, 8, *Q, 8, 6.28, 7, U, None) == _lib.EINVAL
    assert f(None, A + 4096, A + 8192, 8, *Q, 8, 6.28, 1, U, None) == _lib.EINVAL
    assert f(*P, 8, None, *Q[1:], 8, 6.28, 1, U, None) == _lib.EINVAL
    assert f(*P, 8, *Q, 8, 6.28, 1, A + 4, None) == _lib.EOVERLAP      # u over px
    assert f(*P, 0, *Q, 8, 6.28, 1, U, None) == _lib.OK


def test_misaligned_pointers_are_rejected(lib):
    """A pointer not aligned to its element type is an invalid argument: the
    kernels' vector paths assume element alignment, so such a call must not
    reach the device."""
    stream = None
    assert lib.sincos_pairs_ex(A + 2, A + 4096, A + 8192, 8, 0, 0, 0, stream) == _lib.EINVAL
    assert lib.sincos_pairs_ex(A, A + 4097, A + 8192, 8, 0, 0, 0, stream) == _lib.EINVAL
    assert lib.sincos_pairs_ex(A, A + 4096, A + 8193, 8, 1, 0, 0, stream) == _lib.EINVAL  # bf16
    assert lib.sincos_pairs(A + 1, A + 4096, A + 8192, 8, stream) == _lib.EINVAL
    assert lib.sincos_backward(A + 1, None, A + 8192, A + 12288, A + 16384, 8, stream) == _lib.EINVAL
    assert lib.sincos_backward(A, A + 4096, A + 8192, A + 12288, A + 16386, 8, stream) == _lib.EINVAL
    assert lib.sincos_expi(A, A + 4098, 8, 0, 0, stream) == _lib.EINVAL
    assert lib.sincos_batched(A + 4, A + 4096, 4, stream) == _lib.EINVAL       # descriptors: 8 B
    assert lib.sincos_batched(A, A + 4100, 4, stream) == _lib.EINVAL          # lengths: 8 B
    assert lib.sincos_batched_noalloc(A + 4, A + 4096, 4, 0, 0, 0, stream) == _lib.EINVAL
    ws = A
    assert lib.sincos_pairs_host(A + 2, A + 4096, A + 8192, 8, 0, 0, 0, ws, 1 << 20, stream) == \
        _lib.EINVAL
    best = _lib.sincos_plan()
    assert lib.sincos_autotune_pairs(A + 2, A + 4096, A + 8192, 8, 0, 0, 0, stream,
                                     ctypes.byref(best)) == _lib.EINVAL


VALID_CACHE = ('{"version": 1, "plans": [\n'
               '  {"device": "test device \\"q\\":1", "op": 0, "dtype": 1, "bucket": 29, '
               '"block": 512, "unroll": 2, "ctas_per_sm": 2, "vec_bytes": 0},\n'
               '  {"device": "test device:1", "op": 4, "dtype": 0, "bucket": 19, '
               '"block": 256, "unroll": 1, "ctas_per_sm": 8, "vec_bytes": 32}\n]}\n')


@pytest.mark.parametrize("text,want", [
    (VALID_CACHE, "OK"),
    ('{"version": 1, "plans": []}', "OK"),
    ('{"version": 1}', "EINVAL"),                                     # no plans
    ('{"plans": {}}', "EINVAL"),                                      # plans not a list
    ('{"plans": [{"device": "d", "op": 0, "dtype": 0, "bucket": 3, '
     '"block": 100, "unroll": 2, "ctas_per_sm": 1, "vec_bytes": 16}]}', "EINVAL"),  # bad plan
    ('{"plans": [{"op": 0, "dtype": 0, "bucket": 3, "block": 256, "unroll": 2, '
     '"ctas_per_sm": 1, "vec_bytes": 16}]}', "EINVAL"),              # no device
    ('{"plans": [{"device": "d", "op": x}]}', "EINVAL"),              # not a number
    ('{"plans": [{"device" "d"}]}', "EINVAL"),                        # no colon
    ('{"plans": [{device: "d"}]}', "EINVAL"),                         # key not a string
    ('{"plans": [{"device": "unterminated', "EINVAL"),                # truncated string
    ('{"plans": [{"device": "d", "op": 0', "EINVAL"),                 # truncated object
    ('', "EINVAL"),
])
def test_plan_cache_reader(lib, tmp_path, text, want):
    """The plan-cache reader needs no GPU: valid files load, malformed or
    truncated ones are refused with EINVAL (and nothing is read past the end)."""
    path = tmp_path / "plans.json"
    path.write_text(text)
    assert lib.sincos_plan_cache_load(str(path).encode()) == getattr(_lib, want)


def test_seg_check_every_alignment(lib):
    """The descriptor check the batched kernels apply, on the host: for every
    combination of byte offsets 0..7 of x, s and c, null pointers, each output
    dtype and lengths around zero, a descriptor passes exactly when its length
    is <= 0 or all three pointers are non-null with x on a 4-byte and s, c on
    an element boundary of the output dtype."""
    base = 1 << 24
    size = {_lib.F32: 4, _lib.BF16: 2, _lib.F16: 2}
    seg = _lib.sincos_seg()
    checked = 0
    for dt, osz in size.items():
        for length in (-7, -1, 0, 1, 3, 1 << 40):
            for ox in range(8):
                for os_ in range(8):
                    for oc in range(8):
                        for nulls in range(8):
                            x = 0 if nulls & 1 else base + ox
                            s = 0 if nulls & 2 else 2 * base + os_
                            c = 0 if nulls & 4 else 3 * base + oc
                            seg.x, seg.s, seg.c = x, s, c
                            want = length <= 0 or (
                                nulls == 0 and ox % 4 == 0 and os_ % osz == 0 and oc % osz == 0)
                            got = lib.sincos_seg_check(ctypes.byref(seg), length, dt)
                            assert got == (_lib.OK if want else _lib.EINVAL), (dt, length, x, s, c)
                            checked += 1
    assert checked == 3 * 6 * 8 ** 4
    assert lib.sincos_seg_check(None, 1, _lib.F32) == _lib.EINVAL
    seg.x, seg.s, seg.c = base, base, base
    assert lib.sincos_seg_check(ctypes.byref(seg), 1, 7) == _lib.EINVAL
