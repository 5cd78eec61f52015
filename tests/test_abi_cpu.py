"""C ABI checks that need no GPU: the library builds for sm_103a, exports every
symbol include/rlfc.h declares, and its host-side stream validation rejects
corrupt or unsupported streams before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1805_06019_gb300 import buildlib as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rlfc.h")

E_INVALID_ARG, E_FORMAT, E_UNSUPPORTED = 1, 2, 3


@pytest.fixture(scope="module")
def lib():
    path = pkg_build.build()
    L = ctypes.CDLL(path)
    L.rlfc_load_stream.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]
    L.rlfc_strerror.restype = ctypes.c_char_p
    L.rlfc_last_error.restype = ctypes.c_char_p
    return L


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"RLFC_API\s+[\w\s\*]+?\b(rlfc_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_header(lib):
    from paper_1805_06019_gb300 import rlfc
    assert sorted(rlfc.EXPORTS) == _declared()


def test_binding_chooses_the_debug_library_only_when_asked(monkeypatch):
    from paper_1805_06019_gb300 import rlfc
    monkeypatch.delenv("RLFC_DEBUG_LIBRARY", raising=False)
    assert rlfc.library_path() == pkg_build.LIB
    monkeypatch.setenv("RLFC_DEBUG_LIBRARY", "1")
    assert rlfc.library_path() == pkg_build.LIB_DEBUG
    monkeypatch.setenv("RLFC_DEBUG_LIBRARY", "0")
    assert rlfc.library_path() == pkg_build.LIB
    assert pkg_build.LIB != pkg_build.LIB_DEBUG


def test_debug_build_exports_the_same_symbols_and_refuses_null_arguments(lib):
    """The RLFC_DEBUG build (device bounds checks) has the same C ABI; the
    flag query refuses null arguments before any device call, in both builds."""
    dbg = ctypes.CDLL(pkg_build.build(debug=True))
    for n in _declared():
        assert hasattr(dbg, n), n
    f = ctypes.c_uint32(7)
    for L in (lib, dbg):
        L.rlfc_debug_flags.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        assert L.rlfc_debug_flags(None, ctypes.byref(f), 0) == E_INVALID_ARG
        assert L.rlfc_debug_flags(None, None, 1) == E_INVALID_ARG


def test_strerror_covers_every_code(lib):
    texts = [lib.rlfc_strerror(c).decode() for c in range(8)]
    assert len(set(texts)) == 8
    assert lib.rlfc_strerror(99).decode() == "unknown status"


def _load(lib, data: bytes):
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(data, len(data))
    rc = lib.rlfc_load_stream(buf, len(data), None, ctypes.byref(h))
    return rc, h


def _stream():
    rng = np.random.default_rng(0)
    lf = rng.integers(0, 256, size=(9, 12, 16, 3), dtype=np.uint8)
    return bytearray(oracle.encode(lf, 3, 3, B=4, L=2, c=[0, 3], tau_p=3, tau_b=20))


def test_null_arguments_are_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.rlfc_load_stream(None, 10, None, ctypes.byref(h)) == E_INVALID_ARG
    assert lib.rlfc_decode_all(None, None, None) == E_INVALID_ARG
    assert lib.rlfc_stream_info(None, None) == E_INVALID_ARG
    lib.rlfc_free_stream(None)


def test_corrupt_streams_fail_host_validation(lib):
    s = _stream()
    off_offsets = int.from_bytes(s[48:52], "little")
    off_records = int.from_bytes(s[52:56], "little")
    cases = {}
    b = bytearray(s); b[0] ^= 0xFF; cases["magic"] = b
    b = bytearray(s); b[4] = 2; cases["version"] = b
    cases["truncated"] = s[:-4]
    cases["short"] = s[:40]
    b = bytearray(s); b[off_offsets + 4:off_offsets + 8] = (10 ** 6).to_bytes(4, "little"); cases["offsets"] = b
    b = bytearray(s); b[64 + 8 * 2:64 + 8 * 2 + 4] = (77).to_bytes(4, "little"); cases["parent"] = b
    # first stored block's mode := 31
    b = bytearray(s)
    mask = int.from_bytes(b[off_records:off_records + 4], "little")
    assert mask != 0
    b[off_records + 4] |= 31
    cases["mode"] = b
    # a presence bit beyond the last of the S = 9 nodes
    b = bytearray(s); b[off_records + 1] |= 0x80; cases["mask"] = b
    for name, data in cases.items():
        rc, h = _load(lib, bytes(data))
        assert rc == E_FORMAT, (name, rc, lib.rlfc_last_error())
        assert not h.value


def test_block_size_other_than_four_is_unsupported(lib):
    rng = np.random.default_rng(1)
    lf = rng.integers(0, 256, size=(4, 8, 8, 3), dtype=np.uint8)
    data = oracle.encode(lf, 2, 2, B=2, L=2, c=[0, 2])
    rc, _ = _load(lib, data)
    assert rc == E_UNSUPPORTED
    assert "4x4" in lib.rlfc_last_error().decode()


def test_values_beyond_the_16_bit_range_are_unsupported(lib):
    # a top value of 6000 exceeds the largest magnitude the kernels hold
    # exactly (5460: the inverse YCoCg-R reaches 3M + 2 < 2^14); the same
    # stream with an in-range value passes validation and fails only later,
    # without a GPU, at the device copy
    s = _stream()
    off_top = int.from_bytes(s[44:48], "little")
    big = bytearray(s); big[off_top:off_top + 2] = (6000).to_bytes(2, "little", signed=True)
    rc, h = _load(lib, bytes(big))
    assert rc == E_UNSUPPORTED and not h.value
    assert "16-bit" in lib.rlfc_last_error().decode()
    ok = bytearray(s); ok[off_top:off_top + 2] = (-300).to_bytes(2, "little", signed=True)
    rc, h = _load(lib, bytes(ok))
    assert rc not in (E_FORMAT, E_UNSUPPORTED), lib.rlfc_last_error()
    if h.value:
        lib.rlfc_free_stream(h)
