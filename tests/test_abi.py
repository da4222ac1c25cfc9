"""The C ABI library loads and exports every entry point include/dtree.h
declares; calls rejected by argument checks never touch a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dtree.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1304_4327_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dtree_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_api():
    names = declared_functions()
    for required in ("dtree_build", "dtree_knn", "dtree_free", "dtree_error_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_argument_checks_need_no_gpu(lib):
    lib.dtree_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p(1)
    assert lib.dtree_build(None, 10, 3, None, None, ctypes.byref(out)) == -1
    assert out.value is None
    assert lib.dtree_build(ctypes.c_void_p(16), 10, 65, None, None, ctypes.byref(out)) == -1
    assert lib.dtree_build(ctypes.c_void_p(16), 0, 3, None, None, ctypes.byref(out)) == -1
    lib.dtree_knn.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int32] + [ctypes.c_void_p] * 5
    assert lib.dtree_knn(None, None, 3, None, None, None, None, None) == -1
    # the other instances reject a missing tree before any CUDA call too
    lib.dtree_kfn.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int32] + [ctypes.c_void_p] * 5
    assert lib.dtree_kfn(None, None, 3, None, None, None, None, None) == -1
    P, D = ctypes.c_void_p, ctypes.c_double
    lib.dtree_range_count.argtypes = [P, P, D, D, P, P, P, P, P]
    assert lib.dtree_range_count(None, None, 0.0, 1.0, None, None, None, None, None) == -1
    lib.dtree_range_fill.argtypes = [P, P, D, D, P, P, P, P, P]
    assert lib.dtree_range_fill(None, None, 0.0, 1.0, None, None, None, None, None) == -1
    lib.dtree_emst.argtypes = [P] * 6
    assert lib.dtree_emst(None, None, None, None, None, None) == -1
    lib.dtree_size.restype = ctypes.c_int64
    lib.dtree_size.argtypes = [ctypes.c_void_p]
    assert lib.dtree_size(None) == -1
    lib.dtree_free.argtypes = [ctypes.c_void_p]
    lib.dtree_free(None)


def test_error_strings(lib):
    lib.dtree_error_string.restype = ctypes.c_char_p
    for code in range(-7, 1):
        assert lib.dtree_error_string(code)
    assert b"k" in lib.dtree_error_string(-2)


def test_oracle_and_library_share_nothing():
    # the oracle never names the CUDA package; the package never names the oracle
    oracle_dir = os.path.join(ROOT, "oracle")
    for f in os.listdir(oracle_dir):
        if f.endswith((".c", ".py", ".h")):
            text = open(os.path.join(oracle_dir, f)).read()
            assert "csrc" not in text and "libdtree" not in text and "dtree_internal" not in text
    pkg = os.path.join(ROOT, "paper_1304_4327_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "liboracle" not in text, f


def _model_file(d=2, level=1, corrupt=False):
    """A well-formed model file (see dtree_model_save) with zero weights."""
    import struct
    H, C, dpad = 256, 1 << level, 16
    body = b"DTRMODL1" + struct.pack("<5i", d, dpad, H, C, level) + struct.pack("<Qq", 12345, 7)
    body += b"\0" * (4 * 2 * d)
    body += b"\0" * (4 * (H * dpad + H + H * H + H + C * H + C))
    h = 1469598103934665603
    for byte in body:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    data = bytearray(body + struct.pack("<Q", h))
    if corrupt:
        data[40] ^= 1
    return bytes(data)


def test_model_file_checks_need_no_gpu(lib, tmp_path):
    P = ctypes.c_void_p
    lib.dtree_model_load.argtypes = [ctypes.c_char_p, P, P, ctypes.POINTER(P)]
    out = P(1)
    assert lib.dtree_model_load(str(tmp_path / "missing.bin").encode(), None, None,
                                ctypes.byref(out)) == -9          # DTREE_ERR_IO
    assert out.value is None
    f = tmp_path / "m.bin"
    f.write_bytes(b"not a model file" * 8)
    assert lib.dtree_model_load(str(f).encode(), None, None, ctypes.byref(out)) == -9
    f.write_bytes(_model_file(corrupt=True))                      # checksum fails
    assert lib.dtree_model_load(str(f).encode(), None, None, ctypes.byref(out)) == -9
    f.write_bytes(_model_file()[:-9] + _model_file()[-8:])        # truncated
    assert lib.dtree_model_load(str(f).encode(), None, None, ctypes.byref(out)) == -9
    # a sound file passes every file check and then needs a tree
    f.write_bytes(_model_file())
    assert lib.dtree_model_load(str(f).encode(), None, None, ctypes.byref(out)) == -1
    lib.dtree_model_save.argtypes = [P, ctypes.c_char_p, P]
    assert lib.dtree_model_save(None, str(f).encode(), None) == -1
