"""CPU checks of the boundary: libxt builds for sm_103a, loads, and exports
every entry point that include/xt.h declares (no compute call: no GPU here)."""
import ctypes
import os
import re

import pytest

import paper_2301_09310_gb300 as xt
from paper_2301_09310_gb300 import build as xbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "xt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(xt_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    path = xbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("xt_ctx_create", "xt_ctx_destroy", "xt_extend_batch", "xt_extend_batch_plain",
              "xt_extend_batch_host", "xt_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"libxt does not export {name}"


def test_binding_names_match_header():
    names = set(declared_functions())
    assert set(xt.EXPORTED) == names
    for n in names:
        assert hasattr(xt, n), f"binding lacks {n}"


def test_status_strings_without_gpu(lib):
    lib.xt_status_str.restype = ctypes.c_char_p
    assert lib.xt_status_str(0) == b"XT_OK"
    assert lib.xt_status_str(1) == b"XT_EINVAL"
    assert lib.xt_status_str(99) == b"XT_UNKNOWN"


def test_null_context_is_rejected(lib):
    # argument checks happen before any CUDA call
    assert lib.xt_ctx_create(None, 0, 0) == 1
    assert lib.xt_ctx_destroy(None) == 1
    assert lib.xt_ctx_set_schedule(None, 4, 8) == 1


def test_pack4_layout():
    # base p is the low nibble of byte p // 2 when p is even, the high one when odd
    import numpy as np
    codes = np.array([0, 1, 2, 3, 4, 3, 2], np.uint8)
    packed = xt.pack4(codes)
    assert packed.tolist() == [0x10, 0x32, 0x34, 0x02]
    unpacked = np.stack([packed & 15, packed >> 4], axis=1).reshape(-1)[:codes.size]
    assert np.array_equal(unpacked, codes)
    assert xt.pack4(np.array([200], np.uint8)).tolist() == [15]


def test_alphabet_values_match_header():
    src = open(os.path.join(ROOT, "include", "xt.h")).read()
    for name in ("XT_ALPHABET_CODES", "XT_ALPHABET_ASCII", "XT_ALPHABET_PACKED4"):
        m = re.search(rf"#define {name} (\d+)", src)
        assert m and int(m.group(1)) == getattr(xt, name)
