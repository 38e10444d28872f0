"""The C-ABI library builds, loads and exports every entry point that
include/ttgb.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2211_08770_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ttgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("tt_add", "tt_dot", "tt_round", "tt_orthogonalize", "tt_round_batched", "tt_norm"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_no_gpu_error_path(lib):
    lib.tt_status_str.restype = ctypes.c_char_p
    assert lib.tt_status_str(0) == b"TT_OK"
    assert lib.tt_status_str(4) == b"TT_ERR_NOT_SPD"


def test_binding_names_match_the_abi():
    from paper_2211_08770_gb300 import ttgb
    for n in ("tt_add", "tt_dot", "tt_dot_many", "tt_norm", "tt_round", "tt_round_batched", "tt_orthogonalize",
              "tt_scale", "tt_tensor_create", "tt_tensor_wrap_device"):
        assert callable(getattr(ttgb, n))
    assert set(ttgb._SIGS) <= set(_declared())
