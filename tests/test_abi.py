"""The C-ABI library loads and exports every entry point include/pv.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

from paper_1709_00700_gb300 import build, pv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pv.h")).read()
    return sorted(set(re.findall(r"^\s*(?:pv_status|const char\*)\s+(pv_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pv_create", "pv_register_column", "pv_build_hash_table", "pv_run_pipeline", "pv_fetch_result"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert sorted(pv.EXPORTS) == _declared()


def test_binding_structs_match_header_sizes():
    # sizes follow from the C declarations with natural alignment
    assert ctypes.sizeof(pv.pv_ref) == 12
    assert ctypes.sizeof(pv.pv_pred) == 24
    assert ctypes.sizeof(pv.pv_term) == 24
    assert ctypes.sizeof(pv.pv_agg) == 8 + 3 * 24
    assert ctypes.sizeof(pv.pv_variant) == 13 * 4 + 4 + 8  # 4 bytes of padding before the uint64 seed
    assert ctypes.sizeof(pv.pv_ht_variant) == 16 + 8 + 8


def test_library_fails_loudly_when_missing(tmp_path):
    with pytest.raises(RuntimeError):
        pv._lib = None
        pv.load(str(tmp_path / "libpv.so"))
    pv._lib = None
