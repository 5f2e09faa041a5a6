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
    assert ctypes.sizeof(pv.pv_variant) == 16 * 4 + 8  # 16 int32 fields, the uint64 seed
    assert ctypes.sizeof(pv.pv_ht_variant) == 16 + 8 + 8


def test_library_fails_loudly_when_missing(tmp_path):
    with pytest.raises(RuntimeError):
        pv._lib = None
        pv.load(str(tmp_path / "libpv.so"))
    pv._lib = None


def _c_layout(tmp_path, structs):
    """sizeof and offsetof of every field of the given structs, as the C
    compiler lays them out from include/pv.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pv.h"', "int main(void) {"]
    for name, st in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


def test_binding_layout_matches_the_c_compiler(tmp_path):
    structs = {n: getattr(pv, n) for n in ("pv_ref", "pv_pred", "pv_term", "pv_agg", "pv_probe", "pv_build_spec",
                                           "pv_ht_variant", "pv_pipeline_spec", "pv_variant")}
    c = _c_layout(tmp_path, structs)
    for name, st in structs.items():
        assert c[(name, "sizeof")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert c[(name, f)] == getattr(st, f).offset, (name, f)
