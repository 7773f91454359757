"""The C ABI library loads and exports every entry point include/*.h declares, and the Python
binding mirrors them by name and struct size.  No compute call: runs without a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:epbr_status|const char\*)\s+(epbr_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["epbr_precompute_ibl", "epbr_shade", "epbr_ssao", "epbr_tonemap"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2012_03325_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol_and_matches_struct_sizes():
    from paper_2012_03325_gb300 import _ffi
    names = set(_ffi.exported_names())
    assert set(declared_functions()) <= names
    # struct sizes of the ctypes mirror (x86-64 / aarch64 LP64 ABI)
    assert ctypes.sizeof(_ffi.epbr_camera) == 76
    assert ctypes.sizeof(_ffi.epbr_light) == 32
    assert ctypes.sizeof(_ffi.epbr_bloom_params) == 20
    assert ctypes.sizeof(_ffi.epbr_shadows) == 32
    assert ctypes.sizeof(_ffi.epbr_edl_params) == 12
    assert ctypes.sizeof(_ffi.epbr_mesh) == 32
    assert ctypes.sizeof(_ffi.epbr_surfels) == 16
    assert ctypes.sizeof(_ffi.epbr_gbuffer) == 16 + 32 + 32
    assert ctypes.sizeof(_ffi.epbr_ssao_params) == 48
    assert ctypes.sizeof(_ffi.epbr_ibl) == 8 + 8 + 8 + 8 + 16 * 8 + 16 * 4 * 2


def test_binding_constants_match_the_header():
    """Every enumerator of include/*.h (EPBR_NAME = value) exists in the binding with its value."""
    from paper_2012_03325_gb300 import _ffi
    consts = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
            for name, val in re.findall(r"\b(EPBR_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
                consts[name] = int(val)
    assert consts.get("EPBR_SHADE_EARLY_START") == 16
    wrong = {n: (v, getattr(_ffi, n, None)) for n, v in consts.items() if getattr(_ffi, n, None) != v}
    assert not wrong, wrong


def test_oracle_is_not_imported_by_the_product():
    for f in glob.glob(os.path.join(ROOT, "paper_2012_03325_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".inc")):
            txt = open(f).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f
            assert "epbr_oracle" not in txt, f


def test_product_fails_loudly_without_library(tmp_path):
    from paper_2012_03325_gb300 import _ffi
    with pytest.raises(OSError):
        ctypes.CDLL(str(tmp_path / "libepbr.so"))
    assert _ffi.LIB_PATH.endswith("libepbr.so")
