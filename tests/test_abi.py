"""The C-ABI library builds, loads and exports every symbol include/fkski.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fkski.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"FKSKI_API\s+[\w\s\*]*?\b(fkski_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_11751_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("fkski_precompute", "fkski_solve", "fkski_predict", "fkski_grad"):
        assert required in names
    assert len(names) >= 16


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    """Calls that touch no device: defaults and status strings."""
    from paper_2101_11751_gb300 import api
    api.load()
    o = api.opts()
    assert o.maxiter == 1000 and abs(o.rtol - 1e-6) < 1e-18 and o.check_every == 16
    lib.fkski_strerror.restype = ctypes.c_char_p
    assert lib.fkski_strerror(0) == b"ok"
    assert b"grid" in lib.fkski_strerror(-2)
    assert lib.fkski_strerror(-99) == b"unknown status"


def test_struct_layouts_match_header():
    """ctypes mirrors of the C structs have the sizes the header implies on LP64."""
    from paper_2101_11751_gb300 import api
    assert ctypes.sizeof(api.CGrid) == 8 + 3 * 8 * 3
    assert ctypes.sizeof(api.CKernel) == 8 + 3 * 8 + 8 + 8
    # rtol, 5 ints, pad, seed, budget, keep_sort, reserved[7]
    assert ctypes.sizeof(api.COpts) == 80


def test_product_path_has_no_cpu_fallback(tmp_path):
    """Loading from a missing path fails loudly instead of falling back."""
    from paper_2101_11751_gb300 import api
    saved = api._lib
    try:
        api._lib = None
        with pytest.raises(RuntimeError):
            api.load(str(tmp_path / "nope.so"))
    finally:
        api._lib = saved
