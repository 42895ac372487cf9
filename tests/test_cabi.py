"""The C-ABI library builds, loads without a GPU and exports every declared symbol (CPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "mm.h")) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(mm_[a-z_A-Z0-9]+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("mm_plan", "mm_apply_A", "mm_precond", "mm_build_coarse", "mm_solve", "mm_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1408_3048_gb300 import build, mm
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(mm.EXPORTS) == _declared()
    assert lib.mm_version
    fn = lib.mm_version
    fn.restype = ctypes.c_char_p
    assert b"sm_103a" in fn()


def test_null_arguments_are_rejected_without_a_gpu():
    from paper_1408_3048_gb300 import mm
    L = mm.lib()
    h = ctypes.c_void_p()
    assert L.mm_plan(ctypes.byref(h), None, 0, 0, None, None, 0, None, None, 0, None) == mm.MM_ERR_ARG
    assert h.value is None
    assert L.mm_apply_A(None, 0, None, None) == mm.MM_ERR_ARG
    L.mm_destroy(None)
