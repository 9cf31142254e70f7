"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point that include/mcc.h declares (no GPU calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mcc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcc_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2501_06910_gb300 import native_build
    lib_path = native_build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings_and_defaults():
    import paper_2501_06910_gb300 as mcc
    p = mcc.params_default()
    assert (p.R1, p.R2, p.C1, p.C2, p.lmax) == (512, 512, 128, 128, 24)
    assert mcc.status_string(mcc.CORRUPT).startswith("corrupt")
