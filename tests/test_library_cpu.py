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


def test_parameter_checks_on_the_host():
    """The library's own parameter checks, through host-only entry points
    (sizes of the 1D coder): the zero-run stage's limits, the 1D coder's
    option limits, and sizes that do not depend on the stage."""
    import pytest
    import paper_2501_06910_gb300 as mcc
    n = 100_000
    base = mcc.compress_bound_1d(n, mcc.params_default())
    assert mcc.compress_bound_1d(n, mcc.params_default(zero_run=True)) == base
    cw0, dw0 = mcc.workspace_size_1d(n, mcc.params_default())
    cw1, dw1 = mcc.workspace_size_1d(n, mcc.params_default(zero_run=True))
    assert cw1 == cw0 and dw1 == dw0
    for kw, status in ((dict(zero_run=2), mcc.INVALID_ARG),
                       (dict(zero_run=True, R1=2048), mcc.UNSUPPORTED),
                       (dict(zero_run=True, R1=8, R2=8, lmax=4), mcc.INVALID_ARG),
                       (dict(R1=2049), mcc.UNSUPPORTED), (dict(C1=257), mcc.UNSUPPORTED),
                       (dict(lmax=25), mcc.UNSUPPORTED), (dict(eb=-1.0), mcc.INVALID_ARG),
                       (dict(f_op=1), mcc.INVALID_ARG), (dict(g_op=1), mcc.INVALID_ARG),
                       (dict(loop=1), mcc.INVALID_ARG)):
        with pytest.raises(mcc.MCCError) as err:
            mcc.compress_bound_1d(n, mcc.params_default(**kw))
        assert err.value.status == status, kw
    mcc.compress_bound_1d(n, mcc.params_default(R1=8, R2=8, lmax=4))  # fits without the stage
