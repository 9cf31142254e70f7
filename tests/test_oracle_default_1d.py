"""Pins of the oracle's 1D coder (the paper's "default": the vertex array in
storage order through the same coder, Sec. V): the codes against an
independent FP64 quantisation with the bin recomputed from its definition,
the reconstruction s (K + Q), the bound at every value with no raw values
(including the inputs that make the method's guard store raw values),
closed forms, errors."""
import math

import numpy as np
import pytest

import oracle
import synth


def _hdr(s):
    return dict(s=float(s[104:112].view(np.float64)[0]), K=int(s[112:120].view(np.int64)[0]),
                flags=int(s[20:24].view(np.uint32)[0]), dim=int(s[16:20].view(np.uint32)[0]))


def _spacing(M, dtype):
    p, tiny = (52, 2.0 ** -1074) if dtype == np.float64 else (23, 2.0 ** -149)
    if M <= 0:
        return tiny
    m, e = math.frexp(M)
    return max(math.ldexp(1.0, e - 1 - p), tiny)


def _tau(x, eb, mode="rel"):
    x = x.astype(np.float64)
    return eb * (x.max() - x.min()) if mode == "rel" and x.max() > x.min() else eb


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
def test_default_1d_codes_and_bound(dtype, eb):
    c, e = synth.mesh2d_jittered(nside=80, seed=4)
    x = synth.field_bumps_noise(c, seed=9).astype(dtype)
    s, Q = oracle.compress_1d(x, debug=True, eb=eb)
    h = _hdr(s)
    assert h["dim"] == 1 and h["flags"] == 32
    # the bin from its definition: 2 (tau - m) (1 - 2^-20)
    xd = x.astype(np.float64)
    tau = _tau(x, eb)
    M = np.abs(xd).max()
    m = 4 * _spacing(M, np.float64) + (2 * _spacing(M, np.float32) if dtype == np.float32 else 0)
    assert h["s"] == (2.0 * (tau - m)) * (1 - 2.0 ** -20)
    inv = 1.0 / h["s"]
    assert h["K"] == int(np.rint(xd.min() * inv))
    assert np.array_equal(Q, np.rint(xd * inv).astype(np.int64) - h["K"])
    y = oracle.decompress_1d(s, x.size)
    assert y.dtype == dtype
    assert np.array_equal(y, (h["s"] * (h["K"] + Q.astype(np.int64)).astype(np.float64)).astype(dtype))
    assert np.abs(y.astype(np.float64) - xd).max() <= tau


@pytest.mark.parametrize("dtype,offset,eb", [(np.float32, 1.2e4, 5e-3), (np.float64, 3.0e9, 1e-1),
                                             (np.float32, 3.0e5, 0.1), (np.float64, 1.0, 1e-7)])
def test_default_1d_bound_without_raw_values(dtype, offset, eb):
    """Large values in bins of the bound, where the method's guard stores raw
    values: the margin keeps every value within tau. Where the value type's
    spacing itself exceeds the margin's room (FP32 at 1.2e4 has spacing
    2^-10 > tau = 9e-4), no bin can keep the bound without raw values and
    the coder reports a range error."""
    c, e = synth.mesh2d_jittered(nside=60, seed=5)
    x = (synth.field_bumps_noise(c, seed=7) + offset).astype(dtype)
    s = oracle.compress_1d(x, eb=eb, eb_mode="abs")
    y = oracle.decompress_1d(s, x.size)
    assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= eb
    assert int(s[160:168].view(np.uint64)[0]) == 0  # no raw values
    xs = (synth.field_bumps_noise(c, seed=7) + 1.2e4).astype(np.float32)
    with pytest.raises(oracle.OracleError) as err:
        oracle.compress_1d(xs, eb=9e-4, eb_mode="abs")
    assert err.value.status == 4


def test_default_1d_binade_edges():
    """Values on both sides of powers of two (where the spacing jumps)."""
    rng = np.random.default_rng(3)
    x = np.concatenate([np.nextafter(2.0 ** k, 0) * rng.choice([-1, 1], 64) for k in range(-3, 12)] +
                       [2.0 ** k + np.zeros(64) for k in range(-3, 12)])
    for dtype, ebs in ((np.float64, (1e-4, 1e-2, 0.5)), (np.float32, (5e-3, 0.05, 0.5))):
        xx = x.astype(dtype)
        for eb in ebs:
            s = oracle.compress_1d(xx, eb=eb, eb_mode="abs")
            y = oracle.decompress_1d(s, xx.size)
            assert np.abs(y.astype(np.float64) - xx.astype(np.float64)).max() <= eb


def test_default_1d_closed_forms():
    # a constant field: every code equal, every difference but the first 0
    x = np.full(5000, 2.5)
    s, Q = oracle.compress_1d(x, debug=True, eb=1e-3)
    assert np.all(Q == Q[0])
    assert np.abs(oracle.decompress_1d(s, x.size) - x).max() <= 1e-3
    # a linear ramp in storage order: constant differences, one symbol
    x = np.arange(10000, dtype=np.float64) * 0.37
    s, Q = oracle.compress_1d(x, debug=True, eb=1.0, eb_mode="abs")
    d = np.diff(Q)
    assert len(np.unique(d)) <= 2
    assert x.nbytes / s.size > 20


def test_default_1d_errors():
    x = np.linspace(0, 1, 1000)
    for bad in (dict(open_loop=True), dict(f_op="cluster"), dict(g_op="nearest")):
        with pytest.raises(oracle.OracleError) as err:
            oracle.compress_1d(x, eb=1e-3, **bad)
        assert err.value.status == 1
    with pytest.raises(oracle.OracleError) as err:  # tau below the value spacing margin
        oracle.compress_1d(x + 1e17, eb=1.0, eb_mode="abs")
    assert err.value.status == 4
    s = oracle.compress_1d(x, eb=1e-3)
    for off, val in ((16, 2), (20, 0), (44, 999)):
        t = s.copy()
        t[off:off + 4] = np.frombuffer(np.uint32(val).tobytes(), np.uint8)
        with pytest.raises(oracle.OracleError) as err:
            oracle.decompress_1d(t, x.size)
        assert err.value.status == 5
    with pytest.raises(oracle.OracleError):
        oracle.decompress_1d(s, x.size + 1)
