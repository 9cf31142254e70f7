"""GPU parity of the 1D coder (the paper's default baseline): streams
bit-exact against the oracle for FP64 / FP32 values, three bounds and sizes
from a few values to the 2M-vertex benchmark field (many chunks of the
scan, a ragged tail); decoded values bit-exact both ways; the bound without
raw values; errors, and streams of the two coders refused by each other's
decoder."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _field(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.random((n, 2))
    return synth.field_bumps_noise(c, seed=seed)


@pytest.mark.parametrize("n", [1, 7, 4096, 100_003, 2_000_000])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
def test_default_1d_bit_exact(n, dtype, eb):
    import paper_2501_06910_gb300 as mcc
    x = _field(n, 3).astype(dtype)
    if n == 1 and eb == 1e-6:
        x[:] = 0.25
    want = oracle.compress_1d(x, eb=eb)
    prm = mcc.params_default(dtype=mcc.F64 if dtype == np.float64 else mcc.F32, eb=eb)
    got = mcc.compress_1d(torch.from_numpy(x).cuda(), prm).cpu().numpy()
    assert got.size == want.size
    assert np.array_equal(got, want)
    y = torch.empty(n, dtype=torch.float64 if dtype == np.float64 else torch.float32, device="cuda")
    mcc.decompress_1d(torch.from_numpy(want).cuda(), y)
    yo = oracle.decompress_1d(want, n)
    assert np.array_equal(y.cpu().numpy(), yo)
    tau = eb * (x.astype(np.float64).max() - x.astype(np.float64).min()) if n > 1 and x.max() > x.min() else eb
    assert np.abs(yo.astype(np.float64) - x.astype(np.float64)).max() <= tau


def test_default_1d_large_offsets():
    import paper_2501_06910_gb300 as mcc
    x = _field(50_000, 5)
    for dtype, off, eb in ((np.float32, 1.2e4, 5e-3), (np.float64, 3.0e9, 1e-1)):
        xx = (x + off).astype(dtype)
        want = oracle.compress_1d(xx, eb=eb, eb_mode="abs")
        prm = mcc.params_default(dtype=mcc.F64 if dtype == np.float64 else mcc.F32, eb=eb,
                                 eb_mode="abs")
        got = mcc.compress_1d(torch.from_numpy(xx).cuda(), prm).cpu().numpy()
        assert np.array_equal(got, want)


def test_default_1d_errors():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    x = torch.from_numpy(_field(1000, 7)).cuda()
    for bad in (dict(open_loop=True), dict(f_op="cluster"), dict(g_op="nearest"), dict(R1=3)):
        with pytest.raises(mcc.MCCError) as err:
            mcc.compress_1d(x, mcc.params_default(eb=1e-3, **bad))
        assert err.value.status in (mcc.INVALID_ARG, mcc.UNSUPPORTED)
    with pytest.raises(mcc.MCCError) as err:  # tau below the spacing margin
        mcc.compress_1d(x + 1e17, mcc.params_default(eb=1.0, eb_mode="abs"))
    assert err.value.status == mcc.RANGE
    # a 1D stream is refused by the method's decoder and the reverse
    c, e = synth.mesh2d_jittered(nside=30, seed=51)
    gp = G.plan(c, e, (23, 17))
    xm = synth.field_sincos(c, seed=61)
    s1d = oracle.compress_1d(xm, eb=1e-3)
    with pytest.raises(mcc.MCCError) as err:
        G.decompress(gp, s1d, np.float64)
    assert err.value.status == mcc.CORRUPT
    smc = G.compress(gp, xm, eb=1e-3)
    y = torch.empty(xm.size, dtype=torch.float64, device="cuda")
    with pytest.raises(mcc.MCCError) as err:
        mcc.decompress_1d(torch.from_numpy(smc).cuda(), y)
    assert err.value.status == mcc.CORRUPT
    t = s1d.copy()
    t[20] = 33  # an extra flag
    with pytest.raises(mcc.MCCError) as err:
        mcc.decompress_1d(torch.from_numpy(t).cuda(), y)
    assert err.value.status == mcc.CORRUPT
