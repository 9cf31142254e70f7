"""GPU parity of the zero-run stage (runs of zero symbols as bijective base-2
digit tokens before the Huffman coder): streams bit-exact against the oracle
over bounds from loose (long runs) to tight (short ones), chunk sizes from 1
(one symbol per lane) to 256, 2D and 3D meshes, both value types, both loops,
the paper's operators, the learned and auto predictors, batches mixing fields
with and without the stage, the 1D coder, the 2M-vertex benchmark field; the
decoded values bit-exact; closed forms; argument errors and corrupted run
token lengths."""
import numpy as np
import pytest
import torch

import oracle
import synth
from mlp_models import pack, random_model

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "jit2d":
        c, e = synth.mesh2d_jittered(nside=30, seed=71); n = (23, 17)
        x = synth.field_sincos(c, seed=81)
    elif name == "ragged2d":
        c, e = synth.mesh2d_jittered(nside=70, seed=72); n = (37, 29)
        x = synth.field_bumps_noise(c, seed=82)
    elif name == "annulus_small":
        c, e = synth.mesh3d_annulus(nr=6, nth=24, nz=8, seed=73); n = (13, 12, 9)
        x = synth.field_vortex(c, seed=83)
    elif name == "graded2d_big":
        c, e = synth.mesh2d_graded(n=400_000, seed=75); n = (640, 640)
        x = synth.field_bumps_noise(c, seed=85)
    else:
        raise KeyError(name)
    return c, e, n, x


_cache = {}


def _setup(name):
    if name not in _cache:
        import gpu_helpers as G
        c, e, n, x = _case(name)
        _cache[name] = (c, e, n, x, oracle.Plan(c, e, n), G.plan(c, e, n))
    return _cache[name]


def _check(name, x, **kw):
    import gpu_helpers as G
    c, e, n, _, op, gp = _setup(name)
    want = oracle.compress(op, x, zero_run=True, **kw)
    got = G.compress(gp, x, zero_run=True, **kw)
    assert got.size == want.size
    assert np.array_equal(got, want)
    assert int(got[20:24].view(np.uint32)[0]) & 64
    y = G.decompress(gp, got, x.dtype)
    assert np.array_equal(y, oracle.decompress(op, want))
    return got, y


@pytest.mark.parametrize("name", ["jit2d", "ragged2d", "annulus_small"])
@pytest.mark.parametrize("eb", [3e-1, 1e-2, 1e-4])
@pytest.mark.parametrize("C", [1, 7, 128, 256])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_zero_run_bit_exact(name, eb, C, dtype):
    x = _setup(name)[3].astype(dtype)
    _check(name, x, eb=eb, C1=C, C2=C)


@pytest.mark.parametrize("kw", [dict(open_loop=True), dict(f_op="cluster", g_op="nearest"),
                                dict(f_op="cluster", open_loop=True), dict(grid_fraction=0.05),
                                dict(grid_fraction=0.95), dict(eb=1e-6), dict(eb=2.0, eb_mode="abs"),
                                dict(R1=4, R2=4), dict(R1=2047, R2=2047), dict(lmax=11)])
@pytest.mark.parametrize("name", ["ragged2d", "annulus_small"])
def test_zero_run_options(name, kw):
    kw = dict(kw)
    kw.setdefault("eb", 1e-2)
    _check(name, _setup(name)[3], **kw)


@pytest.mark.parametrize("eb", [1e-1, 1e-3])
def test_zero_run_large_mesh(eb):
    """400k vertices on a 640 x 640 grid: many groups, lanes whose runs cross
    every part boundary, a ragged last group."""
    _check("graded2d_big", _setup("graded2d_big")[3], eb=eb)


def test_zero_run_constant_field_closed_form():
    """All residual symbols zero: every full lane of 128 is seven one-bit
    tokens, 7 words per group."""
    import gpu_helpers as G
    c, e = synth.mesh2d_jittered(nside=64, seed=2)
    op, gp = oracle.Plan(c, e, (20, 20)), G.plan(c, e, (20, 20))
    x = np.full(op.n_v, 3.25)
    got = G.compress(gp, x, eb=1e-3, zero_run=True)
    assert np.array_equal(got, oracle.compress(op, x, eb=1e-3, zero_run=True))
    assert int(got[176:184].view(np.uint64)[0]) == 7


def test_zero_run_full_alphabet_with_raw_values():
    """R = 4 with every residual symbol but zero in use, raw values and both
    run tokens: 2R + 1 codes, one more than the 2R symbols."""
    rng = np.random.default_rng(3)
    c, e, n, x, op, gp = _setup("ragged2d")
    xx = (synth.field_bumps_noise(c, seed=82) * 0.05 + rng.standard_normal(c.shape[0]) * 0.01
          + 1e5).astype(np.float32)
    got, _ = _check("ragged2d", xx, eb=0.012, eb_mode="abs", R1=4, R2=4)
    lens2 = [int(v) for v in got[392:400]] + [int(got[210]), int(got[211])]
    assert sum(1 for v in lens2 if v) == 9 and int(got[160:168].view(np.uint64)[0]) > 0


def test_zero_run_learned_and_auto():
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("annulus_small")
    blob = pack(random_model(3, 17))
    dblob = torch.from_numpy(blob).cuda()
    for auto in (False, True):
        for eb in (1e-1, 1e-2, 1e-4):
            want = oracle.compress(op, x, eb=eb, model=blob, auto=auto, zero_run=True)
            got = G.compress(gp, x, eb=eb, model=dblob, auto=auto, zero_run=True)
            assert np.array_equal(got, want), (auto, eb)
            assert np.array_equal(G.decompress(gp, got, x.dtype), oracle.decompress(op, want))


def test_zero_run_batch_mixed():
    """A batch of fields with and without the stage (and with the other
    per-field options): every stream equals the oracle's."""
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("ragged2d")
    rng = np.random.default_rng(5)
    fields = [synth.field_bumps_noise(c, seed=200 + i) * rng.uniform(0.5, 3) for i in range(8)]
    blob = pack(random_model(2, 23))
    dblob = torch.from_numpy(blob).cuda()
    kinds = [dict(zero_run=True), {}, dict(zero_run=True, open_loop=True),
             dict(zero_run=True, f_op="cluster", g_op="nearest"), dict(model=True),
             dict(zero_run=True, model=True, auto=True), dict(zero_run=True, model=True), {}]
    prms, okw = [], []
    for i, k in enumerate(kinds):
        base = dict(eb=10.0 ** -(1 + i % 4), grid_fraction=0.2 + 0.08 * i)
        k = dict(k)
        if k.pop("model", False):
            prms.append(G.params(np.float64, model=dblob, **k, **base))
            okw.append(dict(base, model=blob, **k))
        else:
            prms.append(G.params(np.float64, **k, **base))
            okw.append(dict(base, **k))
    xs = [torch.from_numpy(f).cuda() for f in fields]
    slot = (max(mcc.compress_bound(gp, p) for p in prms) + 7) // 8 * 8
    ws = gp.workspace(prms[0])
    wsb = torch.zeros(ws.numel() * len(fields), dtype=torch.uint8, device="cuda")
    out = torch.zeros(slot * len(fields), dtype=torch.uint8, device="cuda")
    sizes = mcc.compress_batch(gp, xs, prms, wsb, out, slot)
    host = out.cpu().numpy()
    for i in range(len(fields)):
        got = host[i * slot: i * slot + sizes[i]]
        want = oracle.compress(op, fields[i], **okw[i])
        assert np.array_equal(got, want), (i, kinds[i])
    ys = [torch.empty_like(t) for t in xs]
    wsd = gp.workspace(mcc.params_default(), "decompress")
    wsdb = torch.zeros(wsd.numel() * len(fields), dtype=torch.uint8, device="cuda")
    mcc.decompress_batch(gp, out, slot, sizes, ys, wsdb)
    for i in range(len(fields)):
        assert np.array_equal(ys[i].cpu().numpy(), oracle.decompress(op, host[i * slot: i * slot + sizes[i]]))


@pytest.mark.parametrize("n", [1, 5000, 100_003])
@pytest.mark.parametrize("sort", [False, True])
def test_zero_run_1d(n, sort):
    import paper_2501_06910_gb300 as mcc
    rng = np.random.default_rng(9)
    x = synth.field_bumps_noise(rng.random((n, 2)), seed=9)
    if sort:
        x = np.sort(x)
    for eb in (1e-2, 1e-4):
        want = oracle.compress_1d(x, eb=eb, zero_run=True)
        prm = mcc.params_default(eb=eb, zero_run=True)
        got = mcc.compress_1d(torch.from_numpy(x).cuda(), prm).cpu().numpy()
        assert np.array_equal(got, want)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        mcc.decompress_1d(torch.from_numpy(want).cuda(), y)
        assert np.array_equal(y.cpu().numpy(), oracle.decompress_1d(want, n))


def test_zero_run_static_decompress():
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("annulus_small")
    s = oracle.compress(op, x, eb=1e-2, zero_run=True)
    out = torch.empty(op.n_v, dtype=torch.float64, device="cuda")
    mcc.decompress_static(gp, torch.from_numpy(s).cuda(), s.size, out)
    assert np.array_equal(out.cpu().numpy(), oracle.decompress(op, s))


def test_zero_run_errors():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("jit2d")
    for bad, status in ((dict(zero_run=2), mcc.INVALID_ARG),
                        (dict(zero_run=True, R1=2048), mcc.UNSUPPORTED),
                        (dict(zero_run=True, R1=8, R2=8, lmax=4), mcc.INVALID_ARG)):
        with pytest.raises(mcc.MCCError) as err:
            G.compress(gp, x, eb=1e-2, **bad)
        assert err.value.status == status
    G.compress(gp, x, eb=1e-2, R1=2048)                  # without the stage: accepted
    G.compress(gp, x, eb=1e-2, R1=8, R2=8, lmax=4)
    s = G.compress(gp, x, eb=1e-2, zero_run=True)
    for off, val in ((208, 30), (211, 25)):  # run token lengths above lmax
        t = s.copy()
        t[off] = val
        with pytest.raises(mcc.MCCError) as err:
            G.decompress(gp, t, x.dtype)
        assert err.value.status == mcc.CORRUPT
    t = s.copy()
    t[20] |= 128
    with pytest.raises(mcc.MCCError) as err:
        G.decompress(gp, t, x.dtype)
    assert err.value.status == mcc.CORRUPT


@pytest.mark.slow
def test_zero_run_full_size_benchmark_field():
    """The 2M-vertex graded mesh on the 1024^2 grid at rel 1e-2, 1e-4: the
    whole stream against the oracle."""
    import gpu_helpers as G
    c, e = synth.mesh2d_graded()
    x = synth.field_bumps_noise(c)
    op, gp = oracle.Plan(c, e, (1024, 1024)), G.plan(c, e, (1024, 1024))
    for eb in (1e-2, 1e-4):
        want = oracle.compress(op, x, eb=eb, zero_run=True)
        got = G.compress(gp, x, eb=eb, zero_run=True)
        assert np.array_equal(got, want)
        assert np.array_equal(G.decompress(gp, got, x.dtype), oracle.decompress(op, want))
