"""GPU parity of the open-loop mode (Algorithm 3 as printed: residual against
g(x1) with the unquantised grid component, bound tau1 + tau2): streams
bit-exact against the oracle, decoded values bit-exact, batches mixing open,
closed and learned fields, the allocation-free decoder, argument errors and
corrupted flags."""
import numpy as np
import pytest
import torch

import oracle
import synth
from mlp_models import pack, random_model

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "jit2d":
        c, e = synth.mesh2d_jittered(nside=30, seed=51); n = (23, 17)
        x = synth.field_sincos(c, seed=61)
    elif name == "ragged2d":
        c, e = synth.mesh2d_jittered(nside=70, seed=52); n = (37, 29)
        x = synth.field_bumps_noise(c, seed=62)
    elif name == "annulus_small":
        c, e = synth.mesh3d_annulus(nr=6, nth=24, nz=8, seed=53); n = (13, 12, 9)
        x = synth.field_vortex(c, seed=63)
    elif name == "annulus_mid":
        c, e = synth.mesh3d_annulus(nr=12, nth=64, nz=20, seed=54); n = (40, 41, 19)
        x = synth.field_vortex(c, seed=64)
    elif name == "graded2d_big":
        c, e = synth.mesh2d_graded(n=400_000, seed=55); n = (640, 640)
        x = synth.field_bumps_noise(c, seed=65)
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


@pytest.mark.parametrize("name", ["jit2d", "ragged2d", "annulus_small", "annulus_mid"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("eb,frac", [(1e-2, 0.5), (1e-4, 0.8), (1e-6, 0.2)])
def test_open_loop_stream_bit_exact(name, dtype, eb, frac):
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup(name)
    x = x.astype(dtype)
    kw = dict(eb=eb, grid_fraction=frac, open_loop=True)
    want = oracle.compress(op, x, **kw)
    got = G.compress(gp, x, **kw)
    assert got.size == want.size
    assert np.array_equal(got, want)
    y = G.decompress(gp, got, dtype)
    assert np.array_equal(y, oracle.decompress(op, want))
    f = oracle.field_params(x, eb=eb, grid_fraction=frac)
    assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= f["tau1"] + f["tau2"]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_open_loop_large_mesh(dtype):
    """A graded mesh of 400k vertices over a 640 x 640 grid: many tiles and
    ragged edges; the whole stream bit-exact."""
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("graded2d_big")
    x = x.astype(dtype)
    kw = dict(eb=1e-4, grid_fraction=0.5, open_loop=True)
    want = oracle.compress(op, x, **kw)
    got = G.compress(gp, x, **kw)
    assert np.array_equal(got, want)
    assert np.array_equal(G.decompress(gp, got, dtype), oracle.decompress(op, want))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_open_loop_guard_raw_values(dtype):
    """Near 1.2e4 the FP32 spacing lies between tau and 2 tau: reconstructions
    more than half a spacing away round outside the bound and are stored raw;
    the FP64 field takes the same path without raw values."""
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("ragged2d")
    x = (x + 1.2e4).astype(dtype)
    kw = dict(eb=9e-4, eb_mode="abs", open_loop=True)
    want, dbg = oracle.compress(op, x, debug=True, **kw)
    if dtype == np.float32:
        assert np.any(dbg["sym2"] == 2 * 512 - 1)
    got = G.compress(gp, x, **kw)
    assert np.array_equal(got, want)
    assert np.array_equal(G.decompress(gp, got, dtype), oracle.decompress(op, want))


def test_batch_mixing_open_closed_learned():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("annulus_small")
    rng = np.random.default_rng(9)
    fields = [synth.field_vortex(c, seed=80 + i) * rng.uniform(0.5, 3) for i in range(6)]
    blob = pack(random_model(3, 31))
    dblob = torch.from_numpy(blob).cuda()
    kinds = ["open", "closed", "learned", "open", "auto", "open"]
    prms, okw = [], []
    for i, k in enumerate(kinds):
        kw = dict(eb=10.0 ** -(2 + i % 3), grid_fraction=0.3 + 0.1 * i)
        if k == "open":
            prms.append(G.params(np.float64, open_loop=True, **kw)); okw.append(dict(kw, open_loop=True))
        elif k == "closed":
            prms.append(G.params(np.float64, **kw)); okw.append(kw)
        else:
            prms.append(G.params(np.float64, model=dblob, auto=k == "auto", **kw))
            okw.append(dict(kw, model=blob, auto=k == "auto"))
    xs = [torch.from_numpy(f).cuda() for f in fields]
    slot = (max(mcc.compress_bound(gp, p) for p in prms) + 7) // 8 * 8
    ws = gp.workspace(prms[0])
    wsb = torch.zeros(ws.numel() * len(fields), dtype=torch.uint8, device="cuda")
    out = torch.zeros(slot * len(fields), dtype=torch.uint8, device="cuda")
    sizes = mcc.compress_batch(gp, xs, prms, wsb, out, slot)
    for i in range(len(fields)):
        got = out[i * slot: i * slot + sizes[i]].cpu().numpy()
        want = oracle.compress(op, fields[i], **okw[i])
        assert np.array_equal(got, want), (i, kinds[i])
        assert np.array_equal(G.decompress(gp, got, np.float64), oracle.decompress(op, want))


def test_batch_decode_of_open_and_closed_streams():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("jit2d")
    streams = [oracle.compress(op, x * (1 + i), eb=1e-3, open_loop=bool(i % 2)) for i in range(4)]
    slot = (max(s.size for s in streams) + 7) // 8 * 8
    buf = np.zeros(slot * 4, np.uint8)
    for i, s in enumerate(streams):
        buf[i * slot: i * slot + s.size] = s
    outs = [torch.empty(op.n_v, dtype=torch.float64, device="cuda") for _ in range(4)]
    ws1 = gp.workspace(mcc.params_default(), "decompress")
    wsb = torch.zeros(ws1.numel() * 4, dtype=torch.uint8, device="cuda")
    mcc.decompress_batch(gp, torch.from_numpy(buf).cuda(), slot, [s.size for s in streams], outs, wsb)
    for i, s in enumerate(streams):
        assert np.array_equal(outs[i].cpu().numpy(), oracle.decompress(op, s)), i


def test_static_decompress_of_open_stream():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("annulus_small")
    s = oracle.compress(op, x, eb=1e-4, grid_fraction=0.7, open_loop=True)
    st = torch.from_numpy(s).cuda()
    out = torch.empty(op.n_v, dtype=torch.float64, device="cuda")
    mcc.decompress_static(gp, st, s.size, out)
    assert np.array_equal(out.cpu().numpy(), oracle.decompress(op, s))


def test_open_loop_errors():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("jit2d")
    dblob = torch.from_numpy(pack(random_model(2, 3))).cuda()
    for bad in (dict(open_loop=True, model=dblob), dict(loop=2), dict(loop=-1)):
        with pytest.raises(mcc.MCCError) as err:
            G.compress(gp, x, eb=1e-3, **bad)
        assert err.value.status == mcc.INVALID_ARG
    s = G.compress(gp, x, eb=1e-3, open_loop=True)
    for flip in (2, 32):
        t = s.copy()
        t[20] |= flip
        with pytest.raises(mcc.MCCError) as err:
            G.decompress(gp, t, x.dtype)
        assert err.value.status == mcc.CORRUPT
