"""GPU parity of the paper's own operators (nearest-node g, Sec. III-B;
cluster-mean f, Sec. III-C): streams bit-exact against the oracle for every
combination with the default operators, both loops and both value types;
decoded values bit-exact; batches mixing operators, loops and predictors;
the allocation-free decoder; argument errors and corrupted flags."""
import numpy as np
import pytest
import torch

import oracle
import synth
from mlp_models import pack, random_model

pytestmark = pytest.mark.gpu

COMBOS = [("barycentric", "nearest"), ("cluster", "multilinear"), ("cluster", "nearest")]


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
@pytest.mark.parametrize("fop,gop", COMBOS)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("open_loop", [False, True])
def test_operator_stream_bit_exact(name, fop, gop, dtype, open_loop):
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup(name)
    x = x.astype(dtype)
    kw = dict(eb=1e-4, grid_fraction=0.4, f_op=fop, g_op=gop, open_loop=open_loop)
    want = oracle.compress(op, x, **kw)
    got = G.compress(gp, x, **kw)
    assert got.size == want.size
    assert np.array_equal(got, want)
    y = G.decompress(gp, got, dtype)
    assert np.array_equal(y, oracle.decompress(op, want))
    f = oracle.field_params(x, eb=1e-4, grid_fraction=0.4)
    bound = f["tau1"] + f["tau2"] if open_loop else f["tau2"]
    assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= bound


@pytest.mark.parametrize("fop,gop", COMBOS)
def test_operator_large_mesh(fop, gop):
    """400k vertices on a 640 x 640 grid: many tiles, ragged edges, nodes with
    large clusters and nodes with none."""
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("graded2d_big")
    kw = dict(eb=1e-4, f_op=fop, g_op=gop)
    want = oracle.compress(op, x, **kw)
    got = G.compress(gp, x, **kw)
    assert np.array_equal(got, want)
    assert np.array_equal(G.decompress(gp, got, np.float64), oracle.decompress(op, want))


def test_operator_guarded_field():
    """Values far from zero in bins of the bound (every vertex checked)."""
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("ragged2d")
    for dtype in (np.float64, np.float32):
        xx = (x + 1.2e4).astype(dtype)
        kw = dict(eb=9e-4, eb_mode="abs", f_op="cluster", g_op="nearest")
        want = oracle.compress(op, xx, **kw)
        got = G.compress(gp, xx, **kw)
        assert np.array_equal(got, want)
        assert np.array_equal(G.decompress(gp, got, dtype), oracle.decompress(op, want))


def test_batch_mixing_operators():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("annulus_small")
    rng = np.random.default_rng(11)
    fields = [synth.field_vortex(c, seed=90 + i) * rng.uniform(0.5, 3) for i in range(7)]
    blob = pack(random_model(3, 41))
    dblob = torch.from_numpy(blob).cuda()
    kinds = [dict(f_op="cluster"), dict(g_op="nearest"), dict(f_op="cluster", g_op="nearest"),
             {}, dict(open_loop=True, g_op="nearest"), dict(model=True),
             dict(f_op="cluster", model=True, auto=True)]
    prms, okw = [], []
    for i, k in enumerate(kinds):
        base = dict(eb=10.0 ** -(2 + i % 3), grid_fraction=0.3 + 0.08 * i)
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
        want = oracle.decompress(op, host[i * slot: i * slot + sizes[i]])
        assert np.array_equal(ys[i].cpu().numpy(), want), i


def test_static_decompress_of_nearest_stream():
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("annulus_small")
    s = oracle.compress(op, x, eb=1e-4, f_op="cluster", g_op="nearest")
    out = torch.empty(op.n_v, dtype=torch.float64, device="cuda")
    mcc.decompress_static(gp, torch.from_numpy(s).cuda(), s.size, out)
    assert np.array_equal(out.cpu().numpy(), oracle.decompress(op, s))


def test_operator_errors():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("jit2d")
    dblob = torch.from_numpy(pack(random_model(2, 3))).cuda()
    for bad in (dict(g_op="nearest", model=dblob), dict(f_op=2), dict(g_op=-1)):
        with pytest.raises(mcc.MCCError) as err:
            G.compress(gp, x, eb=1e-3, **bad)
        assert err.value.status == mcc.INVALID_ARG
    # a learned stream flagged as nearest-node, and an unknown flag
    s = G.compress(gp, x, eb=1e-3, model=dblob)
    for flip in (8, 32):
        t = s.copy()
        t[20] |= flip
        with pytest.raises(mcc.MCCError) as err:
            G.decompress(gp, t, x.dtype)
        assert err.value.status == mcc.CORRUPT
