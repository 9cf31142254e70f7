"""GPU parity of the learned residual predictor: streams with a model (random
valid models and models at the format's edges) bit-exact against the oracle,
decoded values bit-exact, cross decoding, invalid and corrupted models
rejected, mixed batches equal to single fields."""
import numpy as np
import pytest
import torch

import oracle
import synth
from mlp_models import edge_models, pack, random_model

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


def _dev(blob):
    return torch.from_numpy(np.ascontiguousarray(blob)).cuda()


@pytest.mark.parametrize("name", ["jit2d", "ragged2d", "annulus_small", "annulus_mid"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("seed", [1, 2])
def test_learned_stream_bit_exact(name, dtype, seed):
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup(name)
    x = x.astype(dtype)
    blob = pack(random_model(op.dim, seed))
    kw = dict(eb=1e-3, grid_fraction=0.4)
    want = oracle.compress(op, x, model=blob, **kw)
    got = G.compress(gp, x, model=_dev(blob), **kw)
    assert got.size == want.size
    assert np.array_equal(got, want)
    y = G.decompress(gp, got, dtype)
    assert np.array_equal(y, oracle.decompress(op, want))
    f = oracle.field_params(x, **kw)
    assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= f["tau2"]


@pytest.mark.parametrize("name", ["ragged2d", "annulus_mid"])
def test_edge_models_bit_exact(name):
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup(name)
    for label, m in edge_models(op.dim):
        blob = pack(m)
        want = oracle.compress(op, x, model=blob, eb=1e-4)
        got = G.compress(gp, x, model=_dev(blob), eb=1e-4)
        assert np.array_equal(got, want), label
        assert np.array_equal(G.decompress(gp, want, x.dtype), oracle.decompress(op, want)), label


def test_zero_model_streams_decode_like_plain():
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("jit2d")
    from mlp_models import blank
    s0 = G.compress(gp, x, eb=1e-3)
    s1 = G.compress(gp, x, eb=1e-3, model=_dev(pack(blank(2))))
    assert np.array_equal(G.decompress(gp, s0, x.dtype), G.decompress(gp, s1, x.dtype))
    assert s1.size == s0.size + oracle.MODEL_BYTES


def test_invalid_and_corrupted_models():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("jit2d")
    m = random_model(2, 3)
    bad = pack(m)
    bad[0] ^= 1
    with pytest.raises(mcc.MCCError) as err:
        G.compress(gp, x, model=_dev(bad), eb=1e-3)
    assert err.value.status == mcc.INVALID_ARG
    mm = dict(m, dim=3)
    with pytest.raises(mcc.MCCError) as err:
        G.compress(gp, x, model=_dev(pack(mm)), eb=1e-3)
    assert err.value.status == mcc.INVALID_ARG
    s = G.compress(gp, x, model=_dev(pack(m)), eb=1e-3)
    t = s.copy()
    t[-oracle.MODEL_BYTES + 40] = 0x80  # W1 entry -128: outside the format
    with pytest.raises(mcc.MCCError) as err:
        G.decompress(gp, t, x.dtype)
    assert err.value.status == mcc.CORRUPT
    t = s.copy()
    t[192] ^= 1  # model size field
    with pytest.raises(mcc.MCCError) as err:
        G.decompress(gp, t, x.dtype)
    assert err.value.status == mcc.CORRUPT
    # a plain stream flagged as learned, and a learned one flagged as plain
    for stream in (G.compress(gp, x, eb=1e-3), s):
        t = stream.copy()
        t[20] ^= 2
        with pytest.raises(mcc.MCCError) as err:
            G.decompress(gp, t, x.dtype)
        assert err.value.status == mcc.CORRUPT


def test_mixed_batch_equals_single_fields():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("annulus_small")
    rng = np.random.default_rng(7)
    fields = [synth.field_vortex(c, seed=70 + i) * rng.uniform(0.5, 3) for i in range(5)]
    blobs = [pack(random_model(3, 20 + i)) if i % 2 else None for i in range(5)]
    dblobs = [_dev(b) if b is not None else None for b in blobs]
    prms = [G.params(np.float64, eb=10.0 ** -(2 + i % 3), model=dblobs[i]) for i in range(5)]
    xs = [torch.from_numpy(f).cuda() for f in fields]
    bound = max(mcc.compress_bound(gp, p) for p in prms)
    slot = (bound + 7) // 8 * 8
    ws = gp.workspace(prms[0])
    wsb = torch.zeros(ws.numel() * 5, dtype=torch.uint8, device="cuda")
    out = torch.zeros(slot * 5, dtype=torch.uint8, device="cuda")
    sizes = mcc.compress_batch(gp, xs, prms, wsb, out, slot)
    for i in range(5):
        got = out[i * slot: i * slot + sizes[i]].cpu().numpy()
        want = oracle.compress(op, fields[i], eb=10.0 ** -(2 + i % 3), model=blobs[i])
        assert np.array_equal(got, want), i
        assert np.array_equal(G.decompress(gp, got, np.float64), oracle.decompress(op, want))


def test_static_decompress_of_learned_stream():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("annulus_small")
    blob = pack(random_model(3, 9))
    s = G.compress(gp, x, model=_dev(blob), eb=1e-3)
    st = torch.from_numpy(s).cuda()
    out = torch.empty(op.n_v, dtype=torch.float64, device="cuda")
    mcc.decompress_static(gp, st, s.size, out)
    assert np.array_equal(out.cpu().numpy(), oracle.decompress(op, s))


# --------------------------------------------------------------------------- #
# automatic choice between the plain and the learned predictor
# --------------------------------------------------------------------------- #
def _convex_case():
    if "convex" not in _cache:
        import gpu_helpers as G
        c, e = synth.mesh2d_jittered(nside=200, seed=33)
        _cache["convex"] = (c, e, oracle.Plan(c, e, (33, 29)), G.plan(c, e, (33, 29)))
    return _cache["convex"]


@pytest.mark.parametrize("which", ["zero", "random", "convex"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_auto_choice_bit_exact(which, dtype):
    import gpu_helpers as G
    from test_oracle_mlp_pins import _convex_model
    from mlp_models import blank
    c, e, op, gp = _convex_case()
    eb = 2e-6
    s2 = 2 * (0.5 * eb) * (1 - 2.0 ** -20)
    if which == "convex":
        x = c[:, 0] ** 2 + c[:, 1] ** 2
        m = _convex_model((op.grid.h[0] ** 2 / s2, op.grid.h[1] ** 2 / s2))
    else:
        x = 1e-3 * synth.field_bumps_noise(c, seed=14)
        m = blank(2) if which == "zero" else random_model(2, 15)
    x = x.astype(dtype)
    blob = pack(m)
    kw = dict(eb=eb, eb_mode="abs")
    want = oracle.compress(op, x, model=blob, auto=True, **kw)
    got = G.compress(gp, x, model=_dev(blob), auto=True, **kw)
    assert np.array_equal(got, want)
    learned = bool(int(want[20:24].view(np.uint32)[0]) & 2)
    assert learned == (which == "convex")
    assert np.array_equal(G.decompress(gp, got, dtype), oracle.decompress(op, want))


def test_auto_in_a_mixed_batch():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    from test_oracle_mlp_pins import _convex_model
    c, e, op, gp = _convex_case()
    eb = 2e-6
    s2 = 2 * (0.5 * eb) * (1 - 2.0 ** -20)
    blob = pack(_convex_model((op.grid.h[0] ** 2 / s2, op.grid.h[1] ** 2 / s2)))
    fields = [c[:, 0] ** 2 + c[:, 1] ** 2, 1e-3 * synth.field_bumps_noise(c, seed=3),
              c[:, 0] ** 2 + 0.5 * c[:, 1] ** 2, 1e-3 * synth.field_bumps_noise(c, seed=4)]
    modes = [dict(model=_dev(blob), auto=True), dict(model=_dev(blob), auto=True), {},
             dict(model=_dev(blob))]
    okw = [dict(model=blob, auto=True), dict(model=blob, auto=True), {}, dict(model=blob)]
    prms = [G.params(np.float64, eb=eb, eb_mode="abs", **m) for m in modes]
    xs = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in fields]
    slot = (max(mcc.compress_bound(gp, p) for p in prms) + 7) // 8 * 8
    ws1 = gp.workspace(prms[0])
    wsb = torch.zeros(ws1.numel() * 4, dtype=torch.uint8, device="cuda")
    out = torch.zeros(slot * 4, dtype=torch.uint8, device="cuda")
    sizes = mcc.compress_batch(gp, xs, prms, wsb, out, slot)
    for i in range(4):
        got = out[i * slot: i * slot + sizes[i]].cpu().numpy()
        want = oracle.compress(op, fields[i], eb=eb, eb_mode="abs", **okw[i])
        assert np.array_equal(got, want), i


@pytest.mark.parametrize("name", ["jit2d", "ragged2d", "annulus_small", "annulus_mid"])
def test_tcgen05_network_path_bit_exact(name):
    """The tcgen05 tensor-core path of the network (plan tuning net_path):
    learned and automatic streams and decoded values equal the oracle's,
    as with the default mma.sync path; invalid models are still rejected."""
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup(name)
    assert mcc.get_net_path(gp) == mcc.NET_MMA_SYNC
    mcc.set_net_path(gp, mcc.NET_TCGEN05)
    try:
        assert mcc.get_net_path(gp) == mcc.NET_TCGEN05
        for seed, kw in ((1, dict(eb=1e-3, grid_fraction=0.4)), (2, dict(eb=1e-4, auto=True))):
            blob = pack(random_model(op.dim, seed))
            want = oracle.compress(op, x, model=blob, **kw)
            got = G.compress(gp, x, model=_dev(blob), **kw)
            assert np.array_equal(got, want), seed
            assert np.array_equal(G.decompress(gp, got, x.dtype), oracle.decompress(op, want))
        for label, m in edge_models(op.dim)[:2]:
            blob = pack(m)
            want = oracle.compress(op, x, model=blob, eb=1e-4)
            assert np.array_equal(G.compress(gp, x, model=_dev(blob), eb=1e-4), want), label
        bad = pack(random_model(op.dim, 3))
        bad[0] ^= 1
        with pytest.raises(mcc.MCCError) as err:
            G.compress(gp, x, model=_dev(bad), eb=1e-3)
        assert err.value.status == mcc.INVALID_ARG
    finally:
        mcc.set_net_path(gp, mcc.NET_MMA_SYNC)
    with pytest.raises(mcc.MCCError) as err:
        mcc.set_net_path(gp, 2)
    assert err.value.status == mcc.INVALID_ARG
