"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
the same seeded inputs.

Bar: plan tables, quantisation codes and stream bytes bit-exact; decoded
values bit-exact (both sides evaluate the same IEEE operations); the L-inf
bound |x - x'| <= tau2 <= tau holds at every vertex (Sec. III); streams of
either side decode on the other; corrupt streams are rejected without a
fault.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "jit2d":
        c, e = synth.mesh2d_jittered(nside=30, seed=31); n = (23, 17)
        x = synth.field_sincos(c, seed=41)
    elif name == "ragged2d":
        c, e = synth.mesh2d_jittered(nside=40, seed=32); n = (37, 29)
        x = synth.field_bumps_noise(c, seed=42)
    elif name == "c1":
        c, e = synth.mesh2d_jittered(); n = (128, 128)
        x = synth.field_sincos(c)
    elif name == "graded2d":
        c, e = synth.mesh2d_graded(n=50000, seed=33); n = (300, 200)
        x = synth.field_bumps_noise(c, seed=43)
    elif name == "annulus_small":
        c, e = synth.mesh3d_annulus(nr=6, nth=24, nz=8, seed=34); n = (13, 12, 9)
        x = synth.field_vortex(c, seed=44)
    elif name == "annulus_mid":
        c, e = synth.mesh3d_annulus(nr=12, nth=64, nz=20, seed=35); n = (40, 41, 19)
        x = synth.field_vortex(c, seed=45)
    else:
        raise KeyError(name)
    return c, e, n, x


CASES = ["jit2d", "ragged2d", "c1", "graded2d", "annulus_small", "annulus_mid"]
_cache = {}


def _setup(name):
    if name not in _cache:
        import gpu_helpers as G
        c, e, n, x = _case(name)
        _cache[name] = (c, e, n, x, oracle.Plan(c, e, n), G.plan(c, e, n))
    return _cache[name]


@pytest.mark.parametrize("name", CASES)
def test_plan_tables_bit_exact(name):
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup(name)
    t = G.tables(gp)
    assert gp.n_outside == int((op.vid[0] < 0).sum())
    assert np.array_equal(t["vid"], op.vid)
    assert np.array_equal(t["lam"], op.lam)
    assert np.array_equal(t["cell"], op.cell)
    assert np.array_equal(t["frac"], op.frac)


PARAMS = [
    dict(),
    dict(eb=1e-2, grid_fraction=0.2),
    dict(eb=1e-6, grid_fraction=0.8),
    dict(eb_mode="abs", eb=1e-3, grid_fraction=0.5),
    dict(eb=1e-3, R1=37, R2=6, C1=7, C2=13, lmax=12),
    dict(eb=1e-5, grid_fraction=0.3, C1=256, C2=1),
    dict(eb=1e-7, R1=2048, R2=2048, C1=256, C2=256, lmax=24),  # largest alphabet and chunks
    dict(eb=1e-2, R1=4, R2=4, C1=1, C2=2, lmax=3),            # smallest alphabet, 3-bit limit
]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("pi", range(len(PARAMS)))
@pytest.mark.parametrize("name", CASES)
def test_stream_and_values_bit_exact(name, pi, dtype):
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup(name)
    kw = PARAMS[pi]
    xx = x.astype(dtype)
    s_orc = oracle.compress(op, xx, **kw)
    s_gpu = G.compress(gp, xx, **kw)
    assert s_gpu.size == s_orc.size
    if not np.array_equal(s_gpu, s_orc):
        bad = np.flatnonzero(s_gpu != s_orc)
        pytest.fail(f"stream differs at {bad.size} bytes, first at {bad[:8]}")
    y_gpu = G.decompress(gp, s_gpu, dtype)
    y_orc = oracle.decompress(op, s_orc)
    assert np.array_equal(y_gpu.view(np.uint8), y_orc.view(np.uint8))
    f = oracle.field_params(xx, **kw)
    assert np.abs(y_gpu.astype(np.float64) - xx.astype(np.float64)).max() <= f["tau2"]


def test_guarded_field_and_cross_decode():
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("ragged2d")
    xo = x + 3.0e9  # max|x| > 2^28 tau2: every vertex is checked
    kw = dict(eb_mode="abs", eb=0.1)
    assert oracle.field_params(xo, **kw)["guard"] == 1
    s_orc = oracle.compress(op, xo, **kw)
    s_gpu = G.compress(gp, xo, **kw)
    assert np.array_equal(s_gpu, s_orc)
    # each side decodes the other's stream
    assert np.array_equal(oracle.decompress(op, s_gpu), G.decompress(gp, s_orc, np.float64))


def test_constant_and_degenerate_fields():
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("jit2d")
    for xx in (np.full(x.size, 2.5), np.zeros(x.size), np.full(x.size, -1e-300)):
        s_orc = oracle.compress(op, xx, eb=1e-3)
        s_gpu = G.compress(gp, xx, eb=1e-3)
        assert np.array_equal(s_gpu, s_orc)
        assert np.array_equal(G.decompress(gp, s_gpu, np.float64), oracle.decompress(op, s_orc))


def test_device_errors():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("jit2d")
    with pytest.raises(mcc.MCCError) as err:
        G.compress(gp, x, eb=1e-12)
    assert err.value.status == mcc.RANGE
    bad = x.copy(); bad[5] = np.inf
    with pytest.raises(mcc.MCCError) as err:
        G.compress(gp, bad)
    assert err.value.status == mcc.INVALID_ARG
    with pytest.raises(mcc.MCCError) as err:
        G.compress(gp, x, eb=-1.0)
    assert err.value.status == mcc.INVALID_ARG
    # an alphabet of 2R symbols cannot be coded within lmax bits when
    # 2R > 2^lmax: rejected on the host, as by the oracle
    with pytest.raises(mcc.MCCError) as err:
        G.compress(gp, x, R1=512, R2=512, lmax=9)
    assert err.value.status == mcc.INVALID_ARG
    with pytest.raises(oracle.OracleError):
        oracle.compress(op, x, R1=512, R2=512, lmax=9)
    # the context stays usable
    s = G.compress(gp, x)
    assert np.array_equal(s, oracle.compress(op, x))


def test_capacity_and_workspace_checks():
    import torch
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("jit2d")
    prm = G.params(np.float64)
    xt = torch.from_numpy(x).cuda()
    ws = gp.workspace(prm)
    small = torch.zeros(1000, dtype=torch.uint8, device="cuda")
    with pytest.raises(mcc.MCCError) as err:
        mcc.compress(gp, xt, prm, ws, small)
    assert err.value.status == mcc.CAPACITY
    s = oracle.compress(op, x)
    just = torch.zeros(s.size - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(mcc.MCCError) as err:
        mcc.compress(gp, xt, prm, ws, just)
    assert err.value.status == mcc.CAPACITY
    with pytest.raises(mcc.MCCError) as err:
        mcc.compress(gp, xt, prm, ws[:100], torch.zeros(s.size, dtype=torch.uint8, device="cuda"))
    assert err.value.status == mcc.CAPACITY


def test_corrupt_streams_rejected_without_fault():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("ragged2d")
    s = oracle.compress(op, x, eb=1e-5)
    good = oracle.decompress(op, s)
    rng = np.random.default_rng(1)
    cuts = [0, 100, 383, 384, s.size // 2, s.size - 1]
    for cut in cuts:
        with pytest.raises(mcc.MCCError) as err:
            G.decompress(gp, s[:cut] if cut else s[:4], np.float64)
        assert err.value.status == mcc.CORRUPT
    with pytest.raises(mcc.MCCError) as err:  # wrong value type
        G.decompress(gp, s, np.float32)
    assert err.value.status == mcc.CORRUPT
    for _ in range(60):
        t = s.copy()
        pos = int(rng.integers(0, s.size))
        t[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        try:
            ref = oracle.decompress(op, t)
        except oracle.OracleError:
            ref = None
        try:
            got = G.decompress(gp, t, np.float64)
        except mcc.MCCError as err:
            assert err.status == mcc.CORRUPT
            got = None
        if ref is not None and got is not None:
            assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))
    assert np.array_equal(G.decompress(gp, s, np.float64), good)


def test_deterministic_repeat():
    import gpu_helpers as G
    c, e, n, x, op, gp = _setup("annulus_mid")
    a = G.compress(gp, x)
    b = G.compress(gp, x)
    assert np.array_equal(a, b)


def test_stream_independent_of_output_buffer():
    """The stream is a function of the input: output buffers filled with
    garbage give the same bytes as zeroed ones (the alignment gaps between
    sections are written)."""
    import torch
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, op, gp = _setup("annulus_small")
    want = oracle.compress(op, x, eb=1e-3)
    prm = mcc.params_default(eb=1e-3)
    for R in (511, 512, 7):  # odd and even alphabets move the gaps
        prm.R1 = prm.R2 = R
        want = oracle.compress(op, x, eb=1e-3, R1=R, R2=R)
        ws = gp.workspace(prm)
        ws.fill_(0xA5)
        out = torch.full((mcc.compress_bound(gp, prm),), 0xA5, dtype=torch.uint8, device="cuda")
        size = mcc.compress(gp, torch.from_numpy(x).cuda(), prm, ws, out)
        assert np.array_equal(out[:size].cpu().numpy(), want), R


@pytest.mark.slow
def test_full_size_2d_graded_1024():
    """The 2M-vertex graded Delaunay mesh on the 1024^2 grid (the benchmark
    workload): plan tables, streams and decoded values bit-exact at the
    relative bounds 1e-6, 1e-4, 1e-2."""
    import gpu_helpers as G
    c, e = synth.mesh2d_graded()
    x = synth.field_bumps_noise(c)
    op = oracle.Plan(c, e, (1024, 1024))
    gp = G.plan(c, e, (1024, 1024))
    t = G.tables(gp)
    for k in ("vid", "lam", "cell", "frac"):
        assert np.array_equal(t[k], getattr(op, k)), k
    for eb in (1e-6, 1e-4, 1e-2):
        s_orc = oracle.compress(op, x, eb=eb)
        s_gpu = G.compress(gp, x, eb=eb)
        assert np.array_equal(s_gpu, s_orc), eb
        y = G.decompress(gp, s_gpu, np.float64)
        assert np.array_equal(y, oracle.decompress(op, s_orc))
        assert np.abs(y - x).max() <= oracle.field_params(x, eb=eb)["tau2"]


@pytest.mark.slow
def test_full_size_3d_annulus_256():
    """The 8M-vertex annulus (39M tetrahedra) on the 256^3 grid (the 3D
    workload): plan tables, FP64 and FP32 streams at rel 1e-4 (closed loop,
    and open loop at split 0.65) and decoded values bit-exact. The field is
    generated on the device (same formulas as synth) and copied to the host
    for the oracle."""
    import torch
    import gpu_helpers as G
    from synth import torchgen
    c, e = synth.mesh3d_annulus()
    cd = torch.from_numpy(c).cuda()
    x = torchgen.field_vortex(cd, seed=6).cpu().numpy()
    del cd
    n = (256, 256, 256)
    op = oracle.Plan(c, e, n)
    gp = G.plan(c, e, n)
    t = G.tables(gp)
    for k in ("vid", "lam", "cell", "frac"):
        assert np.array_equal(t[k], getattr(op, k)), k
    del t
    for dtype, kw in ((np.float64, {}), (np.float32, {}),
                      (np.float64, dict(open_loop=True, grid_fraction=0.65))):
        xx = x.astype(dtype)
        s_orc = oracle.compress(op, xx, eb=1e-4, **kw)
        s_gpu = G.compress(gp, xx, eb=1e-4, **kw)
        assert np.array_equal(s_gpu, s_orc), (dtype, kw)
        y = G.decompress(gp, s_gpu, dtype)
        assert np.array_equal(y, oracle.decompress(op, s_orc)), (dtype, kw)
        f = oracle.field_params(xx, eb=1e-4, **{k: v for k, v in kw.items() if k != "open_loop"})
        bound = f["tau1"] + f["tau2"] if kw else f["tau2"]
        assert np.abs(y.astype(np.float64) - xx.astype(np.float64)).max() <= bound


@pytest.mark.parametrize("n", [1, 5, 70])
def test_batched_streams_equal_single_field_streams(n):
    """Batched compression (many fields on one plan, per-field bounds) gives
    each field exactly the stream of the oracle's single-field compression;
    batched decompression gives the oracle's values."""
    import torch
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, nn, x, op, gp = _setup("ragged2d")
    rng = np.random.default_rng(n)
    fields, kws = [], []
    for f in range(n):
        fields.append(synth.field_bumps_noise(c, seed=100 + f) * (1 + f % 3))
        kws.append(dict(eb_mode="rel" if f % 2 else "abs", eb=float(10 ** rng.uniform(-5, -2)),
                        grid_fraction=float(rng.uniform(0.2, 0.8))))
    prms = [mcc.params_default(dtype=mcc.F64, **k) for k in kws]
    slot = (mcc.compress_bound(gp, prms[0]) + 7) // 8 * 8
    cws, dws = mcc.workspace_size(gp, prms[0])
    chain = min(n, 7)  # force several launch chains for n = 70
    ws = torch.empty(cws * chain, dtype=torch.uint8, device="cuda")
    out = torch.zeros(slot * n, dtype=torch.uint8, device="cuda")
    xs = [torch.from_numpy(v).cuda() for v in fields]
    sizes = mcc.compress_batch(gp, xs, prms, ws, out, slot)
    host = out.cpu().numpy()
    for f in range(n):
        ref = oracle.compress(op, fields[f], **kws[f])
        assert sizes[f] == ref.size
        assert np.array_equal(host[f * slot:f * slot + sizes[f]], ref), f
    ys = [torch.empty_like(t) for t in xs]
    wsd = torch.empty(dws * chain, dtype=torch.uint8, device="cuda")
    mcc.decompress_batch(gp, out, slot, sizes, ys, wsd)
    for f in range(n):
        want = oracle.decompress(op, host[f * slot:f * slot + sizes[f]])
        assert np.array_equal(ys[f].cpu().numpy(), want), f
