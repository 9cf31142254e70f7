"""Pins of the oracle's learned residual predictor (the integer network, its
place in the stream, the float training network's gradient and the
post-training quantisation) against hand-computed values, closed forms,
finite differences and invariances. No GPU.
"""
import numpy as np
import pytest

import oracle
import synth

H = 64


@pytest.fixture(scope="module")
def plan2d():
    coords, cells = synth.mesh2d_jittered(nside=50, seed=31)
    return coords, oracle.Plan(coords, cells, (33, 29))


@pytest.fixture(scope="module")
def plan3d():
    coords, cells = synth.mesh3d_annulus(nr=6, nth=24, nz=8, seed=32)
    return coords, oracle.Plan(coords, cells, (13, 12, 9))


from mlp_models import blank as _blank, pack as _pack, random_model as _random_model  # noqa: E402


# --------------------------------------------------------------------------- #
# the integer network
# --------------------------------------------------------------------------- #
def test_act8_rounding_and_clamping_hand_computed():
    """Hidden units: round(a / 2^s) half up, clamped to 0..255; output
    (W3 h2 + b3) 2^e3. Values worked out by hand."""
    m = _blank(2, s1=2, s2=1, e3=-1)
    m["b1"][:6] = [100, 102, -6, 2000, -2, -3]   # -> 25, 26 (25.5 up), 0, 255, 0, 0
    m["W2"][0, :6] = [1, 1, 1, 1, 1, 1]
    m["b2"][0] = 1                                # 25 + 26 + 255 + 1 = 307 -> 154
    m["W3"][0] = 3
    m["b3"] = -2                                  # (3 * 154 - 2) / 2 = 230
    corners = np.zeros((3, 8), np.int32)
    fr = np.zeros((3, 3), np.float32)
    _, p = oracle.mlp_predict(2, _pack(m), corners, fr, 1.0)
    assert np.all(p == 230.0)


def test_bias_and_output_exponent():
    m = _blank(3, e3=-3)
    m["b3"] = 5
    _, p = oracle.mlp_predict(3, _pack(m), np.zeros((4, 8), np.int32), np.zeros((4, 3), np.float32), 0.7)
    assert np.all(p == 5.0 / 8.0)
    m["e3"] = 4
    _, p = oracle.mlp_predict(3, _pack(m), np.zeros((1, 8), np.int32), np.zeros((1, 3), np.float32), 0.7)
    assert p[0] == 80.0


def _identity_model(dim, k, sx=0):
    """p = feature k: two ReLU units carry relu(e) and relu(-e) through both
    hidden layers (weight 2 with shift 1 is exact), W3 = (1, -1)."""
    m = _blank(dim, sx=sx)
    m["W1"][0, k] = 2
    m["W1"][1, k] = -2
    m["W2"][0, 0] = 2
    m["W2"][1, 1] = 2
    m["W3"][:2] = [1, -1]
    return m


@pytest.mark.parametrize("dim", [2, 3])
def test_identity_network_returns_corner_differences(dim):
    """With s1/s2 = 1 and sx = 0 the corner features are e_k = c_k - c_000
    (in vertex bins) clamped to [-127, 127]; with sx = 1 they are halved with
    ties to even; the coordinate features are rint(127 f)."""
    rng = np.random.default_rng(dim)
    n = 400
    corners = rng.integers(-300, 300, (n, 8)).astype(np.int32)
    fr = rng.random((n, 3)).astype(np.float32)
    nc = 1 << dim
    for k in range(nc - 1):
        feats, p = oracle.mlp_predict(dim, _pack(_identity_model(dim, k)), corners, fr, 1.0)
        d = corners[:, k + 1].astype(np.int64) - corners[:, 0]
        assert np.array_equal(p, np.clip(d, -127, 127).astype(np.float32))
        assert np.array_equal(feats[:, k], np.clip(d, -127, 127))
        feats, p = oracle.mlp_predict(dim, _pack(_identity_model(dim, k, sx=1)), corners, fr, 1.0)
        half = np.clip(np.round(d / 2.0), -127, 127)   # numpy rounds half to even
        assert np.array_equal(p, half.astype(np.float32))
    for d in range(dim):
        feats, p = oracle.mlp_predict(dim, _pack(_identity_model(dim, nc - 1 + d)), corners, fr, 1.0)
        want = np.round(fr[:, d].astype(np.float64) * 127.0)
        assert np.array_equal(p, want.astype(np.float32))
    assert np.all(feats[:, nc - 1 + dim:] == 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_level_feature(dim):
    """The last feature is the level of corner 000 as a fraction of the value
    range: rint(127 c_000 (s1/s2) / Qhi), clamped to 0..127; 0 when Qhi = 0."""
    nc = 1 << dim
    corners = np.zeros((6, 8), np.int32)
    corners[:, 0] = [0, 50, 100, 199, 400, 1000]
    m = _pack(_identity_model(dim, nc - 1 + dim))
    _, p = oracle.mlp_predict(dim, m, corners, np.zeros((6, 3), np.float32), 2.0, Qhi=400)
    # 127 * 2 c / 400: 0, 31.75, 63.5 (ties to even: 64), 126.365, 254 -> 127, 635 -> 127
    assert list(p) == [0.0, 32.0, 64.0, 126.0, 127.0, 127.0]
    _, p = oracle.mlp_predict(dim, m, corners, np.zeros((6, 3), np.float32), 2.0, Qhi=0)
    assert np.all(p == 0.0)


def test_feature_scale_by_bin_ratio():
    """e_k is measured in vertex bins: grid-code differences times s1/s2."""
    corners = np.array([[10, 14, 0, 0, 0, 0, 0, 0], [10, 9, 0, 0, 0, 0, 0, 0]], np.int32)
    _, p = oracle.mlp_predict(2, _pack(_identity_model(2, 0)), corners,
                              np.zeros((2, 3), np.float32), 2.5)
    assert list(p) == [10.0, -2.0]   # 4 * 2.5 = 10; -1 * 2.5 = -2.5 -> -2 (ties to even)


def test_model_validation():
    m = _random_model(2, 0)
    blob = _pack(m)
    corners = np.zeros((1, 8), np.int32)
    fr = np.zeros((1, 3), np.float32)
    oracle.mlp_predict(2, blob, corners, fr, 1.0)
    bad = []
    b = blob.copy(); b[0] ^= 1; bad.append(b)                    # magic
    b = _pack(dict(m, dim=3)); bad.append(b)                     # dim mismatch
    mm = dict(m); mm["W1"] = m["W1"].copy(); mm["W1"][0, 12] = 1; bad.append(_pack(mm))  # padding
    mm = dict(m); mm["W2"] = m["W2"].copy(); mm["W2"][3, 3] = -128; bad.append(_pack(mm))
    mm = dict(m, s1=0); bad.append(_pack(mm))
    mm = dict(m, s2=31); bad.append(_pack(mm))
    mm = dict(m); mm["b1"] = m["b1"].copy(); mm["b1"][0] = (1 << 22) + 1; bad.append(_pack(mm))
    for b in bad:
        with pytest.raises(oracle.OracleError):
            oracle.mlp_predict(2, b, corners, fr, 1.0)


# --------------------------------------------------------------------------- #
# the predictor inside the method
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_zero_model_equals_plain_method(plan2d, plan3d, which):
    coords, plan = plan2d if which == "2d" else plan3d
    x = synth.field_vortex(coords, seed=4) if which == "3d" else synth.field_bumps_noise(coords, seed=4)
    s0, d0 = oracle.compress(plan, x, debug=True, eb=1e-3)
    s1, d1 = oracle.compress(plan, x, debug=True, eb=1e-3, model=_pack(_blank(plan.dim)))
    for k in ("Q", "q1", "sym1", "sym2"):
        assert np.array_equal(d0[k], d1[k])
    assert np.array_equal(oracle.decompress(plan, s0), oracle.decompress(plan, s1))
    assert s1.size == s0.size + oracle.MODEL_BYTES + (-s0.size % 8)


@pytest.mark.parametrize("which", ["2d", "3d"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_learned_stream_holds_bound_and_embeds_model(plan2d, plan3d, which, dtype):
    coords, plan = plan2d if which == "2d" else plan3d
    x = (synth.field_vortex(coords, seed=5) if which == "3d"
         else synth.field_bumps_noise(coords, seed=5)).astype(dtype)
    blob = _pack(_random_model(plan.dim, 7))
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-3, model=blob)
    f = oracle.field_params(x, eb=1e-3)
    y = oracle.decompress(plan, s)
    assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= f["tau2"]
    assert int(s[20:24].view(np.uint32)[0]) & 2
    assert int(s[192:200].view(np.uint64)[0]) == oracle.MODEL_BYTES
    assert np.array_equal(s[-oracle.MODEL_BYTES:], blob)
    # the stream differs from the plain one (the model moved the residuals)
    _, d0 = oracle.compress(plan, x, debug=True, eb=1e-3)
    assert not np.array_equal(d0["sym2"], dbg["sym2"])
    assert np.array_equal(d0["q1"], dbg["q1"])
    # a corrupted model section is detected
    t = s.copy(); t[-oracle.MODEL_BYTES] ^= 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.decompress(plan, t)
    assert e.value.status == oracle.CORRUPT


def test_learned_prediction_is_interpolation_plus_network(plan2d):
    """P = round(rho12 g + p): the residual codes of a learned stream against
    an independent FP64 interpolation g plus the network output p (taken from
    the corner codes and local coordinates of each vertex)."""
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=6)
    blob = _pack(_random_model(2, 8))
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-3, grid_fraction=0.4, model=blob)
    f = oracle.field_params(x, eb=1e-3, grid_fraction=0.4)
    nx = plan.grid.n[0]
    c = plan.cell.astype(np.int64)
    q1 = dbg["q1"]
    corners = np.zeros((plan.n_v, 8), np.int32)
    corners[:, 0], corners[:, 1] = q1[c], q1[c + 1]
    corners[:, 2], corners[:, 3] = q1[c + nx], q1[c + nx + 1]
    fr32 = np.zeros((plan.n_v, 3), np.float32)
    fr32[:, :2] = (plan.frac.astype(np.float32) * np.float32(2.0 ** -15)).T
    _, p = oracle.mlp_predict(2, blob, corners, fr32, f["rho12_f"], Qhi=f["Qhi"])
    assert int(s[200:208].view(np.int64)[0]) == f["Qhi"]
    fr = plan.frac.astype(np.float64) / 32768.0
    g = ((1 - fr[0]) * (1 - fr[1]) * corners[:, 0] + fr[0] * (1 - fr[1]) * corners[:, 1]
         + (1 - fr[0]) * fr[1] * corners[:, 2] + fr[0] * fr[1] * corners[:, 3])
    rho12 = f["rho12_q"] / 2.0 ** 40
    sym = dbg["sym2"].astype(np.int64)
    ok = (sym != 0) & (sym != 2 * 512 - 1)
    P = dbg["Q"].astype(np.int64) - (sym - 512)
    assert ok.mean() > 0.9 and np.abs(p).max() > 2.0
    assert np.abs(P - (rho12 * g + p))[ok].max() <= 0.5 + 1e-3


# --------------------------------------------------------------------------- #
# training network: gradient
# --------------------------------------------------------------------------- #
def _float_net(seed, dyadic=20):
    rng = np.random.default_rng(seed)
    q = 2.0 ** -dyadic
    W1 = np.round(rng.normal(0, 0.5, (H, 16)) / q) * q
    W1[:, 11:] = 0
    b1 = np.round(rng.normal(0, 0.2, H) / q) * q
    W2 = np.round(rng.normal(0, 0.25, (H, H)) / q) * q
    b2 = np.round(rng.normal(0, 0.2, H) / q) * q
    W3 = np.round(rng.normal(0, 0.25, H) / q) * q
    b3 = np.round(rng.normal(0, 0.2, 1) / q) * q
    return [a.astype(np.float32) for a in (W1, b1, W2, b2, W3, b3)]


def _batch(seed, B=48):
    rng = np.random.default_rng(seed + 100)
    X = np.zeros((B, 16), np.float32)
    X[:, :11] = rng.integers(-127, 128, (B, 11)) / 128.0
    Y = rng.normal(0, 1.0, B).astype(np.float32)
    return X, Y


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_gradient_central_differences(loss):
    """With the ReLU pattern and the error signs fixed, the loss is linear
    (l1) or quadratic (l2) in each single parameter, so the central
    difference is exact up to FP64 rounding. The step is a power of two and
    the parameters are dyadic, so w +- h is exact in float32."""
    net = _float_net(1)
    X, Y = _batch(1)
    L0, g = oracle.mlp_grad(*net, X, Y, loss=loss, rounding=False)
    h = 2.0 ** -14
    rng = np.random.default_rng(2)
    sizes = [a.size for a in net]
    offs = np.cumsum([0] + sizes)
    picks = []
    for t, n in enumerate(sizes):
        idx = np.arange(n) if n <= 64 else rng.choice(n, 48, replace=False)
        if t == 0:
            idx = [i for i in idx if i % 16 < 11]
        picks += [(t, int(i)) for i in idx]
    for t, i in picks:
        up = [a.copy() for a in net]; dn = [a.copy() for a in net]
        up[t].reshape(-1)[i] += np.float32(h)
        dn[t].reshape(-1)[i] -= np.float32(h)
        Lu, _ = oracle.mlp_grad(*up, X, Y, loss=loss, rounding=False)
        Ld, _ = oracle.mlp_grad(*dn, X, Y, loss=loss, rounding=False)
        fd = (Lu - Ld) / (2 * h)
        an = g[offs[t] + i]
        assert abs(fd - an) <= 1e-9 + 1e-7 * abs(an), (t, i, fd, an)
    assert L0 > 0


def test_gradient_padding_columns_are_zero():
    net = _float_net(3)
    X, Y = _batch(3)
    _, g = oracle.mlp_grad(*net, X, Y)
    assert np.all(g[:1024].reshape(H, 16)[:, 11:] == 0)


def test_rounding_mode_is_identity_on_bf16_exact_operands():
    """When every rounded operand is already a bfloat16 value, rounding mode 1
    equals the FP64 definition: inputs are powers of two on one feature,
    weights bfloat16 values, W2 a signed permutation, l1 loss with B = 2^k
    (the output gradients are +-2^-k)."""
    rng = np.random.default_rng(5)
    B = 32
    W1 = np.zeros((H, 16), np.float32)
    W1[:, 0] = rng.choice([-1.5, -0.75, 0.5, 1.0, 1.25], H)
    b1 = np.zeros(H, np.float32)
    perm = rng.permutation(H)
    W2 = np.zeros((H, H), np.float32)
    W2[np.arange(H), perm] = rng.choice([-2.0, -0.5, 0.75, 1.5], H)
    b2 = np.zeros(H, np.float32)
    W3 = rng.choice([-1.0, 0.5, 0.25, 2.0], H).astype(np.float32)
    b3 = np.array([0.375], np.float32)
    X = np.zeros((B, 16), np.float32)
    X[:, 0] = rng.choice([-1.0, -0.5, 0.25, 0.5, 1.0], B)
    Y = rng.normal(0, 3, B).astype(np.float32)
    net = [W1, b1, W2, b2, W3, b3]
    L0, g0 = oracle.mlp_grad(*net, X, Y, rounding=False)
    L1, g1 = oracle.mlp_grad(*net, X, Y, rounding=True)
    assert L0 == L1 and np.array_equal(g0, g1)
    # generic operands: the two modes agree to bfloat16 precision
    net = _float_net(6)
    X, Y = _batch(6, 256)
    _, g0 = oracle.mlp_grad(*net, X, Y, loss="l2", rounding=False)
    _, g1 = oracle.mlp_grad(*net, X, Y, loss="l2", rounding=True)
    assert np.linalg.norm(g1 - g0) <= 0.02 * np.linalg.norm(g0)
    assert not np.array_equal(g0, g1)


# --------------------------------------------------------------------------- #
# post-training quantisation
# --------------------------------------------------------------------------- #
def _float_params(seed):
    net = _float_net(seed)
    return np.concatenate([a.reshape(-1) for a in net]).astype(np.float32)


def _float_forward(params, X):
    W1, b1, W2, b2, W3, b3 = [a.astype(np.float64) for a in oracle.split_params(params)]
    z1 = X.astype(np.float64) @ W1.T + b1
    z2 = np.maximum(z1, 0) @ W2.T + b2
    return np.maximum(z2, 0) @ W3 + b3[0], z1, z2


def test_quantize_dyadic_weights_exactly():
    """Weights that are integers times 2^-a with the largest magnitude in
    64..127 quantise to those integers; biases to b 2^(a+7) (layer 1)."""
    rng = np.random.default_rng(7)
    params = _float_params(7)
    W1, b1, W2, b2, W3, b3 = oracle.split_params(params)
    I1 = rng.integers(-127, 128, (H, 16)); I1[:, 11:] = 0; I1[0, 0] = 127
    W1[:] = I1 * 2.0 ** -9
    b1[:] = rng.integers(-500, 500, H) * 2.0 ** -16
    blob = oracle.mlp_quantize(3, 2, params, 3.0, 5.0)
    m = oracle.unpack_model(blob)
    assert np.array_equal(m["W1"], I1)
    assert np.array_equal(m["b1"], np.rint(b1.astype(np.float64) * 2.0 ** 16).astype(np.int32))
    assert m["sx"] == 2 and m["dim"] == 3 and m["n_in"] == 7 + 3 + 1


def test_quantize_scale_invariances():
    """Moving a power of two from layer 2 into layer 1 leaves the quantised
    model unchanged; scaling the output layer by 2 only raises e3 by 1."""
    params = _float_params(8)
    X = np.zeros((512, 16), np.float32)
    X[:, :11] = np.random.default_rng(8).integers(-127, 128, (512, 11)) / 128.0
    _, z1, z2 = _float_forward(params, X)
    mz1, mz2 = float(np.maximum(z1, 0).max()), float(np.maximum(z2, 0).max())
    base = oracle.mlp_quantize(3, 0, params, mz1, mz2)
    p2 = params.copy()
    W1, b1, W2, b2, W3, b3 = oracle.split_params(p2)
    W1 *= 2; b1 *= 2; W2 *= 0.5
    assert np.array_equal(oracle.mlp_quantize(3, 0, p2, 2 * mz1, mz2), base)
    p3 = params.copy()
    W1, b1, W2, b2, W3, b3 = oracle.split_params(p3)
    W3 *= 2; b3 *= 2
    m0, m3 = oracle.unpack_model(base), oracle.unpack_model(oracle.mlp_quantize(3, 0, p3, mz1, mz2))
    assert m3["e3"] == m0["e3"] + 1
    for k in ("W1", "W2", "W3", "b1", "b2"):
        assert np.array_equal(m3[k], m0[k])
    assert m3["b3"] == m0["b3"] and (m3["s1"], m3["s2"]) == (m0["s1"], m0["s2"])


@pytest.mark.parametrize("seed", [9, 10, 11])
def test_quantized_network_tracks_float_network(seed):
    """The integer model evaluated by the oracle's predictor approximates the
    float network on the integer features (8-bit weights and activations)."""
    params = _float_params(seed)
    rng = np.random.default_rng(seed)
    n = 2000
    corners = rng.integers(-60, 61, (n, 8)).astype(np.int32)
    corners[:, 0] = 0
    fr = rng.random((n, 3)).astype(np.float32)
    Xi = np.zeros((n, 16))
    Xi[:, :7] = corners[:, 1:]
    Xi[:, 7:10] = np.round(fr.astype(np.float64) * 127)
    pf, z1, z2 = _float_forward(params, (Xi / 128.0).astype(np.float32))
    blob = oracle.mlp_quantize(3, 0, params, float(np.maximum(z1, 0).max()),
                               float(np.maximum(z2, 0).max()))
    feats, pq = oracle.mlp_predict(3, blob, corners, fr, 1.0)
    assert np.array_equal(feats, Xi.astype(np.int32))
    err = np.abs(pq - pf)
    assert err.max() <= 0.06 * np.abs(pf).max()
    assert np.corrcoef(pq, pf)[0, 1] > 0.999


def test_quantize_degenerate_and_errors():
    params = np.zeros(oracle.MLP_PARAMS, np.float32)
    m = oracle.unpack_model(oracle.mlp_quantize(2, 0, params, 0.0, 0.0))
    assert 1 <= m["s1"] <= 30 and 1 <= m["s2"] <= 30
    assert not m["W1"].any() and not m["W2"].any() and m["b3"] == 0
    with pytest.raises(oracle.OracleError):
        oracle.mlp_quantize(2, 61, params, 1.0, 1.0)
    with pytest.raises(oracle.OracleError):
        oracle.mlp_quantize(2, 0, params, -1.0, 1.0)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_edge_models_hold_bound(plan2d, plan3d, which):
    """Saturated or zeroed activations, extreme exponents and biases: the
    bound holds whatever the network says (a correction too large for the
    residual codes turns the vertex into a raw value)."""
    from mlp_models import edge_models
    coords, plan = plan2d if which == "2d" else plan3d
    x = synth.field_vortex(coords, seed=9) if which == "3d" else synth.field_bumps_noise(coords, seed=9)
    f = oracle.field_params(x, eb=1e-4)
    for name, m in edge_models(plan.dim):
        s, dbg = oracle.compress(plan, x, debug=True, eb=1e-4, model=_pack(m))
        y = oracle.decompress(plan, s)
        assert np.abs(y - x).max() <= f["tau2"], name
        if name == "e3_max":  # p = 0 only where the output sum is exactly 0
            assert np.mean(dbg["sym2"] == 2 * 512 - 1) > 0.99


def _auto_cost(sym2, R2, vsz, model):
    cnt = np.bincount(sym2, minlength=2 * R2).astype(np.uint64)
    ln = oracle.huffman_lengths(cnt).astype(np.uint64)
    bits = int((cnt * ln).sum()) + 32 * int(cnt[0]) + 8 * vsz * int(cnt[2 * R2 - 1])
    return bits + (8 * oracle.MODEL_BYTES if model else 0)


def _convex_model(B):
    """p ~ -(B[0] f(X) + B[1] f(Y)), f(t) = t (127 - t) / 127^2: the bilinear
    interpolation error of a paraboloid, in vertex bins, as a piecewise-linear
    function of the coordinate features X, Y (knots 0, 32, 64, 96: ReLU units
    relu(X - t) carried exactly through both layers), output scale 2^-4."""
    knots = np.array([0, 32, 64, 96, 127], np.float64)
    f = knots * (127 - knots) / 127.0 ** 2
    slope = np.diff(f) / np.diff(knots)
    c = np.concatenate([[slope[0]], np.diff(slope)])
    m = _blank(2, s1=1, s2=1, e3=-4)
    for a in range(2):
        for k in range(4):
            u = 4 * a + k
            m["W1"][u, 3 + a] = 2
            m["b1"][u] = -2 * int(knots[k])
            m["W2"][u, u] = 2
            m["W3"][u] = int(np.rint(-B[a] * c[k] * 16))
    return m


@pytest.fixture(scope="module")
def plan2d_big():
    coords, cells = synth.mesh2d_jittered(nside=200, seed=33)
    return coords, oracle.Plan(coords, cells, (33, 29))


@pytest.mark.parametrize("which", ["zero", "random", "convex"])
def test_auto_selection_keeps_the_smaller_encoding(plan2d_big, which):
    """Auto selection: both predictors run; the learned one is kept when its
    code bits plus escape and raw values plus the model are fewer than the
    plain predictor's (a tie keeps the plain). Costs recomputed here from the
    two single-predictor runs. For a paraboloid the bilinear interpolation
    error is a known function of the local coordinates, which a hand-built
    network predicts, so there the learned predictor wins."""
    coords, plan = plan2d_big
    eb = 2e-6
    s2 = 2 * (0.5 * eb) * (1 - 2.0 ** -20)
    if which == "convex":
        x = coords[:, 0] ** 2 + coords[:, 1] ** 2
        h = plan.grid.h
        m = _convex_model((h[0] ** 2 / s2, h[1] ** 2 / s2))
    else:
        x = 1e-3 * synth.field_bumps_noise(coords, seed=14)
        m = _blank(2) if which == "zero" else _random_model(2, 15)
    blob = _pack(m)
    kw = dict(eb=eb, eb_mode="abs")
    s0, d0 = oracle.compress(plan, x, debug=True, **kw)
    s1, d1 = oracle.compress(plan, x, debug=True, model=blob, **kw)
    sa = oracle.compress(plan, x, model=blob, auto=True, **kw)
    c0 = _auto_cost(d0["sym2"], 512, 8, False)
    c1 = _auto_cost(d1["sym2"], 512, 8, True)
    want = s1 if c1 < c0 else s0
    assert np.array_equal(sa, want)
    if which == "convex":
        assert c1 < c0
    else:
        assert c1 >= c0
