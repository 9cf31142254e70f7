"""GPU training of the learned predictor: the tensor-core gradient against the
oracle's FP64 gradient (same bf16 operand rounding), quantisation bit-exact
against the oracle, determinism, argument errors, and the gain of a trained
model over the method without it on unseen fields."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _net(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, 0.5 * scale, (64, 16)); W1[:, 11:] = 0
    b1 = rng.normal(0, 0.2, 64)
    W2 = rng.normal(0, 0.25 * scale, (64, 64))
    b2 = rng.normal(0, 0.2, 64)
    W3 = rng.normal(0, 0.25 * scale, 64)
    b3 = rng.normal(0, 0.2, 1)
    return np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float32)


def _batch(seed, B, kind):
    rng = np.random.default_rng(seed + 1000)
    X = np.zeros((B, 16), np.float32)
    if kind == "features":  # integer features times 2^-7, as in training
        X[:, :7] = rng.integers(-127, 128, (B, 7)) / 128.0
        X[:, 7:11] = rng.integers(0, 128, (B, 4)) / 128.0
    else:                   # generic floats (rounded to bf16 by both sides)
        X[:, :11] = rng.normal(0, 0.7, (B, 11))
    Y = rng.normal(0, 2.0, B).astype(np.float32)
    return X, Y


@pytest.mark.parametrize("loss", ["l1", "l2"])
@pytest.mark.parametrize("B,kind", [(128, "features"), (300, "features"), (1000, "generic")])
def test_gradient_matches_oracle(loss, B, kind):
    import paper_2501_06910_gb300 as mcc
    w = _net(B)
    X, Y = _batch(B, B, kind)
    g, lv = mcc.mlp_grad(torch.from_numpy(w).cuda(), torch.from_numpy(X).cuda(),
                         torch.from_numpy(Y).cuda(), loss=loss)
    g = g.cpu().numpy().astype(np.float64)
    Lref, gref = oracle.mlp_grad(*oracle.split_params(w), X, Y, loss=loss, rounding=True)
    assert float(lv.cpu()[0]) == pytest.approx(Lref, rel=2e-5)
    assert np.linalg.norm(g - gref) <= 1e-3 * np.linalg.norm(gref)
    offs = np.cumsum([0, 1024, 64, 4096, 64, 64, 1])
    for t in range(6):
        a, b = g[offs[t]:offs[t + 1]], gref[offs[t]:offs[t + 1]]
        assert np.abs(a - b).max() <= 2e-3 * np.abs(b).max() + 1e-7, t
    assert np.all(g[:1024].reshape(64, 16)[:, 11:] == 0)


def test_gradient_descent_lowers_the_loss():
    import paper_2501_06910_gb300 as mcc
    w = torch.from_numpy(_net(5)).cuda()
    X, Y = _batch(5, 512, "features")
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    losses = []
    for _ in range(50):
        g, lv = mcc.mlp_grad(w, Xd, Yd, loss="l2")
        losses.append(float(lv.cpu()[0]))
        w -= 0.02 * g
    assert losses[-1] < 0.8 * losses[0]
    assert sum(b < a for a, b in zip(losses, losses[1:])) >= 45


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_quantize_bit_exact(seed):
    import paper_2501_06910_gb300 as mcc
    w = _net(seed, scale=[1.0, 1e-3, 40.0][seed - 1])
    for dim, sx, mz1, mz2 in [(3, 0, 3.5, 7.25), (2, -4, 1e-3, 1e4), (3, 7, 0.0, 0.0),
                              (3, 2, 1e6, 1e-6)]:
        want = oracle.mlp_quantize(dim, sx, w, mz1, mz2)
        got, st = mcc.mlp_quantize(dim, sx, torch.from_numpy(w).cuda(), mz1, mz2)
        assert int(st.cpu()[0]) == 0
        assert np.array_equal(got.cpu().numpy(), want), (dim, sx, mz1, mz2)
    bad = w.copy(); bad[7] = np.nan
    got, st = mcc.mlp_quantize(3, 0, torch.from_numpy(bad).cuda(), 1.0, 1.0)
    assert int(st.cpu()[0]) == mcc.INVALID_ARG
    with pytest.raises(oracle.OracleError):
        oracle.mlp_quantize(3, 0, bad, 1.0, 1.0)


# --------------------------------------------------------------------------- #
# training end to end (3D annulus slab at the 256^3-grid spacing)
# --------------------------------------------------------------------------- #
NZ = 8
HZ = 2.0 * (NZ - 1) / 243
_state = {}


def _slab():
    if "plan" not in _state:
        import gpu_helpers as G
        c, e = synth.mesh3d_annulus(nr=64, nth=512, nz=NZ, H=HZ, seed=5)
        n, lo, hi = (256, 256, NZ), (-1.0, -1.0, 0.0), (1.0, 1.0, HZ)
        _state.update(c=c, e=e, n=n, lo=lo, hi=hi, plan=G.plan(c, e, n, lo, hi))
    return _state


def _train(fields, steps=1500, **cfg_kw):
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    s = _slab()
    prm = G.params(np.float64, eb=1e-4)
    cfg = mcc.train_cfg_default(steps=steps, **cfg_kw)
    xs = [torch.from_numpy(f).cuda() for f in fields]
    return mcc.model_train(s["plan"], xs, prm, cfg)


def test_train_gain_on_unseen_fields():
    import gpu_helpers as G
    s = _slab()
    c = s["c"]
    train = [synth.field_vortex(c, seed=100 + i) for i in range(8)]
    model, losses = _train(train)
    assert np.mean(losses[-100:]) < 0.9 * np.mean(losses[:20])
    blob = model.cpu().numpy()
    m = oracle.unpack_model(blob)
    assert m["magic"] == 0x4D43434D and m["dim"] == 3 and m["n_in"] == 11
    op = oracle.Plan(c, s["e"], s["n"], s["lo"], s["hi"])
    total0 = total1 = 0
    for seed in (200, 201):
        x = synth.field_vortex(c, seed=seed)
        s0 = G.compress(s["plan"], x, eb=1e-4)
        s1 = G.compress(s["plan"], x, eb=1e-4, model=model)
        total0 += s0.size
        total1 += s1.size
        # the learned stream is the oracle's, bit for bit, and holds the bound
        assert np.array_equal(s1, oracle.compress(op, x, eb=1e-4, model=blob))
        y = G.decompress(s["plan"], s1, np.float64)
        assert np.abs(y - x).max() <= oracle.field_params(x, eb=1e-4)["tau2"]
    assert total1 < 0.97 * total0, (total0, total1)


def test_train_deterministic_and_seeded():
    s = _slab()
    fields = [synth.field_vortex(s["c"], seed=300 + i) for i in range(2)]
    a, la = _train(fields, steps=40, samples_per_field=8192)
    b, lb = _train(fields, steps=40, samples_per_field=8192)
    c, lc = _train(fields, steps=40, samples_per_field=8192, seed=2)
    assert torch.equal(a, b) and la == lb
    assert not torch.equal(a, c)


def test_train_argument_errors():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    s = _slab()
    x = torch.from_numpy(synth.field_vortex(s["c"], seed=1)).cuda()
    prm = G.params(np.float64, eb=1e-4)
    for bad in (dict(batch=100), dict(steps=0), dict(lr=0.0), dict(samples_per_field=0)):
        cfg = mcc.train_cfg_default(**bad)
        with pytest.raises(mcc.MCCError) as err:
            mcc.model_train(s["plan"], [x], prm, cfg)
        assert err.value.status == mcc.INVALID_ARG
    cfg = mcc.train_cfg_default(steps=5)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(mcc.MCCError) as err:
        mcc.model_train(s["plan"], [x], prm, cfg, workspace=small)
    assert err.value.status == mcc.CAPACITY
    # a bound the field cannot meet is reported, not trained on
    with pytest.raises(mcc.MCCError) as err:
        mcc.model_train(s["plan"], [x], G.params(np.float64, eb=1e-12), cfg)
    assert err.value.status == mcc.RANGE
