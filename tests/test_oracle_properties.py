"""Property tests of the oracle over random meshes, fields and parameters
(with and without the zero-run stage): the bound at every vertex (closed loop tau2, open loop tau1 + tau2), a
deterministic stream, decoding equal to the debug codes' reconstruction,
and the 1D coder's bound. Seeded draws (numpy), so the CPU suite stays
reproducible without extra packages."""
import numpy as np
import pytest

import oracle
import synth


def _draw(seed):
    rng = np.random.default_rng(seed)
    dim = int(rng.choice([2, 3]))
    if dim == 2:
        c, e = synth.mesh2d_jittered(nside=int(rng.integers(6, 40)), jitter=float(rng.uniform(0, 0.45)),
                                     seed=int(rng.integers(1 << 30)))
        n = tuple(int(v) for v in rng.integers(2, 48, 2))
    else:
        c, e = synth.mesh3d_annulus(nr=int(rng.integers(3, 7)), nth=int(rng.integers(8, 24)),
                                    nz=int(rng.integers(3, 8)), seed=int(rng.integers(1 << 30)))
        n = tuple(int(v) for v in rng.integers(2, 14, 3))
    kind = rng.integers(4)
    if kind == 0:
        x = synth.field_bumps_noise(c, seed=int(rng.integers(1 << 30)))
    elif kind == 1:
        x = rng.standard_normal(c.shape[0]) * 10.0 ** rng.uniform(-3, 3)
    elif kind == 2:
        x = np.full(c.shape[0], rng.uniform(-5, 5))
    else:
        x = c[:, 0] * rng.uniform(-4, 4) + rng.uniform(-1e4, 1e4)
    dtype = np.float64 if rng.random() < 0.6 else np.float32
    R = int(rng.choice([4, 7, 64, 512, 2048]))
    lmax = int(rng.integers(max(3, int(np.ceil(np.log2(2 * R)))), 25))
    kw = dict(eb=float(10 ** rng.uniform(-6, -1)), eb_mode=str(rng.choice(["rel", "abs"])),
              grid_fraction=float(rng.uniform(0.01, 0.99)), R1=R, R2=int(rng.choice([4, 64, 512])),
              C1=int(rng.integers(1, 257)), C2=int(rng.integers(1, 257)), lmax=lmax,
              f_op=str(rng.choice(["barycentric", "cluster"])),
              g_op=str(rng.choice(["multilinear", "nearest"])), open_loop=bool(rng.random() < 0.3))
    kw["lmax"] = max(kw["lmax"], int(np.ceil(np.log2(2 * max(kw["R1"], kw["R2"])))))
    # the zero-run stage on half of the draws (its alphabets of 2R + 2 tokens
    # take R < 2048 and one more bit of length limit where 2R fills lmax)
    kw["zero_run"] = bool(rng.random() < 0.5) and max(kw["R1"], kw["R2"]) < 2048
    if kw["zero_run"]:
        kw["lmax"] = max(kw["lmax"], int(np.ceil(np.log2(2 * max(kw["R1"], kw["R2"]) + 2))))
    return c, e, n, x.astype(dtype), kw


@pytest.mark.parametrize("seed", range(40))
def test_random_configurations_hold_the_bound(seed):
    c, e, n, x, kw = _draw(seed)
    op = oracle.Plan(c, e, n)
    try:
        s = oracle.compress(op, x, **kw)
    except oracle.OracleError as err:  # only a bound the codes cannot span
        assert err.status == 4
        return
    assert np.array_equal(s, oracle.compress(op, x, **kw))
    y = oracle.decompress(op, s)
    f = oracle.field_params(x, **{k: v for k, v in kw.items()
                                 if k not in ("f_op", "g_op", "open_loop")})
    bound = f["tau1"] + f["tau2"] if kw["open_loop"] else f["tau2"]
    assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= bound


@pytest.mark.parametrize("seed", range(20))
def test_random_1d_coder_holds_the_bound(seed):
    c, e, n, x, kw = _draw(1000 + seed)
    kw1 = {k: v for k, v in kw.items() if k not in ("f_op", "g_op", "open_loop", "grid_fraction")}
    try:
        s = oracle.compress_1d(x, **kw1)
    except oracle.OracleError as err:
        assert err.status == 4
        return
    y = oracle.decompress_1d(s, x.size)
    xd = x.astype(np.float64)
    tau = kw1["eb"] * (xd.max() - xd.min()) if kw1["eb_mode"] == "rel" and xd.max() > xd.min() else kw1["eb"]
    assert np.abs(y.astype(np.float64) - xd).max() <= tau


@pytest.mark.parametrize("seed", range(12))
def test_random_coarsened_plans_hold_the_bound(seed):
    """Grid_Coarsen on random meshes and grids finer than them: the plan on
    the kept planes holds the bound and decodes deterministically, for the
    g the planes were kept for."""
    c, e, n, x, kw = _draw(2000 + seed)
    rng = np.random.default_rng(seed)
    n = tuple(int(v) * int(rng.integers(1, 4)) for v in n)  # up to 3x finer
    op = oracle.Plan(c, e, n)
    g_op = str(rng.choice(["multilinear", "nearest"]))
    keep = oracle.grid_coarsen(op, g_op)
    for d in range(op.dim):
        assert keep[d].size >= 2 and np.all(np.diff(keep[d]) > 0)
    kp = oracle.Plan(c, e, n, keep=keep)
    kw = dict(kw, g_op=g_op, f_op=kw["f_op"])
    if g_op == "nearest":
        kw.pop("model", None)
    try:
        s = oracle.compress(kp, x, **kw)
    except oracle.OracleError as err:
        assert err.status == 4
        return
    assert np.array_equal(s, oracle.compress(kp, x, **kw))
    y = oracle.decompress(kp, s)
    f = oracle.field_params(x, **{k: v for k, v in kw.items()
                                 if k not in ("f_op", "g_op", "open_loop")})
    bound = f["tau1"] + f["tau2"] if kw["open_loop"] else f["tau2"]
    assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= bound
