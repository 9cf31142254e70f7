"""Pins of the oracle's open-loop mode (Algorithm 3 as printed: the residual
is taken against g(x1) with the unquantised grid component x1, and the vertex
bound is tau1 + tau2, Sec. III), checked against independent FP64
evaluations of the definitions and the bound theorem."""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import _x1_in_node_units


@pytest.fixture(scope="module")
def plans():
    c2, e2 = synth.mesh2d_jittered(nside=60, seed=21)
    c3, e3 = synth.mesh3d_annulus(nr=6, nth=24, nz=8, seed=22)
    return {"2d": (c2, oracle.Plan(c2, e2, (41, 37))),
            "3d": (c3, oracle.Plan(c3, e3, (13, 12, 9)))}


def _field(which, coords, seed):
    return (synth.field_bumps_noise(coords, seed=seed) if which == "2d"
            else synth.field_vortex(coords, seed=seed))


def _flags(stream):
    return int(stream[20:24].view(np.uint32)[0])


def _multilinear(plan, values):
    """g at every vertex: the bilinear / trilinear interpolation of grid
    ``values`` over the vertex's cell, product form, FP64."""
    nx, ny = plan.grid.n[0], plan.grid.n[1]
    fr = plan.frac.astype(np.float64) / 32768.0
    c = plan.cell.astype(np.int64)
    g = np.zeros(plan.n_v)
    for corner in range(1 << plan.dim):
        off = 0
        w = np.ones(plan.n_v)
        for d, stride in enumerate([1, nx, nx * ny][:plan.dim]):
            bit = (corner >> d) & 1
            off += bit * stride
            w *= fr[d] if bit else 1.0 - fr[d]
        g += w * values[c + off]
    return g


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("eb,frac", [(1e-2, 0.5), (1e-3, 0.2), (1e-4, 0.8), (1e-6, 0.5)])
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_open_loop_bound(plans, which, dtype, eb, frac):
    """Sec. III: |x - x'| <= tau1 + tau2 <= tau at every vertex; the grid
    component is the closed-loop one, code for code."""
    coords, plan = plans[which]
    x = _field(which, coords, 5).astype(dtype)
    s, dbg = oracle.compress(plan, x, debug=True, eb=eb, grid_fraction=frac, open_loop=True)
    sc, dbc = oracle.compress(plan, x, debug=True, eb=eb, grid_fraction=frac)
    assert _flags(s) & 5 == 5 and _flags(sc) & 4 == 0
    assert np.array_equal(dbg["q1"], dbc["q1"]) and np.array_equal(dbg["sym1"], dbc["sym1"])
    assert np.array_equal(dbg["Q"], dbc["Q"])
    f = oracle.field_params(x, eb=eb, grid_fraction=frac)
    y = oracle.decompress(plan, s)
    assert y.dtype == dtype
    err = np.abs(y.astype(np.float64) - x.astype(np.float64))
    assert err.max() <= f["tau1"] + f["tau2"]
    assert f["tau1"] + f["tau2"] <= f["tau"] * (1 + 1e-15)


@pytest.mark.parametrize("which", ["2d", "3d"])
@pytest.mark.parametrize("frac", [0.3, 0.8])
def test_open_loop_residual_is_against_unquantised_x1(plans, which, frac):
    """q2 = round(x / s2 - g(x1)) with x1 = f(x) before quantisation: checked
    against an independent FP64 evaluation of x1 (barycentric) and g
    (multilinear); reconstruction s2 (q2 + g(x1')) with x1' = s1 q1."""
    coords, plan = plans[which]
    x = _field(which, coords, 12)
    eb = 1e-3
    s, dbg = oracle.compress(plan, x, debug=True, eb=eb, grid_fraction=frac, open_loop=True)
    f = oracle.field_params(x, eb=eb, grid_fraction=frac)
    x1 = _x1_in_node_units(plan, dbg["Q"].astype(np.int64), f["fill_u"])
    g = _multilinear(plan, x1)
    r = x * f["inv2"] - f["K"] - g
    sym = dbg["sym2"].astype(np.int64)
    ok = (sym != 0) & (sym != 2 * 512 - 1)
    assert ok.mean() > 0.9
    q2 = sym - 512
    assert np.abs(q2 - r)[ok].max() <= 0.5 + 1e-4
    # the decoder's reconstruction: s2 (K + q2 + g(x1')), x1' in vertex bins
    gq = _multilinear(plan, dbg["q1"].astype(np.float64) * (f["rho12_q"] / 2.0 ** 40))
    y = oracle.decompress(plan, s)
    xr = f["s2"] * (f["K"] + q2 + gq)
    assert np.abs(y - xr)[ok].max() <= 1e-9 * np.abs(x).max()


def test_open_loop_error_reaches_past_tau2(plans):
    """Open loop carries the grid component's error into the vertices: with a
    large grid share the error exceeds tau2 somewhere (the closed loop never
    does), while both stay within tau."""
    coords, plan = plans["2d"]
    x = _field("2d", coords, 9)
    f = oracle.field_params(x, eb=1e-3, grid_fraction=0.8)
    yo = oracle.decompress(plan, oracle.compress(plan, x, eb=1e-3, grid_fraction=0.8,
                                                 open_loop=True))
    yc = oracle.decompress(plan, oracle.compress(plan, x, eb=1e-3, grid_fraction=0.8))
    eo, ec = np.abs(yo - x).max(), np.abs(yc - x).max()
    assert ec <= f["tau2"] < eo <= f["tau"]


def test_open_loop_guard_large_offset(plans):
    """Values far from zero in bins of the bound: every vertex is checked after
    the cast to the output type and violators are stored raw. Near 1.2e4 the
    FP32 spacing 2^-10 lies between tau and 2 tau, so a reconstruction more
    than half a spacing away rounds to a neighbour outside the bound."""
    coords, plan = plans["2d"]
    for dtype in (np.float64, np.float32):
        x = (synth.field_bumps_noise(coords, seed=7) + 1.2e4).astype(dtype)
        kw = dict(eb=9e-4, eb_mode="abs", open_loop=True)
        s, dbg = oracle.compress(plan, x, debug=True, **kw)
        f = oracle.field_params(x, **kw)
        y = oracle.decompress(plan, s)
        assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= f["tau1"] + f["tau2"]
        if dtype == np.float32:
            assert np.any(dbg["sym2"] == 2 * 512 - 1)


def test_open_loop_errors(plans):
    from mlp_models import pack, random_model
    coords, plan = plans["2d"]
    x = _field("2d", coords, 3)
    with pytest.raises(oracle.OracleError) as err:
        oracle.compress(plan, x, eb=1e-3, open_loop=True, model=pack(random_model(2, 1)))
    assert err.value.status == 1  # invalid argument
    s = oracle.compress(plan, x, eb=1e-3, open_loop=True)
    for bad in (s[20] | 2, s[20] | 32):
        t = s.copy()
        t[20] = bad
        with pytest.raises(oracle.OracleError) as err:
            oracle.decompress(plan, t)
        assert err.value.status == 5  # corrupt
    # clearing the flag decodes the same codes closed-loop: a different field
    t = s.copy()
    t[20] &= 0xFB
    assert not np.array_equal(oracle.decompress(plan, t), oracle.decompress(plan, s))


def test_open_loop_deterministic(plans):
    coords, plan = plans["3d"]
    x = _field("3d", coords, 4)
    a = oracle.compress(plan, x, eb=1e-4, open_loop=True)
    assert np.array_equal(a, oracle.compress(plan, x, eb=1e-4, open_loop=True))
