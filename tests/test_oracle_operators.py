"""Pins of the paper's own operators in the oracle: the nearest-node g
(Sec. III-B: x2[k] = x[k] - x1[m_k]) and the cluster-mean f (Sec. III-C:
x1[j] = mean of the vertices whose nearest node is j), each checked against
an independent numpy evaluation, the geometry, the mean's least-squares
property and the bound theorem (Sec. III, a linear g with sum |a_j| = 1)."""
import numpy as np
import pytest

import oracle
import synth

COMBOS = [("barycentric", "multilinear"), ("barycentric", "nearest"),
          ("cluster", "multilinear"), ("cluster", "nearest")]


@pytest.fixture(scope="module")
def plans():
    c2, e2 = synth.mesh2d_jittered(nside=60, seed=21)
    c3, e3 = synth.mesh3d_annulus(nr=6, nth=24, nz=8, seed=22)
    return {"2d": (c2, oracle.Plan(c2, e2, (41, 37))),
            "3d": (c3, oracle.Plan(c3, e3, (13, 12, 9)))}


def _field(which, coords, seed):
    return (synth.field_bumps_noise(coords, seed=seed) if which == "2d"
            else synth.field_vortex(coords, seed=seed))


def _nearest(plan):
    """m_k from the plan's cell and local coordinates (half goes up)."""
    nx, ny = plan.grid.n[0], plan.grid.n[1]
    m = plan.cell.astype(np.int64).copy()
    for d, stride in enumerate([1, nx, nx * ny][:plan.dim]):
        m += stride * (plan.frac[d] >= 16384)
    return m


def _node_coords(plan, j):
    g = plan.grid
    n = list(g.n[:plan.dim])
    idx = np.unravel_index(j, n[::-1])[::-1]  # x fastest
    return np.stack([g.lo[d] + idx[d] * g.h[d] for d in range(plan.dim)], axis=1)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_nearest_node_is_the_geometric_nearest_corner(plans, which):
    """m_k is the grid node closest to vertex k (among its cell's corners,
    hence among all nodes of a rectilinear grid), up to the 2^-15 rounding of
    the local coordinates at the midplanes."""
    coords, plan = plans[which]
    m = _nearest(plan)
    nx, ny = plan.grid.n[0], plan.grid.n[1]
    c = plan.cell.astype(np.int64)
    best = np.full(plan.n_v, np.inf)
    arg = np.zeros(plan.n_v, np.int64)
    for corner in range(1 << plan.dim):
        off = sum(((corner >> d) & 1) * s for d, s in enumerate([1, nx, nx * ny][:plan.dim]))
        p = _node_coords(plan, c + off)
        dist = ((p - coords[:, :plan.dim]) ** 2).sum(axis=1)
        better = dist < best
        best[better] = dist[better]
        arg[better] = (c + off)[better]
    fr = plan.frac.astype(np.float64) / 32768.0
    near_tie = (np.abs(fr - 0.5) < 2.0 ** -14).any(axis=0)
    assert np.array_equal(m[~near_tie], arg[~near_tie])
    assert near_tie.mean() < 0.01


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_nearest_node_prediction(plans, which):
    """g nearest: P = round((s1/s2) q1[m_k]) at every vertex (q2 = Q - P)."""
    coords, plan = plans[which]
    x = _field(which, coords, 3)
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-3, g_op="nearest")
    f = oracle.field_params(x, eb=1e-3)
    m = _nearest(plan)
    sym = dbg["sym2"].astype(np.int64)
    ok = (sym != 0) & (sym != 2 * 512 - 1)
    assert ok.mean() > 0.8
    P = dbg["Q"].astype(np.int64) - (sym - 512)
    want = dbg["q1"].astype(np.float64)[m] * (f["rho12_q"] / 2.0 ** 40)
    assert np.abs(P - want)[ok].max() <= 0.5 + 1e-6


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_cluster_mean_grid_codes(plans, which):
    """f cluster: q1[j] = round((s2/s1) mean(Q over the vertices nearest to
    j)), and nodes no vertex is nearest to take the fill value."""
    coords, plan = plans[which]
    x = _field(which, coords, 4)
    for frac in (0.3, 0.7):
        s, dbg = oracle.compress(plan, x, debug=True, eb=1e-3, grid_fraction=frac, f_op="cluster")
        f = oracle.field_params(x, eb=1e-3, grid_fraction=frac)
        m = _nearest(plan)
        Q = dbg["Q"].astype(np.float64)
        cnt = np.bincount(m, minlength=plan.n_g)
        mean = np.bincount(m, weights=Q, minlength=plan.n_g) / np.maximum(cnt, 1)
        mean[cnt == 0] = f["fill_u"]
        rho21 = f["rho21_q"] / 2.0 ** 40
        assert np.abs(dbg["q1"] - rho21 * mean).max() <= 0.5 + 1e-4
        assert (cnt == 0).any() and (cnt > 1).any()


def test_cluster_mean_least_squares(plans):
    """Sec. III-C: the cluster mean minimises the sum of squared residuals of
    its cluster; the oracle's grid values (its q1 back in vertex bins) are
    within a grid bin of the minimiser, and moving them by a bin or more makes
    the sum larger."""
    coords, plan = plans["2d"]
    x = _field("2d", coords, 5)
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-4, grid_fraction=0.05, f_op="cluster")
    f = oracle.field_params(x, eb=1e-4, grid_fraction=0.05)
    m = _nearest(plan)
    Q = dbg["Q"].astype(np.float64)
    x1 = dbg["q1"].astype(np.float64) * (f["rho12_q"] / 2.0 ** 40)  # vertex bins
    sse = lambda v: np.bincount(m, weights=(Q - v[m]) ** 2, minlength=plan.n_g)
    base = sse(x1)
    step = f["rho12_q"] / 2.0 ** 40  # one grid bin in vertex bins
    used = np.bincount(m, minlength=plan.n_g) > 0
    for d in (-2 * step, 2 * step):
        assert np.all(sse(x1 + d)[used] > base[used])


@pytest.mark.parametrize("fop,gop", COMBOS)
@pytest.mark.parametrize("which", ["2d", "3d"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("open_loop", [False, True])
def test_operator_bound(plans, fop, gop, which, dtype, open_loop):
    """Every combination keeps the bound (closed loop tau2, open loop
    tau1 + tau2) and records the operators in the header flags."""
    coords, plan = plans[which]
    x = _field(which, coords, 6).astype(dtype)
    kw = dict(eb=1e-3, grid_fraction=0.4, f_op=fop, g_op=gop, open_loop=open_loop)
    s = oracle.compress(plan, x, **kw)
    flags = int(s[20:24].view(np.uint32)[0])
    assert bool(flags & 8) == (gop == "nearest") and bool(flags & 16) == (fop == "cluster")
    assert bool(flags & 4) == open_loop
    y = oracle.decompress(plan, s)
    f = oracle.field_params(x, eb=1e-3, grid_fraction=0.4)
    bound = f["tau1"] + f["tau2"] if open_loop else f["tau2"]
    assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= bound


def test_default_operators_unchanged(plans):
    """The default operators give the same stream as before the options."""
    coords, plan = plans["3d"]
    x = _field("3d", coords, 7)
    a = oracle.compress(plan, x, eb=1e-4)
    b = oracle.compress(plan, x, eb=1e-4, f_op="barycentric", g_op="multilinear")
    assert np.array_equal(a, b)
    assert int(a[20:24].view(np.uint32)[0]) & 24 == 0


def test_operator_errors(plans):
    from mlp_models import pack, random_model
    coords, plan = plans["2d"]
    x = _field("2d", coords, 8)
    with pytest.raises(oracle.OracleError) as err:
        oracle.compress(plan, x, eb=1e-3, g_op="nearest", model=pack(random_model(2, 1)))
    assert err.value.status == 1  # invalid argument
    for bad in (dict(f_op=2), dict(g_op=-1)):
        with pytest.raises(oracle.OracleError) as err:
            oracle.compress(plan, x, eb=1e-3, **bad)
        assert err.value.status == 1
    # a learned stream flagged as nearest-node
    s = oracle.compress(plan, x, eb=1e-3, model=pack(random_model(2, 1)))
    t = s.copy()
    t[20] |= 8
    with pytest.raises(oracle.OracleError) as err:
        oracle.decompress(plan, t)
    assert err.value.status == 5  # corrupt
    # the f flag is informative only: clearing it decodes the same values
    s = oracle.compress(plan, x, eb=1e-3, f_op="cluster")
    t = s.copy()
    t[20] &= 0xEF
    assert np.array_equal(oracle.decompress(plan, t), oracle.decompress(plan, s))
