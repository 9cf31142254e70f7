"""Pins of the oracle's Grid_Coarsen (Algorithm 2) and of plans on coarsened
grids. Every vertex marks the grid nodes its g uses (the nearest node, or all
corners of its cell); a plane (a line in 2D) normal to an axis stays when one
of its nodes is marked. Checked against an independent numpy restatement
from the coordinates; the coarsened grid's points are the base grid's points
(identical location and weights); the vertices' cells and local coordinates
on the kept planes against numpy; the nearest node keeps its physical node
(the paper's update of {m_i} is a renumbering); keeping every plane changes
nothing; the bound on coarsened grids; closed forms (a gap between two
blocks of mesh, a domain wider than the mesh)."""
import numpy as np
import pytest

import oracle
import synth


def _numpy_cells(coords, lo, h, kept):
    """Cell (per axis) and u16 local coordinate of every vertex on the kept
    planes, from the definition: t = (p - lo) / h in base spacings, the last
    kept interval starting at or below t, f = (t - k_c) / (k_(c+1) - k_c)."""
    dim = coords.shape[1]
    cells, fracs = [], []
    for d in range(dim):
        t = (coords[:, d] - lo[d]) * (1.0 / h[d])
        kp = kept[d].astype(np.float64)
        c = np.searchsorted(kp[:-1], t, side="right") - 1
        c = np.clip(c, 0, kp.size - 2)
        f = (t - kp[c]) / (kp[c + 1] - kp[c])
        u = np.where(f > 0, np.where(f >= 1.0, 32768, np.rint(f * 32768.0)), 0).astype(np.int64)
        cells.append(c)
        fracs.append(u)
    return cells, fracs


def _numpy_kept(plan, g_op):
    """Marked planes per axis from the uniform plan's geometry (numpy)."""
    g = plan.grid
    coords = plan._coords
    dim = g.dim
    full = [np.arange(g.n[d]) for d in range(dim)]
    cells, fracs = _numpy_cells(coords, g.lo, g.h, full)
    kept = []
    for d in range(dim):
        if g_op == "nearest":
            marks = cells[d] + (fracs[d] >= 16384)
        else:
            marks = np.concatenate([cells[d], cells[d] + 1])
        k = np.unique(marks)
        kept.append(k if k.size >= 2 else np.arange(g.n[d]))
    return kept


def _plan(coords, cells, n, **kw):
    p = oracle.Plan(coords, cells, n, **kw)
    p._coords = np.ascontiguousarray(coords, dtype=np.float64)
    return p


def _two_blocks():
    """Two blocks of mesh side by side with an empty band between them."""
    c, e = synth.mesh2d_jittered(nside=24, seed=5)
    c2 = c.copy()
    c2[:, 0] += 1.6
    coords = np.concatenate([c, c2])
    cells = np.concatenate([e, e + c.shape[0]])
    return coords, cells


CASES = {
    "fine2d": lambda: (*synth.mesh2d_jittered(nside=30, seed=3), (200, 190)),
    "blocks": lambda: (*_two_blocks(), (120, 60)),
    "annulus": lambda: (*synth.mesh3d_annulus(nr=5, nth=20, nz=6, seed=4), (40, 38, 30)),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    coords, cells, n = CASES[request.param]()
    return request.param, coords, cells, n, _plan(coords, cells, n)


@pytest.mark.parametrize("g_op", ["multilinear", "nearest"])
def test_kept_planes_match_numpy(case, g_op):
    name, coords, cells, n, plan = case
    kept = oracle.grid_coarsen(plan, g_op)
    want = _numpy_kept(plan, g_op)
    for d in range(plan.dim):
        assert np.array_equal(kept[d], want[d]), (name, d)
    if name in ("fine2d", "blocks"):
        assert any(kept[d].size < n[d] for d in range(plan.dim))


@pytest.mark.parametrize("g_op", ["multilinear", "nearest"])
def test_coarse_grid_points_are_base_points(case, g_op):
    """Location, vertex ids and weights of every kept node equal the base
    grid's at the same point."""
    name, coords, cells, n, plan = case
    kept = oracle.grid_coarsen(plan, g_op)
    cp = _plan(coords, cells, n, keep=kept)
    base_idx = np.ix_(*[k for k in kept[::-1]])  # (z,) y, x order of the flat index
    shape = tuple(n[::-1])
    sel = np.arange(plan.n_g).reshape(shape)[base_idx].ravel()
    assert np.array_equal(cp.owner, plan.owner[sel])
    assert np.array_equal(cp.vid, plan.vid[:, sel])
    assert np.array_equal(cp.lam, plan.lam[:, sel])
    assert np.array_equal(cp.lam64, plan.lam64[:, sel])
    # the grid's coordinates along each axis are the base grid's kept ones
    for d in range(plan.dim):
        assert np.array_equal(cp.grid.coords_of_axis(d), plan.grid.lo[d] + kept[d] * plan.grid.h[d])


@pytest.mark.parametrize("g_op", ["multilinear", "nearest"])
def test_vertex_tables_on_kept_planes(case, g_op):
    name, coords, cells, n, plan = case
    kept = oracle.grid_coarsen(plan, g_op)
    cp = _plan(coords, cells, n, keep=kept)
    cl, fr = _numpy_cells(cp._coords, cp.grid.lo, cp.grid.h, kept)
    strides = [1, kept[0].size, kept[0].size * (kept[1].size if cp.dim > 1 else 1)]
    cell = sum(cl[d] * strides[d] for d in range(cp.dim))
    assert np.array_equal(cp.cell.astype(np.int64), cell)
    for d in range(cp.dim):
        assert np.array_equal(cp.frac[d].astype(np.int64), fr[d])


def test_nearest_node_keeps_its_node(case):
    """With the nearest-node g, every vertex's nearest node on the coarsened
    grid is the same point as on the base grid (away from exact midplane
    ties of the 2^-15 local coordinates)."""
    name, coords, cells, n, plan = case
    kept = oracle.grid_coarsen(plan, "nearest")
    cp = _plan(coords, cells, n, keep=kept)
    full = [np.arange(n[d]) for d in range(plan.dim)]
    cb, fb = _numpy_cells(plan._coords, plan.grid.lo, plan.grid.h, full)
    cc, fc = _numpy_cells(cp._coords, cp.grid.lo, cp.grid.h, kept)
    same = np.ones(plan.n_v, bool)
    for d in range(plan.dim):
        nb = cb[d] + (fb[d] >= 16384)
        nc = kept[d][cc[d] + (fc[d] >= 16384)]
        same &= nb == nc
    assert same.mean() > 0.999


def test_keeping_every_plane_changes_nothing():
    c, e = synth.mesh2d_jittered(nside=40, seed=8)
    p0 = _plan(c, e, (57, 43))
    p1 = _plan(c, e, (57, 43), keep=[np.arange(57), np.arange(43)])
    for a in ("owner", "vid", "lam", "cell", "frac"):
        assert np.array_equal(getattr(p0, a), getattr(p1, a))
    x = synth.field_bumps_noise(c, seed=2)
    assert np.array_equal(oracle.compress(p0, x, eb=1e-4), oracle.compress(p1, x, eb=1e-4))


@pytest.mark.parametrize("g_op", ["multilinear", "nearest"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_bound_on_coarsened_grids(case, g_op, dtype):
    name, coords, cells, n, plan = case
    kept = oracle.grid_coarsen(plan, g_op)
    cp = _plan(coords, cells, n, keep=kept)
    x = (synth.field_bumps_noise(coords, seed=9) if coords.shape[1] == 2
         else synth.field_vortex(coords, seed=9)).astype(dtype)
    fop = "cluster" if g_op == "nearest" else "barycentric"
    for eb in (1e-2, 1e-4):
        s1 = oracle.compress(cp, x, eb=eb, g_op=g_op, f_op=fop)
        y = oracle.decompress(cp, s1)
        f = oracle.field_params(x, eb=eb)
        assert np.abs(y.astype(np.float64) - x.astype(np.float64)).max() <= f["tau2"]


def test_coarsening_shrinks_fine_grids():
    coords, cells, n = CASES["fine2d"]()
    plan = _plan(coords, cells, n)
    x = synth.field_bumps_noise(coords, seed=1)
    for g_op, fop in (("multilinear", "barycentric"), ("nearest", "cluster")):
        cp = _plan(coords, cells, n, keep=oracle.grid_coarsen(plan, g_op))
        a = oracle.compress(plan, x, eb=1e-3, g_op=g_op, f_op=fop)
        b = oracle.compress(cp, x, eb=1e-3, g_op=g_op, f_op=fop)
        assert b.size < a.size


def test_gap_between_blocks_closed_form():
    """The grid lines strictly inside the empty band between the blocks
    carry no node of any vertex's cell."""
    coords, cells = _two_blocks()
    plan = _plan(coords, cells, (120, 60))
    kept = oracle.grid_coarsen(plan, "multilinear")
    g = plan.grid
    xs = g.lo[0] + np.arange(120) * g.h[0]
    right_of_left = coords[: coords.shape[0] // 2, 0].max()
    left_of_right = coords[coords.shape[0] // 2:, 0].min()
    inner = np.nonzero((xs > right_of_left + g.h[0]) & (xs < left_of_right - g.h[0]))[0]
    assert inner.size > 10 and not np.isin(inner, kept[0]).any()
    assert kept[1].size == 60


def test_domain_wider_than_mesh():
    """User corners outside the mesh: the planes beyond the vertices go."""
    c, e = synth.mesh2d_jittered(nside=20, seed=6)
    lo, hi = c.min(axis=0) - 1.0, c.max(axis=0) + 1.0
    plan = _plan(c, e, (80, 80), lo=lo, hi=hi)
    kept = oracle.grid_coarsen(plan, "nearest")
    g = plan.grid
    for d in range(2):
        pts = g.lo[d] + kept[d] * g.h[d]
        assert pts.min() >= c[:, d].min() - g.h[d] and pts.max() <= c[:, d].max() + g.h[d]
        assert kept[d].size < 80


def test_errors():
    c, e = synth.mesh2d_jittered(nside=20, seed=6)
    plan = _plan(c, e, (30, 30))
    kept = oracle.grid_coarsen(plan, "nearest")
    cp = _plan(c, e, (30, 30), keep=kept)
    with pytest.raises(ValueError):
        oracle.grid_coarsen(cp, "nearest")
    with pytest.raises(oracle.OracleError) as err:
        oracle.grid_coarsen(plan, 2)
    assert err.value.status == 1
    for bad in ([np.array([3]), np.arange(30)], [np.array([5, 4, 9]), np.arange(30)],
                [np.array([0, 30]), np.arange(30)]):
        with pytest.raises(ValueError):
            oracle.Plan(c, e, (30, 30), keep=bad)
