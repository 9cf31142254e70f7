"""Pins of the oracle's Grid_Init (Algorithm 1): the spacing per axis is the
bottom k-th percentile (nearest rank) of the cells' edge extents, checked
against numpy's inverted-CDF percentile of independently enumerated edges;
k grows by delta while the axis would need gmax or more intervals, carrying
over to the next axis; error cases."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


def _extents(coords, cells, d):
    pairs = list(itertools.combinations(range(cells.shape[1]), 2))
    return np.concatenate([np.abs(coords[cells[:, a], d] - coords[cells[:, b], d]) for a, b in pairs])


def _numpy_grid_init(coords, cells, k, delta, gmax):
    dim = coords.shape[1]
    n, lo, hi, gs_all = [], [], [], []
    for d in range(dim):
        ext = _extents(coords, cells, d)
        mn, mx = coords[:, d].min(), coords[:, d].max()
        while True:
            gs = np.percentile(ext, k, method="inverted_cdf")
            gn = (mx - mn) / gs if gs > 0 else math.inf
            if gn < gmax:
                break
            assert k < 100
            k = min(100.0, k + delta)
        n.append(math.ceil(gn) + 1); lo.append(mn); hi.append(mx); gs_all.append(gs)
    return tuple(n), tuple(lo), tuple(hi), tuple(gs_all)


@pytest.mark.parametrize("mesh", ["jit2d", "graded2d", "annulus"])
@pytest.mark.parametrize("k,gmax", [(1, 4096), (10, 4096), (37.5, 200), (99, 32767), (5, 30)])
def test_grid_init_matches_numpy(mesh, k, gmax):
    if mesh == "jit2d":
        c, e = synth.mesh2d_jittered(nside=40, seed=3)
    elif mesh == "graded2d":
        c, e = synth.mesh2d_graded(n=20_000, seed=4)
    else:
        c, e = synth.mesh3d_annulus(nr=6, nth=32, nz=10, seed=5)
    got = oracle.grid_init(c, e, k, 2.5, gmax)
    want = _numpy_grid_init(c, e, k, 2.5, gmax)
    assert got[0] == want[0]
    assert got[1:] == want[1:]
    for d, nd in enumerate(got[0]):
        assert 2 <= nd <= gmax + 1
        # the spacing covers the axis: (n - 1) gs >= max - min
        assert (nd - 1) * got[3][d] >= got[2][d] - got[1][d]


def test_grid_init_structured_closed_form():
    """An unjittered lattice with spacing h along both axes: every edge extent
    is 0 or h, so any percentile above the share of zero extents is h and
    the grid reproduces the lattice."""
    c, e = synth.mesh2d_jittered(nside=33, jitter=0.0, seed=1)
    h = 1.0 / 32
    ext = _extents(c, e, 0)
    zero_share = np.mean(ext == 0) * 100
    n, lo, hi, gs = oracle.grid_init(c, e, zero_share + 1, 1.0, 4096)
    assert gs == pytest.approx((h, h), rel=1e-12)
    assert n == (33, 33) and lo == (0.0, 0.0) and hi == (1.0, 1.0)
    # below that share the percentile is 0 and k climbs to it
    n2, _, _, gs2 = oracle.grid_init(c, e, 1, 1.0, 4096)
    assert gs2[0] == pytest.approx(h, rel=1e-12) and n2 == (33, 33)


def test_grid_init_k_carries_over_axes():
    """Warp x (x -> x^3) so that x needs a large k to stay under gmax: the k
    found on x is kept for y (Algorithm 1 does not reset it), which gives a
    coarser y than restarting from the initial k."""
    c, e = synth.mesh2d_jittered(nside=40, seed=3)
    c = c.copy()
    c[:, 0] = c[:, 0] ** 3
    got = oracle.grid_init(c, e, 1, 1.0, 60)
    assert got == _numpy_grid_init(c, e, 1, 1.0, 60)
    reset = tuple(_numpy_grid_init(c[:, [d]], e, 1, 1.0, 60)[0][0] for d in range(2))
    assert got[0][0] == reset[0] and got[0][1] < reset[1]


def test_grid_init_errors():
    c, e = synth.mesh2d_jittered(nside=20, seed=2)
    for bad in (dict(k_pct=0.0), dict(k_pct=101.0), dict(delta_pct=0.0), dict(gmax=1),
                dict(gmax=40000)):
        kw = dict(k_pct=10.0, delta_pct=1.0, gmax=100)
        kw.update(bad)
        with pytest.raises(oracle.OracleError) as err:
            oracle.grid_init(c, e, **kw)
        assert err.value.status == 1
    with pytest.raises(oracle.OracleError) as err:  # even the longest edge gives >= gmax
        oracle.grid_init(c, e, 10.0, 1.0, 2)
    assert err.value.status == 4
    bad_cells = e.copy()
    bad_cells[3, 1] = c.shape[0]
    with pytest.raises(oracle.OracleError) as err:
        oracle.grid_init(c, bad_cells, 10.0, 1.0, 100)
    assert err.value.status == 1
