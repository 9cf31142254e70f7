"""GPU Grid_Init (Algorithm 1) against the oracle: the same points per axis
and corners (the percentile is an exact selection on both sides), on 2D and
3D meshes, several percentiles and node limits, the 2M-vertex benchmark mesh;
a plan built from the result compresses bit-exactly; argument errors."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _mesh(name):
    if name == "jit2d":
        return synth.mesh2d_jittered(nside=40, seed=3)
    if name == "graded2d":
        return synth.mesh2d_graded(n=100_000, seed=4)
    if name == "annulus":
        return synth.mesh3d_annulus(nr=12, nth=64, nz=20, seed=54)
    raise KeyError(name)


def _dev(c, e):
    return torch.from_numpy(np.ascontiguousarray(c)).cuda(), torch.from_numpy(np.ascontiguousarray(e)).cuda()


@pytest.mark.parametrize("name", ["jit2d", "graded2d", "annulus"])
@pytest.mark.parametrize("k,delta,gmax", [(1, 1.0, 4096), (10, 2.5, 4096), (37.5, 1.0, 200),
                                          (99, 1.0, 32767), (5, 0.5, 30)])
def test_grid_init_matches_oracle(name, k, delta, gmax):
    import paper_2501_06910_gb300 as mcc
    c, e = _mesh(name)
    n, lo, hi = mcc.grid_init(*_dev(c, e), k, delta, gmax)
    want = oracle.grid_init(c, e, k, delta, gmax)
    assert n == want[0]
    assert lo == want[1] and hi == want[2]


@pytest.mark.slow
def test_grid_init_benchmark_mesh_and_plan():
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e = synth.mesh2d_graded()
    cd, ed = _dev(c, e)
    n, lo, hi = mcc.grid_init(cd, ed, 30.0, 1.0, 4096)
    want = oracle.grid_init(c, e, 30.0, 1.0, 4096)
    assert (n, lo, hi) == want[:3]
    # a plan on that grid: streams bit-exact against the oracle's plan
    op = oracle.Plan(c, e, n, lo, hi)
    gp = G.plan(c, e, n, lo, hi)
    x = synth.field_bumps_noise(c)
    for kw in (dict(eb=1e-4), dict(eb=1e-4, f_op="cluster", g_op="nearest")):
        want_s = oracle.compress(op, x, **kw)
        got_s = G.compress(gp, x, **kw)
        assert np.array_equal(got_s, want_s), kw


def test_grid_init_errors():
    import paper_2501_06910_gb300 as mcc
    c, e = _mesh("jit2d")
    cd, ed = _dev(c, e)
    for k, delta, gmax in ((0.0, 1.0, 100), (101.0, 1.0, 100), (10.0, 0.0, 100), (10.0, 1.0, 1),
                           (10.0, 1.0, 40000)):
        with pytest.raises(mcc.MCCError) as err:
            mcc.grid_init(cd, ed, k, delta, gmax)
        assert err.value.status == mcc.INVALID_ARG
    with pytest.raises(mcc.MCCError) as err:
        mcc.grid_init(cd, ed, 10.0, 1.0, 2)
    assert err.value.status == mcc.RANGE
    bad = e.copy()
    bad[3, 1] = c.shape[0]
    with pytest.raises(mcc.MCCError) as err:
        mcc.grid_init(cd, torch.from_numpy(bad).cuda(), 10.0, 1.0, 100)
    assert err.value.status == mcc.INVALID_ARG
