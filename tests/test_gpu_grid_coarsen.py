"""GPU parity of Grid_Coarsen (Algorithm 2) and of plans on kept planes:
the kept planes equal the oracle's for both gs on a fine 2D grid, two blocks
of mesh with an empty band between them and a 3D annulus; the plan tables on
the kept planes equal the oracle's element by element; streams on those
plans are bit-exact with the oracle's and decode to the oracle's values;
errors."""
import numpy as np
import pytest

import oracle
from test_oracle_grid_coarsen import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    import gpu_helpers as G
    coords, cells, n = CASES[request.param]()
    return request.param, coords, cells, n, oracle.Plan(coords, cells, n), G.plan(coords, cells, n)


@pytest.mark.parametrize("g_op", ["multilinear", "nearest"])
def test_kept_planes_and_tables(case, g_op):
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    name, coords, cells, n, op, gp = case
    want = oracle.grid_coarsen(op, g_op)
    got = mcc.grid_coarsen(gp, g_op)
    assert len(got) == len(want)
    for d in range(len(want)):
        assert np.array_equal(got[d], want[d]), (name, d)
    ok = oracle.Plan(coords, cells, n, keep=want)
    gk = G.plan(coords, cells, n, keep=got)
    assert gk.n == ok.grid.n[:ok.dim] and gk.n_grid == ok.n_g
    t = G.tables(gk)
    assert np.array_equal(t["vid"], ok.vid)
    assert np.array_equal(t["lam"], ok.lam)
    assert np.array_equal(t["cell"], ok.cell)
    assert np.array_equal(t["frac"], ok.frac)


@pytest.mark.parametrize("g_op", ["multilinear", "nearest"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_streams_on_kept_planes(case, g_op, dtype):
    import gpu_helpers as G
    import synth
    name, coords, cells, n, op, gp = case
    keep = oracle.grid_coarsen(op, g_op)
    ok, gk = oracle.Plan(coords, cells, n, keep=keep), G.plan(coords, cells, n, keep=keep)
    x = (synth.field_bumps_noise(coords, seed=9) if coords.shape[1] == 2
         else synth.field_vortex(coords, seed=9)).astype(dtype)
    fop = "cluster" if g_op == "nearest" else "barycentric"
    for eb in (1e-2, 1e-4):
        want = oracle.compress(ok, x, eb=eb, g_op=g_op, f_op=fop)
        got = G.compress(gk, x, eb=eb, g_op=g_op, f_op=fop)
        assert np.array_equal(got, want)
        assert np.array_equal(G.decompress(gk, got, dtype), oracle.decompress(ok, want))


def test_errors(case):
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    name, coords, cells, n, op, gp = case
    keep = mcc.grid_coarsen(gp, "nearest")
    gk = G.plan(coords, cells, n, keep=keep)
    with pytest.raises(mcc.MCCError) as err:
        mcc.grid_coarsen(gk, "nearest")
    assert err.value.status == mcc.INVALID_ARG
    with pytest.raises(mcc.MCCError) as err:
        mcc.grid_coarsen(gp, 2)
    assert err.value.status == mcc.INVALID_ARG
    bad = [k.copy() for k in keep]
    bad[0] = bad[0][::-1].copy()
    with pytest.raises(mcc.MCCError) as err:
        G.plan(coords, cells, n, keep=bad)
    assert err.value.status == mcc.INVALID_ARG
