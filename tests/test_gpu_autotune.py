"""The autotuner on the GPU: the launch configuration it picks is one of its
candidates and is set on the plan; no configuration changes a stream or a
decoded value (the tuner checks that itself, this test checks it again
against the default configuration); invalid configurations are refused."""
import pytest
import torch

import paper_2501_06910_gb300 as mcc
import synth
from paper_2501_06910_gb300 import autotune

pytestmark = pytest.mark.gpu


def _round_trip(plan, x, prm):
    wsc = plan.workspace(prm, "compress")
    wsd = plan.workspace(prm, "decompress")
    out = torch.zeros(mcc.compress_bound(plan, prm), dtype=torch.uint8, device=x.device)
    size = mcc.compress(plan, x, prm, wsc, out)
    y = torch.empty_like(x)
    mcc.decompress(plan, out, size, y, wsd)
    return out[:size].clone(), y


@pytest.mark.parametrize("dim", [2, 3])
def test_tuned_launch_keeps_the_result(dim):
    if dim == 2:
        coords, cells = synth.mesh2d_jittered(nside=90, seed=5)
        x = synth.field_sincos(coords, seed=6)
        n = (100, 90)
    else:
        coords, cells = synth.mesh3d_annulus(nr=10, nth=48, nz=12, seed=4)
        x = synth.field_vortex(coords, seed=7)
        n = (40, 40, 24)
    dev = torch.device("cuda", 0)
    plan = mcc.plan_create(torch.from_numpy(coords).to(dev), torch.from_numpy(cells).to(dev), n)
    xd = torch.from_numpy(x).to(dev)
    assert mcc.get_tuning(plan) == (mcc.TILE_64x16, 0, 0)
    base = dict(dtype=mcc.F64, eb=1e-3, grid_fraction=0.5)
    ref = _round_trip(plan, xd, mcc.params_default(**base))
    params, table = autotune.tune(plan, xd, base, candidates=[(512, 128)], reps=2)
    rows = autotune.tune.launch_table
    assert len(rows) == (12 if dim == 2 else 4)
    chosen = mcc.get_tuning(plan)
    assert chosen[:2] in {(r[0], r[1]) for r in rows} and chosen[2] == 0
    assert min(rows, key=lambda r: r[2])[:2] == chosen[:2]
    got = _round_trip(plan, xd, mcc.params_default(**params))
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
    for bad in ((3, 8, 0), (-1, 8, 0), (0, 1, 0), (0, -1, 0), (0, 33, 0), (0, 8, -1), (0, 8, 65)):
        with pytest.raises(mcc.MCCError) as e:
            mcc.set_tuning(plan, *bad)
        assert e.value.status == mcc.INVALID_ARG
    assert mcc.get_tuning(plan) == chosen
    plan.close()


def test_tuned_batch_chain_keeps_the_result():
    """tune_batch times every fields-per-chain candidate on a batch of fields
    with uneven bounds; each gives the same streams and values (it checks),
    and the fastest is set."""
    coords, cells = synth.mesh2d_jittered(nside=70, seed=9)
    dev = torch.device("cuda", 0)
    plan = mcc.plan_create(torch.from_numpy(coords).to(dev), torch.from_numpy(cells).to(dev),
                           (64, 64))
    xs = [torch.from_numpy(synth.field_sincos(coords, seed=20 + k)).to(dev) for k in range(6)]
    prms = [mcc.params_default(dtype=mcc.F64, eb=eb) for eb in (1e-5, 1e-4, 1e-3) * 2]
    rows = autotune.tune_batch(plan, xs, prms, chains=(0, 1, 2, 6), reps=2)
    assert [r[0] for r in rows] == [0, 1, 2, 6]
    assert mcc.get_tuning(plan)[2] == min(rows, key=lambda r: r[1])[0]
    plan.close()
