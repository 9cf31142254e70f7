"""The allocation-free decompression entry point (mcc_decompress_static).

It serves callers that cannot allocate device memory: its scratch is a fixed
array inside the library. Its output must equal that of mcc_decompress (the
existing entry point, whose parity with the CPU oracle the other GPU tests
establish), bit for bit, on two calls in a row (the second call reuses the
array the first one left behind). This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _compress(gp, x, **kw):
    import gpu_helpers as G
    return G.compress(gp, x, **kw)


def test_static_decompress_matches_workspace_decompress_twice():
    import torch
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    coords, cells = synth.mesh2d_jittered(nside=80, seed=71)
    gp = G.plan(coords, cells, (61, 53))
    for seed, kw, dt in ((72, dict(eb=1e-4), np.float64), (73, dict(eb=1e-6, grid_fraction=0.3), np.float64),
                         (74, dict(eb=1e-3), np.float32)):
        x = synth.field_bumps_noise(coords, seed=seed).astype(dt)
        s = _compress(gp, x, **kw)
        ref = G.decompress(gp, s, dt)
        st = torch.from_numpy(s).cuda()
        tdt = torch.float64 if dt == np.float64 else torch.float32
        for _ in range(2):
            y = torch.full((gp.n_vertices,), float("nan"), dtype=tdt, device="cuda")
            mcc.decompress_static(gp, st, s.size, y)
            assert np.array_equal(y.cpu().numpy().view(np.uint8), ref.view(np.uint8))


def test_static_decompress_rejects_plans_beyond_the_scratch():
    import torch
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    coords, cells = synth.mesh2d_jittered(nside=20, seed=75)
    gp = G.plan(coords, cells, (3000, 3000))  # decompression workspace > 32 MiB
    _, dws = mcc.workspace_size(gp, mcc.params_default())
    assert dws > mcc.static_scratch_bytes()
    x = synth.field_sincos(coords, seed=76)
    s = _compress(gp, x, eb=1e-3)
    y = torch.empty(gp.n_vertices, dtype=torch.float64, device="cuda")
    with pytest.raises(mcc.MCCError) as err:
        mcc.decompress_static(gp, torch.from_numpy(s).cuda(), s.size, y)
    assert err.value.status == mcc.CAPACITY
