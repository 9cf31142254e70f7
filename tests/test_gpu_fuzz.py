"""GPU against the oracle over the seeded random configurations of
test_oracle_properties (meshes, fields, value types, bounds, splits, radii,
chunk sizes, length limits, operators, loops, the zero-run stage): the same stream byte for
byte and the same decoded values, or the same error; the 1D coder likewise."""
import numpy as np
import pytest
import torch

import oracle
from test_oracle_properties import _draw

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(40))
def test_random_configuration_parity(seed):
    import gpu_helpers as G
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, kw = _draw(seed)
    op = oracle.Plan(c, e, n)
    gp = G.plan(c, e, n)
    try:
        want = oracle.compress(op, x, **kw)
    except oracle.OracleError as err:
        with pytest.raises(mcc.MCCError) as gerr:
            G.compress(gp, x, **kw)
        assert gerr.value.status == err.status
        return
    got = G.compress(gp, x, **kw)
    assert np.array_equal(got, want)
    assert np.array_equal(G.decompress(gp, got, x.dtype), oracle.decompress(op, want))


@pytest.mark.parametrize("seed", range(20))
def test_random_1d_parity(seed):
    import paper_2501_06910_gb300 as mcc
    c, e, n, x, kw = _draw(1000 + seed)
    kw1 = {k: v for k, v in kw.items() if k not in ("f_op", "g_op", "open_loop", "grid_fraction")}
    prm = mcc.params_default(dtype=mcc.F64 if x.dtype == np.float64 else mcc.F32, **kw1)
    try:
        want = oracle.compress_1d(x, **kw1)
    except oracle.OracleError as err:
        with pytest.raises(mcc.MCCError) as gerr:
            mcc.compress_1d(torch.from_numpy(x).cuda(), prm)
        assert gerr.value.status == err.status
        return
    got = mcc.compress_1d(torch.from_numpy(x).cuda(), prm).cpu().numpy()
    assert np.array_equal(got, want)
    y = torch.empty(x.size, dtype=torch.float64 if x.dtype == np.float64 else torch.float32, device="cuda")
    mcc.decompress_1d(torch.from_numpy(want).cuda(), y)
    assert np.array_equal(y.cpu().numpy(), oracle.decompress_1d(want, x.size))
