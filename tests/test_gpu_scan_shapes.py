"""The decoder's prefix passes over grid shapes that take each of its paths:
the fused row and y pass per z-plane with rows of up to 256, 512 and 1024
codes and row counts that are not a multiple of its batch, and rows whose
length is not a multiple of 4 (separate row and y passes); streams and
decoded values bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [(40, 41, 19), (256, 7, 5), (300, 9, 6), (600, 5, 4), (1024, 3, 3),
                               (1028, 3, 3), (61, 17, 9), (13, 12, 9)])
def test_decoder_prefix_passes_bit_exact(n):
    import gpu_helpers as G
    c, e = synth.mesh3d_annulus(nr=6, nth=24, nz=8, seed=57)
    x = synth.field_vortex(c, seed=58)
    op = oracle.Plan(c, e, n)
    gp = G.plan(c, e, n)
    for eb in (1e-4, 1e-2):
        want = oracle.compress(op, x, eb=eb)
        got = G.compress(gp, x, eb=eb)
        assert np.array_equal(got, want), eb
        assert np.array_equal(G.decompress(gp, got, np.float64), oracle.decompress(op, want)), eb
