"""The device-side field generators reproduce the numpy ones (run here on the
CPU): the lattice hash bit for bit, the fields to rounding."""
import numpy as np
import torch

import synth
from synth import torchgen


def test_hash_bit_exact():
    rng = np.random.default_rng(0)
    a = rng.integers(-(1 << 40), 1 << 40, 5000)
    b = rng.integers(-1000, 1000, 5000)
    want = synth._hash_u01(a, b, np.int64(7042))
    got = torchgen.hash_u01(torch.from_numpy(a), torch.from_numpy(b), 7042).numpy()
    assert np.array_equal(got, want)


def test_fields_match_numpy():
    c, _ = synth.mesh3d_annulus(nr=5, nth=16, nz=6, seed=3)
    ct = torch.from_numpy(c)
    assert np.allclose(torchgen.field_vortex(ct, seed=4).numpy(), synth.field_vortex(c, seed=4),
                       rtol=0, atol=1e-12)
    c2, _ = synth.mesh2d_jittered(nside=20, seed=5)
    want = [v for _, _, v in synth.fields_advected(c2, nvars=2, nsteps=3, seed=9)]
    got = [v.numpy() for _, _, v in torchgen.fields_advected(torch.from_numpy(c2), nvars=2,
                                                              nsteps=3, seed=9)]
    for a, b in zip(got, want):
        assert np.allclose(a, b, rtol=0, atol=1e-12)
