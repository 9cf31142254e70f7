"""The benchmark's host-side helpers on oracle streams (CPU): the component
sizes read from a stream header add up with the stream's other sections to
its total, and follow the header's word and value counts."""
import numpy as np

import oracle
import synth


def test_component_bytes_from_header():
    import bench
    c, e = synth.mesh2d_jittered(nside=50, seed=3)
    plan = oracle.Plan(c, e, (33, 31))
    x = synth.field_bumps_noise(c, seed=4)
    for kw in (dict(eb=1e-4), dict(eb=1e-2, zero_run=True), dict(eb=9e-4, eb_mode="abs")):
        for xx in (x, (x + 1.2e4).astype(np.float32)):
            s = oracle.compress(plan, xx, **kw)
            g, r = bench.component_bytes(s[:208])
            u64 = lambda o: int(s[o:o + 8].view(np.uint64)[0])
            vsz = xx.dtype.itemsize
            assert g == 4 * (u64(168) + u64(144))
            assert r == 4 * (u64(176) + u64(152)) + vsz * u64(160)
            assert 0 < g + r < s.size
            # what is left is the header, code lengths, group and lane tables
            # (and alignment): at most a few bytes per group plus 2 KB
            ng = -(-plan.n_g // (32 * 128)) + -(-plan.n_v // (32 * 128))
            assert s.size - (g + r) <= 384 + 4 * 512 + ng * 64 + 64
