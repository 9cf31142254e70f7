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


def test_algorithmic_bytes_model():
    """The per-launch byte model: each kernel's streamed inputs and outputs
    once (gathers as cache hits), the second stream's launches split per
    component, the fused 3D plane scan one read and one write of q1."""
    import bench
    n_v, n_g, cb, c1 = 7_995_392, 256 ** 3, 10_600_136, 5_000_000
    alg = bench.algorithmic_bytes(3, n_v, n_g, 8, cb, c1,
                                  launched=("k_group_len_grid", "k_dec_syms_res"))
    assert alg["k_node"] == (4 + 6 + 4 + 2) * n_v       # cell, local coordinates, Q in; symbols out
    assert alg["k_recon"] == (4 + 6 + 4 + 8) * n_v      # cell, local coordinates, q2 in; values out
    assert alg["k_grid_codes"] == 28 * n_g               # 24 B of plan records in; q1 out
    assert alg["k_grid3d_grid"] == alg["k_grid3d"] == 6 * n_g
    assert alg["k_scan_xy"] == alg["k_scan_axis"] == 8 * n_g
    assert alg["k_group_len"] == 2 * n_v and alg["k_group_len_grid"] == 2 * n_g
    assert alg["k_dec_syms"] == c1 + 4 * n_g and alg["k_dec_syms_res"] == (cb - c1) + 4 * n_v
    # 2D: two local coordinates
    alg2 = bench.algorithmic_bytes(2, 1000, 2000, 8, 500)
    assert alg2["k_node"] == (4 + 4 + 4 + 2) * 1000 and alg2["k_recon"] == (4 + 4 + 4 + 8) * 1000
    # one step: every kernel's bytes times its launches per step
    per = {"k_node": {"launches_per_step": 1.0}, "k_scan_axis": {"launches_per_step": 2.0}}
    assert bench.step_bytes(alg, per) == alg["k_node"] + 2 * alg["k_scan_axis"]
