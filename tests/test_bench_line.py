"""The benchmark's output contract on the CPU: the headline (last stdout line)
is one JSON object under 2 KB with the metric, the dominant kernel's roofline
and the whole step's, and the CPU baseline; the oracle's all-core timing
runs one spawned process per core on the workload's sample."""
import json

import pytest


def _stub_prof(steps):
    # name: (total ms over `steps` replays, launches)
    per = {"k_reduce": 0.015, "k_prequant": 0.02, "k_grid_codes": 0.25, "k_grid3d": 0.03, "k_node": 0.16,
           "k_codebook": 0.033, "k_group_len": 0.03, "k_pack": 0.04, "k_dec_prep": 0.012,
           "k_dec_syms": 0.12, "k_scan_rows": 0.03, "k_predict": 0.002, "k_recon": 0.16}
    prof = {k: (v * steps, steps) for k, v in per.items()}
    prof["k_scan_axis"] = (0.035 * 2 * steps, 2 * steps)  # two axes in 3D
    return prof


def test_headline_is_compact_json_with_rooflines():
    import bench
    steps = 20
    n_v, n_g = 7_995_392, 256 ** 3
    alg = bench.algorithmic_bytes(3, n_v, n_g, 8, 10_000_000)
    prof = _stub_prof(steps)
    cpu = {"value": 0.2, "unit": "GB/s", "cores": 16, "kind": "oracle", "sample": "s" * 200,
           "single_core": {"value": 0.016, "cores": 1, "ms_per_step": 280.0}, "nproc": 16}
    e2e = {"value": 20.0, "unit": "GB/s", "h2d_bytes_per_step": 74_000_000,
           "d2h_bytes_per_step": 74_000_000}
    config = {"workload": "3d-annulus", "n_vertices": n_v, "grid": [256, 256, 256]}
    line = bench.build_headline(world=1, steps=steps, warmup=5, ms=1.0, nbytes=n_v * 8,
                                config=config, prof=prof, alg=alg, peaks={"hbm_gbs": 6780.0},
                                cpu=cpu, e2e=e2e, clocks={"sm_mhz": 2070.0, "reasons": []},
                                traffic=lambda k: 123)
    s = bench.headline_json(line)
    assert len(s) <= bench.HEADLINE_MAX_BYTES
    d = json.loads(s)
    assert d["value"] == pytest.approx(n_v * 8 / 1e-3 / 1e9, rel=1e-4)
    r = d["roofline"]
    assert r["kernel"] == "k_grid_codes" and r["traffic"] == 123 and r["bound"] == "hbm"
    assert r["frac"] == pytest.approx(alg["k_grid_codes"] / 0.25e-3 / 1e9 / 6780.0, rel=1e-4)
    # the whole step: every kernel's bytes times its launches, over the step time
    sb = sum(alg[k] * (2 if k == "k_scan_axis" else 1) for k in prof)
    assert r["step_alg_bytes"] == pytest.approx(sb, rel=1e-4)
    assert r["step_frac"] == pytest.approx(sb / 1e-3 / 1e9 / 6780.0, rel=1e-4)
    assert d["gpu_launches"] == 15 * steps
    for key in ("metric", "unit", "n_gpus", "ms_per_step", "cpu_baseline", "e2e", "clocks"):
        assert key in d
    assert d["cpu_baseline"]["cores"] == 16


def test_headline_drops_the_kernel_table_before_overflowing():
    import bench
    prof = {f"k_kernel_with_a_long_name_{i}": (1.0, 1) for i in range(60)}
    line = bench.build_headline(world=1, steps=1, warmup=3, ms=1.0, nbytes=8, config={},
                                prof=prof, alg={}, peaks={}, cpu=None, e2e=None, clocks={})
    s = bench.headline_json(line)
    d = json.loads(s)
    assert len(s) <= bench.HEADLINE_MAX_BYTES
    kept = list(d.get("kernels_us", {}))
    assert 0 < len(kept) < 60 and kept == list(line["kernels_us"])[:len(kept)]  # a prefix
    assert d["roofline"]["peak_source"].startswith("fallback")


def test_annulus_sample_keeps_the_full_grid_spacing():
    import bench
    coords, cells, n, x, desc = bench.cpu_sample("c3")
    assert n[:2] == (256, 256) and n[2] == 18
    assert coords.shape[0] == 64 * 512 * bench.SLAB_LAYERS and cells.shape[1] == 4
    hz = (coords[:, 2].max() - coords[:, 2].min()) / (n[2] - 1)
    assert hz == pytest.approx(2.0 / 255.0, rel=0.02)
    assert x.dtype.name == "float64" and "17 of 244" in desc


def test_oracle_on_all_cores_with_spawned_processes():
    import bench
    gbs, walls, procs, nbytes, size, _ = bench.oracle_all_cores("c1", 1e-4, steps=1, warmup=0,
                                                                procs=2)
    assert procs == 2 and len(walls) == 1 and gbs > 0 and 0 < size < nbytes
