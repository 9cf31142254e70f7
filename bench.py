#!/usr/bin/env python
"""Throughput benchmark of the GB300 multi-component compressor.

Metric: compress + decompress GB/s of input values (n_v x sizeof(value) bytes
per field) at relative bound 1e-4 (grid / residual split 0.5), together with
the compression ratio, on the 2D graded workload: 2,000,000 vertices with
density ~ exp(-4 |p - c|) around c = (0.3, 0.6), Delaunay triangulated, a
float64 field of 20 Gaussian bumps plus 6-octave value noise, on a 1024^2
grid (the stand-in for the paper's OpenFOAM airfoil-large, Table I). The
plan (mesh -> grid mapping) is built once and excluded, as in Sec. IV-A.

One step = mcc_compress + mcc_decompress of one device-resident field,
enqueued without host synchronisation and replayed as one CUDA graph. The L2
(129 MB) is flushed (256 MiB write, untimed) before every step; each step is
timed with CUDA events on the launch stream. Under torchrun every rank runs an
independent replica on its own GPU (the method has no exchange step); value is
the sum over ranks of the input bytes divided by the slowest rank's time.

``--impl reference`` times the CPU oracle (single core) on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "compress+decompress GB/s at eb=1e-4 rel"


def max_over_ranks(ms, world, device):
    """The step time of the job: the slowest rank's (all-reduce MAX over the
    process group when there is more than one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, nbytes, ms):
    """Whole-job throughput in GB/s: the bytes every rank processed in one
    step over the slowest rank's step time (replicas: weak scaling)."""
    return world * nbytes / (ms * 1e-3) / 1e9


def component_bytes(header):
    """Bytes of each component in a stream, from its header (uint8 array of
    at least 208 bytes): the grid component's bitstream and escape values,
    and the residual component's bitstream, escape values and raw values
    (the shared header, code lengths and group tables are left out). The
    paper's Fig. 5a/c compression ratios of the grid data and of the
    residuals divide the components' raw bytes by these."""
    u32 = lambda o: int(header[o:o + 4].view(np.uint32)[0])
    u64 = lambda o: int(header[o:o + 8].view(np.uint64)[0])
    vsz = 8 if u32(12) == 0 else 4
    grid = 4 * (u64(168) + u64(144))
    residual = 4 * (u64(176) + u64(152)) + vsz * u64(160)
    return grid, residual


def algorithmic_bytes(dim, n_v, n_g, vsz, w1, w2, cbytes):
    """HBM bytes each kernel must move at least once per launch (inputs read,
    outputs written). Gathers of the vertex codes and of the grid codes are
    counted as cache hits: both arrays fit in L2."""
    k1 = dim + 1
    return {
        "k_reduce": vsz * n_v,
        "k_prequant": (vsz + 4) * n_v,
        "k_grid2d": (4 * k1 + 2 * dim + 4 + 2) * n_g,
        "k_grid3d": (4 * k1 + 2 * dim + 4 + 2) * n_g,
        "k_node": (4 + 2 * dim + 4 + 2) * n_v,
        "k_codebook": 0,
        "k_group_len": 2 * (n_g + n_v),
        "k_scan": 0,
        "k_pack": 2 * (n_g + n_v) + cbytes,
        "k_runs": 2 * (n_g + n_v),
        "k_dec_prep": 0,
        "k_dec_syms": 4 * (w1 + w2) + 4 * (n_g + n_v),
        "k_scan_rows": 8 * n_g,
        "k_scan_axis": 12 * n_g,
        "k_recon": 4 * n_v + (4 + 2 * dim) * n_v + vsz * n_v,
    }


def load_workload(config):
    if config == "c2":
        coords, cells = synth.mesh2d_graded()
        return dict(name="2d-graded-2M-delaunay-grid1024^2", coords=coords, cells=cells,
                    x=synth.field_bumps_noise(coords), n=(1024, 1024))
    if config == "c1":
        coords, cells = synth.mesh2d_jittered()
        return dict(name="2d-jittered-20k-grid128^2", coords=coords, cells=cells,
                    x=synth.field_sincos(coords), n=(128, 128))
    if config == "c3":
        coords, cells = synth.mesh3d_annulus()
        return dict(name="3d-annulus-8M-tets39M-grid256^3", coords=coords, cells=cells,
                    x=synth.field_vortex(coords), n=(256, 256, 256))
    raise SystemExit(f"unknown config {config}")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms into a file."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                p = [v.strip() for v in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "window": "0.5 s pre-roll of the same step plus the timed region"}


def run_reference(args, wl):
    """The CPU oracle (single-threaded C) timed on the same workload."""
    import oracle
    if int(os.environ.get("RANK", "0")) != 0:
        return
    plan = oracle.Plan(wl["coords"], wl["cells"], wl["n"])
    x = wl["x"]
    kw = dict(eb=args.eb, grid_fraction=0.5)
    for _ in range(args.warmup):
        oracle.decompress(plan, oracle.compress(plan, x, **kw))
    times, size = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s = oracle.compress(plan, x, **kw)
        oracle.decompress(plan, s)
        times.append(time.perf_counter() - t0)
        size = s.size
    t = statistics.mean(times)
    gbs = x.nbytes / t / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "eb_rel": args.eb, "grid_fraction": 0.5,
                   "compression_ratio": x.nbytes / size},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"full workload, {args.steps} steps, plan excluded"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(wl, eb, budget_s=12.0):
    """The oracle's compress + decompress, repeated over a bounded time budget."""
    import oracle
    plan = oracle.Plan(wl["coords"], wl["cells"], wl["n"])
    x = wl["x"]
    reps, t_total = 0, 0.0
    while t_total < budget_s and reps < 200:
        t0 = time.perf_counter()
        s = oracle.compress(plan, x, eb=eb)
        oracle.decompress(plan, s)
        t_total += time.perf_counter() - t0
        reps += 1
    return {"value": x.nbytes * reps / t_total / 1e9, "unit": "GB/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{reps} x compress+decompress of the full {x.size}-vertex field, "
                      f"{t_total:.1f} s, plan excluded"}


def time_replays(fn, flush, steps, warmup, stream):
    """fn captured in one CUDA graph; mean ms of `steps` replays, each after an
    L2 flush and bracketed by events on the launch stream."""
    import torch
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    for _ in range(warmup):
        flush.fill_(1)
        g.replay()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(ev):
        flush.fill_(k & 0xFF)
        a.record(stream)
        g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    del g
    return ms


def learned_line(args, dev, flush, stream):
    """The learned residual predictor on the 3D annulus (8M vertices, 256^3
    grid): trained on the GPU on 16 seeds of vortex + noise fields, evaluated
    on 2 unseen seeds at rel 1e-4 against the plain predictor (auto choice
    per field)."""
    import torch
    import paper_2501_06910_gb300 as mcc
    from synth import torchgen
    t0 = time.perf_counter()
    coords, cells = synth.mesh3d_annulus()
    cd = torch.from_numpy(coords).to(dev)
    plan = mcc.plan_create(cd, torch.from_numpy(cells).to(dev), (256, 256, 256))
    del cells
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    eb = 1e-4
    base = dict(dtype=mcc.F64, eb=eb, grid_fraction=0.5)
    train = [torchgen.field_vortex(cd, seed=1000 + i) for i in range(16)]
    cfg = mcc.train_cfg_default()
    t0 = time.perf_counter()
    model, losses = mcc.model_train(plan, train, mcc.params_default(**base), cfg)
    t_train = time.perf_counter() - t0
    del train
    res = {"workload": "3d-annulus-8M-tets39M-grid256^3, vortex + 4-octave noise, FP64, "
                       "train seeds 1000-1015, eval seeds 2000-2001, rel 1e-4",
           "train_s": t_train, "train_steps": cfg.steps, "train_batch": cfg.batch,
           "samples_per_field": int(cfg.samples_per_field),
           "loss_first_100": float(np.mean(losses[:100])),
           "loss_last_100": float(np.mean(losses[-100:])), "setup_s": t_setup}
    n = coords.shape[0]
    out = {}
    for label, prm in (("plain", mcc.params_default(**base)),
                       ("learned", mcc.params_default(model=model, auto=True, **base))):
        cws, dws = mcc.workspace_size(plan, prm)
        wsc = torch.empty(cws, dtype=torch.uint8, device=dev)
        wsd = torch.empty(dws, dtype=torch.uint8, device=dev)
        cap = mcc.compress_bound(plan, prm)
        buf = torch.empty(cap, dtype=torch.uint8, device=dev)
        sizes, mss, chosen = [], [], []
        for seed in (2000, 2001):
            x = torchgen.field_vortex(cd, seed=seed)
            y = torch.empty_like(x)
            size = mcc.compress(plan, x, prm, wsc, buf)
            mcc.decompress(plan, buf, size, y, wsd)
            tau = eb * float(x.max() - x.min())
            if not float((y - x).abs().max()) <= tau:
                raise SystemExit(f"learned line: bound violated ({label})")
            chosen.append("learned" if int(buf[20].item()) & 2 else "plain")
            sizes.append(size)

            def step():
                mcc.compress(plan, x, prm, wsc, buf, sync=False)
                mcc.decompress(plan, buf, cap, y, wsd, sync=False)

            mss.append(time_replays(step, flush, max(5, args.steps // 4), args.warmup, stream))
        out[label] = {"compression_ratio": 2 * n * 8 / sum(sizes), "stream_bytes": sizes,
                      "ms_per_field": statistics.mean(mss),
                      "GBps": n * 8 / (statistics.mean(mss) * 1e-3) / 1e9,
                      "chosen": chosen}
        del wsc, wsd, buf
    res.update(out)
    res["ratio_gain"] = out["learned"]["compression_ratio"] / out["plain"]["compression_ratio"]
    # the 3D configuration itself: grid / residual split swept 0.2 .. 0.8,
    # FP64 and FP32 fields (seed 6), plain predictor, rel 1e-4, closed loop
    # (residual against the decompressed grid) and open loop (against the
    # grid before quantisation, Algorithm 3 as printed)
    sweep = []
    x64 = torchgen.field_vortex(cd, seed=6)
    cases = [(dt, xx, loop, frac) for dt, xx in (("f64", x64), ("f32", x64.float()))
             for loop in ("closed", "open") for frac in (0.2, 0.35, 0.5, 0.65, 0.8)]
    for dt, xx, loop, frac in cases:
        yy = torch.empty_like(xx)
        prm = mcc.params_default(dtype=mcc.F64 if dt == "f64" else mcc.F32, eb=eb,
                                 grid_fraction=frac, open_loop=loop == "open")
        cws, dws = mcc.workspace_size(plan, prm)
        wsc = torch.empty(cws, dtype=torch.uint8, device=dev)
        wsd = torch.empty(dws, dtype=torch.uint8, device=dev)
        cap = mcc.compress_bound(plan, prm)
        buf = torch.empty(cap, dtype=torch.uint8, device=dev)
        size = mcc.compress(plan, xx, prm, wsc, buf)
        mcc.decompress(plan, buf, size, yy, wsd)
        tau = eb * float(xx.max() - xx.min())
        err = float((yy.double() - xx.double()).abs().max())
        if not err <= tau:
            raise SystemExit(f"split sweep: bound violated ({dt}, {frac})")

        def sstep(prm=prm, xx=xx, yy=yy, wsc=wsc, wsd=wsd, buf=buf, cap=cap):
            mcc.compress(plan, xx, prm, wsc, buf, sync=False)
            mcc.decompress(plan, buf, cap, yy, wsd, sync=False)

        ms = time_replays(sstep, flush, 5, args.warmup, stream)
        nb = xx.numel() * xx.element_size()
        sweep.append({"dtype": dt, "loop": loop, "grid_fraction": frac,
                      "compression_ratio": nb / size,
                      "ms_per_field": ms, "GBps": nb / (ms * 1e-3) / 1e9,
                      "max_abs_err_over_tau": err / tau})
        del wsc, wsd, buf
    res["c3_split_sweep"] = sweep
    plan.close()
    return res


def grid_init_line(args, dev, flush, stream, wl, x):
    """Grid_Init (Algorithm 1) on the benchmark mesh: the grid from the
    bottom k-th percentile of the edge extents (gmax 4096, delta 1), for
    several k; ratio and compress+decompress rate at rel 1e-4 with the
    default operators and with the paper's (cluster-mean f, nearest-node g),
    on the uniform grid and on its planes kept by Grid_Coarsen (Algorithm 2,
    for the same g). The plans are built outside the timed region."""
    import torch
    import paper_2501_06910_gb300 as mcc
    cd = torch.from_numpy(wl["coords"]).to(dev)
    ed = torch.from_numpy(wl["cells"]).to(dev)
    rows = []
    for k in (30.0, 50.0, 70.0, 90.0, 99.0):
        t0 = time.perf_counter()
        n, lo, hi = mcc.grid_init(cd, ed, k, 1.0, 4096)
        t_init = time.perf_counter() - t0
        plan = mcc.plan_create(cd, ed, n, lo, hi)

        def measure(pl, prm, what):
            wsc = pl.workspace(prm, "compress")
            wsd = pl.workspace(prm, "decompress")
            cap = mcc.compress_bound(pl, prm)
            out = torch.empty(cap, dtype=torch.uint8, device=dev)
            y = torch.empty_like(x)
            size = mcc.compress(pl, x, prm, wsc, out)
            mcc.decompress(pl, out, size, y, wsd)
            tau = 1e-4 * (float(x.max()) - float(x.min()))
            if not float((y - x).abs().max()) <= tau:
                raise SystemExit(f"grid_init line: bound violated (k {k}, {what})")

            def gstep():
                mcc.compress(pl, x, prm, wsc, out, sync=False)
                mcc.decompress(pl, out, cap, y, wsd, sync=False)

            ms = time_replays(gstep, flush, 5, args.warmup, stream)
            g_bytes, r_bytes = component_bytes(out[:208].cpu().numpy())
            comp = {"grid_component_ratio": pl.n_grid * 8 / max(g_bytes, 1),
                    "residual_component_ratio": x.numel() * 8 / max(r_bytes, 1)}
            return x.numel() * 8 / size, ms, comp

        for fop, gop in (("barycentric", "multilinear"), ("cluster", "nearest")):
            prm = mcc.params_default(dtype=mcc.F64, eb=1e-4, grid_fraction=0.5, f_op=fop, g_op=gop)
            ratio, ms, comp = measure(plan, prm, f"{fop}, {gop}")
            row = {"k_pct": k, "grid": list(n), "grid_init_s": t_init, "f": fop, "g": gop,
                   "compression_ratio": ratio, "ms_per_step": ms,
                   "GBps": x.numel() * 8 / (ms * 1e-3) / 1e9, **comp}
            try:  # the same on the planes Grid_Coarsen keeps (recorded, never fatal here)
                keep = mcc.grid_coarsen(plan, gop)
                kplan = mcc.plan_create(cd, ed, n, lo, hi, keep=keep)
                ratio_k, ms_k, _ = measure(kplan, prm, f"{fop}, {gop}, coarsened")
                kplan.close()
                row.update({"coarsened_grid": [int(v.size) for v in keep],
                            "coarsened_compression_ratio": ratio_k, "coarsened_ms_per_step": ms_k,
                            "coarsened_GBps": x.numel() * 8 / (ms_k * 1e-3) / 1e9})
            except (Exception, SystemExit) as err:
                row["coarsened_error"] = str(err)
            rows.append(row)
        plan.close()
    return {"workload": wl["name"] + ", grid from Grid_Init (gmax 4096, delta 1)", "rows": rows}


def batched_c4_line(args, dev, flush, stream):
    """Many variables x timesteps on one mesh: 1M-vertex 2D mesh, 4 variables
    x 64 timesteps of advected Gaussian bumps (FP64), per-variable rel bounds
    1e-6, 1e-4, 1e-3, 1e-2; R and C per variable from the autotuner; every
    variable's 64 fields in one batched compress + decompress chain, all four
    in one CUDA graph; against the same fields one call at a time."""
    import torch
    import paper_2501_06910_gb300 as mcc
    from paper_2501_06910_gb300 import autotune
    from synth import torchgen
    coords, cells = synth.mesh2d_jittered(nside=1000, seed=41)
    cd = torch.from_numpy(coords).to(dev)
    plan = mcc.plan_create(cd, torch.from_numpy(cells).to(dev), (1024, 1024))
    del cells
    nvars, nsteps = 4, 64
    ebs = [1e-6, 1e-4, 1e-3, 1e-2]
    fields = [[None] * nsteps for _ in range(nvars)]
    for v, t, f in torchgen.fields_advected(cd, nvars=nvars, nsteps=nsteps, seed=8):
        fields[v][t] = f
    n = coords.shape[0]
    tuned, tables, prms = [], [], []
    for v in range(nvars):
        best, table = autotune.tune(plan, fields[v][0], dict(dtype=mcc.F64, eb=ebs[v]))
        tuned.append(best)
        tables.append(table)
        prms.append(mcc.params_default(**best))
    slots, outs, wscs, wsds, ys = [], [], [], [], []
    for v in range(nvars):
        cws, dws = mcc.workspace_size(plan, prms[v])
        slot = (mcc.compress_bound(plan, prms[v]) + 7) // 8 * 8
        slots.append(slot)
        outs.append(torch.empty(slot * nsteps, dtype=torch.uint8, device=dev))
        wscs.append(torch.empty(cws * nsteps, dtype=torch.uint8, device=dev))
        wsds.append(torch.empty(dws * nsteps, dtype=torch.uint8, device=dev))
        ys.append([torch.empty_like(fields[v][0]) for _ in range(nsteps)])
    sizes = []
    for v in range(nvars):
        sz = mcc.compress_batch(plan, fields[v], [prms[v]] * nsteps, wscs[v], outs[v], slots[v])
        mcc.decompress_batch(plan, outs[v], slots[v], sz, ys[v], wsds[v])
        for t in (0, nsteps - 1):
            x = fields[v][t]
            if not float((ys[v][t] - x).abs().max()) <= ebs[v] * float(x.max() - x.min()):
                raise SystemExit("batched c4 line: bound violated")
        sizes.append(sz)

    def bstep():
        for v in range(nvars):
            mcc.compress_batch(plan, fields[v], [prms[v]] * nsteps, wscs[v], outs[v], slots[v],
                               sync=False)
            mcc.decompress_batch(plan, outs[v], slots[v], [slots[v]] * nsteps, ys[v], wsds[v],
                                 sync=False)

    reps = max(3, args.steps // 10)
    bms = time_replays(bstep, flush, reps, args.warmup, stream)
    # the same 256 fields one call at a time (the plain form), one graph
    cws1, dws1 = mcc.workspace_size(plan, prms[0])
    ws1c = torch.empty(max(mcc.workspace_size(plan, p)[0] for p in prms), dtype=torch.uint8,
                       device=dev)
    ws1d = torch.empty(max(mcc.workspace_size(plan, p)[1] for p in prms), dtype=torch.uint8,
                       device=dev)

    def sstep():
        for v in range(nvars):
            for t in range(nsteps):
                o = outs[v][t * slots[v]:(t + 1) * slots[v]]
                mcc.compress(plan, fields[v][t], prms[v], ws1c, o, sync=False)
                mcc.decompress(plan, o, slots[v], ys[v][t], ws1d, sync=False)

    sms = time_replays(sstep, flush, reps, args.warmup, stream)
    total = nvars * nsteps * n * 8
    res = {"workload": "2d-jittered-1M-grid1024^2, 4 vars x 64 steps advected bumps FP64, "
                       "rel bounds 1e-6/1e-4/1e-3/1e-2",
           "fields": nvars * nsteps, "input_bytes": total,
           "ms_per_step": bms, "GBps": total / (bms * 1e-3) / 1e9,
           "one_call_per_field": {"ms_per_step": sms, "GBps": total / (sms * 1e-3) / 1e9},
           "per_var": [{"eb_rel": ebs[v], "R": tuned[v]["R1"], "C": tuned[v]["C1"],
                        "compression_ratio": nsteps * n * 8 / sum(sizes[v]),
                        "autotune": [list(r) for r in tables[v]]} for v in range(nvars)]}
    plan.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mcc", choices=["mcc", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--eb", type=float, default=1e-4)
    ap.add_argument("--zero-run", action="store_true",
                    help="main line with the zero-run stage (the other lines as they are)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-kernel-times", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--preroll", type=float, default=0.5, help="seconds of untimed steps")
    ap.add_argument("--batch", type=int, default=16, help="fields per step of the batched line")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-predictor line")
    ap.add_argument("--no-c4", action="store_true", help="skip the variables x timesteps line")
    ap.add_argument("--no-grid-init", action="store_true", help="skip the Grid_Init line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = load_workload(args.config)
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    import torch.distributed as dist
    import paper_2501_06910_gb300 as mcc

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    plan = mcc.plan_create(torch.from_numpy(wl["coords"]).to(dev),
                           torch.from_numpy(wl["cells"]).to(dev), wl["n"])
    x_np = wl["x"]
    x = torch.from_numpy(x_np).to(dev)
    prm = mcc.params_default(dtype=mcc.F64, eb=args.eb, grid_fraction=0.5,
                             zero_run=1 if args.zero_run else 0)
    wsc = plan.workspace(prm, "compress")
    wsd = plan.workspace(prm, "decompress")
    cap = mcc.compress_bound(plan, prm)
    out = torch.zeros(cap, dtype=torch.uint8, device=dev)
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        mcc.compress(plan, x, prm, wsc, out, sync=False)
        mcc.decompress(plan, out, cap, y, wsd, sync=False)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    st, size = mcc.workspace_result(wsc)
    st2, _ = mcc.workspace_result(wsd)
    if st != 0 or st2 != 0:
        raise SystemExit(f"device status {st}/{st2}")
    # the main line's bitstream sizes (words) for the algorithmic bytes; the
    # other lines below reuse `out`
    hdr = out[:192].cpu().numpy()
    W1 = int(hdr[168:176].view(np.uint64)[0])
    W2 = int(hdr[176:184].view(np.uint64)[0])
    tau = args.eb * (float(x.max()) - float(x.min()))
    err = float((y - x).abs().max())
    if not err <= tau:
        raise SystemExit(f"bound violated: {err} > {tau}")

    graph = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()

    def run_step():
        if graph is not None:
            graph.replay()
        else:
            step()

    for _ in range(args.warmup):
        flush.fill_(1)
        run_step()
    y.zero_()
    run_step()
    torch.cuda.synchronize()
    if float((y - x).abs().max()) != err:
        raise SystemExit("graph replay differs from the eager step")

    # timed region: K steps, each bracketed by events, L2 flushed before each
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        t_end = time.perf_counter() + args.preroll
        while time.perf_counter() < t_end:  # pre-roll under the same load
            flush.fill_(3)
            run_step()
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            run_step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = max_over_ranks(statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends)), world, dev)
    clocks = clk.summary()

    # per-kernel device times: the same step captured with an event pair
    # around every kernel, replayed K times (L2 flushed before each)
    prof = {}
    if not args.no_kernel_times:
        mcc.profile_reset()
        mcc.profile_enable(True)
        pgraph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(pgraph):
            step()
        mcc.profile_enable(False)
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            pgraph.replay()
            torch.cuda.synchronize()
            for name, (t, n) in mcc.profile_read().items():
                a = prof.setdefault(name, [0.0, 0])
                a[0] += t
                a[1] += n
        mcc.profile_reset()
    launches_per_step = (sum(n for _, n in prof.values()) / args.steps) if prof else None

    # batched: B fields of the same workload per step through mcc_compress_batch
    # and mcc_decompress_batch (one graph; plan shared; L2 flushed per step)
    batched = None
    if args.batch > 1:
        B = args.batch
        xs = [x.clone() for _ in range(B)]
        ys = [torch.empty_like(x) for _ in range(B)]
        prms = [mcc.params_default(dtype=mcc.F64, eb=args.eb, grid_fraction=0.5) for _ in range(B)]
        slot = (cap + 7) // 8 * 8
        bout = torch.zeros(slot * B, dtype=torch.uint8, device=dev)
        cws, dws = mcc.workspace_size(plan, prm)
        chain = min(B, 64)
        bwsc = torch.empty(cws * chain, dtype=torch.uint8, device=dev)
        bwsd = torch.empty(dws * chain, dtype=torch.uint8, device=dev)

        def bstep():
            mcc.compress_batch(plan, xs, prms, bwsc, bout, slot, sync=False)
            mcc.decompress_batch(plan, bout, slot, [slot] * B, ys, bwsd, sync=False)

        bstep()
        sizes = mcc.compress_batch(plan, xs, prms, bwsc, bout, slot, sync=True)
        mcc.decompress_batch(plan, bout, slot, sizes, ys, bwsd, sync=True)
        if any(not torch.equal(ys[f], y) for f in range(B)):
            raise SystemExit("batched result differs from the single-field result")
        bgraph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(bgraph):
            bstep()
        for _ in range(args.warmup):
            flush.fill_(1)
            bgraph.replay()
        bs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        be = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            bs[k].record(stream)
            bgraph.replay()
            be[k].record(stream)
        torch.cuda.synchronize()
        bms = max_over_ranks(statistics.mean(s.elapsed_time(e) for s, e in zip(bs, be)), world, dev)
        batched = {"fields_per_step": B, "ms_per_step": bms,
                   "value": job_value(world, B * x_np.nbytes, bms), "unit": "GB/s",
                   "compression_ratio": x_np.nbytes / sizes[0]}
        del bgraph, bout, bwsc, bwsd, xs, ys

    # end to end through the API with host buffers (pinned)
    e2e = None
    h2d = d2h = 0
    if not args.no_e2e:
        x_host = torch.from_numpy(x_np).pin_memory()
        out_host = torch.empty(cap, dtype=torch.uint8).pin_memory()
        y_host = torch.empty_like(x_host).pin_memory()
        x_dev = torch.empty_like(x)
        in_dev = torch.empty_like(out)
        e2e_ms = []
        for k in range(args.warmup + args.steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x_dev.copy_(x_host, non_blocking=True)
            n_out = mcc.compress(plan, x_dev, prm, wsc, out, sync=True)
            out_host[:n_out].copy_(out[:n_out])
            in_dev[:n_out].copy_(out_host[:n_out], non_blocking=True)
            mcc.decompress(plan, in_dev, n_out, y, wsd, sync=False)
            y_host.copy_(y)
            torch.cuda.synchronize()
            if k >= args.warmup:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
            h2d, d2h = x_np.nbytes + n_out, n_out + x_np.nbytes
        if not torch.equal(y_host, y.cpu()):
            raise SystemExit("e2e mismatch")
        e2e = max_over_ranks(statistics.mean(e2e_ms), world, dev)

    # the other bounds of the 2D graded configuration (1e-6, 1e-2): ratio and
    # compress+decompress time of the same field
    bounds = {}
    for eb in (1e-6, 1e-2):
        prm_b = mcc.params_default(dtype=mcc.F64, eb=eb, grid_fraction=0.5)
        size_b = mcc.compress(plan, x, prm_b, wsc, out)
        mcc.decompress(plan, out, size_b, y, wsd)
        tau_b = eb * (float(x.max()) - float(x.min()))
        if not float((y - x).abs().max()) <= tau_b:
            raise SystemExit(f"bound violated at eb {eb}")

        def bstep_b(prm_b=prm_b):
            mcc.compress(plan, x, prm_b, wsc, out, sync=False)
            mcc.decompress(plan, out, cap, y, wsd, sync=False)

        ms_b = time_replays(bstep_b, flush, max(5, args.steps // 4), args.warmup, stream)
        bounds[str(eb)] = {"compression_ratio": x_np.nbytes / size_b, "ms_per_step": ms_b,
                           "GBps": x_np.nbytes / (ms_b * 1e-3) / 1e9}

    # the operators (Sec. III-B, III-C) on the same field: barycentric or
    # cluster-mean f, bi/trilinear or nearest-node g, at the three bounds
    operators = []
    for eb in (1e-6, 1e-4, 1e-2):
        for fop, gop in (("barycentric", "multilinear"), ("barycentric", "nearest"),
                         ("cluster", "multilinear"), ("cluster", "nearest")):
            prm_o = mcc.params_default(dtype=mcc.F64, eb=eb, grid_fraction=0.5, f_op=fop,
                                       g_op=gop)
            size_o = mcc.compress(plan, x, prm_o, wsc, out)
            mcc.decompress(plan, out, size_o, y, wsd)
            tau_o = eb * (float(x.max()) - float(x.min()))
            err_o = float((y - x).abs().max())
            if not err_o <= tau_o:
                raise SystemExit(f"bound violated ({fop}, {gop}, {eb})")

            def ostep(prm_o=prm_o):
                mcc.compress(plan, x, prm_o, wsc, out, sync=False)
                mcc.decompress(plan, out, cap, y, wsd, sync=False)

            ms_o = time_replays(ostep, flush, max(5, args.steps // 4), args.warmup, stream)
            operators.append({"eb_rel": eb, "f": fop, "g": gop,
                              "compression_ratio": x_np.nbytes / size_o, "ms_per_step": ms_o,
                              "GBps": x_np.nbytes / (ms_o * 1e-3) / 1e9,
                              "max_abs_err_over_tau": err_o / tau_o})

    # the zero-run stage (runs of zero symbols as digit tokens before the
    # Huffman coder) against the plain coder on the same field, from tight
    # bounds (short runs) to loose ones (long runs)
    zero_run = []
    for eb in (1e-6, 1e-4, 1e-3, 1e-2, 1e-1):
        row = {"eb_rel": eb}
        for zr in (0, 1):
            prm_z = mcc.params_default(dtype=mcc.F64, eb=eb, grid_fraction=0.5, zero_run=zr)
            size_z = mcc.compress(plan, x, prm_z, wsc, out)
            mcc.decompress(plan, out, size_z, y, wsd)
            tau_z = eb * (float(x.max()) - float(x.min()))
            if not float((y - x).abs().max()) <= tau_z:
                raise SystemExit(f"bound violated (zero_run {zr}, {eb})")

            def zstep(prm_z=prm_z):
                mcc.compress(plan, x, prm_z, wsc, out, sync=False)
                mcc.decompress(plan, out, cap, y, wsd, sync=False)

            ms_z = time_replays(zstep, flush, max(5, args.steps // 4), args.warmup, stream)
            key = "zero_run" if zr else "plain"
            row[key] = {"compression_ratio": x_np.nbytes / size_z, "ms_per_step": ms_z,
                        "GBps": x_np.nbytes / (ms_z * 1e-3) / 1e9}
        zero_run.append(row)

    # the paper's default baseline (Sec. V): the same coder on the vertex
    # array in 1D, in storage order (shuffled ids) and in Morton order of the
    # vertex positions (a file with spatial locality); the improvement is the
    # method's ratio over it at the same bound
    default_1d = []
    orders = [("storage", None)]
    if len(wl["n"]) == 2:
        cxy = wl["coords"]
        lo_c, span_c = cxy.min(axis=0), np.maximum(np.ptp(cxy, axis=0), 1e-300)
        kk = np.minimum(((cxy - lo_c) / span_c * 65535.0).astype(np.int64), 65535)
        orders.append(("morton", np.argsort(synth._morton2(kk[:, 0], kk[:, 1]), kind="stable")))
    mc_ratio = {1e-6: bounds["1e-06"]["compression_ratio"], 1e-4: x_np.nbytes / size,
                1e-2: bounds["0.01"]["compression_ratio"]}
    for oname, perm in orders:
        xo_d = x if perm is None else torch.from_numpy(np.ascontiguousarray(x_np[perm])).to(dev)
        for eb in (1e-6, 1e-4, 1e-2):
            prm_1 = mcc.params_default(dtype=mcc.F64, eb=eb)
            s1 = mcc.compress_1d(xo_d, prm_1)
            y1 = torch.empty_like(xo_d)
            mcc.decompress_1d(s1, y1)
            tau_1 = eb * (float(xo_d.max()) - float(xo_d.min()))
            if not float((y1 - xo_d).abs().max()) <= tau_1:
                raise SystemExit(f"1D coder: bound violated ({oname}, {eb})")
            ws1c, ws1d = mcc.workspace_size_1d(xo_d.numel(), prm_1)
            w1c = torch.empty(ws1c, dtype=torch.uint8, device=dev)
            w1d = torch.empty(ws1d, dtype=torch.uint8, device=dev)
            o1 = torch.empty(mcc.compress_bound_1d(xo_d.numel(), prm_1), dtype=torch.uint8, device=dev)

            def step1(prm_1=prm_1, xo_d=xo_d, y1=y1, w1c=w1c, w1d=w1d, o1=o1):
                mcc.compress_1d_into(xo_d, prm_1, w1c, o1, sync=False)
                mcc.decompress_1d_into(o1, o1.numel(), y1, w1d, sync=False)

            ms_1 = time_replays(step1, flush, max(5, args.steps // 4), args.warmup, stream)
            r1 = x_np.nbytes / s1.numel()
            default_1d.append({"order": oname, "eb_rel": eb, "compression_ratio": r1,
                               "ms_per_step": ms_1, "GBps": x_np.nbytes / (ms_1 * 1e-3) / 1e9,
                               "method_ratio": mc_ratio[eb], "improvement": mc_ratio[eb] / r1})
            del w1c, w1d, o1

    grid_init = None
    if not args.no_grid_init and len(wl["n"]) == 2:
        grid_init = grid_init_line(args, dev, flush, stream, wl, x)

    learned = batched_c4 = None
    if not args.no_learned:
        learned = learned_line(args, dev, flush, stream)
    if not args.no_c4:
        batched_c4 = batched_c4_line(args, dev, flush, stream)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    nbytes = x_np.nbytes
    alg = algorithmic_bytes(len(wl["n"]), x_np.size, int(np.prod(wl["n"])), 8, W1, W2, size)
    per_kernel = {}
    if prof:
        tot = sum(t for t, _ in prof.values())
        per_kernel = {k: {"ms_per_launch": v[0] / v[1], "launches_per_step": v[1] / args.steps,
                          "share": v[0] / tot,
                          "alg_GBps": alg.get(k, 0) / (v[0] / v[1] * 1e-3) / 1e9}
                      for k, v in prof.items() if v[1]}
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    roofline = None
    if per_kernel:
        dom = max(per_kernel,
                  key=lambda k: per_kernel[k]["ms_per_launch"] * per_kernel[k]["launches_per_step"])
        achieved = alg.get(dom, 0) / (per_kernel[dom]["ms_per_launch"] * 1e-3) / 1e9
        traffic = None
        tfile = os.path.join(ROOT, "profiles", "dram_traffic.json")
        if os.path.exists(tfile):  # counters count only while the kernel is unchanged
            ent = json.load(open(tfile)).get(dom)
            if isinstance(ent, dict):
                src = os.path.join(ROOT, "paper_2501_06910_gb300", "csrc", ent["source"])
                if os.path.exists(src) and \
                        hashlib.sha1(open(src, "rb").read()).hexdigest() == ent["sha1"]:
                    traffic = ent["bytes"]
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": traffic, "kernel": dom,
                    "peak_source": "measured" if peaks else "fallback"}
    cpu = None if args.no_cpu_baseline else cpu_baseline(wl, args.eb)
    line = {
        "metric": METRIC,
        "value": job_value(world, nbytes, ms),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "n_vertices": int(x_np.size),
                   "grid": list(wl["n"]), "eb_rel": args.eb, "grid_fraction": 0.5,
                   "zero_run": bool(args.zero_run),
                   "compression_ratio": nbytes / size, "stream_bytes": int(size),
                   "max_abs_err_over_tau": err / tau,
                   "l2": "flushed before every step (256 MiB write, untimed)",
                   "cuda_graph": graph is not None, "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "kernels": per_kernel,
        "cpu_baseline": cpu,
        "e2e": None if e2e is None else {
            "value": world * nbytes / (e2e * 1e-3) / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": None if launches_per_step is None else int(round(launches_per_step * args.steps)),
        "other_bounds": bounds,
        "operators": operators,
        "zero_run": zero_run,
        "default_1d": default_1d,
        "grid_init": grid_init,
        "batched": batched,
        "learned": learned,
        "batched_c4": batched_c4,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
