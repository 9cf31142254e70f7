#!/usr/bin/env python
"""Throughput benchmark of the GB300 multi-component compressor.

Metric: compress + decompress GB/s of input values (n_v x sizeof(value) bytes
per field) at relative bound 1e-4 (grid / residual split 0.5), with the
compression ratio. Headline workload (default ``--config c3``): the 3D
tetrahedral annulus, a cylinder of radius 1 and height 2 with a coaxial hole
of radius 0.3, (64, 512, 244) jittered structured nodes (7,995,392 vertices)
split into 39,191,040 tetrahedra, vertex and cell order shuffled; a float64
swirling vortex plus 4-octave value noise; a 256^3 grid (the stand-in for
the paper's Nek5000 pipe / VKI blade meshes, Table I). The plan (mesh -> grid
mapping) is built once and excluded, as in Sec. IV-A.

One step = mcc_compress + mcc_decompress of one device-resident field,
enqueued without host synchronisation and replayed as one CUDA graph. The L2
(129 MB) is flushed (256 MiB write, then 256 MiB read, untimed) before every
step; each step is timed with CUDA events on the launch stream. Under
torchrun every rank runs an independent replica on its own GPU (the method
has no exchange step); value is the sum over ranks of the input bytes
divided by the slowest rank's time.

Output: one compact JSON object per side measurement ({"side": name, ...};
other bounds, operators, the zero-run stage, the 1D default, Grid_Init, the
2D graded mesh, batches, the learned predictor, the split sweep, many
variables x timesteps), then, as the LAST line, the headline (metric, value,
roofline, cpu_baseline, e2e, clocks). ``--side-out PATH`` also writes the
side objects to a file.

``--impl reference`` times the CPU oracle on the machine's host cores (one
process per core, each compressing and decompressing a bounded sample of the
same workload) and prints the same headline keys with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
HEADLINE_MAX_BYTES = 2048


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


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def rnd(v, digits=4):
    """Round floats to `digits` significant digits (compact side lines)."""
    if isinstance(v, float):
        if not math.isfinite(v) or v == 0.0:
            return v if math.isfinite(v) else None
        return float(f"{v:.{digits}g}")
    if isinstance(v, dict):
        return {k: rnd(x, digits) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [rnd(x, digits) for x in v]
    return v


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


def algorithmic_bytes(dim, n_v, n_g, vsz, cbytes, c1bytes=None, launched=()):
    """HBM bytes each kernel must move at least once per LAUNCH (inputs read,
    outputs written), for a plain-predictor field. Gathers of the vertex
    codes Q (4 n_v bytes) and of the grid codes q1 (4 n_g bytes) are counted
    as cache hits (each array is read from HBM once by its streaming
    producer or consumer). cbytes = the compressed stream, c1bytes = its grid
    component's share. Names ending in _grid / _res are the launches of one
    component on the plan's second stream; the plain name then covers the
    other component."""
    c1 = cbytes // 2 if c1bytes is None else c1bytes
    alg = {
        "k_group_len_grid": 2 * n_g,
        "k_runs_grid": 2 * n_g,
        "k_codebook_grid": 0,
        "k_grid3d_grid": (4 + 2) * n_g,
        "k_dec_syms_res": (cbytes - c1) + 4 * n_v,
        **_alg_both(dim, n_v, n_g, vsz, cbytes),
    }
    if "k_group_len_grid" in launched:  # the caller's stream kept the residual groups
        alg["k_group_len"] = 2 * n_v
        alg["k_runs"] = 2 * n_v
        alg["k_pack"] = 2 * (n_g + n_v) + cbytes
    if "k_dec_syms_res" in launched:  # ... and the grid component's decoding
        alg["k_dec_syms"] = c1 + 4 * n_g
    return alg


def _alg_both(dim, n_v, n_g, vsz, cbytes):
    return {
        "k_reduce": vsz * n_v,                                 # x
        "k_prequant": (vsz + 4) * n_v,                         # x in, Q out
        "k_grid2d": (16 + 4 + 2) * n_g,                        # 16-byte plan record in; q1, symbols out
        "k_grid_codes": (16 + 8 + 4) * n_g,                    # 3D: ids, weights in; q1 out
        "k_grid3d": (4 + 2) * n_g,                             # 3D: q1 in; symbols out
        "k_node": (4 + 2 * dim + 4 + 2) * n_v,                 # cell, local coords, Q in; symbols out
        "k_codebook": 0,
        "k_group_len": 2 * (n_g + n_v),                        # symbols in
        "k_pack": 2 * (n_g + n_v) + cbytes,                    # symbols in, stream out
        "k_runs": 2 * (n_g + n_v),
        "k_dec_prep": 0,
        "k_dec_syms": cbytes + 4 * (n_g + n_v),                # stream in; deltas, q2 out
        "k_scan_rows": 8 * n_g,                                # one read + one write per pass
        "k_scan_axis": 8 * n_g,
        "k_scan_xy": 8 * n_g,                                  # 3D: rows and y in one pass
        "k_predict": 0,                                        # plain streams: returns at once
        "k_recon": (4 + 2 * dim + 4 + vsz) * n_v,              # cell, local coords, q2 in; x' out
    }


def step_bytes(alg, per_kernel):
    """Algorithmic bytes of one whole step: every kernel's per-launch bytes
    times its launches per step."""
    return sum(alg.get(k, 0) * v["launches_per_step"] for k, v in per_kernel.items())


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
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- #
# workloads
# --------------------------------------------------------------------------- #
WORKLOADS = {
    "c3": "3d-annulus-8M-tets39M-grid256^3-f64",
    "c2": "2d-graded-2M-delaunay-grid1024^2-f64",
    "c1": "2d-jittered-20k-grid128^2-f64",
}


def load_mesh(config, layers=None):
    """(coords, cells, grid) of a workload (the field is made separately);
    for the 3D annulus, ``layers`` < 244 keeps only its bottom node layers
    (the same spacings, and a grid of the full grid's spacing over them: a
    small case of the same kernels for profiling)."""
    if config == "c3":
        if layers and layers < 244:
            coords, cells = synth.mesh3d_annulus_slab(layers)
            nz = int(round(float(coords[:, 2].max() - coords[:, 2].min()) / (2.0 / 255.0))) + 1
            return coords, cells, (256, 256, nz)
        coords, cells = synth.mesh3d_annulus()
        return coords, cells, (256, 256, 256)
    if config == "c2":
        coords, cells = synth.mesh2d_graded()
        return coords, cells, (1024, 1024)
    if config == "c1":
        coords, cells = synth.mesh2d_jittered()
        return coords, cells, (128, 128)
    raise SystemExit(f"unknown config {config}")


def field_on_device(config, coords, cd):
    """The workload's FP64 field, on the device (numpy for the 2D ones)."""
    import torch
    if config == "c3":
        from synth import torchgen
        return torchgen.field_vortex(cd, seed=6)
    x = synth.field_bumps_noise(coords) if config == "c2" else synth.field_sincos(coords)
    return torch.from_numpy(x).to(cd.device)


# --------------------------------------------------------------------------- #
# CPU baseline: the oracle on the host cores (one process per core)
# --------------------------------------------------------------------------- #
SLAB_LAYERS = 17


def cpu_sample(config):
    """A bounded sample of the workload for the CPU oracle: (coords, cells,
    grid, x, description). The 3D annulus: its bottom 17 node layers (same
    radial / angular resolution and z spacing) with an 18-plane grid of the
    full grid's spacing; the 2D workloads: the full mesh."""
    if config == "c3":
        coords, cells = synth.mesh3d_annulus_slab(SLAB_LAYERS)
        h = 2.0 / 255.0
        nz = int(round(float(coords[:, 2].max() - coords[:, 2].min()) / h)) + 1
        x = synth.field_vortex(coords)
        return coords, cells, (256, 256, nz), x, (
            f"z-slab of the annulus: {SLAB_LAYERS} of 244 node layers, {x.size} vertices, "
            f"{cells.shape[0]} tets, grid 256x256x{nz} (same spacings), FP64 vortex, "
            "rel 1e-4, plan excluded")
    coords, cells, n = load_mesh(config)
    x = synth.field_bumps_noise(coords) if config == "c2" else synth.field_sincos(coords)
    return coords, cells, n, x, f"full workload ({x.size} vertices), plan excluded"


_W = {}


def _oracle_init(config, eb):
    import oracle
    coords, cells, n, x, _ = cpu_sample(config)
    _W.update(plan=oracle.Plan(coords, cells, n), x=x, eb=eb)


def _oracle_task(_):
    import oracle
    t0 = time.perf_counter()
    s = oracle.compress(_W["plan"], _W["x"], eb=_W["eb"])
    oracle.decompress(_W["plan"], s)
    return time.perf_counter() - t0, int(s.size)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_all_cores(config, eb, steps, warmup, procs=None):
    """One process per host core (spawned: none inherits a CUDA context);
    a step = every process compresses and decompresses the sample once.
    Returns (GB/s over all processes, per-step seconds, processes, nbytes,
    stream bytes, description)."""
    import multiprocessing as mp
    procs = procs or host_cores()
    _, _, _, x, desc = cpu_sample(config)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_oracle_init, initargs=(config, eb)) as pool:
        for _ in range(warmup):
            pool.map(_oracle_task, range(procs), chunksize=1)
        walls, size = [], 0
        for _ in range(steps):
            t0 = time.perf_counter()
            res = pool.map(_oracle_task, range(procs), chunksize=1)
            walls.append(time.perf_counter() - t0)
            size = res[0][1]
    t = statistics.mean(walls)
    return procs * x.nbytes / t / 1e9, walls, procs, x.nbytes, size, desc


def oracle_one_core(config, eb, steps, warmup):
    """The oracle in this process (one thread): GB/s and seconds per step."""
    import oracle
    coords, cells, n, x, desc = cpu_sample(config)
    plan = oracle.Plan(coords, cells, n)
    for _ in range(warmup):
        oracle.decompress(plan, oracle.compress(plan, x, eb=eb))
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        s = oracle.compress(plan, x, eb=eb)
        oracle.decompress(plan, s)
        ts.append(time.perf_counter() - t0)
    t = statistics.mean(ts)
    return x.nbytes / t / 1e9, t, x.nbytes, int(s.size), desc


def cpu_baseline(config, eb, steps=6, warmup=1):
    """The oracle as it stands on the host cores: all cores (one process
    each) and one core, on the bounded sample (10-30 s of CPU work)."""
    v1, t1, nbytes, size, desc = oracle_one_core(config, eb, steps, warmup)
    vn, walls, procs, _, _, _ = oracle_all_cores(config, eb, steps, warmup)
    return {"value": vn, "unit": "GB/s", "cores": procs, "kind": "oracle",
            "sample": f"{desc}; {steps} steps of one compress+decompress per process",
            "single_core": {"value": v1, "cores": 1, "ms_per_step": t1 * 1e3},
            "nproc": host_cores(), "compression_ratio": nbytes / size}


def run_reference(args):
    """The CPU oracle timed on the host cores: every step, one process per
    core compresses and decompresses the bounded sample once (rank 0 only;
    other ranks exit without work)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    vn, walls, procs, nbytes, size, desc = oracle_all_cores(args.config, args.eb, args.steps,
                                                            args.warmup)
    v1, t1, _, _, _ = oracle_one_core(args.config, args.eb, max(3, min(args.steps, 10)), 1)
    ms = statistics.mean(walls) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": vn, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config], "eb_rel": args.eb, "grid_fraction": 0.5,
                   "compression_ratio": nbytes / size, "l2": "n/a (host)"},
        "cpu_baseline": {"value": vn, "unit": "GB/s", "cores": procs, "kind": "oracle",
                         "sample": f"{desc}; a step = one compress+decompress per process",
                         "single_core": {"value": v1, "cores": 1, "ms_per_step": t1 * 1e3},
                         "nproc": host_cores()},
        "e2e": {"value": vn, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(rnd(line, 6), allow_nan=False), flush=True)


class L2Flush:
    """Evicts the L2 (129 MB) between timed steps: a write of a 256 MiB
    buffer, then a read of a second one, so that a timed step starts with no
    line of its data in L2 and no dirty line of the flush itself left to
    write back to HBM inside the timed region."""

    def __init__(self, dev, nbytes=256 << 20):
        import torch
        self.w = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.r = torch.zeros(nbytes // 8, dtype=torch.int64, device=dev)

    def fill_(self, v):
        self.w.fill_(v)
        self.r.max()  # a device-side reduction: reads the buffer, no host sync


def time_replays(fn, flush, steps, warmup, stream, world=1):
    """fn captured in one CUDA graph; mean ms of `steps` replays, each after an
    L2 flush and bracketed by events on the launch stream (a barrier on both
    sides of the timed loop when there are several ranks)."""
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
    barrier(world)
    for k, (a, b) in enumerate(ev):
        flush.fill_(k & 0xFF)
        a.record(stream)
        g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    del g
    return ms


class Field:
    """One field on one plan with its workspaces and buffers."""

    def __init__(self, mcc, plan, x, prm):
        import torch
        self.mcc, self.plan, self.x, self.prm = mcc, plan, x, prm
        self.wsc = plan.workspace(prm, "compress")
        self.wsd = plan.workspace(prm, "decompress")
        self.cap = mcc.compress_bound(plan, prm)
        self.out = torch.zeros(self.cap, dtype=torch.uint8, device=x.device)
        self.y = torch.empty_like(x)

    def step(self):
        self.mcc.compress(self.plan, self.x, self.prm, self.wsc, self.out, sync=False)
        self.mcc.decompress(self.plan, self.out, self.cap, self.y, self.wsd, sync=False)

    def check(self, eb, what):
        """One synchronous round trip; the bound at every vertex. Returns
        (stream bytes, max |x - x'| / tau)."""
        size = self.mcc.compress(self.plan, self.x, self.prm, self.wsc, self.out)
        self.mcc.decompress(self.plan, self.out, size, self.y, self.wsd)
        x = self.x.double()
        tau = eb * (float(x.max()) - float(x.min()))
        err = float((self.y.double() - x).abs().max())
        if not err <= tau:
            raise RuntimeError(f"{what}: bound violated ({err} > {tau})")
        return size, err / tau


def kernel_times(mcc, step, flush, steps):
    """Per-kernel device times: the step captured with an event pair around
    every kernel, replayed `steps` times (L2 flushed before each). Returns
    {name: [total ms, launches]}."""
    import torch
    prof = {}
    mcc.profile_reset()
    mcc.profile_enable(True)
    pgraph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(pgraph):
        step()
    mcc.profile_enable(False)
    for k in range(steps):
        flush.fill_(k & 0xFF)
        pgraph.replay()
        torch.cuda.synchronize()
        for name, (t, n) in mcc.profile_read().items():
            a = prof.setdefault(name, [0.0, 0])
            a[0] += t
            a[1] += n
    mcc.profile_reset()
    del pgraph
    return prof


def dram_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, only
    while the kernel's source file is the one the counters were taken on."""
    tfile = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(tfile):
        return None
    ent = json.load(open(tfile)).get(kernel)
    if not isinstance(ent, dict):
        return None
    src = os.path.join(ROOT, "paper_2501_06910_gb300", "csrc", ent["source"])
    if os.path.exists(src) and hashlib.sha1(open(src, "rb").read()).hexdigest() == ent["sha1"]:
        return ent["bytes"]
    return None


def build_headline(*, world, steps, warmup, ms, nbytes, config, prof, alg, peaks, cpu, e2e,
                   clocks, traffic=None):
    """The headline JSON object (the last stdout line, under 2 KB): metric and
    value, the dominant kernel's roofline and the whole step's, the CPU
    oracle baseline, the end-to-end figure and the clocks."""
    per_kernel = {}
    if prof:
        tot = sum(t for t, _ in prof.values()) or 1.0
        per_kernel = {k: {"ms_per_launch": t / n, "launches_per_step": n / steps, "share": t / tot}
                      for k, (t, n) in prof.items() if n}
    hbm = peaks.get("hbm_gbs")
    peak_source = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    roofline = None
    if per_kernel:
        dom = max(per_kernel, key=lambda k: per_kernel[k]["share"])
        achieved = alg.get(dom, 0) / (per_kernel[dom]["ms_per_launch"] * 1e-3) / 1e9
        sb = step_bytes(alg, per_kernel)
        step_gbs = sb / (ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": traffic(dom) if traffic else None,
                    "kernel": dom, "alg_bytes_per_launch": alg.get(dom, 0),
                    "step_alg_bytes": sb, "step_achieved": step_gbs, "step_frac": step_gbs / hbm,
                    "peak_source": f"{peak_source} (hbm_gbs, copy)"}
    launches = sum(n for _, n in prof.values()) if prof else None
    line = {
        "metric": METRIC,
        "value": job_value(world, nbytes, ms),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": config,
        "roofline": roofline,
        "kernels_us": {k: [v["ms_per_launch"] * 1e3, v["launches_per_step"]]
                       for k, v in sorted(per_kernel.items(), key=lambda kv: -kv[1]["share"])},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": None if launches is None else int(launches),
        "clocks": clocks,
    }
    return rnd(line, 5)


def headline_json(line):
    """The compact last line: the per-kernel table (the longest-running
    kernels first) is cut from its tail, then dropped, before anything else
    would push the line past HEADLINE_MAX_BYTES (the whole table goes on its
    own earlier line)."""
    s = json.dumps(line, allow_nan=False, separators=(",", ":"))
    ks = list((line.get("kernels_us") or {}).items())
    while len(s) > HEADLINE_MAX_BYTES and "kernels_us" in line:
        line = dict(line)
        ks = ks[:-1]
        if ks:
            line["kernels_us"] = dict(ks)
        else:
            line.pop("kernels_us")
        s = json.dumps(line, allow_nan=False, separators=(",", ":"))
    return s


class Sides:
    """Side measurements: each printed as one compact JSON line as it
    completes (and collected for --side-out); a failing one records its
    error and the run goes on."""

    def __init__(self, path):
        self.path = path
        self.rows = []

    def run(self, name, fn, *a, **kw):
        t0 = time.perf_counter()
        try:
            res = fn(*a, **kw)
        except Exception as err:  # noqa: BLE001 -- recorded, never fatal
            res = {"error": f"{type(err).__name__}: {err}"}
        row = {"side": name, "wall_s": time.perf_counter() - t0, **(res or {})}
        row = rnd(row, 4)
        self.rows.append(row)
        print(json.dumps(row, allow_nan=False, separators=(",", ":")), flush=True)
        import torch
        torch.cuda.empty_cache()

    def write(self):
        if self.path:
            with open(self.path, "w") as f:
                for r in self.rows:
                    f.write(json.dumps(r, allow_nan=False) + "\n")


# --------------------------------------------------------------------------- #
# side measurements
# --------------------------------------------------------------------------- #
def rate(nbytes, ms):
    return nbytes / (ms * 1e-3) / 1e9


def side_bounds(mcc, plan, x, flush, stream, args, ebs=(1e-6, 1e-2)):
    """Other bounds on the headline field: ratio and compress+decompress rate."""
    rows = []
    for eb in ebs:
        f = Field(mcc, plan, x, mcc.params_default(dtype=mcc.F64, eb=eb, grid_fraction=0.5))
        size, e = f.check(eb, f"eb {eb}")
        ms = time_replays(f.step, flush, max(5, args.steps // 4), args.warmup, stream)
        rows.append({"eb_rel": eb, "ratio": x.numel() * 8 / size, "ms": ms,
                     "GBps": rate(x.numel() * 8, ms), "err_over_tau": e})
    return {"rows": rows}


def side_batched(mcc, plan, x, flush, stream, args, world):
    """B copies of the headline field per step through mcc_compress_batch /
    mcc_decompress_batch (one graph; plan shared; L2 flushed per step)."""
    import torch
    B = args.batch
    xs = [x.clone() for _ in range(B)]
    ys = [torch.empty_like(x) for _ in range(B)]
    prm = mcc.params_default(dtype=mcc.F64, eb=args.eb, grid_fraction=0.5)
    prms = [prm] * B
    cap = mcc.compress_bound(plan, prm)
    slot = (cap + 7) // 8 * 8
    bout = torch.zeros(slot * B, dtype=torch.uint8, device=x.device)
    cws, dws = mcc.workspace_size(plan, prm)
    chain = min(B, 64)
    bwsc = torch.empty(cws * chain, dtype=torch.uint8, device=x.device)
    bwsd = torch.empty(dws * chain, dtype=torch.uint8, device=x.device)

    def bstep():
        mcc.compress_batch(plan, xs, prms, bwsc, bout, slot, sync=False)
        mcc.decompress_batch(plan, bout, slot, [slot] * B, ys, bwsd, sync=False)

    sizes = mcc.compress_batch(plan, xs, prms, bwsc, bout, slot, sync=True)
    mcc.decompress_batch(plan, bout, slot, sizes, ys, bwsd, sync=True)
    ref = Field(mcc, plan, x, prm)
    ref.check(args.eb, "batched reference")
    if any(not torch.equal(ys[f], ref.y) for f in range(B)):
        raise RuntimeError("batched result differs from the single-field result")
    ms = time_replays(bstep, flush, max(5, args.steps // 2), args.warmup, stream, world)
    ms = max_over_ranks(ms, world, x.device)
    return {"fields_per_step": B, "ms_per_step": ms,
            "GBps": job_value(world, B * x.numel() * 8, ms),
            "ratio": x.numel() * 8 / sizes[0]}


def side_split(mcc, plan, cd, flush, stream, args):
    """The 3D configuration's grid / residual split swept 0.2 .. 0.8, FP64
    and FP32 fields (seed 6), rel 1e-4, closed loop (residual against the
    decompressed grid) and open loop (against the grid before quantisation,
    Algorithm 3 as printed): ratio / GB/s / max error over tau."""
    from synth import torchgen
    x64 = torchgen.field_vortex(cd, seed=6)
    rows = []
    for dt, xx in (("f64", x64), ("f32", x64.float())):
        for loop in ("closed", "open"):
            for frac in (0.2, 0.35, 0.5, 0.65, 0.8):
                prm = mcc.params_default(dtype=mcc.F64 if dt == "f64" else mcc.F32, eb=1e-4,
                                         grid_fraction=frac, open_loop=loop == "open")
                f = Field(mcc, plan, xx, prm)
                size, e = f.check(1e-4, f"split {dt} {loop} {frac}")
                ms = time_replays(f.step, flush, 5, args.warmup, stream)
                nb = xx.numel() * xx.element_size()
                rows.append([dt, loop, frac, nb / size, rate(nb, ms), e])
                del f
    return {"cols": ["dtype", "loop", "grid_fraction", "ratio", "GBps", "err_over_tau"],
            "rows": rows}


def side_learned(mcc, plan, cd, flush, stream, args):
    """The learned residual predictor on the 3D annulus: trained on the GPU on
    16 seeds of vortex + noise fields, evaluated on 2 unseen seeds at rel
    1e-4 against the plain predictor (auto choice per field); then one field
    with the network on the tcgen05 path."""
    import torch
    from synth import torchgen
    eb = 1e-4
    base = dict(dtype=mcc.F64, eb=eb, grid_fraction=0.5)
    train = [torchgen.field_vortex(cd, seed=1000 + i) for i in range(16)]
    cfg = mcc.train_cfg_default()
    t0 = time.perf_counter()
    model, losses = mcc.model_train(plan, train, mcc.params_default(**base), cfg)
    t_train = time.perf_counter() - t0
    del train
    res = {"train_s": t_train, "train_steps": cfg.steps, "train_batch": cfg.batch,
           "loss_first_100": float(np.mean(losses[:100])),
           "loss_last_100": float(np.mean(losses[-100:]))}
    n = cd.shape[0]
    for label, prm in (("plain", mcc.params_default(**base)),
                       ("learned", mcc.params_default(model=model, auto=True, **base))):
        sizes, mss, chosen = [], [], []
        for seed in (2000, 2001):
            f = Field(mcc, plan, torchgen.field_vortex(cd, seed=seed), prm)
            size, _ = f.check(eb, f"learned line ({label})")
            chosen.append("learned" if int(f.out[20].item()) & 2 else "plain")
            sizes.append(size)
            mss.append(time_replays(f.step, flush, max(5, args.steps // 4), args.warmup, stream))
            del f
        res[label] = {"ratio": 2 * n * 8 / sum(sizes), "ms_per_field": statistics.mean(mss),
                      "GBps": rate(n * 8, statistics.mean(mss)), "chosen": chosen}
    res["ratio_gain"] = res["learned"]["ratio"] / res["plain"]["ratio"]
    # the same learned field with the network on tcgen05 (plan tuning): the
    # stream must not change
    prm = mcc.params_default(model=model, auto=True, **base)
    f = Field(mcc, plan, torchgen.field_vortex(cd, seed=2000), prm)
    size0, _ = f.check(eb, "learned line (mma.sync)")
    ref = f.out[:size0].clone()
    mcc.set_net_path(plan, mcc.NET_TCGEN05)
    try:
        size1, _ = f.check(eb, "learned line (tcgen05)")
        same = size1 == size0 and bool(torch.equal(f.out[:size1], ref))
        ms = time_replays(f.step, flush, max(5, args.steps // 4), args.warmup, stream)
    finally:
        mcc.set_net_path(plan, mcc.NET_MMA_SYNC)
    res["learned_tcgen05"] = {"ms_per_field": ms, "GBps": rate(n * 8, ms), "same_stream": same}
    del f
    return res


def side_c2(mcc, dev, flush, stream, args, sides):
    """The 2D graded workload (2M vertices, 1024^2 grid, FP64): the main
    figures at rel 1e-6 / 1e-4 / 1e-2, the operators (Sec. III-B, III-C),
    the zero-run stage, the paper's 1D default (Sec. V) and Grid_Init
    (Algorithm 1) with Grid_Coarsen (Algorithm 2); one side line each."""
    import torch
    coords, cells, n = load_mesh("c2")
    cd = torch.from_numpy(coords).to(dev)
    ed = torch.from_numpy(cells).to(dev)
    plan = mcc.plan_create(cd, ed, n)
    x = field_on_device("c2", coords, cd)
    nb = x.numel() * 8
    ratios = {}

    def main_rows():
        rows = []
        for eb in (1e-6, 1e-4, 1e-2):
            f = Field(mcc, plan, x, mcc.params_default(dtype=mcc.F64, eb=eb, grid_fraction=0.5))
            size, e = f.check(eb, f"c2 eb {eb}")
            ms = time_replays(f.step, flush, max(5, args.steps // 2), args.warmup, stream)
            ratios[eb] = nb / size
            rows.append({"eb_rel": eb, "ratio": nb / size, "ms": ms, "GBps": rate(nb, ms),
                         "err_over_tau": e})
        return {"workload": WORKLOADS["c2"], "rows": rows}

    def operators():
        rows = []
        for eb in (1e-6, 1e-4, 1e-2):
            for fop, gop in (("barycentric", "multilinear"), ("barycentric", "nearest"),
                             ("cluster", "multilinear"), ("cluster", "nearest")):
                prm = mcc.params_default(dtype=mcc.F64, eb=eb, grid_fraction=0.5, f_op=fop,
                                         g_op=gop)
                f = Field(mcc, plan, x, prm)
                size, e = f.check(eb, f"operators {fop} {gop} {eb}")
                ms = time_replays(f.step, flush, 5, args.warmup, stream)
                rows.append([eb, fop, gop, nb / size, rate(nb, ms), e])
        return {"cols": ["eb_rel", "f", "g", "ratio", "GBps", "err_over_tau"], "rows": rows}

    def zero_run():
        rows = []
        for eb in (1e-6, 1e-4, 1e-3, 1e-2, 1e-1):
            row = [eb]
            for zr in (0, 1):
                f = Field(mcc, plan, x, mcc.params_default(dtype=mcc.F64, eb=eb,
                                                           grid_fraction=0.5, zero_run=zr))
                size, _ = f.check(eb, f"zero_run {zr} {eb}")
                ms = time_replays(f.step, flush, 5, args.warmup, stream)
                row += [nb / size, rate(nb, ms)]
            rows.append(row)
        return {"cols": ["eb_rel", "plain_ratio", "plain_GBps", "zr_ratio", "zr_GBps"],
                "rows": rows}

    def default_1d():
        rows = []
        lo_c, span_c = coords.min(axis=0), np.maximum(np.ptp(coords, axis=0), 1e-300)
        kk = np.minimum(((coords - lo_c) / span_c * 65535.0).astype(np.int64), 65535)
        morton = np.argsort(synth._morton2(kk[:, 0], kk[:, 1]), kind="stable")
        for oname, perm in (("storage", None), ("morton", morton)):
            xo = x if perm is None else x[torch.from_numpy(morton).to(dev)].contiguous()
            for eb in (1e-6, 1e-4, 1e-2):
                prm = mcc.params_default(dtype=mcc.F64, eb=eb)
                s1 = mcc.compress_1d(xo, prm)
                y1 = torch.empty_like(xo)
                mcc.decompress_1d(s1, y1)
                tau = eb * float(xo.max() - xo.min())
                if not float((y1 - xo).abs().max()) <= tau:
                    raise RuntimeError(f"1D coder: bound violated ({oname}, {eb})")
                ws1c, ws1d = mcc.workspace_size_1d(xo.numel(), prm)
                w1c = torch.empty(ws1c, dtype=torch.uint8, device=dev)
                w1d = torch.empty(ws1d, dtype=torch.uint8, device=dev)
                o1 = torch.empty(mcc.compress_bound_1d(xo.numel(), prm), dtype=torch.uint8,
                                 device=dev)

                def step1(prm=prm, xo=xo, y1=y1, w1c=w1c, w1d=w1d, o1=o1):
                    mcc.compress_1d_into(xo, prm, w1c, o1, sync=False)
                    mcc.decompress_1d_into(o1, o1.numel(), y1, w1d, sync=False)

                ms = time_replays(step1, flush, 5, args.warmup, stream)
                r1 = nb / s1.numel()
                rows.append([oname, eb, r1, rate(nb, ms), ratios.get(eb), ratios.get(eb, 0) / r1])
        return {"cols": ["order", "eb_rel", "ratio", "GBps", "method_ratio", "improvement"],
                "rows": rows}

    def grid_init():
        rows = []
        for k in (30.0, 50.0, 70.0, 90.0, 99.0):
            t0 = time.perf_counter()
            gn, lo, hi = mcc.grid_init(cd, ed, k, 1.0, 4096)
            t_init = time.perf_counter() - t0
            gplan = mcc.plan_create(cd, ed, gn, lo, hi)
            for fop, gop in (("barycentric", "multilinear"), ("cluster", "nearest")):
                prm = mcc.params_default(dtype=mcc.F64, eb=1e-4, grid_fraction=0.5, f_op=fop,
                                         g_op=gop)
                f = Field(mcc, gplan, x, prm)
                size, _ = f.check(1e-4, f"grid_init {k} {fop}")
                ms = time_replays(f.step, flush, 5, args.warmup, stream)
                g_bytes, r_bytes = component_bytes(f.out[:208].cpu().numpy())
                row = [k, list(gn), t_init, fop, gop, nb / size, rate(nb, ms),
                       gplan.n_grid * 8 / max(g_bytes, 1), nb / max(r_bytes, 1)]
                try:  # the same on the planes Grid_Coarsen keeps
                    keep = mcc.grid_coarsen(gplan, gop)
                    kplan = mcc.plan_create(cd, ed, gn, lo, hi, keep=keep)
                    fk = Field(mcc, kplan, x, prm)
                    size_k, _ = fk.check(1e-4, f"grid_init {k} {fop} coarsened")
                    ms_k = time_replays(fk.step, flush, 5, args.warmup, stream)
                    row += [[int(v.size) for v in keep], nb / size_k, rate(nb, ms_k)]
                    del fk
                    kplan.close()
                except Exception as err:  # noqa: BLE001
                    row += [str(err), None, None]
                rows.append(row)
                del f
            gplan.close()
        return {"cols": ["k_pct", "grid", "grid_init_s", "f", "g", "ratio", "GBps",
                         "grid_component_ratio", "residual_component_ratio", "coarsened_grid",
                         "coarsened_ratio", "coarsened_GBps"], "rows": rows}

    sides.run("c2_main", main_rows)
    sides.run("c2_operators", operators)
    sides.run("c2_zero_run", zero_run)
    sides.run("c2_default_1d", default_1d)
    if not args.no_grid_init:
        sides.run("c2_grid_init", grid_init)
    plan.close()


def side_c4(mcc, dev, flush, stream, args):
    """Many variables x timesteps on one mesh: 1M-vertex 2D mesh, 4 variables
    x 64 timesteps of advected Gaussian bumps (FP64), per-variable rel bounds
    1e-6, 1e-4, 1e-3, 1e-2; R and C per variable from the autotuner; every
    variable's 64 fields in one batched compress + decompress chain, all four
    in one CUDA graph; against the same fields one call at a time."""
    import torch
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
    tuned, prms = [], []
    launch_table = []
    for v in range(nvars):
        # R and C per variable; the plan's launch configuration (shared by
        # the variables) from the 1e-4 variable's first timestep
        best, _ = autotune.tune(plan, fields[v][0], dict(dtype=mcc.F64, eb=ebs[v]),
                                launch=v == 1)
        if v == 1:
            launch_table = autotune.tune.launch_table
        tuned.append(best)
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
                raise RuntimeError("batched c4 line: bound violated")
        sizes.append(sz)

    def bstep():
        for v in range(nvars):
            mcc.compress_batch(plan, fields[v], [prms[v]] * nsteps, wscs[v], outs[v], slots[v],
                               sync=False)
            mcc.decompress_batch(plan, outs[v], slots[v], [slots[v]] * nsteps, ys[v], wsds[v],
                                 sync=False)

    # fields per launch chain: timed on the 1e-4 variable's 64 timesteps
    chain_table = autotune.tune_batch(plan, fields[1], [prms[1]] * nsteps, chains=(0, 8, 16, 64))
    reps = max(3, args.steps // 10)
    bms = time_replays(bstep, flush, reps, args.warmup, stream)
    # the same step recorded by the library's own graph API (mcc_graph_*) on a
    # second stream and replayed through mcc_graph_launch
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)

    def bstep_on(s_):
        for v in range(nvars):
            mcc.compress_batch(plan, fields[v], [prms[v]] * nsteps, wscs[v], outs[v], slots[v],
                               sync=False, stream=s_)
            mcc.decompress_batch(plan, outs[v], slots[v], [slots[v]] * nsteps, ys[v], wsds[v],
                                 sync=False, stream=s_)

    graph = mcc.graph_capture(lambda: bstep_on(gs), gs)
    for _ in range(args.warmup):
        graph.launch(gs)
    gms = []
    for k in range(reps):
        flush.fill_(k & 0xFF)
        gs.wait_stream(stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(gs)
        graph.launch(gs)
        b.record(gs)
        b.synchronize()
        gms.append(a.elapsed_time(b))
    graph.close()
    lms = statistics.mean(gms)
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
                       "rel 1e-6/1e-4/1e-3/1e-2",
           "fields": nvars * nsteps, "ms_per_step": bms, "GBps": rate(total, bms),
           "library_graph_GBps": rate(total, lms),
           "launch_tuning": [list(r) for r in launch_table],
           "chain_tuning": [list(r) for r in chain_table],
           "launch_chosen": list(mcc.get_tuning(plan)),
           "one_call_per_field_GBps": rate(total, sms),
           "per_var": [[ebs[v], tuned[v]["R1"], tuned[v]["C1"], nsteps * n * 8 / sum(sizes[v])]
                       for v in range(nvars)], "per_var_cols": ["eb_rel", "R", "C", "ratio"]}
    plan.close()
    return res


def measure_e2e(mcc, F, x_host, flush, steps, warmup, world, nlanes=2):
    """End to end through the API with host buffers (pinned), `nlanes` fields
    in flight: steps rotate over that many streams, each with its own device
    buffers and workspaces, so one step's copies (on the copy engines) and
    host-side size read overlap the others' kernels. Every step copies its field in, compresses
    (the stream size is read back on that step's stream), copies the stream
    out and back in, decompresses and copies the values out. Returns (ms per
    step over the timed steps, h2d bytes, d2h bytes per step)."""
    import torch
    plan, prm = F.plan, F.prm
    lanes = []
    for _ in range(nlanes):
        lanes.append(dict(
            s=torch.cuda.Stream(), x=torch.empty_like(F.x), out=torch.empty_like(F.out),
            inb=torch.empty_like(F.out), y=torch.empty_like(F.x),
            wsc=plan.workspace(prm, "compress"), wsd=plan.workspace(prm, "decompress"),
            out_host=torch.empty(F.cap, dtype=torch.uint8).pin_memory(),
            y_host=torch.empty_like(x_host).pin_memory()))
    h2d = d2h = 0

    def one(L):
        nonlocal h2d, d2h
        s = L["s"]
        with torch.cuda.stream(s):
            L["x"].copy_(x_host, non_blocking=True)
            mcc.compress(plan, L["x"], prm, L["wsc"], L["out"], sync=False, stream=s)
            st, n_out = mcc.workspace_result(L["wsc"], stream=s)  # waits for this stream only
            if st != 0:
                raise SystemExit(f"e2e: compression status {st}")
            L["out_host"][:n_out].copy_(L["out"][:n_out], non_blocking=True)
            L["inb"][:n_out].copy_(L["out_host"][:n_out], non_blocking=True)
            mcc.decompress(plan, L["inb"], n_out, L["y"], L["wsd"], sync=False, stream=s)
            L["y_host"].copy_(L["y"], non_blocking=True)
        h2d = x_host.numel() * x_host.element_size() + n_out
        d2h = n_out + L["y_host"].numel() * L["y_host"].element_size()

    for k in range(max(warmup, nlanes)):
        one(lanes[k % nlanes])
    torch.cuda.synchronize()
    flush.fill_(1)  # the fields and streams are larger than L2 together; one flush up front
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for k in range(steps):
        one(lanes[k % nlanes])
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    barrier(world)
    for L in lanes:
        if not torch.equal(L["y_host"], F.y.cpu()):
            raise SystemExit("e2e mismatch")
    return ms, h2d, d2h


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mcc", choices=["mcc", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--layers", type=int, default=None,
                    help="3D annulus cut to its bottom node layers (a small profiling case)")
    ap.add_argument("--eb", type=float, default=1e-4)
    ap.add_argument("--zero-run", action="store_true", help="headline with the zero-run stage")
    ap.add_argument("--side", default="all",
                    help="comma list of side lines (bounds,batched,split,learned,c2,c4), "
                         "'all' or 'none'")
    ap.add_argument("--side-out", default=None, help="also write the side lines to this file")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-lanes", type=int, default=2,
                    help="steps in flight in the end-to-end measurement (streams)")
    ap.add_argument("--no-kernel-times", action="store_true")
    ap.add_argument("--no-grid-init", action="store_true")
    ap.add_argument("--preroll", type=float, default=0.5, help="seconds of untimed steps")
    ap.add_argument("--batch", type=int, default=16, help="fields per step of the batched line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    import paper_2501_06910_gb300 as mcc

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    coords, cells, n = load_mesh(args.config, args.layers)
    n_cells = int(cells.shape[0])
    cd = torch.from_numpy(coords).to(dev)
    ed = torch.from_numpy(cells).to(dev)
    del cells
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = mcc.plan_create(cd, ed, n)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    del ed
    x = field_on_device(args.config, coords, cd)
    prm = mcc.params_default(dtype=mcc.F64, eb=args.eb, grid_fraction=0.5,
                             zero_run=1 if args.zero_run else 0)
    F = Field(mcc, plan, x, prm)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.fill_(1)
        F.step()
    st, _ = mcc.workspace_result(F.wsc)
    st2, _ = mcc.workspace_result(F.wsd)
    if st != 0 or st2 != 0:
        raise SystemExit(f"device status {st}/{st2}")
    size, err_over_tau = F.check(args.eb, "headline")
    g_bytes, _ = component_bytes(F.out[:208].cpu().numpy())  # the grid component's share
    y_ref = F.y.clone()

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        F.step()
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        flush.fill_(1)
        graph.replay()
    F.y.zero_()
    graph.replay()
    torch.cuda.synchronize()
    if not torch.equal(F.y, y_ref):
        raise SystemExit("graph replay differs from the eager step")

    # timed region: K steps, each bracketed by events, L2 flushed before each
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        t_end = time.perf_counter() + args.preroll
        while time.perf_counter() < t_end:  # pre-roll under the same load
            flush.fill_(3)
            graph.replay()
            torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            graph.replay()
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
    ms = max_over_ranks(statistics.mean(s.elapsed_time(e) for s, e in zip(starts, ends)), world, dev)
    clocks = clk.summary()
    del graph

    prof = {} if args.no_kernel_times else kernel_times(mcc, F.step, flush, args.steps)

    e2e = None
    if not args.no_e2e:
        x_host = x.cpu().pin_memory()
        e_ms, h2d, d2h = measure_e2e(mcc, F, x_host, flush, args.steps, args.warmup, world,
                                     args.e2e_lanes)
        e_ms = max_over_ranks(e_ms, world, dev)
        e2e = {"value": job_value(world, x.numel() * 8, e_ms), "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e_ms,
               "how": "pinned host field in, compress, stream out and in, decompress, "
                      f"values out; C-ABI calls, {args.e2e_lanes} steps in flight"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.config, args.eb)

    sides = Sides(args.side_out)
    want = set() if args.side == "none" or world > 1 else (
        {"bounds", "batched", "split", "learned", "c2", "c4"} if args.side == "all"
        else set(args.side.split(",")))
    if "bounds" in want:
        sides.run("bounds", side_bounds, mcc, plan, x, flush, stream, args)
    if "batched" in want and args.batch > 1:
        sides.run("batched", side_batched, mcc, plan, x, flush, stream, args, world)
    if args.config == "c3":
        if "split" in want:
            sides.run("split_sweep_c3", side_split, mcc, plan, cd, flush, stream, args)
        if "learned" in want:
            sides.run("learned_c5", side_learned, mcc, plan, cd, flush, stream, args)
    del F
    plan.close()
    torch.cuda.empty_cache()
    if "c2" in want and args.config != "c2":
        side_c2(mcc, dev, flush, stream, args, sides)
    if "c4" in want:
        sides.run("c4_vars_x_steps", side_c4, mcc, dev, flush, stream, args)
    sides.write()

    if rank == 0:
        peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
        nbytes = x.numel() * 8
        alg = algorithmic_bytes(len(n), x.numel(), int(np.prod(n)), 8, size, g_bytes, tuple(prof))
        wname = WORKLOADS[args.config] if not args.layers else \
            f"3d-annulus-slab-{args.layers}-layers-grid{n[0]}x{n[1]}x{n[2]}-f64"
        config = {"workload": wname, "n_vertices": int(x.numel()),
                  "n_cells": n_cells, "grid": list(n), "eb_rel": args.eb, "grid_fraction": 0.5,
                  "zero_run": bool(args.zero_run), "compression_ratio": nbytes / size,
                  "stream_bytes": int(size), "max_abs_err_over_tau": err_over_tau,
                  "plan_s": t_plan,
                  "l2": "flushed before every step (256 MiB write + 256 MiB read, untimed)",
                  "cuda_graph": True, "parallelism": f"replicas x{world}"}
        line = build_headline(world=world, steps=args.steps, warmup=args.warmup, ms=ms,
                              nbytes=nbytes, config=config, prof=prof, alg=alg, peaks=peaks,
                              cpu=cpu, e2e=e2e, clocks=clocks, traffic=dram_traffic)
        if line.get("kernels_us"):  # the whole table, on its own line
            print(json.dumps({"side": "kernels_us", "kernels_us": line["kernels_us"]},
                             allow_nan=False, separators=(",", ":")), flush=True)
        print(headline_json(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
