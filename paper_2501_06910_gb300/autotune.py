"""Autotuner of one variable on one plan, in two stages:

1. the alphabet radius R (2R quantisation-code symbols per component) and the
   lane chunk C (symbols per lane of a 32-lane group), which are part of the
   stream: every candidate compresses a representative field (e.g. the
   first timestep) and the smallest stream wins, ties to the faster;
2. the plan's launch configuration, which is not part of the stream: the 2D
   grid kernel's tile (64 x 16, 32 x 32, 128 x 8) and the blocks per SM of
   the vertex-streaming kernels; every candidate times compress AND
   decompress of the field with the chosen R and C (median of the repeats,
   CUDA events on the stream) and the fastest is set on the plan;
3. (tune_batch) the fields per launch chain of the batched calls, timing a
   batched compress + decompress of the caller's fields.

Host logic over the C ABI; every compression and decompression runs in the
library's kernels, and the result of every candidate is checked against the
first one (the tuning never changes a stream or a decoded value)."""
from __future__ import annotations

import itertools
import statistics

import torch

from . import (TILE_128x8, TILE_32x32, TILE_64x16, compress, compress_batch, compress_bound,
               decompress, decompress_batch, get_tuning, params_default, set_tuning,
               workspace_size)

CANDIDATES = list(itertools.product((128, 512, 2048), (64, 128, 256)))
TILES = (TILE_64x16, TILE_32x32, TILE_128x8)
VERTEX_BLOCKS = (0, 4, 8, 16)  # 0: one full wave of resident blocks


def _time_round_trip(plan, x, prm, wsc, wsd, out, y, reps):
    """Median ms of `reps` compress + decompress round trips (no host sync
    inside a round trip)."""
    cap = out.numel()
    ms = []
    for _ in range(reps):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        compress(plan, x, prm, wsc, out, sync=False)
        decompress(plan, out, cap, y, wsd, sync=False)
        t1.record()
        torch.cuda.synchronize()
        ms.append(t0.elapsed_time(t1))
    return statistics.median(ms)


def tune(plan, x: torch.Tensor, base: dict, candidates=CANDIDATES, reps: int = 3,
         tiles=TILES, vertex_blocks=VERTEX_BLOCKS, launch: bool = True):
    """Returns (best parameter dict, table of (R, C, stream bytes, ms)); with
    ``launch`` also sets the fastest launch configuration on the plan and
    records its table as ``tune.launch_table`` rows (tile, blocks per SM, ms)."""
    table = []
    for R, C in candidates:
        kw = dict(base, R1=R, R2=R, C1=C, C2=C)
        prm = params_default(**kw)
        cws, _ = workspace_size(plan, prm)
        ws = torch.empty(cws, dtype=torch.uint8, device=x.device)
        out = torch.empty(compress_bound(plan, prm), dtype=torch.uint8, device=x.device)
        size = compress(plan, x, prm, ws, out)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            compress(plan, x, prm, ws, out, sync=False)
        t1.record()
        torch.cuda.synchronize()
        table.append((R, C, int(size), t0.elapsed_time(t1) / reps))
    best = min(table, key=lambda r: (r[2], r[3]))
    params = dict(base, R1=best[0], R2=best[0], C1=best[1], C2=best[1])
    tune.launch_table = []
    if launch:
        tune.launch_table = tune_launch(plan, x, params, reps=max(reps, 5), tiles=tiles,
                                        vertex_blocks=vertex_blocks)
    return params, table


def tune_launch(plan, x: torch.Tensor, params: dict, reps: int = 5, tiles=TILES,
                vertex_blocks=VERTEX_BLOCKS):
    """Time compress + decompress for every launch configuration, set the
    fastest on the plan; returns rows (tile, blocks per SM, ms). Raises if a
    configuration changes the stream or the decoded values."""
    prm = params_default(**params)
    cws, dws = workspace_size(plan, prm)
    wsc = torch.empty(cws, dtype=torch.uint8, device=x.device)
    wsd = torch.empty(dws, dtype=torch.uint8, device=x.device)
    out = torch.zeros(compress_bound(plan, prm), dtype=torch.uint8, device=x.device)
    y = torch.empty_like(x)
    dims = plan.dim
    bf = get_tuning(plan)[2]  # the batch chain length stays
    rows, ref = [], None
    for tile in (tiles if dims == 2 else tiles[:1]):  # the tile is a 2D kernel's
        for vb in vertex_blocks:
            set_tuning(plan, tile, vb, bf)
            size = compress(plan, x, prm, wsc, out)
            decompress(plan, out, size, y, wsd)
            got = (out[:size].clone(), y.clone())
            if ref is None:
                ref = got
            elif not (torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])):
                raise RuntimeError(f"launch configuration {tile}/{vb} changed the result")
            ms = _time_round_trip(plan, x, prm, wsc, wsd, out, y, reps)
            rows.append((tile, vb, ms))
    best = min(rows, key=lambda r: r[2])
    set_tuning(plan, best[0], best[1], bf)
    assert get_tuning(plan) == (best[0], best[1], bf)
    return rows


def tune_batch(plan, xs, params, chains=(0, 1, 4, 16, 64), reps: int = 3):
    """Time a batched compress + decompress of the fields ``xs`` (with the
    parameter structures ``params``) for every fields-per-chain candidate (0:
    the library's L2 rule), set the fastest on the plan; returns rows
    (batch_fields, ms). Raises if a candidate changes a stream or a value."""
    n = len(xs)
    cws = max(workspace_size(plan, p)[0] for p in params)
    dws = max(workspace_size(plan, p)[1] for p in params)
    slot = (max(compress_bound(plan, p) for p in params) + 7) // 8 * 8
    dev = xs[0].device
    chain_max = min(max(chains), n)
    wsc = torch.empty(cws * chain_max, dtype=torch.uint8, device=dev)
    wsd = torch.empty(dws * chain_max, dtype=torch.uint8, device=dev)
    out = torch.zeros(slot * n, dtype=torch.uint8, device=dev)
    ys = [torch.empty_like(x) for x in xs]
    tile, vb, _ = get_tuning(plan)
    rows, ref = [], None
    for bf in chains:
        set_tuning(plan, tile, vb, bf)
        sizes = compress_batch(plan, xs, params, wsc, out, slot)
        decompress_batch(plan, out, slot, sizes, ys, wsd)
        got = (sizes, out.clone(), [y.clone() for y in ys])
        if ref is None:
            ref = got
        elif got[0] != ref[0] or not torch.equal(got[1], ref[1]) or \
                any(not torch.equal(a, b) for a, b in zip(got[2], ref[2])):
            raise RuntimeError(f"batch chain length {bf} changed the result")
        ms = []
        for _ in range(reps):
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            compress_batch(plan, xs, params, wsc, out, slot, sync=False)
            decompress_batch(plan, out, slot, [slot] * n, ys, wsd, sync=False)
            t1.record()
            torch.cuda.synchronize()
            ms.append(t0.elapsed_time(t1))
        rows.append((bf, statistics.median(ms)))
    best = min(rows, key=lambda r: r[1])
    set_tuning(plan, tile, vb, best[0])
    return rows
