"""Autotuner for the alphabet radius R (quantisation bins: 2R symbols) and the
lane chunk C (symbols per lane of a 32-lane group) of one variable: every
candidate compresses a representative field (e.g. the first timestep) and
the smallest stream wins; ties go to the faster candidate. Host logic over
the C ABI; every compression runs in the library's kernels."""
from __future__ import annotations

import itertools

import torch

from . import compress, compress_bound, params_default, workspace_size

CANDIDATES = list(itertools.product((128, 512, 2048), (64, 128, 256)))


def tune(plan, x: torch.Tensor, base: dict, candidates=CANDIDATES, reps: int = 3):
    """Returns (best parameter dict, table of (R, C, stream bytes, ms))."""
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
    return dict(base, R1=best[0], R2=best[0], C1=best[1], C2=best[1]), table
