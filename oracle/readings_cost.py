"""What each of the oracle's readings costs in compressed size, measured on
the benchmark workloads with the oracle and its plain FP64 definition layer.

TEST INFRASTRUCTURE ONLY (calls only ``oracle/`` and the seeded input
generators). Usage:

    python -m oracle.readings_cost [c2] [c3]

For each workload (FP64 field, rel 1e-4, grid / residual split 0.5, R = 512)
it prints the coded bits of the grid component (Lorenzo differences of the
grid codes) and of the residual component under the plain definition, then
with the readings switched on one after another (u16 weights, f on the
vertex codes, u16 local coordinates, bins shrunk by 2^-20, the dual
residual form), then the oracle's own stream; the compression ratio of each
adds the oracle stream's fixed part (header, code lengths, group tables).
"""
from __future__ import annotations

import sys
import time

import numpy as np

import oracle
import synth
from oracle import plain

R = 512


def symbol_bits(sym, R, raw_bits):
    """Coded bits of a symbol array as the oracle codes it: an optimal
    24-bit-limited prefix code over the symbol counts, plus 32 bits per
    escape (symbol 0) and raw_bits per raw value (symbol 2R - 1)."""
    counts = np.bincount(np.asarray(sym, np.int64), minlength=2 * R).astype(np.uint64)
    lens = oracle.huffman_lengths(np.concatenate([counts, np.zeros(2, np.uint64)]), 24)
    bits = int(np.sum(counts * lens[:2 * R].astype(np.uint64)))
    return bits + 32 * int(counts[0]) + raw_bits * int(counts[2 * R - 1])


def workload(name):
    if name == "c2":
        c, e = synth.mesh2d_graded()
        return "2D graded, 2M vertices, 1024^2", c, e, (1024, 1024), synth.field_bumps_noise(c)
    if name == "c3":
        c, e = synth.mesh3d_annulus()
        return "3D annulus, 8M vertices, 256^3", c, e, (256, 256, 256), synth.field_vortex(c)
    raise SystemExit(f"unknown workload {name}")


def run(name, eb=1e-4):
    label, c, e, n, x = workload(name)
    t0 = time.perf_counter()
    p = oracle.Plan(c, e, n)
    del e
    t_plan = time.perf_counter() - t0
    s, dbg = oracle.compress(p, x, debug=True, eb=eb)
    n_in = x.nbytes
    nn = p.grid.n[:p.dim]
    b1 = symbol_bits(dbg["sym1"], R, 0)
    b2 = symbol_bits(dbg["sym2"], R, 64)
    fixed = s.size - (b1 + b2) / 8.0  # header, code lengths, group / lane tables, padding
    rows = []
    steps = [("plain definition", plain.Readings()),
             ("+ u16 weights", plain.Readings(u16_weights=True)),
             ("+ f on vertex codes", plain.Readings(u16_weights=True, f_on_codes=True)),
             ("+ u16 local coordinates", plain.Readings(True, True, True)),
             ("+ bins shrunk by 2^-20", plain.Readings(True, True, True, True)),
             ("+ dual residual form (all readings, FP64)", plain.Readings.production())]
    for what, rd in steps:
        r = plain.compress_codes(x, p, eb, readings=rd, vertex_coords=c)
        g_bits = plain.coded_bits(plain.lorenzo(r["q1"], nn), R)
        r_bits = plain.coded_bits(r["q2"], R)
        rows.append((what, g_bits, r_bits, n_in / (fixed + (g_bits + r_bits) / 8.0),
                     float(np.max(np.abs(x - r["xr"])) / r["tau2"])))
    rows.append(("oracle stream (FP32 / 2^-40 arithmetic)", b1, b2, n_in / s.size, None))
    print(f"{label}: FP64, rel {eb:g}, split 0.5, plan {t_plan:.1f} s, stream {s.size} bytes "
          f"(fixed part {fixed:.0f})")
    base = rows[0][3]
    print(f"  {'reading':44s} {'grid bits':>12s} {'residual bits':>14s} {'ratio':>8s} "
          f"{'vs plain':>9s} {'err/tau2':>9s}")
    for what, g_bits, r_bits, ratio, err in rows:
        e_s = f"{err:9.4f}" if err is not None else " " * 9
        print(f"  {what:44s} {g_bits:12d} {r_bits:14d} {ratio:8.4f} {ratio / base - 1:+9.4%} {e_s}")
    return rows


if __name__ == "__main__":
    for w in (sys.argv[1:] or ["c2", "c3"]):
        run(w)
