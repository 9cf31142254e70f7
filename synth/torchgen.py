"""Device-side generators of the same synthetic fields as ``synth`` (PyTorch on
the GPU), for workloads too large to generate with numpy in a benchmark run
(hundreds of fields of millions of vertices).

Same formulas, same lattice hash (bit for bit: 64-bit wrapping arithmetic),
same random bump parameters (drawn with numpy from the same seeds); the
transcendental functions are the device's, so values may differ from the
numpy versions in the last bits. Like ``synth`` this module only produces
inputs and holds none of the compressor's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np
import torch

_GOLD = 0x9E3779B97F4A7C15
_MIX = 0xBF58476D1CE4E5B9


def _s64(u: int) -> int:
    """An unsigned 64-bit constant as the int64 with the same bits."""
    return u - (1 << 64) if u >= 1 << 63 else u


def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def hash_u01(*ints_and_seed) -> torch.Tensor:
    """The lattice hash of ``synth`` on int64 tensors -> float64 in [-1, 1)."""
    acc = None
    for k, v in enumerate(ints_and_seed):
        x = v if isinstance(v, torch.Tensor) else torch.tensor(int(v), dtype=torch.int64)
        t = x * _s64(_MIX + 2 * k + 1)
        acc = t if acc is None else acc ^ t
        acc = (acc ^ _srl(acc, 31)) * _s64(_GOLD)
        acc = acc ^ _srl(acc, 29)
    return _srl(acc, 11).to(torch.float64) * (2.0 / 2.0 ** 53) - 1.0


def value_noise(p: torch.Tensor, octaves: int, base_freq: float, persistence: float,
                seed: int) -> torch.Tensor:
    dim = p.shape[1]
    out = torch.zeros(p.shape[0], dtype=torch.float64, device=p.device)
    amp, freq = 1.0, base_freq
    for o in range(octaves):
        q = p * freq
        i0f = torch.floor(q)
        f = q - i0f
        i0 = i0f.to(torch.int64)
        w = f * f * (3.0 - 2.0 * f)
        acc = torch.zeros_like(out)
        for corner in range(1 << dim):
            wt = torch.ones_like(out)
            idx = []
            for d in range(dim):
                bit = (corner >> d) & 1
                wt = wt * (w[:, d] if bit else (1.0 - w[:, d]))
                idx.append(i0[:, d] + bit)
            acc += wt * hash_u01(*idx, seed * 1000 + o)
        out += amp * acc
        amp *= persistence
        freq *= 2.0
    return out


def field_vortex(coords: torch.Tensor, seed: int = 6) -> torch.Tensor:
    """Swirling vortex exp(-((r-0.65)/0.2)^2) sin(3 theta - pi z + 4 r) plus
    0.05 x 4-octave value noise (``synth.field_vortex`` on the device)."""
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    r = torch.sqrt(x * x + y * y)
    t = torch.atan2(y, x)
    psi = torch.exp(-(((r - 0.65) / 0.2) ** 2)) * torch.sin(3 * t - math.pi * z + 4 * r)
    return psi + 0.05 * value_noise(coords, 4, 2.0, 0.5, seed)


def fields_advected(coords: torch.Tensor, nvars: int = 4, nsteps: int = 64, seed: int = 8,
                    nbumps: int = 8):
    """``synth.fields_advected`` on the device: yields (var, step, values)."""
    rng = np.random.default_rng(seed)
    xy = coords[:, :2]
    for v in range(nvars):
        cen = rng.random((nbumps, 2))
        vel = rng.uniform(-0.3, 0.3, (nbumps, 2)) / nsteps
        sig = rng.uniform(0.03, 0.15, nbumps)
        amp = rng.standard_normal(nbumps)
        for s in range(nsteps):
            out = torch.zeros(coords.shape[0], dtype=torch.float64, device=coords.device)
            c = (cen + s * vel) % 1.0
            for k in range(nbumps):
                d2 = ((xy[:, 0] - c[k, 0]) ** 2 + (xy[:, 1] - c[k, 1]) ** 2)
                out += amp[k] * torch.exp(-d2 / (2 * sig[k] ** 2))
            yield v, s, out
