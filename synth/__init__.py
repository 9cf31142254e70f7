"""Seeded synthetic meshes and fields shaped like the workloads of Gong et al.,
"A General Framework for Error-controlled Unstructured Scientific Data
Compression" (Sec. V, Table I).

The paper's datasets (OpenFOAM airfoils, Nek5000 turbPipe, VKI blade) are not
available, so every input here is synthetic and seeded. This module only
PRODUCES inputs (vertex coordinates, simplex connectivity, vertex values); it
holds none of the compressor's arithmetic, and both the CPU oracle and the CUDA
library consume what it returns.

Workloads:
  * ``mesh2d_jittered``  -- jittered lattice in the unit square, Delaunay
    triangulated (the 20k-vertex 2D case).
  * ``mesh2d_graded``    -- points with density ~ exp(-4 |p - c|) around
    c = (0.3, 0.6), Delaunay triangulated (stands in for airfoil-large,
    1,994,776 vertices, Table I).
  * ``mesh3d_annulus``   -- a cylinder with an annular hole, structured
    (r, theta, z) hexahedra split into 5 tetrahedra each (stands in for the
    turbPipe / VKI 3D meshes).
  * fields: ``field_sincos``, ``field_bumps_noise``, ``field_vortex``,
    ``fields_advected``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "mesh2d_jittered",
    "mesh2d_graded",
    "mesh3d_annulus",
    "mesh3d_annulus_slab",
    "mesh2d_two_triangles",
    "field_sincos",
    "field_linear",
    "field_bumps_noise",
    "field_vortex",
    "fields_advected",
    "value_noise",
]


# --------------------------------------------------------------------------- #
# helpers
# --------------------------------------------------------------------------- #
def _morton2(ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0xFFFF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x55555555)
        return v

    return spread(ix) | (spread(iy) << np.uint64(1))


def _delaunay(points: np.ndarray) -> np.ndarray:
    """Delaunay triangles (int32, counter-clockwise not enforced).

    Points are handed to qhull in Morton order (about 2x faster for millions of
    points); the returned indices refer to the caller's order.
    """
    from scipy.spatial import Delaunay

    lo = points.min(axis=0)
    span = np.maximum(points.max(axis=0) - lo, 1e-300)
    k = np.minimum(((points - lo) / span * 65535.0).astype(np.int64), 65535)
    order = np.argsort(_morton2(k[:, 0], k[:, 1]), kind="stable")
    tri = Delaunay(points[order]).simplices
    return order[tri].astype(np.int32)


def _relabel(coords, cells, rng):
    """Shuffle vertex ids and cell order (meshes from files carry no locality
    guarantee, so the library must not rely on one)."""
    n = coords.shape[0]
    perm = rng.permutation(n)  # new id of old vertex i is inv[i]
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    coords = coords[perm]
    cells = inv[cells].astype(np.int32)
    cells = cells[rng.permutation(cells.shape[0])]
    return np.ascontiguousarray(coords), np.ascontiguousarray(cells)


# --------------------------------------------------------------------------- #
# meshes
# --------------------------------------------------------------------------- #
def mesh2d_jittered(nside: int = 142, jitter: float = 0.35, seed: int = 1):
    """Jittered ``nside x nside`` lattice in [0,1]^2, Delaunay triangulated.

    Interior points move by U(-jitter*h, +jitter*h) per axis; points on the
    square's edges only move along the edge, so the convex hull is the unit
    square. Returns (coords float64 [n,2], cells int32 [m,3]).
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / (nside - 1)
    g = np.arange(nside) * h
    X, Y = np.meshgrid(g, g, indexing="xy")
    p = np.stack([X.ravel(), Y.ravel()], axis=1)
    d = rng.uniform(-jitter * h, jitter * h, size=p.shape)
    on_x = (np.isclose(p[:, 0], 0.0)) | (np.isclose(p[:, 0], 1.0))
    on_y = (np.isclose(p[:, 1], 0.0)) | (np.isclose(p[:, 1], 1.0))
    d[on_x, 0] = 0.0
    d[on_y, 1] = 0.0
    p = np.clip(p + d, 0.0, 1.0)
    cells = _delaunay(p)
    return _relabel(p, cells, rng)


def mesh2d_graded(n: int = 2_000_000, center=(0.3, 0.6), rate: float = 4.0, seed: int = 3):
    """``n`` points in [0,1]^2 with density proportional to exp(-rate*|p-c|),
    drawn by rejection sampling, plus the 4 corners; Delaunay triangulated."""
    rng = np.random.default_rng(seed)
    c = np.asarray(center, dtype=np.float64)
    need = n - 4
    out = []
    got = 0
    while got < need:
        m = max(1024, int((need - got) * 3.2))
        p = rng.random((m, 2))
        r = np.sqrt(((p - c) ** 2).sum(axis=1))
        keep = rng.random(m) < np.exp(-rate * r)
        p = p[keep]
        out.append(p)
        got += p.shape[0]
    p = np.concatenate(out)[:need]
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    p = np.concatenate([corners, p])
    cells = _delaunay(p)
    return _relabel(p, cells, rng)


def mesh2d_two_triangles():
    """Unit square split along its diagonal into two triangles (hand case)."""
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    cells = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return coords, cells


def mesh3d_annulus(nr: int = 64, nth: int = 512, nz: int = 244, R: float = 1.0,
                   r0: float = 0.3, H: float = 2.0, jitter: float = 0.2, seed: int = 5):
    """Cylinder of radius ``R`` and height ``H`` with a coaxial hole of radius
    ``r0``; nodes on an (nr, nth, nz) structured grid in (r, theta, z)
    (theta periodic), jittered by U(+-jitter) of the local spacing (boundary
    nodes stay on their boundary surfaces), each hexahedron split into 5
    tetrahedra with alternating (checkerboard) orientation so faces match.
    Vertex and tetrahedron order are shuffled. Returns (coords float64 [n,3],
    cells int32 [m,4]).
    """
    rng = np.random.default_rng(seed)
    rr = np.linspace(r0, R, nr)
    th = np.arange(nth) * (2 * np.pi / nth)
    zz = np.linspace(0.0, H, nz)
    ir, it, iz = np.meshgrid(np.arange(nr), np.arange(nth), np.arange(nz), indexing="ij")
    ir = ir.ravel(); it = it.ravel(); iz = iz.ravel()
    dr = (R - r0) / (nr - 1)
    dth = 2 * np.pi / nth
    dz = H / (nz - 1)
    jr = rng.uniform(-jitter, jitter, ir.size) * dr
    jt = rng.uniform(-jitter, jitter, ir.size) * dth
    jz = rng.uniform(-jitter, jitter, ir.size) * dz
    jr[(ir == 0) | (ir == nr - 1)] = 0.0
    jz[(iz == 0) | (iz == nz - 1)] = 0.0
    r = rr[ir] + jr
    t = th[it] + jt
    z = zz[iz] + jz
    coords = np.stack([r * np.cos(t), r * np.sin(t), z], axis=1)

    def vid(a, b, c):
        return (a * nth + (b % nth)) * nz + c

    a, b, c = np.meshgrid(np.arange(nr - 1), np.arange(nth), np.arange(nz - 1), indexing="ij")
    a = a.ravel(); b = b.ravel(); c = c.ravel()
    v = [vid(a + (k & 1), b + ((k >> 1) & 1), c + ((k >> 2) & 1)) for k in range(8)]
    # hexahedron corners v[k], k = bit0 (r) | bit1 (theta) | bit2 (z)
    even = ((a + b + c) & 1) == 0
    # 5-tet split: a central tet plus 4 corner tets; the two parities use the
    # two complementary central tets so neighbouring hexes share face diagonals.
    split_even = [(0, 1, 2, 4), (1, 3, 2, 7), (1, 4, 5, 7), (2, 4, 7, 6), (1, 2, 4, 7)]
    split_odd = [(0, 1, 3, 5), (0, 3, 2, 6), (0, 4, 5, 6), (3, 5, 6, 7), (0, 3, 5, 6)]
    tets = []
    for s_even, s_odd in zip(split_even, split_odd):
        te = np.stack([v[i] for i in s_even], axis=1)
        to = np.stack([v[i] for i in s_odd], axis=1)
        tets.append(np.where(even[:, None], te, to))
    cells = np.concatenate(tets).astype(np.int32)
    return _relabel(coords, cells, rng)


def mesh3d_annulus_slab(layers: int = 17, nz_full: int = 244, H_full: float = 2.0,
                        seed: int = 5):
    """The bottom ``layers`` node layers of ``mesh3d_annulus(nz=nz_full,
    H=H_full)``: the same radial / angular resolution and the same z spacing,
    jitter and tetrahedral split, over a height of H_full (layers - 1) /
    (nz_full - 1). A bounded sample of the 3D workload with its structure
    (a CPU-sized piece of the same mesh shape). Returns (coords, cells)."""
    H = H_full * (layers - 1) / (nz_full - 1)
    return mesh3d_annulus(nz=layers, H=H, seed=seed)


# --------------------------------------------------------------------------- #
# fields
# --------------------------------------------------------------------------- #
def _hash_u01(*ints_and_seed):
    """Deterministic lattice hash -> float64 in [-1, 1)."""
    h = np.uint64(0x9E3779B97F4A7C15)
    acc = np.zeros(np.broadcast(*ints_and_seed).shape, dtype=np.uint64)
    for k, v in enumerate(ints_and_seed):
        x = np.asarray(v).astype(np.int64).astype(np.uint64)
        acc = acc ^ (x * np.uint64(0xBF58476D1CE4E5B9 + 2 * k + 1))
        acc = (acc ^ (acc >> np.uint64(31))) * h
        acc = acc ^ (acc >> np.uint64(29))
    return (acc >> np.uint64(11)).astype(np.float64) * (2.0 / 2.0 ** 53) - 1.0


def value_noise(p: np.ndarray, octaves: int, base_freq: float, persistence: float,
                seed: int) -> np.ndarray:
    """Fractal value noise: hashed lattice values, smoothstep-interpolated,
    summed over ``octaves`` with frequency doubling and amplitude x persistence."""
    p = np.asarray(p, dtype=np.float64)
    dim = p.shape[1]
    out = np.zeros(p.shape[0])
    amp = 1.0
    freq = base_freq
    for o in range(octaves):
        q = p * freq
        i0 = np.floor(q).astype(np.int64)
        f = q - i0
        w = f * f * (3.0 - 2.0 * f)
        acc = np.zeros(p.shape[0])
        for corner in range(1 << dim):
            wt = np.ones(p.shape[0])
            idx = []
            for d in range(dim):
                bit = (corner >> d) & 1
                wt = wt * (w[:, d] if bit else (1.0 - w[:, d]))
                idx.append(i0[:, d] + bit)
            acc += wt * _hash_u01(*idx, np.int64(seed * 1000 + o))
        out += amp * acc
        amp *= persistence
        freq *= 2.0
    return out


def field_linear(coords: np.ndarray, a: float = 0.25, b=(1.5, -0.75, 0.5)) -> np.ndarray:
    """a + b . p (exact linear field)."""
    b = np.asarray(b[: coords.shape[1]], dtype=np.float64)
    return a + coords @ b


def field_sincos(coords: np.ndarray, seed: int = 2, noise: float = 0.01) -> np.ndarray:
    """sin(4 pi x) cos(3 pi y) + noise * N(0, 1)."""
    rng = np.random.default_rng(seed)
    x, y = coords[:, 0], coords[:, 1]
    return np.sin(4 * np.pi * x) * np.cos(3 * np.pi * y) + noise * rng.standard_normal(x.size)


def field_bumps_noise(coords: np.ndarray, seed: int = 4, nbumps: int = 20) -> np.ndarray:
    """Sum of ``nbumps`` Gaussian bumps (centres U[0,1]^2, sigma U[0.01,0.2],
    amplitudes N(0,1)) plus 6-octave value noise (base frequency 4,
    persistence 0.5, amplitude 0.3)."""
    rng = np.random.default_rng(seed)
    cen = rng.random((nbumps, 2))
    sig = rng.uniform(0.01, 0.2, nbumps)
    amp = rng.standard_normal(nbumps)
    out = np.zeros(coords.shape[0])
    for k in range(nbumps):
        d2 = ((coords[:, :2] - cen[k]) ** 2).sum(axis=1)
        out += amp[k] * np.exp(-d2 / (2 * sig[k] ** 2))
    out += 0.3 * value_noise(coords[:, :2], 6, 4.0, 0.5, seed)
    return out


def field_vortex(coords: np.ndarray, seed: int = 6) -> np.ndarray:
    """Swirling vortex exp(-((r-0.65)/0.2)^2) sin(3 theta - pi z + 4 r) plus
    0.05 x 4-octave value noise."""
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    r = np.sqrt(x * x + y * y)
    t = np.arctan2(y, x)
    psi = np.exp(-(((r - 0.65) / 0.2) ** 2)) * np.sin(3 * t - np.pi * z + 4 * r)
    return psi + 0.05 * value_noise(coords, 4, 2.0, 0.5, seed)


def fields_advected(coords: np.ndarray, nvars: int = 4, nsteps: int = 64, seed: int = 8,
                    nbumps: int = 8):
    """``nvars`` x ``nsteps`` fields of Gaussian bumps advected with constant
    per-bump velocities U(+-0.3)/nsteps per step. Yields (var, step, values)."""
    rng = np.random.default_rng(seed)
    xy = coords[:, :2]
    for v in range(nvars):
        cen = rng.random((nbumps, 2))
        vel = rng.uniform(-0.3, 0.3, (nbumps, 2)) / nsteps
        sig = rng.uniform(0.03, 0.15, nbumps)
        amp = rng.standard_normal(nbumps)
        for s in range(nsteps):
            out = np.zeros(coords.shape[0])
            c = (cen + s * vel) % 1.0
            for k in range(nbumps):
                d2 = ((xy - c[k]) ** 2).sum(axis=1)
                out += amp[k] * np.exp(-d2 / (2 * sig[k] ** 2))
            yield v, s, out
