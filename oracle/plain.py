"""The method's definition in plain FP64 (numpy), beside the oracle's
production arithmetic, for Gong et al., "A General Framework for
Error-controlled Unstructured Scientific Data Compression" (Sec. III, IV;
Algorithms 3 and 4).

TEST INFRASTRUCTURE ONLY. Only ``tests/`` and the oracle's own scripts use
this module; it never imports the CUDA library. It restates, with no blocking,
fusion or reordering, what the oracle's C code computes through fixed-point
and reduced-precision shortcuts:

  point location   every grid point P = lo + i h tested against every
                   simplex (brute force, no single-precision pre-filter):
                   barycentric coordinates by Cramer's rule on the edge
                   vectors from the first vertex, inside when every
                   coordinate is >= -1e-12, the smallest simplex id owns P.
  f (Sec. IV-D)    x1[j] = sum_k lam_jk x[v_jk], FP64 weights on the values
                   (not the codes), summed left to right; points outside the
                   mesh take the fill value (zero clamped to [min x, max x]).
  C(x1)            q1 = rint((x1 - x_min) / (2 tau1)), x1' = x_min + 2 tau1 q1.
  g (Sec. III)     bilinear / trilinear interpolation of x1' at each vertex:
                   t_d = (p_d - lo_d) / h_d, cell i_d = clamp(floor t_d, 0,
                   n_d - 2), local coordinate f_d = clamp(t_d - i_d, 0, 1),
                   corner weights prod_d (f_d or 1 - f_d), corners in the
                   order 000, 100, 010, 110, 001, 101, 011, 111 (x fastest).
  C(x2)            q2 = rint((x - g) / (2 tau2)), x' = g + 2 tau2 q2.

Each of the oracle's readings can be switched on one at a time
(``Readings``), so a test can bound the distance each one adds, element by
element, and a script can measure what each costs in compressed size.
"""
from __future__ import annotations

import dataclasses

import numpy as np

TOL_INSIDE = 1e-12


# --------------------------------------------------------------------------- #
# grid
# --------------------------------------------------------------------------- #
def grid_points(lo, h, n):
    """Coordinates of every grid point, P = lo + i h per axis (FP64; the
    product i h rounded, then the sum), in the array order x fastest.
    Returns [n_g, dim]."""
    dim = len(n)
    axes = [np.float64(lo[d]) + np.arange(n[d], dtype=np.float64) * np.float64(h[d])
            for d in range(dim)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")  # [z][y][x] / [y][x]
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


# --------------------------------------------------------------------------- #
# point location, brute force (Sec. IV-C; the minimum simplex id on ties)
# --------------------------------------------------------------------------- #
def barycentric(P, V):
    """Barycentric coordinates of points P [m, dim] in simplices V [m, dim+1,
    dim] (FP64): Cramer's rule on the edge vectors from V[:, 0]. 2D:
    den = v0x v1y - v1x v0y, lb = (v2x v1y - v1x v2y) / den,
    lc = (v0x v2y - v2x v0y) / den, la = (1 - lb) - lc. 3D: with c = v1 x v2,
    den = v0 . c, lb = vp . (v1 x v2) / den, lc = v0 . (vp x v2) / den,
    ld = v0 . (v1 x vp) / den, la = ((1 - lb) - lc) - ld; every product and
    sum rounded in this order. Returns (lam [m, dim+1], den [m])."""
    A = V[:, 0]
    dim = P.shape[1]
    if dim == 2:
        v0x, v0y = V[:, 1, 0] - A[:, 0], V[:, 1, 1] - A[:, 1]
        v1x, v1y = V[:, 2, 0] - A[:, 0], V[:, 2, 1] - A[:, 1]
        v2x, v2y = P[:, 0] - A[:, 0], P[:, 1] - A[:, 1]
        den = v0x * v1y - v1x * v0y
        with np.errstate(divide="ignore", invalid="ignore"):
            lb = (v2x * v1y - v1x * v2y) / den
            lc = (v0x * v2y - v2x * v0y) / den
        la = (1.0 - lb) - lc
        return np.stack([la, lb, lc], axis=1), den

    def cross(u, w):
        return np.stack([u[:, 1] * w[:, 2] - u[:, 2] * w[:, 1],
                         u[:, 2] * w[:, 0] - u[:, 0] * w[:, 2],
                         u[:, 0] * w[:, 1] - u[:, 1] * w[:, 0]], axis=1)

    def dot(u, w):
        return (u[:, 0] * w[:, 0] + u[:, 1] * w[:, 1]) + u[:, 2] * w[:, 2]

    v0, v1, v2 = V[:, 1] - A, V[:, 2] - A, V[:, 3] - A
    vp = P - A
    c = cross(v1, v2)
    den = dot(v0, c)
    nb = dot(vp, c)
    nc = dot(v0, cross(vp, v2))
    nd = dot(v0, cross(v1, vp))
    with np.errstate(divide="ignore", invalid="ignore"):
        lb, lc, ld = nb / den, nc / den, nd / den
    la = ((1.0 - lb) - lc) - ld
    return np.stack([la, lb, lc, ld], axis=1), den


def locate_brute(coords, cells, P):
    """For every point of P [n_g, dim]: the smallest id of a simplex holding
    it (every barycentric coordinate >= -1e-12, non-degenerate), or -1, and
    its barycentric coordinates (zeros outside). Tests every (point, simplex)
    pair: tiny meshes only."""
    coords = np.asarray(coords, np.float64)
    cells = np.asarray(cells, np.int64)
    n_g, dim = P.shape
    owner = np.full(n_g, -1, np.int64)
    lam = np.zeros((n_g, dim + 1))
    for t in range(cells.shape[0]):  # increasing id: the first hit is the minimum
        free = np.nonzero(owner < 0)[0]
        if free.size == 0:
            break
        V = np.broadcast_to(coords[cells[t]], (free.size, dim + 1, dim))
        l, den = barycentric(P[free], V)
        hit = (den != 0.0) & np.all(l >= -TOL_INSIDE, axis=1)
        owner[free[hit]] = t
        lam[free[hit]] = l[hit]
    return owner, lam


# --------------------------------------------------------------------------- #
# the readings of the oracle's production arithmetic, one switch each
# --------------------------------------------------------------------------- #
@dataclasses.dataclass(frozen=True)
class Readings:
    """Which of the oracle's readings to apply (all False = the plain
    definition above):
      u16_weights  barycentric weights rounded to 2^-15 units (the first one
                   implied: x1 = x_a + sum_{k>=1} lam_k (x_k - x_a));
      f_on_codes   f interpolates the vertex codes Q = rint(x / s2) - K (in
                   value units s2 (Q + K)) instead of x;
      u16_local    local coordinates rounded to 2^-15 units;
      shrunk_bins  bins 2 tau (1 - 2^-20) instead of 2 tau;
      dual         residual codes in dual form q2 = Q - rint(g / s2 - K)
                   instead of rint((x - g) / s2), and the grid codes offset
                   by K s2 (the vertex codes' origin) instead of x_min."""
    u16_weights: bool = False
    f_on_codes: bool = False
    u16_local: bool = False
    shrunk_bins: bool = False
    dual: bool = False

    @staticmethod
    def production():
        return Readings(True, True, True, True, True)


def bounds(x, eb, grid_fraction=0.5, rel=True):
    """tau = eb (absolute) or eb (max x - min x) (relative; a constant field
    uses eb); tau1 = f tau, tau2 = (1 - f) tau."""
    lo, hi = float(np.min(x)), float(np.max(x))
    tau = eb * (hi - lo) if rel and hi > lo else eb
    return tau, grid_fraction * tau, (1.0 - grid_fraction) * tau


def u16(v):
    """Clamp to [0, 1] and round to 2^-15 units (ties to even)."""
    return np.rint(np.clip(v, 0.0, 1.0) * 32768.0) / 32768.0


def f_interp(x_at_vertices, vid, lam64, readings):
    """f at every grid point inside the mesh: sum_k lam_k x[v_k] (FP64,
    left to right), or, with u16 weights, x[v_0] + sum_{k>=1} u16(lam_k)
    (x[v_k] - x[v_0]). vid, lam64: [(dim+1), n_g] with vid[0] < 0 outside
    (returned as NaN there)."""
    k1 = vid.shape[0]
    inside = vid[0] >= 0
    vv = np.where(inside, vid, 0)
    xs = [x_at_vertices[vv[k]] for k in range(k1)]
    if readings.u16_weights:
        acc = xs[0].copy()
        for k in range(1, k1):
            acc = acc + u16(lam64[k]) * (xs[k] - xs[0])
    else:
        acc = lam64[0] * xs[0]
        for k in range(1, k1):
            acc = acc + lam64[k] * xs[k]
    return np.where(inside, acc, np.nan)


def local_coords(coords, lo, h, n):
    """Per vertex: the lower corner index per axis i_d = clamp(floor(t_d), 0,
    n_d - 2) and the local coordinate f_d = clamp(t_d - i_d, 0, 1),
    t_d = (p_d - lo_d) / h_d (FP64)."""
    coords = np.asarray(coords, np.float64)
    dim = coords.shape[1]
    idx = np.empty((coords.shape[0], dim), np.int64)
    fr = np.empty((coords.shape[0], dim))
    for d in range(dim):
        t = (coords[:, d] - lo[d]) / h[d]
        i = np.clip(np.floor(t), 0, n[d] - 2).astype(np.int64)
        idx[:, d] = i
        fr[:, d] = np.clip(t - i, 0.0, 1.0)
    return idx, fr


def g_interp(x1p, n, idx, fr):
    """Bilinear / trilinear interpolation of the grid values x1p (flat, x
    fastest) at every vertex: sum over the corners in the order 000, 100,
    010, 110 (, 001, 101, 011, 111) of prod_d (f_d or 1 - f_d) times the
    corner value, left to right (FP64)."""
    dim = len(n)
    out = np.zeros(idx.shape[0])
    for corner in range(1 << dim):
        w = np.ones(idx.shape[0])
        j = np.zeros(idx.shape[0], np.int64)
        stride = 1
        for d in range(dim):
            b = (corner >> d) & 1
            w = w * (fr[:, d] if b else (1.0 - fr[:, d]))
            j = j + (idx[:, d] + b) * stride
            stride *= n[d]
        out = out + w * x1p[j]
    return out


def compress_codes(x, plan, eb, grid_fraction=0.5, readings=Readings(), vertex_coords=None):
    """The method on one field with the given readings (closed loop: the
    residual is taken against g of the DECOMPRESSED grid). ``plan`` supplies
    the grid (lo, h, n) and the point location (vid, lam64: FP64 weights
    from the plain barycentric solve; the oracle's tables, pinned against
    ``locate_brute``); ``vertex_coords`` the mesh coordinates for the local
    coordinates. Returns a dict: x1 (f, NaN outside), q1 (grid codes), x1p
    (decompressed grid values), g (at the vertices), q2 (residual codes),
    xr (reconstruction), s1, s2, tau1, tau2, off (grid code origin)."""
    x = np.asarray(x, np.float64)
    tau, tau1, tau2 = bounds(x, eb, grid_fraction)
    shrink = (1.0 - 2.0 ** -20) if readings.shrunk_bins else 1.0
    s1 = (2.0 * tau1) * shrink
    s2 = (2.0 * tau2) * shrink
    lo_x, hi_x = float(x.min()), float(x.max())
    K = float(np.rint(lo_x * (1.0 / s2))) if readings.f_on_codes or readings.dual else 0.0
    if readings.f_on_codes:
        Q = np.rint(x * (1.0 / s2)) - K
        xin = s2 * (Q + K)
    else:
        xin = x
    g_plan = plan.grid
    dim = plan.dim
    n, glo, gh = tuple(g_plan.n[:dim]), g_plan.lo[:dim], g_plan.h[:dim]
    x1 = f_interp(xin, plan.vid, plan.lam64, readings)
    fill = min(max(0.0, lo_x), hi_x)
    x1 = np.where(np.isnan(x1), fill, x1)
    off = K * s2 if readings.dual else lo_x
    q1 = np.rint((x1 - off) / s1)
    x1p = off + s1 * q1
    idx, fr = local_coords(vertex_coords, glo, gh, n)
    if readings.u16_local:
        fr = u16(fr)
    g = g_interp(x1p, n, idx, fr)
    if readings.dual:
        Qv = np.rint(x * (1.0 / s2)) - K
        P = np.rint(g / s2 - K)
        q2 = Qv - P
        xr = s2 * (Qv + K)
    else:
        q2 = np.rint((x - g) / s2)
        xr = g + s2 * q2
    return dict(x1=x1, q1=q1, x1p=x1p, g=g, q2=q2, xr=xr, s1=s1, s2=s2, tau1=tau1, tau2=tau2,
                off=off, idx=idx, fr=fr)


def lorenzo(q, n):
    """N-D Lorenzo difference of a flat grid array (x fastest), zero outside:
    2D q(i,j) - q(i-1,j) - q(i,j-1) + q(i-1,j-1); 3D the 7-neighbour
    inclusion-exclusion."""
    a = np.asarray(q, np.int64).reshape(tuple(n[::-1]))
    p = np.pad(a, [(1, 0)] * a.ndim)
    if a.ndim == 2:
        d = p[1:, 1:] - p[1:, :-1] - p[:-1, 1:] + p[:-1, :-1]
    else:
        d = (p[1:, 1:, 1:] - p[1:, 1:, :-1] - p[1:, :-1, 1:] - p[:-1, 1:, 1:]
             + p[1:, :-1, :-1] + p[:-1, 1:, :-1] + p[:-1, :-1, 1:] - p[:-1, :-1, :-1])
    return d.ravel()


def coded_bits(values, R, lmax=24):
    """Bits of one component under the coder: symbols v + R for
    -(R-1) <= v <= R-2, else an escape (symbol 0) plus 32 bits for the value;
    an optimal length-limited prefix code over the symbol counts."""
    import oracle
    v = np.asarray(values, np.int64)
    esc = (v < -(R - 1)) | (v > R - 2)
    sym = np.where(esc, 0, v + R)
    counts = np.bincount(sym, minlength=2 * R).astype(np.uint64)
    lens = oracle.huffman_lengths(np.concatenate([counts, np.zeros(2, np.uint64)]), lmax)
    return int(np.sum(counts * lens[:2 * R].astype(np.uint64))) + 32 * int(esc.sum())
