"""The oracle's production arithmetic against the method's plain FP64
definition (``oracle/plain.py``), element by element.

The plain layer is pinned on its own first (brute-force point location with
no single-precision pre-filter; linear fields reproduced to 1e-12 relative;
the bound of each component). Then every reading of the oracle is bounded
against it with a tolerance derived from the reading alone:

  u16 weights   |dx1| <= 2^-16 sum_{k>=1} |x_k - x_0|          (+ FP64 rounding)
  f on codes    |dx1| <= s2 / 2                                 (+ FP64 rounding)
  u16 local     |dg|  <= 2^-16 sum_d |dg/df_d| <= 2^-16 D (max - min corner)
  shrunk bins   s = 2 tau (1 - 2^-20) exactly; both bounds hold
  FP32 / 2^-40  the oracle's grid and vertex codes equal rint of the FP64
                reading wherever that value is farther than the FP32 and
                fixed-point error bound from a rounding boundary
(Sec. III: the bound |x - x'| <= tau2 in closed loop; Sec. IV-D: f the
linear interpolation of the vertex values.)"""
import numpy as np
import pytest

import oracle
import synth
from oracle import plain

U64 = 2.0 ** -53


def _cases():
    c2, e2 = synth.mesh2d_jittered(nside=30, seed=3)
    g2, f2 = synth.mesh2d_graded(n=2500, seed=5)
    c3, e3 = synth.mesh3d_annulus(nr=6, nth=24, nz=6, seed=2)
    return [("jittered", c2, e2, (40, 36)), ("graded", g2, f2, (33, 31)),
            ("annulus", c3, e3, (14, 13, 12))]


CASES = _cases()


def _field(c):
    return synth.field_sincos(c[:, :2]) if c.shape[1] == 2 else synth.field_vortex(c)


def _plan(c, e, n):
    return oracle.Plan(c, e, n)


def _points(p):
    d = p.dim
    return plain.grid_points(p.grid.lo[:d], p.grid.h[:d], p.grid.n[:d])


# --------------------------------------------------------------------------- #
# the plain layer, pinned on its own
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("name,c,e,n", CASES, ids=[k[0] for k in CASES])
def test_brute_force_location_without_prefilter_equals_oracle(name, c, e, n):
    """Every (point, simplex) pair in FP64 with no pre-filter: the same owner
    (minimum id) and the same FP64 barycentric weights, bit for bit."""
    p = _plan(c, e, n)
    own, lam = plain.locate_brute(c, e, _points(p))
    assert np.array_equal(own, p.owner)
    ins = own >= 0
    assert ins.any() and np.array_equal(lam[ins].T, p.lam64[:, ins])


def test_brute_force_ties_go_to_the_smaller_simplex():
    """Points on the shared diagonal of two triangles belong to both; the
    smaller id owns them, also when the cell order is reversed."""
    coords, cells = synth.mesh2d_two_triangles()
    P = plain.grid_points((0.0, 0.0), (0.25, 0.25), (5, 5))
    diag = np.isclose(P[:, 0], P[:, 1])
    for order in ([0, 1], [1, 0]):
        own, _ = plain.locate_brute(coords, cells[order], P)
        assert np.all(own >= 0) and np.all(own[diag] == 0)
        l, _ = plain.barycentric(P[diag], np.broadcast_to(coords[cells[order][1]],
                                                          (diag.sum(), 3, 2)))
        assert np.all(l >= -plain.TOL_INSIDE)  # also inside the other triangle


@pytest.mark.parametrize("name,c,e,n", CASES, ids=[k[0] for k in CASES])
def test_plain_interpolations_reproduce_linear_fields_to_1e12(name, c, e, n):
    """f (barycentric, FP64 weights) at every inside grid point and g
    (multilinear, FP64 local coordinates) at every vertex reproduce a linear
    field a + b.p to 1e-12 relative."""
    p = _plan(c, e, n)
    b = np.array([1.5, -0.75, 0.5])[: p.dim]
    a = 0.25
    x = a + c @ b
    P = _points(p)
    x1 = plain.f_interp(x, p.vid, p.lam64, plain.Readings())
    ins = p.vid[0] >= 0
    exact = a + P @ b
    assert np.max(np.abs(x1[ins] - exact[ins]) / np.abs(exact[ins]).max()) <= 1e-12
    d = p.dim
    idx, fr = plain.local_coords(c, p.grid.lo[:d], p.grid.h[:d], p.grid.n[:d])
    g = plain.g_interp(exact, p.grid.n[:d], idx, fr)
    assert np.max(np.abs(g - x)) / np.abs(x).max() <= 1e-12


def test_plain_g_is_multilinear_and_a_partition_of_unity():
    """g of the field xy(z) on the grid nodes equals it at the vertices (the
    multilinear interpolant reproduces every multilinear function); g of
    the constant 1 is 1."""
    _, c, e, n = CASES[2]
    p = _plan(c, e, n)
    d = p.dim
    P = _points(p)
    idx, fr = plain.local_coords(c, p.grid.lo[:d], p.grid.h[:d], p.grid.n[:d])
    inside_box = np.all((c >= P.min(axis=0)) & (c <= P.max(axis=0)), axis=1)
    g = plain.g_interp(np.prod(P, axis=1), p.grid.n[:d], idx, fr)
    assert np.max(np.abs(g - np.prod(c, axis=1))[inside_box]) <= 1e-12
    one = plain.g_interp(np.ones(P.shape[0]), p.grid.n[:d], idx, fr)
    assert np.max(np.abs(one - 1.0)) <= 4 * U64


@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
@pytest.mark.parametrize("name,c,e,n", CASES, ids=[k[0] for k in CASES])
def test_plain_components_hold_their_bounds(name, c, e, n, eb):
    """Closed loop, plain definition: |x1 - x1'| <= tau1 at every grid point
    and |x - x'| <= tau2 at every vertex (up to the FP64 rounding of the
    quotient and the reconstruction, a few units in the last place)."""
    p = _plan(c, e, n)
    x = _field(c)
    r = plain.compress_codes(x, p, eb, readings=plain.Readings(), vertex_coords=c)
    M = np.abs(x).max() + r["tau1"]
    assert np.max(np.abs(r["x1"] - r["x1p"])) <= r["tau1"] + 8 * U64 * M
    assert np.max(np.abs(x - r["xr"])) <= r["tau2"] + 8 * U64 * M


# --------------------------------------------------------------------------- #
# each reading against the plain definition
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("name,c,e,n", CASES, ids=[k[0] for k in CASES])
def test_u16_weights_move_f_by_at_most_a_2_16_share_of_the_spread(name, c, e, n):
    p = _plan(c, e, n)
    x = _field(c)
    ins = p.vid[0] >= 0
    x0 = plain.f_interp(x, p.vid, p.lam64, plain.Readings())
    x1 = plain.f_interp(x, p.vid, p.lam64, plain.Readings(u16_weights=True))
    xs = [x[np.where(ins, p.vid[k], 0)] for k in range(p.dim + 1)]
    spread = sum(np.abs(xs[k] - xs[0]) for k in range(1, p.dim + 1))
    tol = 2.0 ** -16 * spread + 16 * U64 * np.abs(x).max()
    assert np.all(np.abs(x1 - x0)[ins] <= tol[ins])
    # the oracle's u16 table is exactly this rounding of the FP64 solve
    assert np.array_equal(p.lam.astype(np.float64) / 32768.0, plain.u16(p.lam64[1:]))


@pytest.mark.parametrize("name,c,e,n", CASES, ids=[k[0] for k in CASES])
def test_f_on_codes_moves_f_by_at_most_half_a_residual_bin(name, c, e, n):
    """Interpolating the vertex codes' values s2 (Q + K) instead of x: each
    vertex value moves by at most s2 / 2 and the weights are convex."""
    p = _plan(c, e, n)
    x = _field(c)
    for eb in (1e-2, 1e-4):
        r0 = plain.compress_codes(x, p, eb, readings=plain.Readings(), vertex_coords=c)
        r1 = plain.compress_codes(x, p, eb, readings=plain.Readings(f_on_codes=True),
                                  vertex_coords=c)
        ins = p.vid[0] >= 0
        tol = r1["s2"] / 2 + 16 * U64 * np.abs(x).max()
        assert np.max(np.abs(r1["x1"] - r0["x1"])[ins]) <= tol


@pytest.mark.parametrize("name,c,e,n", CASES, ids=[k[0] for k in CASES])
def test_u16_local_coordinates_move_g_by_at_most_2_16_of_the_corner_spread(name, c, e, n):
    p = _plan(c, e, n)
    x = _field(c)
    d = p.dim
    nn = p.grid.n[:d]
    idx, fr = plain.local_coords(c, p.grid.lo[:d], p.grid.h[:d], nn)
    r = plain.compress_codes(x, p, 1e-3, readings=plain.Readings(), vertex_coords=c)
    g0 = plain.g_interp(r["x1p"], nn, idx, fr)
    g1 = plain.g_interp(r["x1p"], nn, idx, plain.u16(fr))
    corners = []
    for corner in range(1 << d):
        j = np.zeros(c.shape[0], np.int64)
        stride = 1
        for a in range(d):
            j = j + (idx[:, a] + ((corner >> a) & 1)) * stride
            stride *= nn[a]
        corners.append(r["x1p"][j])
    corners = np.stack(corners)
    spread = corners.max(axis=0) - corners.min(axis=0)
    tol = 2.0 ** -16 * d * spread + 16 * U64 * np.abs(r["x1p"]).max()
    assert np.all(np.abs(g1 - g0) <= tol)
    # the oracle's table: the same rounding (t from the reciprocal spacing,
    # so a rare tie may land one unit away)
    assert np.max(np.abs(p.frac.astype(np.float64).T / 32768.0 - plain.u16(fr))) <= 2.0 ** -15


@pytest.mark.parametrize("name,c,e,n", CASES, ids=[k[0] for k in CASES])
def test_shrunk_bins_keep_both_bounds_with_a_margin(name, c, e, n):
    """Bins 2 tau (1 - 2^-20): the reconstruction error stays below
    tau2 (1 - 2^-20) + the FP64 rounding, and the oracle's field parameters
    carry exactly these bins."""
    p = _plan(c, e, n)
    x = _field(c)
    for eb in (1e-2, 1e-5):
        r = plain.compress_codes(x, p, eb, readings=plain.Readings(shrunk_bins=True, dual=True,
                                                                   f_on_codes=True),
                                 vertex_coords=c)
        fp = oracle.field_params(x, eb=eb)
        assert r["s1"] == fp["s1"] and r["s2"] == fp["s2"]
        assert fp["s2"] == (2.0 * fp["tau2"]) * (1.0 - 2.0 ** -20)
        M = np.abs(x).max()
        assert np.max(np.abs(x - r["xr"])) <= fp["tau2"] * (1 - 2.0 ** -20) + 4 * U64 * M


@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
@pytest.mark.parametrize("name,c,e,n", CASES, ids=[k[0] for k in CASES])
def test_oracle_codes_equal_the_fp64_readings_away_from_rounding_ties(name, c, e, n, eb):
    """The oracle's FP32 interpolation on integer code differences and its
    2^-40 fixed-point rescale give the grid codes q1 and the vertex
    predictions P = Q - q2 of the FP64 reading, except where the FP64 value
    lies within the FP32 / fixed-point error bound of a rounding boundary
    (there both neighbours are allowed)."""
    p = _plan(c, e, n)
    x = _field(c)
    _, dbg = oracle.compress(p, x, debug=True, eb=eb)
    fp = oracle.field_params(x, eb=eb)
    rd = plain.Readings.production()
    r = plain.compress_codes(x, p, eb, readings=rd, vertex_coords=c)
    s1, s2, K = r["s1"], r["s2"], fp["K"]
    # grid: u = (s2 / s1) (a + sum lam16_k d_k) in code units (exact integers
    # a, d_k; the FP32 sum errs by <= 4 2^-24 sum |lam d|, the ratio's 2^-40
    # quantisation by 2^-41 |a + acc|)
    ins = p.vid[0] >= 0
    Q = dbg["Q"].astype(np.float64)
    vv = np.where(ins, p.vid, 0)
    a = np.where(ins, Q[vv[0]], float(fp["fill_u"]))
    lam16 = p.lam.astype(np.float64) / 32768.0
    acc = sum(lam16[k - 1] * (Q[vv[k]] - Q[vv[0]]) for k in range(1, p.dim + 1))
    acc_abs = sum(lam16[k - 1] * np.abs(Q[vv[k]] - Q[vv[0]]) for k in range(1, p.dim + 1))
    acc = np.where(ins, acc, 0.0)
    acc_abs = np.where(ins, acc_abs, 0.0)
    u = (s2 / s1) * (a + acc)
    err = (s2 / s1) * (4 * 2.0 ** -24 * acc_abs) + 2.0 ** -41 * np.abs(a + acc) + \
        2.0 ** -24 * (np.abs(u - np.floor(u)) + 1) + 1e-9
    q1 = dbg["q1"].astype(np.float64)
    near = np.abs((u - np.floor(u)) - 0.5) <= err
    assert np.array_equal(q1[~near], np.rint(u[~near]))
    assert np.all(np.abs(q1[near] - u[near]) <= 0.5 + err[near])
    assert np.array_equal(np.rint(r["q1"]), q1) or near.any()
    # vertices: P = round((s1/s2) g(q1)) against the FP64 interpolation of the
    # grid codes at the u16 local coordinates (FP32 sum: 8 2^-24 of the
    # corner spread per term; a u16 tie may move a coordinate by 2^-15)
    R = 512
    sym2 = dbg["sym2"].astype(np.int64)
    plain_sym = (sym2 != 0) & (sym2 != 2 * R - 1)
    q2 = sym2 - R
    P_or = dbg["Q"].astype(np.int64) - q2
    d = p.dim
    nn = p.grid.n[:d]
    fr16 = p.frac.astype(np.float64).T / 32768.0
    cells = p.cell.astype(np.int64)
    idx = np.stack([(cells // int(np.prod(nn[:a]))) % nn[a] for a in range(d)], axis=1)
    gq = plain.g_interp(q1, nn, idx, fr16) * (s1 / s2)
    corner_spread = np.zeros(c.shape[0])
    cq = []
    for corner in range(1 << d):
        j = np.zeros(c.shape[0], np.int64)
        stride = 1
        for ax in range(d):
            j = j + (idx[:, ax] + ((corner >> ax) & 1)) * stride
            stride *= nn[ax]
        cq.append(q1[j])
    cq = np.stack(cq)
    corner_spread = (cq.max(axis=0) - cq.min(axis=0)) * (s1 / s2)
    # the oracle's own u16 local coordinates are used on both sides, so only
    # the FP32 products and sums (and integer differences beyond 2^24) differ
    errv = 16 * 2.0 ** -24 * corner_spread * (1 << d) + 2.0 ** -41 * np.abs(gq) + \
        2.0 ** -24 * (np.abs(gq - np.floor(gq)) + 1) + 1e-9
    nearv = np.abs((gq - np.floor(gq)) - 0.5) <= errv
    ok = plain_sym & ~nearv
    if eb >= 1e-4:
        assert ok.sum() >= 0.5 * plain_sym.sum() > 0
    assert np.array_equal(P_or[ok], np.rint(gq[ok]).astype(np.int64))
    assert np.all(np.abs(P_or[plain_sym & nearv] - gq[plain_sym & nearv]) <= 0.5 + errv[
        plain_sym & nearv])
