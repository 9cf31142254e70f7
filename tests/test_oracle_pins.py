"""Pins of the CPU oracle against things other than itself: textbook values,
closed forms, invariants, brute force and independent numpy restatements.

Each test names the property of Gong et al. (Sec. III-IV) or of the textbook
building block it checks. No GPU; runs in the CPU suite.
"""
import heapq
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- #
# Huffman (canonical, length limited)
# --------------------------------------------------------------------------- #
def _read_textbook():
    syms, freq, want, cost = [], [], [], None
    for line in open(os.path.join(GOLDEN, "huffman_textbook.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "cost":
            cost = int(parts[1])
            continue
        syms.append(parts[0]); freq.append(int(parts[1])); want.append(int(parts[2]))
    return freq, want, cost


def test_huffman_textbook_lengths():
    freq, want, cost = _read_textbook()
    ln = oracle.huffman_lengths(np.array(freq, dtype=np.uint64))
    assert list(ln) == want
    assert int(np.dot(freq, ln)) == cost


def _heap_huffman_cost(counts):
    """Optimal prefix-code cost = sum of the weights of all merged nodes."""
    h = [int(c) for c in counts if c > 0]
    if len(h) <= 1:
        return sum(h)
    heapq.heapify(h)
    total = 0
    while len(h) > 1:
        a = heapq.heappop(h); b = heapq.heappop(h)
        total += a + b
        heapq.heappush(h, a + b)
    return total


@pytest.mark.parametrize("seed", range(8))
def test_huffman_optimal_cost_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 600))
    counts = rng.geometric(rng.uniform(0.01, 0.6), size=n).astype(np.uint64)
    counts[rng.random(n) < 0.3] = 0
    counts[0] += 1
    counts[-1] += 1
    ln = oracle.huffman_lengths(counts)
    assert int(np.dot(counts, ln.astype(np.uint64))) == _heap_huffman_cost(counts)
    used = counts > 0
    assert np.all(ln[used] > 0) and np.all(ln[~used] == 0)
    kraft = np.sum(2.0 ** -ln[used].astype(np.float64))
    assert kraft == pytest.approx(1.0, abs=0)


def test_huffman_infeasible_limit_rejected():
    """m used symbols need m <= 2^lmax; the halving loop would never end."""
    with pytest.raises(oracle.OracleError):
        oracle.huffman_lengths(np.ones(9, dtype=np.uint64), lmax=3)
    ln = oracle.huffman_lengths(np.ones(8, dtype=np.uint64), lmax=3)
    assert list(ln) == [3] * 8


def test_huffman_length_limit_fibonacci():
    fib = [1, 1]
    while len(fib) < 26:
        fib.append(fib[-1] + fib[-2])
    counts = np.array(fib, dtype=np.uint64)
    free = oracle.huffman_lengths(counts, lmax=32)
    assert free.max() == 26 - 1  # the classic worst case: a chain
    ln = oracle.huffman_lengths(counts, lmax=24)
    assert ln.max() <= 24
    assert np.sum(2.0 ** -ln.astype(np.float64)) <= 1.0


def test_huffman_degenerate():
    c = np.zeros(16, dtype=np.uint64)
    assert oracle.huffman_lengths(c).sum() == 0
    c[7] = 1000
    ln = oracle.huffman_lengths(c)
    assert ln[7] == 1 and ln.sum() == 1


def test_canonical_codes_prefix_free():
    rng = np.random.default_rng(3)
    counts = rng.integers(0, 5000, 300).astype(np.uint64)
    ln = oracle.huffman_lengths(counts)
    code = oracle.canonical_codes(ln)
    words = {}
    for s in np.flatnonzero(ln):
        words[s] = format(int(code[s]), "0%db" % ln[s])
    ws = sorted(words.values())
    for a, b in zip(ws, ws[1:]):
        assert not b.startswith(a)
    # same-length codes are consecutive integers in symbol order
    for L in np.unique(ln[ln > 0]):
        syms = np.flatnonzero(ln == L)
        assert np.all(np.diff(code[syms].astype(np.int64)) == 1)


# --------------------------------------------------------------------------- #
# Lorenzo (N-D difference) and its inverse (prefix sums)
# --------------------------------------------------------------------------- #
def test_lorenzo_linear_ramp_2d():
    y, x = np.mgrid[0:23, 0:31]
    q = (5 + 3 * x - 7 * y).astype(np.int32)
    d = oracle.lorenzo(q)
    assert np.all(d[1:, 1:] == 0)
    assert d[0, 0] == 5 and np.all(d[0, 1:] == 3) and np.all(d[1:, 0] == -7)


def test_lorenzo_bilinear_2d_is_mixed_difference():
    y, x = np.mgrid[0:9, 0:13]
    d = oracle.lorenzo((x * y).astype(np.int32))
    assert np.all(d[1:, 1:] == 1) and np.all(d[0, :] == 0) and np.all(d[:, 0] == 0)


def test_lorenzo_linear_ramp_3d():
    z, y, x = np.mgrid[0:7, 0:9, 0:11]
    q = (2 + x + 4 * y - 3 * z).astype(np.int32)
    d = oracle.lorenzo(q)
    assert np.all(d[1:, 1:, 1:] == 0)
    # trilinear xyz -> third mixed difference 1
    d = oracle.lorenzo((x * y * z).astype(np.int32))
    assert np.all(d[1:, 1:, 1:] == 1) and np.all(d[0] == 0)


@pytest.mark.parametrize("shape", [(17, 29), (5, 6, 7), (1, 40), (2, 2)])
def test_lorenzo_inverse_roundtrip(shape):
    rng = np.random.default_rng(0)
    q = rng.integers(-10 ** 6, 10 ** 6, shape).astype(np.int32)
    d = oracle.lorenzo(q)
    assert np.array_equal(oracle.lorenzo_inverse(d), q)
    # the inverse is the N-D inclusive prefix sum
    ref = d.astype(np.int64)
    for ax in range(d.ndim):
        ref = np.cumsum(ref, axis=ax)
    assert np.array_equal(ref, q)


# --------------------------------------------------------------------------- #
# point location and barycentric weights (plan)
# --------------------------------------------------------------------------- #
def _small_mesh(name):
    if name == "jit2d":
        return synth.mesh2d_jittered(nside=12, seed=11) + ((23, 17),)
    if name == "graded2d":
        return synth.mesh2d_graded(n=300, seed=12) + ((19, 21),)
    return synth.mesh3d_annulus(nr=4, nth=12, nz=4, seed=13) + ((9, 10, 7),)


@pytest.mark.parametrize("name", ["jit2d", "graded2d", "annulus3d"])
def test_locate_brute_force_equals_raster(name):
    coords, cells, n = _small_mesh(name)
    g = oracle.Grid(coords, n)
    a = oracle.locate(g, coords, cells, brute=True)
    b = oracle.locate(g, coords, cells, brute=False)
    assert np.array_equal(a, b)


def _numpy_bary(P, V):
    """Independent barycentric coordinates by a linear solve."""
    A = (V[1:] - V[0]).T
    lam = np.linalg.solve(A, P - V[0])
    return np.concatenate([[1.0 - lam.sum()], lam])


@pytest.mark.parametrize("name", ["jit2d", "annulus3d"])
def test_locate_matches_definition(name):
    coords, cells, n = _small_mesh(name)
    g = oracle.Grid(coords, n)
    owner = oracle.locate(g, coords, cells)
    dim = coords.shape[1]
    idx = np.stack(np.unravel_index(np.arange(g.n_g), g.n[:dim][::-1]), 1)[:, ::-1]
    P = g.lo[:dim] + idx * g.h[:dim]
    for j in range(g.n_g):
        lams = np.array([_numpy_bary(P[j], coords[c]) for c in cells])
        mins = lams.min(axis=1)
        clear_in = np.flatnonzero(mins > 1e-9)
        maybe = np.flatnonzero(mins >= -1e-9)
        if clear_in.size:
            assert owner[j] == min(maybe), j
        elif maybe.size == 0:
            assert owner[j] == -1, j
        else:  # on a shared face / edge / vertex: the minimum candidate id
            assert owner[j] in maybe, j


def test_two_triangles_shared_diagonal():
    coords, cells = synth.mesh2d_two_triangles()
    g = oracle.Grid(coords, (5, 5))
    owner = oracle.locate(g, coords, cells).reshape(5, 5)
    y, x = np.mgrid[0:5, 0:5]
    # triangle 0 = (0,0),(1,0),(1,1) holds y <= x (diagonal included: min id)
    assert np.all(owner[y <= x] == 0) and np.all(owner[y > x] == 1)


@pytest.mark.parametrize("name", ["jit2d", "graded2d", "annulus3d"])
def test_barycentric_reproduces_points_and_linear_fields(name):
    coords, cells, n = _small_mesh(name)
    plan = oracle.Plan(coords, cells, n)
    dim = coords.shape[1]
    inside = plan.vid[0] >= 0
    idx = np.stack(np.unravel_index(np.arange(plan.n_g), plan.grid.n[:dim][::-1]), 1)[:, ::-1]
    P = plan.grid.lo[:dim] + idx * plan.grid.h[:dim]
    V = coords[plan.vid.T]  # [n_g, dim+1, dim]
    lam = plan.lam64.T      # [n_g, dim+1]
    rec = np.einsum("gk,gkd->gd", lam, V)
    assert np.abs(rec - P)[inside].max() <= 1e-14 * max(1.0, np.abs(P).max())
    assert np.abs(lam.sum(1) - 1.0)[inside].max() <= 1e-15
    # a linear field is reproduced by the FP64 weights to rounding ...
    f = synth.field_linear(coords)
    exact = synth.field_linear(P)
    got = np.einsum("gk,gk->g", lam, f[plan.vid.T])
    assert np.abs(got - exact)[inside].max() <= 1e-14 * np.abs(exact).max()
    # ... and by the stored 2^-15 weights within half a unit per weight
    l16 = plan.lam.T.astype(np.float64) / 32768.0
    w = np.concatenate([1.0 - l16.sum(1, keepdims=True), l16], 1)
    got16 = np.einsum("gk,gk->g", w, f[plan.vid.T])
    fv = f[plan.vid.T]
    bound = (np.abs(fv[:, 1:] - fv[:, :1]).sum(1)) * 2.0 ** -16 + 1e-14
    assert np.all((np.abs(got16 - exact) <= bound)[inside])


@pytest.mark.parametrize("name", ["jit2d", "annulus3d"])
def test_vertex_cells_and_local_coordinates(name):
    coords, cells, n = _small_mesh(name)
    plan = oracle.Plan(coords, cells, n)
    g = plan.grid
    dim = coords.shape[1]
    nn = np.array(g.n[:dim])
    c = plan.cell.astype(np.int64)
    ci = []
    for d in range(dim):
        ci.append(c % nn[d]); c //= nn[d]
    ci = np.stack(ci, 1)
    assert np.all(ci >= 0) and np.all(ci <= nn - 2)
    t = (coords - g.lo[:dim]) / g.h[:dim]
    f = np.clip(t - ci, 0.0, 1.0)
    assert np.abs(plan.frac.T / 32768.0 - f).max() <= 2.0 ** -16 + 1e-12


# --------------------------------------------------------------------------- #
# compression: the bound theorem (Sec. III) and the allocation
# --------------------------------------------------------------------------- #
@pytest.fixture(scope="module")
def plan2d():
    coords, cells = synth.mesh2d_jittered(nside=60, seed=21)
    return coords, oracle.Plan(coords, cells, (41, 37))


@pytest.fixture(scope="module")
def plan3d():
    coords, cells = synth.mesh3d_annulus(nr=6, nth=24, nz=8, seed=22)
    return coords, oracle.Plan(coords, cells, (13, 12, 9))


def _x1_in_node_units(plan, Q, fill_u):
    """x1 = f(x) on the vertex codes, evaluated independently in FP64."""
    l16 = plan.lam.astype(np.float64) / 32768.0
    out = np.empty(plan.n_g)
    inside = plan.vid[0] >= 0
    qa = Q[np.where(inside, plan.vid[0], 0)].astype(np.float64)
    acc = np.zeros(plan.n_g)
    for k in range(1, plan.dim + 1):
        acc += l16[k - 1] * (Q[plan.vid[k]].astype(np.float64) - qa)
    out[inside] = (qa + acc)[inside]
    out[~inside] = fill_u
    return out


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("eb,frac", [(1e-2, 0.5), (1e-3, 0.2), (1e-4, 0.8), (1e-5, 0.5)])
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_bound_and_allocation(plan2d, plan3d, dtype, eb, frac, which):
    coords, plan = plan2d if which == "2d" else plan3d
    x = (synth.field_bumps_noise(coords, seed=5) if which == "2d"
         else synth.field_vortex(coords, seed=6)).astype(dtype)
    s, dbg = oracle.compress(plan, x, debug=True, eb=eb, grid_fraction=frac)
    y = oracle.decompress(plan, s)
    f = oracle.field_params(x, eb=eb, grid_fraction=frac)
    err = np.abs(y.astype(np.float64) - x.astype(np.float64))
    # Sec. III: |x - x'| <= tau1 + tau2 = tau at every vertex; closed loop
    # puts the whole vertex error in the residual component: <= tau2.
    assert err.max() <= f["tau2"]
    assert f["tau1"] + f["tau2"] <= f["tau"] * (1 + 1e-15)
    # grid component: |x1 - x1'| <= tau1 (x1' = s1 q1, x1 in value units)
    x1u = _x1_in_node_units(plan, dbg["Q"].astype(np.int64), f["fill_u"])
    gerr = np.abs(f["s1"] * dbg["q1"] - f["s2"] * x1u)
    assert gerr.max() <= f["tau1"] * (1 + 1e-5)
    # vertex codes: Q = round(x / s2) - K
    Qref = np.rint(x.astype(np.float64) * f["inv2"]).astype(np.int64) - f["K"]
    assert np.array_equal(dbg["Q"], Qref)


def test_guard_path_large_offset(plan2d):
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=7) + 3.0e9
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-1, eb_mode="abs")
    f = oracle.field_params(x, eb=1e-1, eb_mode="abs")
    assert f["guard"] == 1
    y = oracle.decompress(plan, s)
    assert np.abs(y - x).max() <= f["tau2"]


def test_unguarded_fields_never_need_raw_values(plan2d):
    """When max|x| <= 2^28 tau2 the product bound proves every vertex holds the
    bound without a check, so the oracle's check never fires."""
    coords, plan = plan2d
    for eb in (1e-2, 1e-4, 1e-6):
        x = synth.field_bumps_noise(coords, seed=8)
        s, dbg = oracle.compress(plan, x, debug=True, eb=eb)
        assert oracle.field_params(x, eb=eb)["guard"] == 0
        assert np.all(dbg["sym2"] != 2 * 512 - 1)


def test_constant_field_closed_form(plan2d):
    coords, plan = plan2d
    x = np.full(plan.n_v, 2.5)
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-3)
    # range 0 -> tau = eb; every vertex code equal; grid codes constant, so
    # the Lorenzo difference is the code at the origin and 0 elsewhere
    assert np.all(dbg["Q"] == dbg["Q"][0])
    q1 = dbg["q1"]
    assert np.all(q1 == q1[0])
    y = oracle.decompress(plan, s)
    assert np.abs(y - x).max() <= 0.5e-3


def test_huge_bound_one_bit_floor(plan2d):
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=9)
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e3, eb_mode="abs")
    assert np.all(dbg["sym2"] == 512)  # every residual code is 0
    hdr_words2 = int(s[176:184].view(np.uint64)[0])
    groups = -(-plan.n_v // (32 * 128))
    # one used symbol -> 1 bit per vertex, groups padded to 32-bit words
    assert hdr_words2 == sum(-(-min(32 * 128, plan.n_v - g * 32 * 128) // 32) for g in range(groups))


def test_errors_and_corruption(plan2d):
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=10)
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(plan, x, eb=0.0)
    assert e.value.status == oracle.INVALID_ARG
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(plan, x, grid_fraction=1.0)
    assert e.value.status == oracle.INVALID_ARG
    bad = x.copy(); bad[3] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(plan, bad)
    assert e.value.status == oracle.INVALID_ARG
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(plan, x, eb=1e-12)
    assert e.value.status == oracle.RANGE
    # 2R symbols need 2R <= 2^lmax; otherwise no length-limited code exists
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress(plan, x, R1=512, R2=512, lmax=9)
    assert e.value.status == oracle.INVALID_ARG
    s = oracle.compress(plan, x)
    for cut in (0, 100, s.size - 1):
        with pytest.raises(oracle.OracleError) as e:
            oracle.decompress(plan, s[:cut])
        assert e.value.status == oracle.CORRUPT
    t = s.copy(); t[0] ^= 1
    with pytest.raises(oracle.OracleError):
        oracle.decompress(plan, t)
    # random bit flips: either detected or decoded, never a crash
    rng = np.random.default_rng(0)
    for _ in range(50):
        t = s.copy()
        pos = int(rng.integers(0, s.size))
        t[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        try:
            oracle.decompress(plan, t)
        except oracle.OracleError as err:
            assert err.status == oracle.CORRUPT


def test_deterministic(plan2d):
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=11)
    assert np.array_equal(oracle.compress(plan, x), oracle.compress(plan, x))


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_vertex_predictor_is_multilinear_interpolation(plan2d, plan3d, which):
    """g(x1') at a vertex is the bilinear / trilinear interpolation of the grid
    codes of its cell (Sec. III: piecewise linear g, weights >= 0 summing to
    1); the residual code is q2 = Q - round(rho12 g). Checked against an
    independent FP64 evaluation."""
    coords, plan = plan2d if which == "2d" else plan3d
    x = (synth.field_bumps_noise(coords, seed=12) if which == "2d"
         else synth.field_vortex(coords, seed=13))
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-3, grid_fraction=0.3)
    f = oracle.field_params(x, eb=1e-3, grid_fraction=0.3)
    dim = plan.dim
    nx, ny = plan.grid.n[0], plan.grid.n[1]
    fr = plan.frac.astype(np.float64) / 32768.0
    q1 = dbg["q1"].astype(np.float64)
    c = plan.cell.astype(np.int64)
    g = np.zeros(plan.n_v)
    for corner in range(1 << dim):
        off = 0
        w = np.ones(plan.n_v)
        for d, stride in enumerate([1, nx, nx * ny][:dim]):
            bit = (corner >> d) & 1
            off += bit * stride
            w *= fr[d] if bit else 1.0 - fr[d]
        g += w * q1[c + off]
    rho12 = f["rho12_q"] / 2.0 ** 40
    sym = dbg["sym2"].astype(np.int64)
    ok = (sym != 0) & (sym != 2 * 512 - 1)
    P = dbg["Q"].astype(np.int64) - (sym - 512)
    assert ok.mean() > 0.9
    assert np.abs(P - rho12 * g)[ok].max() <= 0.5 + 1e-3


def test_lane_table_padding(plan2d):
    """Lane tables store u16 base + u8 deltas; a group whose lane lengths
    spread over more than 255 bits pads its short lanes up to max - 255 (zero
    bits after their codes). Half the vertices of every 32 noisy, half
    constant, so lane lengths differ widely: the stream still decodes within
    the bound and the table shows the clamped spread."""
    coords, plan = plan2d
    rng = np.random.default_rng(17)
    i = np.arange(plan.n_v)
    x = np.where(i % 32 < 16, rng.normal(0, 1, plan.n_v), 0.25)
    kw = dict(eb=1e-4, eb_mode="abs", C2=64, R2=2048, lmax=24)
    s = oracle.compress(plan, x, **kw)
    y = oracle.decompress(plan, s)
    assert np.abs(y - x).max() <= 0.5e-4
    # residual lane table: after the grid's, header fields give the sizes
    hdr32 = s[:64].view(np.uint32)
    R1, R2, C1, C2 = (int(v) for v in hdr32[6:10])
    ng1 = -(-plan.n_g // (32 * C1))
    ng2 = -(-plan.n_v // (32 * C2))
    o = 384 + 2 * R1 + 2 * R2
    o = (o + 3) // 4 * 4 + 4 * (ng1 + 1) * 2 + 4 * (ng2 + 1) * 3
    lt2 = s[o + 34 * ng1: o + 34 * ng1 + 34 * ng2].reshape(ng2, 34)
    deltas = lt2[0, 2:]
    # the longest lane sits at base + 255; the lanes padded up to base have 0
    assert deltas.max() == 255 and (deltas == 0).sum() >= 8
