"""Pins of the oracle's zero-run stage (an option, not in the paper): within
each lane chunk, a maximal run of r zero symbols (difference or residual 0,
symbol R) becomes the digits of r in bijective base 2, least significant
first (token 2R for a digit 1, 2R + 1 for a digit 2), and the canonical
Huffman code is built over these tokens.

The stream is read here by an independent decoder written from the layout
(header, code lengths, group tables, lane tables, bitstreams): it rebuilds the
canonical codes from the lengths, decodes every lane's tokens bit by bit and
expands the runs; the symbols must equal the oracle's symbols from before the
stage, and the code lengths must be an optimal length-limited code of the
token counts taken from this file's own tokenisation. Closed forms: a lane of
128 zeros is the seven tokens 2, 1, 1, 1, 1, 1, 1; the decoded values never
depend on the stage."""
import numpy as np
import pytest

import oracle
import synth


def _u32(s, o):
    return int(s[o:o + 4].view(np.uint32)[0])


def _u64(s, o):
    return int(s[o:o + 8].view(np.uint64)[0])


def _up(v, a):
    return (v + a - 1) // a * a


def _layout(s):
    """Section offsets from the header, following the written layout."""
    R1, R2, C1, C2 = _u32(s, 24), _u32(s, 28), _u32(s, 32), _u32(s, 36)
    n_v, n_g = _u64(s, 56), _u64(s, 64)
    dim = _u32(s, 16)
    nout1, nout2, nraw, w1, w2 = (_u64(s, o) for o in (144, 152, 160, 168, 176))
    vsz = 8 if _u32(s, 12) == 0 else 4
    ng1 = -(-n_g // (32 * C1))
    ng2 = 0 if dim == 1 else -(-n_v // (32 * C2))
    L = {}
    o = 384
    L["lens1"] = o; o += 2 * R1
    L["lens2"] = o; o += 2 * R2
    o = _up(o, 4)
    L["gtab1"] = o; o += 4 * (ng1 + 1)
    L["gtab2"] = o; o += 4 * (ng2 + 1)
    L["etab1"] = o; o += 4 * (ng1 + 1)
    L["etab2"] = o; o += 4 * (ng2 + 1)
    L["rtab2"] = o; o += 4 * (ng2 + 1)
    L["ltab1"] = o; o += 34 * ng1
    L["ltab2"] = o; o += 34 * ng2
    o = _up(o, 4)
    L["out1"] = o; o += 4 * nout1
    L["out2"] = o; o += 4 * nout2
    o = _up(o, 8)
    L["raw"] = o; o += vsz * nraw
    o = _up(o, 4)
    L["bits1"] = o; o += 4 * w1
    L["bits2"] = o; o += 4 * w2
    return L, dict(R1=R1, R2=R2, C1=C1, C2=C2, n_g=n_g, n_v=n_v, ng1=ng1, ng2=ng2)


def _canonical(lens):
    """Code of every symbol: symbols sorted by (length, symbol), codes counted
    up within a length and shifted left at each longer length."""
    order = sorted((l, s) for s, l in enumerate(lens) if l > 0)
    codes, code, prev = {}, 0, order[0][0] if order else 0
    for l, s in order:
        code <<= l - prev
        prev = l
        codes[(l, code)] = s
        code += 1
    return codes


def _decode_component(s, which, zr):
    L, h = _layout(s)
    R, C = (h["R1"], h["C1"]) if which == 1 else (h["R2"], h["C2"])
    n, ng = (h["n_g"], h["ng1"]) if which == 1 else (h["n_v"], h["ng2"])
    lens = [int(v) for v in s[L[f"lens{which}"]: L[f"lens{which}"] + 2 * R]]
    tl = [int(s[208 + 2 * (which - 1)]), int(s[209 + 2 * (which - 1)])] if zr else [0, 0]
    codes = _canonical(lens + tl)
    raw = s[L[f"bits{which}"]:L[f"bits{which}"] + 4 * (_u64(s, 168) if which == 1 else _u64(s, 176))]
    bits = np.unpackbits(raw.view(np.uint32).astype(">u4").view(np.uint8))
    sym = np.full(n, -1, np.int64)
    tokens = []
    for g in range(ng):
        w0 = _u32(s, L[f"gtab{which}"] + 4 * g)
        lt = s[L[f"ltab{which}"] + 34 * g: L[f"ltab{which}"] + 34 * (g + 1)]
        base = int(lt[0]) | (int(lt[1]) << 8)
        pos = 32 * w0
        for lane in range(32):
            lb = base + int(lt[2 + lane])
            b = pos
            cnt = sum(1 for k in range(C) if g * 32 * C + 32 * k + lane < n)
            k, digit = 0, 0
            while k < cnt:
                code, l = 0, 0
                while (l, code) not in codes:
                    code = (code << 1) | int(bits[b]); b += 1; l += 1
                    assert l <= 24
                t = codes[(l, code)]
                tokens.append(t)
                if t >= 2 * R:
                    z = (t - 2 * R + 1) << digit
                    for e in range(z):
                        sym[g * 32 * C + 32 * (k + e) + lane] = R
                    k += z
                    digit += 1
                else:
                    sym[g * 32 * C + 32 * k + lane] = t
                    k += 1
                    digit = 0
            assert k == cnt and b - pos <= lb
            pos += lb
    return sym, np.array(tokens), lens + tl


def _tokens(sym, n, C, R):
    """This file's tokenisation: lane by lane, runs of R as bijective base-2
    digits, least significant first."""
    out = []
    ng = -(-n // (32 * C))
    for g in range(ng):
        for lane in range(32):
            run = 0
            for k in range(C):
                p = g * 32 * C + 32 * k + lane
                if p >= n:
                    break
                if sym[p] == R:
                    run += 1
                    continue
                while run:
                    d = 1 if run % 2 else 2
                    out.append(2 * R + d - 1); run = (run - d) // 2
                out.append(int(sym[p]))
            while run:
                d = 1 if run % 2 else 2
                out.append(2 * R + d - 1); run = (run - d) // 2
    return np.array(out, np.int64)


@pytest.fixture(scope="module")
def plan2d():
    c, e = synth.mesh2d_jittered(nside=70, seed=31)
    return c, oracle.Plan(c, e, (45, 41))


def test_bijective_digits_closed_form():
    """The digit sequence of r = 1..9 and 128 (d_0 first)."""
    want = {1: [1], 2: [2], 3: [1, 1], 4: [2, 1], 5: [1, 2], 6: [2, 2], 7: [1, 1, 1],
            8: [2, 1, 1], 9: [1, 2, 1], 128: [2, 1, 1, 1, 1, 1, 1]}
    for r, d in want.items():
        toks = _tokens(np.full(32 * r, 5), 32 * r, 4096, 5)  # every lane holds r zeros
        assert toks.size == 32 * len(d)
        assert list(toks[:len(d)] - 10 + 1) == d
        assert sum(x << i for i, x in enumerate(d)) == r


def test_digits_are_the_bits_of_r_plus_one():
    """The identity the GPU coder uses to cost and write a run: the bijective
    base-2 digits of r, least significant first, are the bits of r + 1
    below its leading one, each plus one."""
    for r in range(1, 20000):
        d, t = [], r
        while t:
            x = 1 if t % 2 else 2
            d.append(x)
            t = (t - x) // 2
        v = r + 1
        bits = [(v >> i) & 1 for i in range(v.bit_length() - 1)]
        assert d == [b + 1 for b in bits]


@pytest.mark.parametrize("eb", [1e-1, 1e-2, 1e-4])
@pytest.mark.parametrize("C", [1, 5, 128])
def test_stream_decodes_independently(plan2d, eb, C):
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=3)
    s, dbg = oracle.compress(plan, x, debug=True, eb=eb, C1=C, C2=C, zero_run=True)
    assert _u32(s, 20) & 64
    for which, key, R in ((1, "sym1", 512), (2, "sym2", 512)):
        sym, toks, lens = _decode_component(s, which, True)
        assert np.array_equal(sym, dbg[key].astype(np.int64))
        mine = _tokens(dbg[key].astype(np.int64), sym.size, C, R)
        assert np.array_equal(toks, mine)
        # the code book is an optimal 24-bit-limited code of the token counts
        cnt = np.bincount(mine, minlength=2 * R + 2)
        assert cnt[R] == 0
        assert np.array_equal(np.array(lens), oracle.huffman_lengths(cnt, 24))


@pytest.mark.parametrize("eb", [1e-1, 1e-3])
def test_stream_decodes_independently_3d(eb):
    """The same reader on a 3D annulus (tetrahedra, trilinear g) and on a
    plan of kept planes (Grid_Coarsen): the stage sees only symbols."""
    c, e = synth.mesh3d_annulus(nr=5, nth=20, nz=6, seed=4)
    x = synth.field_vortex(c, seed=5)
    base = oracle.Plan(c, e, (21, 19, 15))
    for plan in (base, oracle.Plan(c, e, (21, 19, 15), keep=oracle.grid_coarsen(base, "nearest"))):
        s, dbg = oracle.compress(plan, x, debug=True, eb=eb, C1=17, C2=64, zero_run=True)
        for which, key in ((1, "sym1"), (2, "sym2")):
            sym, toks, lens = _decode_component(s, which, True)
            assert np.array_equal(sym, dbg[key].astype(np.int64))
            C = 17 if which == 1 else 64
            assert np.array_equal(toks, _tokens(dbg[key].astype(np.int64), sym.size, C, 512))


def test_stage_off_decodes_independently(plan2d):
    """The same reader without the stage (tokens are the symbols)."""
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=4)
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-3, C1=9, C2=33)
    assert not _u32(s, 20) & 64 and s[208:212].sum() == 0
    for which, key in ((1, "sym1"), (2, "sym2")):
        sym, toks, _ = _decode_component(s, which, False)
        assert np.array_equal(sym, dbg[key].astype(np.int64))
        assert np.array_equal(toks, dbg[key].astype(np.int64)[_lane_order(sym.size, 9 if which == 1 else 33)])


def _lane_order(n, C):
    idx = []
    for g in range(-(-n // (32 * C))):
        for lane in range(32):
            for k in range(C):
                p = g * 32 * C + 32 * k + lane
                if p < n:
                    idx.append(p)
    return np.array(idx)


def test_all_zero_residual_closed_form():
    """A field the grid reproduces exactly (a constant): every residual lane
    of 128 zeros is the seven tokens B A A A A A A; with one code bit each a
    full group takes 7 words."""
    c, e = synth.mesh2d_jittered(nside=64, seed=2)   # 4096 vertices: one full group
    plan = oracle.Plan(c, e, (20, 20))
    x = np.full(plan.n_v, 3.25)
    s, dbg = oracle.compress(plan, x, debug=True, eb=1e-3, zero_run=True)
    assert np.all(dbg["sym2"] == 512) and plan.n_v == 4096
    assert _u64(s, 176) == 7
    assert s[210] == 1 and s[211] == 1
    sym, toks, _ = _decode_component(s, 2, True)
    assert list(toks[:7]) == [1025, 1024, 1024, 1024, 1024, 1024, 1024]
    y = oracle.decompress(plan, s)
    assert np.all(y == y[0]) and abs(y[0] - 3.25) <= 0.5e-3


@pytest.mark.parametrize("kw", [dict(), dict(open_loop=True), dict(f_op="cluster", g_op="nearest"),
                                dict(eb=1e-6), dict(dtype32=True)])
def test_values_independent_of_stage(plan2d, kw):
    coords, plan = plan2d
    kw = dict(kw)
    x = synth.field_bumps_noise(coords, seed=5)
    if kw.pop("dtype32", False):
        x = x.astype(np.float32)
    kw.setdefault("eb", 1e-2)
    a = oracle.compress(plan, x, **kw)
    b = oracle.compress(plan, x, zero_run=True, **kw)
    assert np.array_equal(oracle.decompress(plan, a), oracle.decompress(plan, b))
    # identical up to the flag, the token lengths and the coded sections
    assert _u32(b, 20) == _u32(a, 20) | 64


def test_learned_auto_with_stage(plan2d):
    from mlp_models import pack, random_model
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=6)
    blob = pack(random_model(2, 7))
    for auto in (False, True):
        s, dbg = oracle.compress(plan, x, debug=True, eb=1e-2, model=blob, auto=auto, zero_run=True)
        sym, _, _ = _decode_component(s, 2, True)
        assert np.array_equal(sym, dbg["sym2"].astype(np.int64))
        y = oracle.decompress(plan, s)
        assert np.array_equal(y, oracle.decompress(plan, oracle.compress(plan, x, eb=1e-2, model=blob,
                                                                         auto=auto)))


def test_stage_shrinks_sparse_components(plan2d):
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=7)
    a = oracle.compress(plan, x, eb=1e-1)
    b = oracle.compress(plan, x, eb=1e-1, zero_run=True)
    assert b.size < a.size


def test_default_1d_with_stage():
    c, e = synth.mesh2d_jittered(nside=90, seed=8)
    x = np.sort(synth.field_bumps_noise(c, seed=9))   # sorted: long runs of equal codes
    for eb in (1e-2, 1e-4):
        a = oracle.compress_1d(x, eb=eb)
        b = oracle.compress_1d(x, eb=eb, zero_run=True)
        assert _u32(b, 20) == 32 | 64 and _u32(a, 20) == 32
        assert np.array_equal(oracle.decompress_1d(a, x.size), oracle.decompress_1d(b, x.size))
        s, Q = oracle.compress_1d(x, debug=True, eb=eb, zero_run=True)
        sym, toks, _ = _decode_component(s, 1, True)
        d = np.diff(Q.astype(np.int64), prepend=0)
        assert np.array_equal(sym[np.abs(d) < 511], d[np.abs(d) < 511] + 512)
        if eb == 1e-2:
            assert b.size < a.size


def test_errors(plan2d):
    coords, plan = plan2d
    x = synth.field_bumps_noise(coords, seed=10)
    with pytest.raises(oracle.OracleError) as err:
        oracle.compress(plan, x, eb=1e-2, zero_run=2)
    assert err.value.status == 1
    # 2R + 2 symbols must fit in lmax bits
    oracle.compress(plan, x, eb=1e-2, R1=8, R2=8, lmax=4)
    with pytest.raises(oracle.OracleError) as err:
        oracle.compress(plan, x, eb=1e-2, R1=8, R2=8, lmax=4, zero_run=True)
    assert err.value.status == 1
    s = oracle.compress(plan, x, eb=1e-2, zero_run=True)
    for off, val in ((208, 30), (211, 25)):   # token lengths above lmax
        t = s.copy()
        t[off] = val
        with pytest.raises(oracle.OracleError) as err:
            oracle.decompress(plan, t)
        assert err.value.status == 5
    t = s.copy()
    t[20] |= 128   # an unknown flag
    with pytest.raises(oracle.OracleError) as err:
        oracle.decompress(plan, t)
    assert err.value.status == 5
