"""CPU oracle of the multi-component unstructured-mesh compressor (Gong et al.,
Sec. III-IV, Algorithms 3 and 4), as a ctypes binding over ``mcc_oracle.c``.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. It shares no code with
the CUDA library and never imports it. Everything here is plain single-threaded
C on host arrays; the library's product path never falls back to it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcc_oracle.c")
_HDR = os.path.join(_HERE, "mcc_oracle.h")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

OK, INVALID_ARG, CUDA, OOM, RANGE, CORRUPT, CAPACITY, TIMEOUT, UNSUPPORTED = range(9)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile liborc.so with gcc (plain C11, no FMA contraction)."""
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("h", C.c_double * 3), ("inv_h", C.c_double * 3), ("keep", C.c_void_p * 3)]


class _Params(C.Structure):
    _fields_ = [("dtype", C.c_int), ("eb_mode", C.c_int), ("eb", C.c_double),
                ("grid_fraction", C.c_double), ("R1", C.c_int), ("R2", C.c_int),
                ("C1", C.c_int), ("C2", C.c_int), ("lmax", C.c_int),
                ("model", C.c_void_p), ("model_bytes", C.c_size_t), ("auto_select", C.c_int),
                ("open_loop", C.c_int), ("f_op", C.c_int), ("g_op", C.c_int),
                ("zero_run", C.c_int)]


class _Field(C.Structure):
    _fields_ = [("lo", C.c_double), ("hi", C.c_double), ("M", C.c_double),
                ("tau", C.c_double), ("tau1", C.c_double), ("tau2", C.c_double),
                ("s1", C.c_double), ("s2", C.c_double), ("inv2", C.c_double),
                ("K", C.c_int64), ("Qhi", C.c_int64), ("fill_u", C.c_int64),
                ("rho21_q", C.c_int64), ("rho12_q", C.c_int64),
                ("rho21_f", C.c_float), ("rho12_f", C.c_float), ("guard", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_grid_resolve.argtypes = [C.c_int, C.c_int64, P, P, P, P, C.POINTER(_Grid)]
            lib.orc_compress_bound_1d.argtypes = [C.c_int64, C.POINTER(_Params)]
            lib.orc_compress_bound_1d.restype = C.c_size_t
            lib.orc_compress_1d.argtypes = [C.c_int64, P, C.POINTER(_Params), P, C.c_size_t,
                                            C.POINTER(C.c_size_t), P]
            lib.orc_decompress_1d.argtypes = [C.c_int64, P, C.c_size_t, P]
            lib.orc_grid_init.argtypes = [C.c_int, C.c_int64, P, C.c_int64, P, C.c_double,
                                          C.c_double, C.c_int32, P, P, P, P]
            lib.orc_point_in_simplex.argtypes = [C.POINTER(_Grid), P, P, P, P]
            lib.orc_locate.argtypes = [C.POINTER(_Grid), C.c_int64, P, C.c_int64, P, C.c_int, P]
            lib.orc_plan_tables.argtypes = [C.POINTER(_Grid), C.c_int64, P, P, P, P, P, P, P, P]
            lib.orc_field_params.argtypes = [C.POINTER(_Params), C.c_int64, P, C.POINTER(_Field)]
            lib.orc_compress_bound.argtypes = [C.POINTER(_Grid), C.c_int64, C.POINTER(_Params)]
            lib.orc_compress_bound.restype = C.c_size_t
            lib.orc_compress.argtypes = [C.POINTER(_Grid), C.c_int64, P, P, P, P, P,
                                         C.POINTER(_Params), P, C.c_size_t,
                                         C.POINTER(C.c_size_t), P, P, P, P]
            lib.orc_decompress.argtypes = [C.POINTER(_Grid), C.c_int64, P, P, P, C.c_size_t, P, P]
            lib.orc_huffman_lengths.argtypes = [P, C.c_int, C.c_int, P]
            lib.orc_canonical_codes.argtypes = [P, C.c_int, P]
            lib.orc_lorenzo.argtypes = [C.c_int, P, P, P]
            lib.orc_lorenzo_inverse.argtypes = [C.c_int, P, P, P]
            lib.orc_mlp_predict.argtypes = [C.c_int, P, C.c_size_t, P, P, C.c_float, C.c_int64, C.c_int64, P, P]
            lib.orc_mlp_quantize.argtypes = [C.c_int, C.c_int, P, C.c_float, C.c_float, P]
            lib.orc_mlp_grad.argtypes = [P, P, P, P, P, P, P, P, C.c_int64, C.c_int, C.c_int, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------- #
# grid and plan
# --------------------------------------------------------------------------- #
class Grid:
    """Resolved rectilinear grid (corners, spacing) -- Sec. IV-C. ``keep``
    (one increasing index array per axis) keeps only those planes of the
    uniform grid (Grid_Coarsen, Algorithm 2)."""

    def __init__(self, coords, n, lo=None, hi=None, keep=None):
        coords = _c(coords, np.float64)
        dim = coords.shape[1]
        nn = np.ones(3, dtype=np.int32)
        nn[:dim] = n
        lo3 = np.zeros(3); hi3 = np.zeros(3)  # lo >= hi selects the mesh bounding box
        if lo is not None:
            lo3[:dim] = lo
            hi3[:dim] = hi
        g = _Grid()
        st = _load().orc_grid_resolve(dim, coords.shape[0], _ptr(coords), _ptr(nn),
                                      _ptr(lo3), _ptr(hi3), C.byref(g))
        if st:
            raise OracleError(st, "grid_resolve")
        self.base_n = tuple(int(v) for v in g.n)
        self._keep = None
        if keep is not None:
            self._keep = []
            for d in range(dim):
                k = np.ascontiguousarray(keep[d], dtype=np.int32)
                if k.size < 2 or np.any(np.diff(k) <= 0) or k[0] < 0 or k[-1] >= g.n[d]:
                    raise ValueError("keep: increasing base indices, at least two per axis")
                self._keep.append(k)
                g.keep[d] = k.ctypes.data
                g.n[d] = k.size
        self._g = g
        self.dim = dim
        self.n = tuple(int(v) for v in g.n)
        self.lo = np.array(g.lo[:])
        self.h = np.array(g.h[:])
        self.n_g = int(np.prod(self.n))

    def coords_of_axis(self, d):
        """Coordinates of the grid's points along axis d."""
        idx = self._keep[d] if self._keep is not None else np.arange(self.n[d])
        return self.lo[d] + idx.astype(np.float64) * self.h[d]


def point_in_simplex(grid: Grid, coords, cell, idx):
    coords = _c(coords, np.float64)
    cell = _c(cell, np.int32)
    idx3 = np.zeros(3, dtype=np.int32)
    idx3[: len(idx)] = idx
    lam = np.zeros(4)
    inside = _load().orc_point_in_simplex(C.byref(grid._g), _ptr(coords), _ptr(cell),
                                          _ptr(idx3), _ptr(lam))
    return bool(inside), lam[: grid.dim + 1]


def locate(grid: Grid, coords, cells, brute=False):
    coords = _c(coords, np.float64)
    cells = _c(cells, np.int32)
    owner = np.empty(grid.n_g, dtype=np.int32)
    st = _load().orc_locate(C.byref(grid._g), coords.shape[0], _ptr(coords), cells.shape[0],
                            _ptr(cells), 1 if brute else 0, _ptr(owner))
    if st:
        raise OracleError(st, "locate")
    return owner


def grid_init(coords, cells, k_pct, delta_pct=1.0, gmax=4096):
    """Grid_Init (Algorithm 1): returns (n, lo, hi, gs) per axis."""
    coords = _c(coords, np.float64)
    cells = _c(cells, np.int32)
    dim = coords.shape[1]
    n = (C.c_int32 * 3)()
    lo, hi, gs = (C.c_double * 3)(), (C.c_double * 3)(), (C.c_double * 3)()
    st = _load().orc_grid_init(dim, coords.shape[0], _ptr(coords), cells.shape[0], _ptr(cells),
                               C.c_double(k_pct), C.c_double(delta_pct), int(gmax), n, lo, hi, gs)
    if st:
        raise OracleError(st, "grid_init")
    return tuple(n[:dim]), tuple(lo[:dim]), tuple(hi[:dim]), tuple(gs[:dim])


def grid_coarsen(plan, g_op="multilinear"):
    """Grid_Coarsen (Algorithm 2) on a plan of a uniform grid: the kept
    plane indices per axis (a list of int32 arrays) for ``Plan(..., n,
    keep=...)`` with the same n, lo, hi."""
    g = plan.grid
    if g._keep is not None:
        raise ValueError("grid_coarsen takes a uniform grid")
    gop = {"multilinear": 0, "nearest": 1}[g_op] if isinstance(g_op, str) else int(g_op)
    outs = [np.empty(max(g.n[d], 1), dtype=np.int32) for d in range(3)]
    keep_p = (C.c_void_p * 3)(*[o.ctypes.data for o in outs])
    n_out = (C.c_int32 * 3)()
    lib = _load()
    lib.orc_grid_coarsen.argtypes = [C.POINTER(_Grid), C.c_int64, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_void_p * 3, C.c_int32 * 3]
    st = lib.orc_grid_coarsen(C.byref(g._g), plan.n_v, _ptr(plan.cell), _ptr(plan.frac), gop,
                              keep_p, n_out)
    if st:
        raise OracleError(st, "grid_coarsen")
    return [outs[d][: n_out[d]].copy() for d in range(g.dim)]


class Plan:
    """Mesh -> grid mapping tables: per grid point vertex ids ``vid``
    [(dim+1), n_g] (vid[0] = -1 outside the mesh) and u16 weights ``lam``
    [dim, n_g]; per vertex the cell index ``cell`` [n_v] and u16 local
    coordinates ``frac`` [dim, n_v]."""

    def __init__(self, coords, cells, n, lo=None, hi=None, brute=False, keep=None):
        coords = _c(coords, np.float64)
        cells = _c(cells, np.int32)
        self.grid = Grid(coords, n, lo, hi, keep)
        g = self.grid
        self.dim = g.dim
        self.n_v = coords.shape[0]
        self.n_g = g.n_g
        self.owner = locate(g, coords, cells, brute)
        self.vid = np.empty((g.dim + 1, g.n_g), dtype=np.int32)
        self.lam = np.empty((g.dim, g.n_g), dtype=np.uint16)
        self.lam64 = np.empty((g.dim + 1, g.n_g), dtype=np.float64)
        self.cell = np.empty(self.n_v, dtype=np.uint32)
        self.frac = np.empty((g.dim, self.n_v), dtype=np.uint16)
        st = _load().orc_plan_tables(C.byref(g._g), self.n_v, _ptr(coords), _ptr(cells),
                                     _ptr(self.owner), _ptr(self.vid), _ptr(self.lam),
                                     _ptr(self.lam64), _ptr(self.cell), _ptr(self.frac))
        if st:
            raise OracleError(st, "plan_tables")


# --------------------------------------------------------------------------- #
# compression
# --------------------------------------------------------------------------- #
DEFAULTS = dict(eb_mode="rel", eb=1e-4, grid_fraction=0.5, R1=512, R2=512, C1=128, C2=128,
                lmax=24)


def make_params(dtype, model=None, auto=False, open_loop=False, f_op="barycentric",
                g_op="multilinear", zero_run=False, **kw):
    """Parameters; ``model`` is a learned-predictor blob (uint8 array) or None;
    ``auto`` keeps whichever predictor encodes smaller; ``zero_run`` turns on
    the zero-run stage before the Huffman coder. The returned structure keeps
    a reference to the blob."""
    p = dict(DEFAULTS)
    p.update(kw)
    out = _Params()
    out.auto_select = 1 if auto else 0
    out.open_loop = 1 if open_loop else 0
    out.zero_run = int(zero_run) if not isinstance(zero_run, bool) else (1 if zero_run else 0)
    out.f_op = {"barycentric": 0, "cluster": 1}[f_op] if isinstance(f_op, str) else int(f_op)
    out.g_op = {"multilinear": 0, "nearest": 1}[g_op] if isinstance(g_op, str) else int(g_op)
    if model is not None:
        blob = np.ascontiguousarray(model, dtype=np.uint8)
        out._blob = blob
        out.model = blob.ctypes.data
        out.model_bytes = blob.size
    out.dtype = 0 if np.dtype(dtype) == np.float64 else 1
    out.eb_mode = 1 if p["eb_mode"] in ("rel", 1) else 0
    out.eb = float(p["eb"])
    out.grid_fraction = float(p["grid_fraction"])
    for k in ("R1", "R2", "C1", "C2", "lmax"):
        setattr(out, k, int(p[k]))
    return out


def field_params(x, **kw):
    x = np.ascontiguousarray(x)
    p = make_params(x.dtype, **kw)
    f = _Field()
    st = _load().orc_field_params(C.byref(p), x.size, _ptr(x), C.byref(f))
    if st:
        raise OracleError(st, "field_params")
    return {k: getattr(f, k) for k, _ in _Field._fields_}


def compress_bound(plan: Plan, dtype, **kw):
    p = make_params(dtype, **kw)
    return int(_load().orc_compress_bound(C.byref(plan.grid._g), plan.n_v, C.byref(p)))


def compress(plan: Plan, x, debug=False, **kw):
    """Algorithm 3 (closed loop). Returns the stream as a uint8 array, plus a
    dict of intermediates (Q, q1, sym1, sym2) when ``debug``."""
    x = np.ascontiguousarray(x)
    if x.dtype not in (np.float64, np.float32):
        raise TypeError("values must be float64 or float32")
    p = make_params(x.dtype, **kw)
    cap = compress_bound(plan, x.dtype, **kw)
    out = np.zeros(cap, dtype=np.uint8)
    size = C.c_size_t(0)
    dbg = None
    if debug:
        dbg = dict(Q=np.empty(plan.n_v, np.int32), q1=np.empty(plan.n_g, np.int32),
                   sym1=np.empty(plan.n_g, np.uint16), sym2=np.empty(plan.n_v, np.uint16))
    st = _load().orc_compress(C.byref(plan.grid._g), plan.n_v, _ptr(plan.vid), _ptr(plan.lam),
                              _ptr(plan.cell), _ptr(plan.frac), _ptr(x), C.byref(p), _ptr(out),
                              cap, C.byref(size),
                              _ptr(dbg["Q"]) if dbg else None, _ptr(dbg["q1"]) if dbg else None,
                              _ptr(dbg["sym1"]) if dbg else None,
                              _ptr(dbg["sym2"]) if dbg else None)
    if st:
        raise OracleError(st, "compress")
    out = out[: size.value].copy()
    return (out, dbg) if debug else out


def decompress(plan: Plan, stream, debug=False):
    """Algorithm 4. Returns the reconstructed vertex values (dtype from the
    stream header), plus the decoded grid codes when ``debug``."""
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    dtype = np.float64
    if stream.size >= 16 and int(stream[12:16].view(np.uint32)[0]) == 1:
        dtype = np.float32
    x = np.empty(plan.n_v, dtype=dtype)
    q1 = np.empty(plan.n_g, np.int32) if debug else None
    st = _load().orc_decompress(C.byref(plan.grid._g), plan.n_v, _ptr(plan.cell),
                                _ptr(plan.frac), _ptr(stream), stream.size, _ptr(x), _ptr(q1))
    if st:
        raise OracleError(st, "decompress")
    return (x, q1) if debug else x


def compress_1d(x, debug=False, **kw):
    """The paper's default: the vertex array in storage order through the
    same coder in 1D. Returns the stream (and the codes Q when ``debug``)."""
    x = np.ascontiguousarray(x)
    if x.dtype not in (np.float64, np.float32):
        raise TypeError("values must be float64 or float32")
    p = make_params(x.dtype, **kw)
    cap = int(_load().orc_compress_bound_1d(x.size, C.byref(p)))
    out = np.zeros(cap, dtype=np.uint8)
    size = C.c_size_t(0)
    Q = np.empty(x.size, np.int32) if debug else None
    st = _load().orc_compress_1d(x.size, _ptr(x), C.byref(p), _ptr(out), cap, C.byref(size),
                                 _ptr(Q) if debug else None)
    if st:
        raise OracleError(st, "compress_1d")
    out = out[: size.value].copy()
    return (out, Q) if debug else out


def decompress_1d(stream, n):
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    dtype = np.float32 if stream.size >= 16 and int(stream[12:16].view(np.uint32)[0]) == 1 \
        else np.float64
    x = np.empty(n, dtype=dtype)
    st = _load().orc_decompress_1d(n, _ptr(stream), stream.size, _ptr(x))
    if st:
        raise OracleError(st, "decompress_1d")
    return x


# --------------------------------------------------------------------------- #
# building blocks (pin tests)
# --------------------------------------------------------------------------- #
def huffman_lengths(counts, lmax=24):
    counts = _c(counts, np.uint64)
    ln = np.zeros(counts.size, dtype=np.uint8)
    st = _load().orc_huffman_lengths(_ptr(counts), counts.size, lmax, _ptr(ln))
    if st:
        raise OracleError(st, "huffman_lengths")
    return ln


def canonical_codes(lengths):
    lengths = _c(lengths, np.uint8)
    code = np.zeros(lengths.size, dtype=np.uint32)
    _load().orc_canonical_codes(_ptr(lengths), lengths.size, _ptr(code))
    return code


def lorenzo(q):
    q = _c(q, np.int32)
    dim = q.ndim
    n = np.ones(3, dtype=np.int32)
    n[:dim] = q.shape[::-1]  # array is [z][y][x] / [y][x]; x fastest
    d = np.empty_like(q)
    _load().orc_lorenzo(dim, _ptr(n), _ptr(q), _ptr(d))
    return d


def lorenzo_inverse(d):
    d = _c(d, np.int32)
    dim = d.ndim
    n = np.ones(3, dtype=np.int32)
    n[:dim] = d.shape[::-1]
    q = np.empty_like(d)
    _load().orc_lorenzo_inverse(dim, _ptr(n), _ptr(d), _ptr(q))
    return q


# --------------------------------------------------------------------------- #
# learned predictor
# --------------------------------------------------------------------------- #
MODEL_BYTES = 5736
MLP_PARAMS = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def pack_model(dim, sx, s1, s2, e3, W1, W2, W3, b1, b2, b3):
    """Model blob from its integer fields (the byte format the stream embeds):
    magic, version 1, dim, n_in, sx, s1, s2, e3, W1 int8 [64][16],
    W2 int8 [64][64], W3 int8 [64], b1, b2 int32 [64], b3 int32."""
    blob = np.zeros(MODEL_BYTES, np.uint8)
    head = np.array([0x4D43434D, 1, dim, (1 << dim) + dim, sx, s1, s2, e3], np.int64)
    blob[0:32] = head.astype(np.uint32).view(np.uint8)
    blob[32:1056] = np.asarray(W1, np.int8).reshape(-1).view(np.uint8)
    blob[1056:5152] = np.asarray(W2, np.int8).reshape(-1).view(np.uint8)
    blob[5152:5216] = np.asarray(W3, np.int8).reshape(-1).view(np.uint8)
    blob[5216:5472] = np.asarray(b1, np.int32).view(np.uint8)
    blob[5472:5728] = np.asarray(b2, np.int32).view(np.uint8)
    blob[5728:5732] = np.asarray([b3], np.int32).view(np.uint8)
    return blob


def unpack_model(blob):
    """Inverse of pack_model: dict of the integer fields."""
    blob = np.asarray(blob, np.uint8)
    head = blob[0:32].view(np.int32)
    return dict(magic=int(np.uint32(head[0])), version=int(head[1]), dim=int(head[2]),
                n_in=int(head[3]), sx=int(head[4]), s1=int(head[5]), s2=int(head[6]),
                e3=int(head[7]), W1=blob[32:1056].view(np.int8).reshape(64, 16).copy(),
                W2=blob[1056:5152].view(np.int8).reshape(64, 64).copy(),
                W3=blob[5152:5216].view(np.int8).copy(), b1=blob[5216:5472].view(np.int32).copy(),
                b2=blob[5472:5728].view(np.int32).copy(), b3=int(blob[5728:5732].view(np.int32)[0]))


def split_params(params):
    """Float parameter vector (5313) -> W1 [64,16], b1, W2 [64,64], b2, W3, b3."""
    params = np.asarray(params)
    o = np.cumsum([0, 1024, 64, 4096, 64, 64, 1])
    W1, b1, W2, b2, W3, b3 = (params[o[i]:o[i + 1]] for i in range(6))
    return W1.reshape(64, 16), b1, W2.reshape(64, 64), b2, W3, b3


def mlp_quantize(dim, sx, params, max_z1, max_z2):
    """Post-training quantisation of the float network into a model blob."""
    params = _c(params, np.float32)
    assert params.size == MLP_PARAMS
    blob = np.zeros(MODEL_BYTES, np.uint8)
    st = _load().orc_mlp_quantize(dim, sx, _ptr(params), float(max_z1), float(max_z2), _ptr(blob))
    if st:
        raise OracleError(st, "mlp_quantize")
    return blob


def mlp_predict(dim, model, corners, fr, rho12_f, Qhi=0):
    """Integer-exact predictor: corners int32 [n, 8], fr float32 [n, 3], s1/s2
    in FP32 and the largest vertex code -> (features int32 [n, 16], p float32
    [n])."""
    model = _c(model, np.uint8)
    corners = _c(corners, np.int32)
    fr = _c(fr, np.float32)
    n = corners.shape[0]
    feats = np.zeros((n, 16), np.int32)
    p = np.zeros(n, np.float32)
    st = _load().orc_mlp_predict(dim, _ptr(model), model.size, _ptr(corners), _ptr(fr),
                                 float(rho12_f), int(Qhi), n, _ptr(feats), _ptr(p))
    if st:
        raise OracleError(st, "mlp_predict")
    return feats, p


def mlp_grad(W1, b1, W2, b2, W3, b3, X, Y, loss="l1", rounding=True):
    """FP64 loss and gradient of the training network. loss: "l1" (mean
    absolute error) or "l2" (mean squared error); rounding: round the
    tensor-core operands to bfloat16 as the GPU does."""
    arrs = [_c(a, np.float32) for a in (W1, b1, W2, b2, W3, b3, X, Y)]
    grad = np.zeros(MLP_PARAMS)
    lossv = np.zeros(1)
    st = _load().orc_mlp_grad(*[_ptr(a) for a in arrs], arrs[6].shape[0],
                              {"l2": 0, "l1": 1}[loss], 1 if rounding else 0, _ptr(grad),
                              _ptr(lossv))
    if st:
        raise ValueError(f"orc_mlp_grad: status {st}")
    return float(lossv[0]), grad
