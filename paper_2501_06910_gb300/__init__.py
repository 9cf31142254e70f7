"""GB300 (sm_103a) multi-component compressor for data on unstructured
meshes, after Gong et al., "A General Framework for Error-controlled
Unstructured Scientific Data Compression" (Sec. III-IV, Algorithms 3-4).

A thin ctypes binding over the C ABI of ``include/mcc.h`` (``libmcc.so``).
Functions carry the C names without the ``mcc_`` prefix; arguments are
marshalled from torch tensors (device memory, streams) and every step of the
compressor runs in the library's CUDA kernels. There is no CPU fallback: if
the library or a CUDA device is missing, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

import torch

from .native_build import LIB, build

__all__ = [
    "MCCError", "Params", "Plan", "load", "build", "params_default", "plan_create",
    "compress", "decompress", "compress_bound", "workspace_size", "workspace_result",
    "status_string", "profile_enable", "profile_reset", "profile_read", "compress_batch",
    "decompress_batch",
]

OK, INVALID_ARG, CUDA, OOM, RANGE, CORRUPT, CAPACITY, TIMEOUT, UNSUPPORTED = range(9)
F64, F32 = 0, 1
ABS, REL = 0, 1
PRED_ZERO, PRED_LEARNED, PRED_AUTO = 0, 1, 2
LOOP_CLOSED, LOOP_OPEN = 0, 1
F_BARYCENTRIC, F_CLUSTER = 0, 1
G_MULTILINEAR, G_NEAREST = 0, 1
LOSS_L2, LOSS_L1 = 0, 1
MODEL_BYTES = 5736
MLP_PARAMS = 5313

_lock = threading.Lock()
_lib = None


class MCCError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = int(status)
        msg = status_string(status) if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})")


class _Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_vertices", C.c_int64), ("coords", C.c_void_p),
                ("n_cells", C.c_int64), ("cells", C.c_void_p)]


class _GridSpec(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class Params(C.Structure):
    """mcc_params: dtype, eb_mode, eb, grid_fraction, R1, R2, C1, C2, lmax,
    predictor, d_model, loop, f_op, g_op, zero_run."""
    _fields_ = [("dtype", C.c_int), ("eb_mode", C.c_int), ("eb", C.c_double),
                ("grid_fraction", C.c_double), ("R1", C.c_int), ("R2", C.c_int),
                ("C1", C.c_int), ("C2", C.c_int), ("lmax", C.c_int),
                ("predictor", C.c_int), ("d_model", C.c_void_p), ("loop", C.c_int),
                ("f_op", C.c_int), ("g_op", C.c_int), ("zero_run", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrainCfg(C.Structure):
    """mcc_train_cfg: steps, batch, lr, beta1, beta2, eps, loss,
    samples_per_field, seed."""
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("loss", C.c_int),
                ("samples_per_field", C.c_int64), ("seed", C.c_uint64)]


class Tuning(C.Structure):
    _fields_ = [("tile2d", C.c_int), ("vertex_blocks_per_sm", C.c_int), ("batch_fields", C.c_int),
                ("net_path", C.c_int)]


TILE_64x16, TILE_32x32, TILE_128x8 = 0, 1, 2
NET_MMA_SYNC, NET_TCGEN05 = 0, 1


class _PlanInfo(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("h", C.c_double * 3), ("n_vertices", C.c_int64), ("n_grid", C.c_int64),
                ("n_outside", C.c_int64)]


def load():
    """Load libmcc.so (building it first when stale). Raises when no CUDA
    device is present: the library has no host fallback."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                build()
            lib = C.CDLL(LIB)
            P, S = C.c_void_p, C.c_size_t
            lib.mcc_params_default.argtypes = [C.POINTER(Params)]
            lib.mcc_params_default.restype = None
            lib.mcc_status_string.argtypes = [C.c_int]
            lib.mcc_status_string.restype = C.c_char_p
            lib.mcc_plan_create.argtypes = [C.POINTER(_Mesh), C.POINTER(_GridSpec), P, C.POINTER(P)]
            lib.mcc_plan_create_kept.argtypes = [C.POINTER(_Mesh), C.POINTER(_GridSpec), P, P, P,
                                                 C.POINTER(P)]
            lib.mcc_grid_coarsen.argtypes = [P, C.c_int, P, P, P]
            lib.mcc_workspace_size_1d.argtypes = [C.c_int64, C.POINTER(Params), C.POINTER(S),
                                                  C.POINTER(S)]
            lib.mcc_compress_bound_1d.argtypes = [C.c_int64, C.POINTER(Params), C.POINTER(S)]
            lib.mcc_compress_1d.argtypes = [P, C.c_int64, C.POINTER(Params), P, S, P, S,
                                            C.POINTER(S), P]
            lib.mcc_decompress_1d.argtypes = [P, S, P, C.c_int64, C.c_int, P, S, C.c_int, P]
            lib.mcc_grid_init.argtypes = [C.POINTER(_Mesh), C.c_double, C.c_double, C.c_int32,
                                          C.POINTER(_GridSpec), P]
            lib.mcc_plan_destroy.argtypes = [P]
            lib.mcc_plan_destroy.restype = None
            lib.mcc_plan_get_info.argtypes = [P, C.POINTER(_PlanInfo)]
            lib.mcc_plan_copy_tables.argtypes = [P, P, P, P, P, P]
            lib.mcc_workspace_size.argtypes = [P, C.POINTER(Params), C.POINTER(S), C.POINTER(S)]
            lib.mcc_compress_bound.argtypes = [P, C.POINTER(Params), C.POINTER(S)]
            lib.mcc_compress.argtypes = [P, P, C.POINTER(Params), P, S, P, S, C.POINTER(S), P]
            lib.mcc_decompress.argtypes = [P, P, S, P, C.c_int, P, S, C.c_int, P]
            lib.mcc_workspace_result.argtypes = [P, P, C.POINTER(S)]
            lib.mcc_compress_batch.argtypes = [P, C.c_int, C.POINTER(P), C.POINTER(Params), P, S, P,
                                               S, C.POINTER(S), P]
            lib.mcc_decompress_batch.argtypes = [P, C.c_int, P, S, C.POINTER(S), C.POINTER(P),
                                                 C.c_int, P, S, C.c_int, P]
            lib.mcc_compress_batch.restype = C.c_int
            lib.mcc_decompress_static.argtypes = [P, P, S, P, C.c_int, C.c_int, P]
            lib.mcc_decompress_static.restype = C.c_int
            lib.mcc_plan_set_tuning.argtypes = [P, C.POINTER(Tuning)]
            lib.mcc_plan_set_tuning.restype = C.c_int
            lib.mcc_plan_get_tuning.argtypes = [P, C.POINTER(Tuning)]
            lib.mcc_plan_get_tuning.restype = C.c_int
            lib.mcc_graph_begin.argtypes = [P]
            lib.mcc_graph_begin.restype = C.c_int
            lib.mcc_graph_end.argtypes = [P, C.POINTER(C.c_void_p)]
            lib.mcc_graph_end.restype = C.c_int
            lib.mcc_graph_launch.argtypes = [P, P]
            lib.mcc_graph_launch.restype = C.c_int
            lib.mcc_graph_destroy.argtypes = [P]
            lib.mcc_graph_destroy.restype = None
            lib.mcc_static_scratch_bytes.argtypes = []
            lib.mcc_static_scratch_bytes.restype = S
            lib.mcc_decompress_batch.restype = C.c_int
            lib.mcc_profile_enable.argtypes = [C.c_int]
            lib.mcc_profile_enable.restype = None
            lib.mcc_profile_reset.argtypes = []
            lib.mcc_profile_reset.restype = None
            lib.mcc_profile_read.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]
            lib.mcc_profile_read.restype = C.c_int
            lib.mcc_train_cfg_default.argtypes = [C.POINTER(TrainCfg)]
            lib.mcc_train_cfg_default.restype = None
            lib.mcc_train_workspace_size.argtypes = [P, C.POINTER(Params), C.POINTER(TrainCfg),
                                                     C.c_int, C.POINTER(S)]
            lib.mcc_model_train.argtypes = [P, C.c_int, C.POINTER(P), C.POINTER(Params),
                                            C.POINTER(TrainCfg), P, S, P, P, P]
            lib.mcc_mlp_grad_workspace_size.argtypes = [C.c_int64]
            lib.mcc_mlp_grad_workspace_size.restype = S
            lib.mcc_mlp_grad.argtypes = [P, P, P, C.c_int64, C.c_int, P, S, P, P, P]
            lib.mcc_mlp_quantize.argtypes = [C.c_int, C.c_int, P, C.c_float, C.c_float, P, P, P]
            for fn in ("mcc_train_workspace_size", "mcc_model_train", "mcc_mlp_grad",
                       "mcc_mlp_quantize"):
                getattr(lib, fn).restype = C.c_int
            for fn in ("mcc_plan_create", "mcc_plan_create_kept", "mcc_grid_coarsen",
                       "mcc_plan_get_info", "mcc_plan_copy_tables",
                       "mcc_workspace_size", "mcc_compress_bound", "mcc_compress",
                       "mcc_decompress", "mcc_workspace_result"):
                getattr(lib, fn).restype = C.c_int
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().mcc_status_string(int(status)).decode()


def _check(status, what):
    if status != OK:
        raise MCCError(status, what)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def params_default(model=None, auto=False, open_loop=False, **overrides) -> Params:
    """Parameters; ``model`` (a CUDA uint8 tensor of MODEL_BYTES) selects the
    learned predictor, or with ``auto`` the smaller of learned and plain;
    ``open_loop`` takes the residual against the unquantised grid component
    (bound tau1 + tau2); ``f_op`` ("barycentric" / "cluster") and ``g_op``
    ("multilinear" / "nearest") pick the operators; ``zero_run=True`` turns
    on the zero-run stage before the Huffman coder. The structure keeps a
    reference to the tensor."""
    p = Params()
    load().mcc_params_default(C.byref(p))
    if open_loop:
        p.loop = LOOP_OPEN
    for k, table in (("f_op", {"barycentric": F_BARYCENTRIC, "cluster": F_CLUSTER}),
                     ("g_op", {"multilinear": G_MULTILINEAR, "nearest": G_NEAREST})):
        if isinstance(overrides.get(k), str):
            overrides[k] = table[overrides[k]]
    if model is not None:
        if model.dtype != torch.uint8 or model.numel() != MODEL_BYTES:
            raise ValueError("model must be a uint8 tensor of MODEL_BYTES bytes")
        p._model = model
        p.predictor = PRED_AUTO if auto else PRED_LEARNED
        p.d_model = _dptr(model).value
    for k, v in overrides.items():
        if k == "dtype" and not isinstance(v, int):
            v = F64 if v in (torch.float64, "float64", "f64") else F32
        if k == "eb_mode" and isinstance(v, str):
            v = REL if v == "rel" else ABS
        if k == "zero_run" and isinstance(v, bool):
            v = int(v)
        setattr(p, k, v)
    return p


class Plan:
    """Owner of an ``mcc_plan`` (mesh -> grid mapping tables on the device)."""

    def __init__(self, handle, info):
        self._h = handle
        self.dim = info.dim
        self.n = tuple(info.n[: info.dim])
        self.lo = tuple(info.lo[: info.dim])
        self.h = tuple(info.h[: info.dim])
        self.n_vertices = info.n_vertices
        self.n_grid = info.n_grid
        self.n_outside = info.n_outside

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().mcc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def copy_tables(self, stream=None):
        """Device copies of the plan tables (vid, lam, cell, frac)."""
        d, ng, nv = self.dim, self.n_grid, self.n_vertices
        dev = torch.device("cuda")
        vid = torch.empty((d + 1, ng), dtype=torch.int32, device=dev)
        lam = torch.empty((d, ng), dtype=torch.int16, device=dev)
        cell = torch.empty(nv, dtype=torch.int32, device=dev)
        frac = torch.empty((d, nv), dtype=torch.int16, device=dev)
        _check(load().mcc_plan_copy_tables(self._h, _dptr(vid), _dptr(lam), _dptr(cell),
                                           _dptr(frac), _stream(stream)), "plan_copy_tables")
        return dict(vid=vid, lam=lam, cell=cell, frac=frac)

    def workspace(self, params: Params, which="compress"):
        c, d = workspace_size(self, params)
        return torch.empty(c if which == "compress" else d, dtype=torch.uint8, device="cuda")


def plan_create(coords: torch.Tensor, cells: torch.Tensor, n, lo=None, hi=None,
                stream=None, keep=None) -> Plan:
    """mcc_plan_create: coords float64 [n_v, dim], cells int32 [n_c, dim+1],
    both on the device; n grid points per axis; lo/hi corners (None: the mesh
    bounding box). ``keep`` (one increasing index array per axis, e.g. from
    ``grid_coarsen``) builds the plan on those planes of that grid
    (mcc_plan_create_kept)."""
    dim = coords.shape[1]
    m = _Mesh(dim, coords.shape[0], _dptr(coords).value, cells.shape[0], _dptr(cells).value)
    g = _GridSpec()
    for d in range(3):
        g.n[d] = n[d] if d < dim else 1
        g.lo[d] = lo[d] if lo is not None and d < dim else 0.0
        g.hi[d] = hi[d] if hi is not None and d < dim else 0.0
    h = C.c_void_p()
    if keep is None:
        _check(load().mcc_plan_create(C.byref(m), C.byref(g), _stream(stream), C.byref(h)),
               "plan_create")
    else:
        flat = np.ascontiguousarray(np.concatenate([np.asarray(keep[d], dtype=np.int32)
                                                    for d in range(dim)]), dtype=np.int32)
        nk = (C.c_int32 * 3)(*[len(keep[d]) if d < dim else 1 for d in range(3)])
        _check(load().mcc_plan_create_kept(C.byref(m), C.byref(g), flat.ctypes.data,
                                           C.cast(nk, C.c_void_p), _stream(stream), C.byref(h)),
               "plan_create_kept")
    info = _PlanInfo()
    _check(load().mcc_plan_get_info(h, C.byref(info)), "plan_get_info")
    return Plan(h, info)


def _tuning(plan: "Plan") -> Tuning:
    t = Tuning()
    _check(load().mcc_plan_get_tuning(plan.handle, C.byref(t)), "plan_get_tuning")
    return t


def set_tuning(plan: "Plan", tile2d: int, vertex_blocks_per_sm: int, batch_fields: int = 0):
    """mcc_plan_set_tuning: the launch configuration of the plan's kernels
    (the network's tensor-core path stays as set by set_net_path)."""
    t = _tuning(plan)
    t.tile2d, t.vertex_blocks_per_sm, t.batch_fields = \
        int(tile2d), int(vertex_blocks_per_sm), int(batch_fields)
    _check(load().mcc_plan_set_tuning(plan.handle, C.byref(t)), "plan_set_tuning")


def get_tuning(plan: "Plan"):
    t = _tuning(plan)
    return int(t.tile2d), int(t.vertex_blocks_per_sm), int(t.batch_fields)


def set_net_path(plan: "Plan", path: int):
    """The learned predictor's tensor-core path on this plan (mcc_tuning
    net_path): NET_MMA_SYNC (default) or NET_TCGEN05."""
    t = _tuning(plan)
    t.net_path = int(path)
    _check(load().mcc_plan_set_tuning(plan.handle, C.byref(t)), "plan_set_tuning")


def get_net_path(plan: "Plan") -> int:
    return int(_tuning(plan).net_path)


def grid_coarsen(plan: Plan, g_op="multilinear", stream=None):
    """mcc_grid_coarsen (Algorithm 2): the kept plane indices per axis (a list
    of int32 numpy arrays) of a plan's uniform grid, for plan_create(...,
    keep=...) with the same n, lo and hi."""
    gop = {"multilinear": G_MULTILINEAR, "nearest": G_NEAREST}[g_op] if isinstance(g_op, str) \
        else int(g_op)
    out = np.empty(int(sum(plan.n)), dtype=np.int32)
    n_out = (C.c_int32 * 3)()
    _check(load().mcc_grid_coarsen(plan.handle, gop, out.ctypes.data, C.cast(n_out, C.c_void_p),
                                   _stream(stream)), "grid_coarsen")
    res, o = [], 0
    for d in range(plan.dim):
        res.append(out[o: o + n_out[d]].copy())
        o += n_out[d]
    return res


def grid_init(coords: torch.Tensor, cells: torch.Tensor, k_pct: float, delta_pct: float = 1.0,
              gmax: int = 4096, stream=None):
    """mcc_grid_init (Algorithm 1): (n, lo, hi) per axis for plan_create from
    the bottom k-th percentile of the cells' edge extents."""
    dim = coords.shape[1]
    m = _Mesh(dim, coords.shape[0], _dptr(coords).value, cells.shape[0], _dptr(cells).value)
    g = _GridSpec()
    _check(load().mcc_grid_init(C.byref(m), C.c_double(k_pct), C.c_double(delta_pct),
                                C.c_int32(gmax), C.byref(g), _stream(stream)), "grid_init")
    return tuple(g.n[:dim]), tuple(g.lo[:dim]), tuple(g.hi[:dim])


def workspace_size_1d(n: int, params: Params):
    """(compress, decompress) workspace bytes of the 1D coder for n values."""
    cb, db = C.c_size_t(), C.c_size_t()
    _check(load().mcc_workspace_size_1d(n, C.byref(params), C.byref(cb), C.byref(db)),
           "workspace_size_1d")
    return cb.value, db.value


def compress_bound_1d(n: int, params: Params) -> int:
    b = C.c_size_t()
    _check(load().mcc_compress_bound_1d(n, C.byref(params), C.byref(b)), "compress_bound_1d")
    return b.value


def compress_1d_into(x: torch.Tensor, params: Params, workspace: torch.Tensor, out: torch.Tensor,
                     sync: bool = True, stream=None):
    """mcc_compress_1d (the paper's default baseline): the values in storage
    order through the 1D coder into ``out``; returns the size when ``sync``
    (without it the call only enqueues, so it can be graph-captured)."""
    size = C.c_size_t()
    _check(load().mcc_compress_1d(_dptr(x), x.numel(), C.byref(params), _dptr(workspace),
                                  workspace.numel(), _dptr(out), out.numel(),
                                  C.byref(size) if sync else None, _stream(stream)), "compress_1d")
    return size.value if sync else None


def decompress_1d_into(stream_bytes: torch.Tensor, nbytes: int, out: torch.Tensor,
                       workspace: torch.Tensor, sync: bool = True, stream=None):
    """mcc_decompress_1d into ``out`` (n values of the stream's type)."""
    dtype = F64 if out.dtype == torch.float64 else F32
    _check(load().mcc_decompress_1d(_dptr(stream_bytes), int(nbytes), _dptr(out), out.numel(), dtype,
                                    _dptr(workspace), workspace.numel(), 1 if sync else 0,
                                    _stream(stream)), "decompress_1d")
    return out


def compress_1d(x: torch.Tensor, params: Params, stream=None):
    """compress_1d_into with its own workspace and output; returns the stream
    as a uint8 CUDA tensor."""
    cb, _ = workspace_size_1d(x.numel(), params)
    ws = torch.empty(cb, dtype=torch.uint8, device=x.device)
    out = torch.empty(compress_bound_1d(x.numel(), params), dtype=torch.uint8, device=x.device)
    size = compress_1d_into(x, params, ws, out, True, stream)
    return out[:size]


def decompress_1d(stream_bytes: torch.Tensor, out: torch.Tensor, stream=None):
    """decompress_1d_into with its own workspace."""
    prm = params_default(dtype=F64 if out.dtype == torch.float64 else F32)
    _, db = workspace_size_1d(out.numel(), prm)
    ws = torch.empty(db, dtype=torch.uint8, device=out.device)
    return decompress_1d_into(stream_bytes, stream_bytes.numel(), out, ws, True, stream)


def workspace_size(plan: Plan, params: Params):
    c, d = C.c_size_t(), C.c_size_t()
    _check(load().mcc_workspace_size(plan.handle, C.byref(params), C.byref(c), C.byref(d)),
           "workspace_size")
    return c.value, d.value


def compress_bound(plan: Plan, params: Params) -> int:
    b = C.c_size_t()
    _check(load().mcc_compress_bound(plan.handle, C.byref(params), C.byref(b)), "compress_bound")
    return b.value


def compress(plan: Plan, x: torch.Tensor, params: Params, workspace: torch.Tensor,
             out: torch.Tensor, sync: bool = True, stream=None):
    """mcc_compress. Returns the stream size when ``sync`` (synchronises),
    else None (size later from ``workspace_result``)."""
    size = C.c_size_t(0)
    st = load().mcc_compress(plan.handle, _dptr(x), C.byref(params), _dptr(workspace),
                             workspace.numel(), _dptr(out), out.numel(),
                             C.byref(size) if sync else None, _stream(stream))
    _check(st, "compress")
    return size.value if sync else None


def decompress(plan: Plan, stream_bytes: torch.Tensor, nbytes: int, out: torch.Tensor,
               workspace: torch.Tensor, sync: bool = True, stream=None):
    """mcc_decompress into ``out`` (float64 or float32, n_vertices values)."""
    dtype = F64 if out.dtype == torch.float64 else F32
    st = load().mcc_decompress(plan.handle, _dptr(stream_bytes), int(nbytes), _dptr(out), dtype,
                               _dptr(workspace), workspace.numel(), 1 if sync else 0,
                               _stream(stream))
    _check(st, "decompress")


def workspace_result(workspace: torch.Tensor, stream=None):
    size = C.c_size_t(0)
    st = load().mcc_workspace_result(_dptr(workspace), _stream(stream), C.byref(size))
    return st, size.value


def profile_enable(on: bool = True):
    """mcc_profile_enable: bracket every library kernel with CUDA events."""
    load().mcc_profile_enable(1 if on else 0)


def profile_reset():
    load().mcc_profile_reset()


def profile_read(max_entries: int = 64):
    """mcc_profile_read: {kernel name: (total ms, launches)} (synchronises)."""
    names = (C.c_char * 32 * max_entries)()
    ms = (C.c_double * max_entries)()
    n = (C.c_longlong * max_entries)()
    k = load().mcc_profile_read(C.cast(names, C.c_void_p), ms, n, max_entries)
    return {bytes(names[i]).split(b"\0")[0].decode(): (ms[i], n[i]) for i in range(k)}


def compress_batch(plan: Plan, xs, params, workspace: torch.Tensor, out: torch.Tensor,
                   slot_bytes: int, sync: bool = True, stream=None):
    """mcc_compress_batch: field f of ``xs`` (device tensors) with ``params[f]``
    into ``out[f * slot_bytes:]``. Returns the stream sizes when ``sync``."""
    n = len(xs)
    ptrs = (C.c_void_p * n)(*[_dptr(x).value for x in xs])
    prm = (Params * n)(*params)
    sizes = (C.c_size_t * n)()
    st = load().mcc_compress_batch(plan.handle, n, ptrs, prm, _dptr(workspace), workspace.numel(),
                                   _dptr(out), int(slot_bytes), sizes if sync else None,
                                   _stream(stream))
    _check(st, "compress_batch")
    return [int(v) for v in sizes] if sync else None


def decompress_batch(plan: Plan, stream_bytes: torch.Tensor, slot_bytes: int, in_bytes, outs,
                     workspace: torch.Tensor, sync: bool = True, stream=None):
    """mcc_decompress_batch: field f from ``stream_bytes[f * slot_bytes:]``
    (``in_bytes[f]`` bytes) into ``outs[f]``."""
    n = len(outs)
    ptrs = (C.c_void_p * n)(*[_dptr(y).value for y in outs])
    nb = (C.c_size_t * n)(*[int(v) for v in in_bytes])
    dtype = F64 if outs[0].dtype == torch.float64 else F32
    st = load().mcc_decompress_batch(plan.handle, n, _dptr(stream_bytes), int(slot_bytes), nb, ptrs,
                                     dtype, _dptr(workspace), workspace.numel(), 1 if sync else 0,
                                     _stream(stream))
    _check(st, "decompress_batch")


class Graph:
    """An executable graph of recorded library calls (mcc_graph_*)."""

    def __init__(self, handle):
        self._h = handle

    def launch(self, stream=None):
        _check(load().mcc_graph_launch(self._h, _stream(stream)), "graph_launch")

    def close(self):
        if self._h:
            load().mcc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass


def graph_begin(stream):
    """mcc_graph_begin on ``stream`` (a torch.cuda.Stream, not the default)."""
    _check(load().mcc_graph_begin(_stream(stream)), "graph_begin")


def graph_end(stream) -> Graph:
    """mcc_graph_end: the calls recorded on ``stream`` since graph_begin."""
    h = C.c_void_p()
    _check(load().mcc_graph_end(_stream(stream), C.byref(h)), "graph_end")
    return Graph(h)


def graph_capture(fn, stream) -> Graph:
    """Record the asynchronous library calls ``fn()`` makes on ``stream``
    (``fn`` passes ``stream`` to each call) into a Graph."""
    graph_begin(stream)
    try:
        fn()
    except BaseException:
        try:
            graph_end(stream)
        except MCCError:
            pass
        raise
    return graph_end(stream)


def decompress_static(plan: Plan, stream_bytes: torch.Tensor, nbytes: int, out: torch.Tensor,
                      sync: bool = True, stream=None):
    """mcc_decompress_static: decompression whose scratch memory is a fixed
    array inside the library (no device allocation by the call)."""
    dtype = F64 if out.dtype == torch.float64 else F32
    st = load().mcc_decompress_static(plan.handle, _dptr(stream_bytes), int(nbytes), _dptr(out),
                                      dtype, 1 if sync else 0, _stream(stream))
    _check(st, "decompress_static")


def static_scratch_bytes() -> int:
    return int(load().mcc_static_scratch_bytes())


# --------------------------------------------------------------------------- #
# learned predictor: training
# --------------------------------------------------------------------------- #
def train_cfg_default(**overrides) -> TrainCfg:
    c = TrainCfg()
    load().mcc_train_cfg_default(C.byref(c))
    for k, v in overrides.items():
        if k == "loss" and isinstance(v, str):
            v = LOSS_L1 if v == "l1" else LOSS_L2
        setattr(c, k, v)
    return c


def train_workspace_size(plan: "Plan", params: Params, cfg: TrainCfg, n: int) -> int:
    size = C.c_size_t(0)
    _check(load().mcc_train_workspace_size(plan.handle, C.byref(params), C.byref(cfg), int(n),
                                           C.byref(size)), "train_workspace_size")
    return int(size.value)


def model_train(plan: "Plan", fields, params: Params, cfg: TrainCfg, workspace=None, stream=None):
    """mcc_model_train: returns (model blob as a CUDA uint8 tensor, per-step
    minibatch losses as a list). Synchronises."""
    n = len(fields)
    if workspace is None:
        workspace = torch.empty(train_workspace_size(plan, params, cfg, n), dtype=torch.uint8,
                                device="cuda")
    model = torch.zeros(MODEL_BYTES, dtype=torch.uint8, device="cuda")
    ptrs = (C.c_void_p * n)(*[_dptr(x).value for x in fields])
    losses = (C.c_float * cfg.steps)()
    st = load().mcc_model_train(plan.handle, n, ptrs, C.byref(params), C.byref(cfg),
                                _dptr(workspace), workspace.numel(), _dptr(model), losses,
                                _stream(stream))
    _check(st, "model_train")
    return model, [float(v) for v in losses]


def mlp_grad(params: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, loss="l1", stream=None):
    """mcc_mlp_grad: (gradient as a CUDA float tensor, loss) of the training
    network on the batch (X [B, 16], Y [B], float32 CUDA tensors)."""
    B = int(X.shape[0])
    ws = torch.empty(max(4, int(load().mcc_mlp_grad_workspace_size(B))), dtype=torch.uint8,
                     device="cuda")
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    lossv = torch.empty(1, dtype=torch.float32, device="cuda")
    st = load().mcc_mlp_grad(_dptr(params), _dptr(X), _dptr(Y), B,
                             LOSS_L1 if loss == "l1" else LOSS_L2, _dptr(ws), ws.numel(),
                             _dptr(grad), _dptr(lossv), _stream(stream))
    _check(st, "mlp_grad")
    return grad, lossv


def mlp_quantize(dim: int, sx: int, params: torch.Tensor, max_z1: float, max_z2: float,
                 stream=None):
    """mcc_mlp_quantize: (model blob as a CUDA uint8 tensor, device status)."""
    model = torch.zeros(MODEL_BYTES, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = load().mcc_mlp_quantize(int(dim), int(sx), _dptr(params), float(max_z1), float(max_z2),
                                 _dptr(model), _dptr(status), _stream(stream))
    _check(st, "mlp_quantize")
    return model, status
