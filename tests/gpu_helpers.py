"""Helpers that drive the CUDA library through its C ABI (via the thin
binding) on numpy inputs, for the GPU parity tests."""
import numpy as np
import torch

import paper_2501_06910_gb300 as mcc


def plan(coords, cells, n, lo=None, hi=None, keep=None):
    c = torch.from_numpy(np.ascontiguousarray(coords, dtype=np.float64)).cuda()
    e = torch.from_numpy(np.ascontiguousarray(cells, dtype=np.int32)).cuda()
    p = mcc.plan_create(c, e, n, lo, hi, keep=keep)
    torch.cuda.synchronize()
    return p


def tables(p):
    t = p.copy_tables()
    torch.cuda.synchronize()
    return dict(vid=t["vid"].cpu().numpy(), lam=t["lam"].cpu().numpy().view(np.uint16),
                cell=t["cell"].cpu().numpy().view(np.uint32),
                frac=t["frac"].cpu().numpy().view(np.uint16))


def params(x_dtype, **kw):
    return mcc.params_default(dtype=mcc.F64 if np.dtype(x_dtype) == np.float64 else mcc.F32, **kw)


def compress(p, x, **kw):
    prm = params(x.dtype, **kw)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ws = p.workspace(prm)
    out = torch.zeros(mcc.compress_bound(p, prm), dtype=torch.uint8, device="cuda")
    size = mcc.compress(p, xt, prm, ws, out)
    return out[:size].cpu().numpy()


def decompress(p, stream, dtype):
    s = torch.from_numpy(np.ascontiguousarray(stream, dtype=np.uint8)).cuda()
    out = torch.empty(p.n_vertices, dtype=torch.float64 if np.dtype(dtype) == np.float64
                      else torch.float32, device="cuda")
    ws = p.workspace(mcc.params_default(), "decompress")
    mcc.decompress(p, s, stream.size, out, ws)
    return out.cpu().numpy()
