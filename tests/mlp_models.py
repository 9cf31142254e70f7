"""Seeded learned-predictor blobs for the tests (inputs, not expected values):
random valid models and models at the edges of the format."""
import numpy as np

import oracle

H = 64


def blank(dim, sx=0, s1=1, s2=1, e3=0):
    return dict(dim=dim, sx=sx, s1=s1, s2=s2, e3=e3, W1=np.zeros((H, 16), np.int8),
                W2=np.zeros((H, H), np.int8), W3=np.zeros(H, np.int8),
                b1=np.zeros(H, np.int32), b2=np.zeros(H, np.int32), b3=0)


def pack(m):
    return oracle.pack_model(**m)


def random_model(dim, seed, sx=0, s1=9, s2=11, e3=-9, bias1=4000, bias2=20000):
    """A valid model whose activations use their 8-bit range."""
    rng = np.random.default_rng(seed)
    n_in = (1 << dim) + dim
    m = blank(dim, sx=sx, s1=s1, s2=s2, e3=e3)
    m["W1"][:, :n_in] = rng.integers(-127, 128, (H, n_in))
    m["W2"][:] = rng.integers(-127, 128, (H, H))
    m["W3"][:] = rng.integers(-127, 128, H)
    m["b1"][:] = rng.integers(-bias1, bias1, H)
    m["b2"][:] = rng.integers(-bias2, bias2, H)
    m["b3"] = int(rng.integers(-1000, 1000))
    return m


def edge_models(dim):
    """Models at the format's edges: saturated activations (shift 1), shifts at
    23 / 24 (the last that passes values, the first that zeroes them), biases
    at +-2^22, the output exponent at both ends."""
    out = []
    m = random_model(dim, 101, s1=1, s2=1, e3=-20)
    out.append(("saturated", m))
    m = random_model(dim, 102, s1=23, s2=24, e3=0, bias1=1 << 22, bias2=1 << 22)
    m["b1"][:4] = [1 << 22, -(1 << 22), (1 << 22) - 1, 1 << 21]
    out.append(("shift23_24", m))
    m = random_model(dim, 103, sx=-3, s1=6, s2=12, e3=-100)
    out.append(("e3_min", m))
    m = random_model(dim, 104, sx=5, s1=7, s2=13, e3=60)
    out.append(("e3_max", m))
    m = random_model(dim, 105, s1=8, s2=14, e3=-12, bias2=1 << 22)
    m["b2"][:8] = (1 << 22)
    out.append(("big_sums", m))
    return out
