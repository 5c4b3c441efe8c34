"""FP64 CPU oracle for the learned-closure network.

TEST INFRASTRUCTURE ONLY: the tests use it; the product library never
imports, links or runs it.  It shares no code with the CUDA path.

The paper has no learned closure; the network it checks is the one the
library defines for its closure extension (a coarse 2D vorticity field in,
the subgrid term out):

* four 3x3 convolutions on a periodic ``H x W`` grid, channels
  1 -> 32 -> 32 -> 32 -> 1, as cross-correlations
  ``z[co](p) = b[co] + sum_ci sum_{dy,dx in -1..1} W[co, ci, dy+1, dx+1] a[ci](p + (dy, dx))``
  with ``p = (y, x)`` taken modulo the grid;
* exact GELU, ``GELU(z) = z Phi(z)`` with the normal CDF ``Phi``, after the
  first three convolutions, none after the last;
* loss = mean over all outputs of ``(y - t)^2``;
* Adam (Kingma & Ba 2015, Algorithm 1) with beta1 = 0.9, beta2 = 0.999,
  eps = 1e-8, bias-corrected moments.

Parameters are one flat vector in the order W0 b0 W1 b1 W2 b2 W3 b3, W_l as
``[Cout][Cin][3][3]`` (C order).  Everything is plain numpy in float64;
gradients follow the chain rule layer by layer, with no fusion.
Parity pins: ``tests/test_oracle_closure.py``.
"""
from __future__ import annotations

import math

import numpy as np

CHANNELS = (1, 32, 32, 32, 1)


def layer_shapes(channels=CHANNELS):
    """[(Cout, Cin)] per layer."""
    return [(channels[i + 1], channels[i]) for i in range(len(channels) - 1)]


def num_params(channels=CHANNELS) -> int:
    return sum(co * ci * 9 + co for co, ci in layer_shapes(channels))


def unpack(p: np.ndarray, channels=CHANNELS):
    """Flat vector -> [(W [Cout, Cin, 3, 3], b [Cout])] (views as float64 copies)."""
    p = np.asarray(p, dtype=np.float64)
    out, off = [], 0
    for co, ci in layer_shapes(channels):
        w = p[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = p[off:off + co]
        off += co
        out.append((w, b))
    assert off == p.size
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def shifted(a: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """a(p + (dy, dx)) on the periodic grid, for arrays [..., H, W]."""
    return np.roll(a, shift=(-dy, -dx), axis=(-2, -1))


def conv(a: np.ndarray, w: np.ndarray, b) -> np.ndarray:
    """Periodic 3x3 cross-correlation: a [B, Cin, H, W], w [Cout, Cin, 3, 3],
    b [Cout] or None -> [B, Cout, H, W]."""
    bsz, cin, h, wd = a.shape
    cout = w.shape[0]
    out = np.zeros((bsz, cout, h, wd))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            s = shifted(a, dy, dx)
            out += np.einsum("oc,bchw->bohw", w[:, :, dy + 1, dx + 1], s)
    if b is not None:
        out += np.asarray(b)[None, :, None, None]
    return out


_erf = np.vectorize(math.erf, otypes=[np.float64])


def normal_cdf(z):
    return 0.5 * (1.0 + _erf(np.asarray(z, dtype=np.float64) / math.sqrt(2.0)))


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return z * normal_cdf(z)


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return normal_cdf(z) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(p: np.ndarray, x: np.ndarray, channels=CHANNELS):
    """x [B, H, W] -> y [B, H, W] and the per-layer (input, pre-activation) cache."""
    layers = unpack(p, channels)
    a = np.asarray(x, dtype=np.float64)[:, None]
    cache = []
    for i, (w, b) in enumerate(layers):
        z = conv(a, w, b)
        cache.append((a, z))
        a = gelu(z) if i < len(layers) - 1 else z
    return a[:, 0], cache


def loss(p: np.ndarray, x: np.ndarray, t: np.ndarray, channels=CHANNELS) -> float:
    y, _ = forward(p, x, channels)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradients(p: np.ndarray, x: np.ndarray, t: np.ndarray, channels=CHANNELS):
    """(flat gradient of the loss, loss), by the chain rule:
    dL/dy = 2 (y - t) / count;  for z = conv(a, W) + b:
    dL/dW[co, ci, k] = sum_{b,p} dz[co](p) a[ci](p + off_k),  dL/db[co] = sum dz[co],
    dL/da[ci](q) = sum_co sum_k W[co, ci, k] dz[co](q - off_k);
    below a GELU, dz = da * GELU'(z)."""
    layers = unpack(p, channels)
    y, cache = forward(p, x, channels)
    t = np.asarray(t, dtype=np.float64)
    n = y.size
    dz = (2.0 * (y - t) / n)[:, None]
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        w, _ = layers[i]
        a, _ = cache[i]
        dw = np.zeros_like(w)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                dw[:, :, dy + 1, dx + 1] = np.einsum("bohw,bchw->oc", dz, shifted(a, dy, dx))
        db = dz.sum(axis=(0, 2, 3))
        grads[i] = (dw, db)
        if i > 0:
            da = np.zeros_like(a)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    da += np.einsum("oc,bohw->bchw", w[:, :, dy + 1, dx + 1], shifted(dz, -dy, -dx))
            dz = da * gelu_grad(cache[i - 1][1])
    return pack(grads), float(np.mean((y - t) ** 2))


def adam_step(p, g, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step counts from 1); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
