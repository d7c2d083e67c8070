"""FP64 reference of the learned-surrogate network (test infrastructure only).

The paper has no learned component; this restates, in plain NumPy, the network the library
trains: 3x3x3 convolutions with padding 1 (first 2 -> C with stride 2, then stride-2 convs
C -> C down to an edge of 2, then one stride-1 conv), ReLU after each, the flattened result
concatenated with per-cell features, a ReLU dense layer to H units and a linear dense layer to
the outputs; loss = mean squared error.  ``round_bf16`` applies the BF16 rounding the library
uses for weights (round to nearest even of the FP32 value) so that GPU and oracle compute the
same function; finite-difference checks use exact weights.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to BF16 (nearest even) through the FP32 bit pattern; returns FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def layout(cell: int, n_feat: int, n_out: int, C: int, H: int) -> List[dict]:
    """Layers in parameter order: conv layers, hidden dense, output dense (weights then bias)."""
    layers, off, d, cin = [], 0, cell, 2
    n2 = int(round(math.log2(cell))) - 1
    for l in range(n2 + 1):
        stride = 2 if l < n2 else 1
        dout = (d + 2 - 3) // stride + 1
        nw = C * cin * 27
        layers.append(dict(kind="conv", cin=cin, cout=C, din=d, dout=dout, stride=stride, relu=True,
                           woff=off, boff=off + nw))
        off += nw + C
        d, cin = dout, C
    nflat = C * d ** 3
    for nin, nout, relu in ((nflat + n_feat, H, True), (H, n_out, False)):
        layers.append(dict(kind="dense", cin=nin, cout=nout, relu=relu, woff=off, boff=off + nin * nout))
        off += nin * nout + nout
    return layers


def n_params(cell, n_feat, n_out, C, H) -> int:
    L = layout(cell, n_feat, n_out, C, H)
    last = L[-1]
    return last["boff"] + last["cout"]


def _conv_fwd(x, W, b, stride):
    B, cin, d = x.shape[0], x.shape[1], x.shape[2]
    cout = W.shape[0]
    dout = (d + 2 - 3) // stride + 1
    xp = np.zeros((B, cin, d + 2, d + 2, d + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((B, cout, dout, dout, dout))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, :, dz:dz + stride * dout:stride, dy:dy + stride * dout:stride, dx:dx + stride * dout:stride]
                out += np.einsum("bcxyz,oc->boxyz", patch, W[:, :, dz, dy, dx])
    return out + b[None, :, None, None, None]


def _conv_bwd(x, W, g, stride):
    """Gradients (dx, dW, db) of sum(g * conv(x))."""
    B, cin, d = x.shape[0], x.shape[1], x.shape[2]
    dout = g.shape[2]
    xp = np.zeros((B, cin, d + 2, d + 2, d + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = (slice(None), slice(None), slice(dz, dz + stride * dout, stride),
                      slice(dy, dy + stride * dout, stride), slice(dx, dx + stride * dout, stride))
                dW[:, :, dz, dy, dx] = np.einsum("boxyz,bcxyz->oc", g, xp[sl])
                dxp[sl] += np.einsum("boxyz,oc->bcxyz", g, W[:, :, dz, dy, dx])
    return dxp[:, :, 1:-1, 1:-1, 1:-1], dW, g.sum(axis=(0, 2, 3, 4))


def forward(params: np.ndarray, x: np.ndarray, f: np.ndarray, cell, n_feat, n_out, C, H, round_bf16=True):
    """Returns (outputs, cache)."""
    L = layout(cell, n_feat, n_out, C, H)
    p = np.asarray(params, dtype=np.float64)
    q = bf16(p) if round_bf16 else p
    B = x.shape[0]
    a = np.asarray(x, dtype=np.float64).reshape(B, 2, cell, cell, cell)
    cache = []
    for l in L:
        W = q[l["woff"]:l["boff"]]
        b = p[l["boff"]:l["boff"] + l["cout"]]
        if l["kind"] == "conv":
            W = W.reshape(l["cout"], l["cin"], 3, 3, 3)
            z = _conv_fwd(a, W, b, l["stride"])
        else:
            if a.ndim > 2:
                a = np.concatenate([a.reshape(B, -1), np.asarray(f, np.float64).reshape(B, -1)], axis=1)
            W = W.reshape(l["cout"], l["cin"])
            z = a @ W.T + b
        out = np.maximum(z, 0) if l["relu"] else z
        cache.append((a, W, out))
        a = out
    return a, cache


def backward(params, x, f, dy, cell, n_feat, n_out, C, H, round_bf16=True) -> np.ndarray:
    """Gradient of sum(dy * forward(...)) with respect to the parameter vector."""
    L = layout(cell, n_feat, n_out, C, H)
    _, cache = forward(params, x, f, cell, n_feat, n_out, C, H, round_bf16)
    grad = np.zeros(len(params))
    g = np.asarray(dy, dtype=np.float64)
    B = g.shape[0]
    for l, (a, W, out) in zip(reversed(L), reversed(cache)):
        if l["relu"]:
            g = g * (out > 0)
        if l["kind"] == "conv":
            dx, dW, db = _conv_bwd(a, W, g, l["stride"])
            grad[l["woff"]:l["boff"]] = dW.ravel()
            grad[l["boff"]:l["boff"] + l["cout"]] = db
            g = dx
        else:
            grad[l["woff"]:l["boff"]] = (g.T @ a).ravel()
            grad[l["boff"]:l["boff"] + l["cout"]] = g.sum(axis=0)
            g = g @ W
            if l is L[-2]:
                last_conv = L[-3]
                nflat = last_conv["cout"] * last_conv["dout"] ** 3
                g = g[:, :nflat].reshape(B, last_conv["cout"], last_conv["dout"], last_conv["dout"], last_conv["dout"])
    return grad


def mse(y, t, mask=None):
    d = (y - t) if mask is None else (y - t) * mask
    return float(np.mean(d * d))
