"""FP64 CPU oracle for the warm-start network (a 3D convolutional encoder-decoder).

TEST INFRASTRUCTURE ONLY: imported by the tests to check the CUDA network kernels; the library
never imports it and shares no code with it.

The network and its training follow the plain definitions:
* 3D convolution with zero padding: y[b,o,v] = bias[o] + sum_i sum_t w[o,i,t] x[b,i,v + off(t)],
  off(t) running over the 3x3x3 neighbourhood (t = 9 dz' + 3 dy' + dx', d' = d + 1) or the
  single centre tap of a 1x1x1 convolution;
* ReLU, 2x average pooling, 2x nearest-neighbour upsampling, channel concatenation;
* mean squared error and Adam (Kingma & Ba 2015), bias-corrected;
* gradients by reverse-mode differentiation of those definitions.
Arrays are float64, activations [B][C][n][n][n], weights [Co][Ci][k^3].
"""
from __future__ import annotations

import numpy as np


def _offsets(k):
    if k == 1:
        return [(0, 0, 0)]
    return [(t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1) for t in range(27)]


def _shift(a, dx, dy, dz):
    """out[..., z, y, x] = a[..., z + dz, y + dy, x + dx], zero outside."""
    n = a.shape[-1]
    out = np.zeros_like(a)
    zs = slice(max(0, -dz), n - max(0, dz))
    ys = slice(max(0, -dy), n - max(0, dy))
    xs = slice(max(0, -dx), n - max(0, dx))
    zs2 = slice(max(0, dz), n - max(0, -dz))
    ys2 = slice(max(0, dy), n - max(0, -dy))
    xs2 = slice(max(0, dx), n - max(0, -dx))
    out[..., zs, ys, xs] = a[..., zs2, ys2, xs2]
    return out


def conv3d(x, w, b=None):
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    Co, Ci, taps = w.shape
    k = 3 if taps == 27 else 1
    B = x.shape[0]
    y = np.zeros((B, Co) + x.shape[2:])
    for t, (dx, dy, dz) in enumerate(_offsets(k)):
        xs = _shift(x, dx, dy, dz)                      # [B][Ci][n^3]
        y += np.einsum("oi,bizyx->bozyx", w[:, :, t], xs)
    if b is not None:
        y += np.asarray(b, np.float64)[None, :, None, None, None]
    return y


def conv3d_dgrad(dy, w):
    """Gradient w.r.t. x of conv3d (the transpose of the convolution)."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    Co, Ci, taps = w.shape
    k = 3 if taps == 27 else 1
    dx = np.zeros((dy.shape[0], Ci) + dy.shape[2:])
    for t, (ox, oy, oz) in enumerate(_offsets(k)):
        # y[v] uses x[v + o]  =>  dx[u] += w * dy[u - o]
        dx += np.einsum("oi,bozyx->bizyx", w[:, :, t], _shift(dy, -ox, -oy, -oz))
    return dx


def conv3d_wgrad(x, dy, k=3):
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    Ci, Co = x.shape[1], dy.shape[1]
    offs = _offsets(k)
    dw = np.zeros((Co, Ci, len(offs)))
    for t, (dx, ddy, dz) in enumerate(offs):
        dw[:, :, t] = np.einsum("bozyx,bizyx->oi", dy, _shift(x, dx, ddy, dz))
    db = dy.sum(axis=(0, 2, 3, 4))
    return dw, db


def pool2(x):
    B, C, n = x.shape[0], x.shape[1], x.shape[-1]
    m = n // 2
    return np.asarray(x, np.float64).reshape(B, C, m, 2, m, 2, m, 2).mean(axis=(3, 5, 7))


def pool2_bwd(dy):
    return np.repeat(np.repeat(np.repeat(np.asarray(dy, np.float64), 2, 2), 2, 3), 2, 4) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(np.asarray(x, np.float64), 2, 2), 2, 3), 2, 4)


def up2_bwd(dy):
    B, C, n = dy.shape[0], dy.shape[1], dy.shape[-1]
    m = n // 2
    return np.asarray(dy, np.float64).reshape(B, C, m, 2, m, 2, m, 2).sum(axis=(3, 5, 7))


def mse(p, t):
    d = np.asarray(p, np.float64) - np.asarray(t, np.float64)
    return float((d * d).mean()), 2.0 * d / d.size


def adam(w, g, m, v, lr, b1, b2, eps, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# ----------------------------------------------------------------------------------------------
# The encoder-decoder: levels l = 0..L-1 with channels chans[l]; encoder: two 3^3 conv+ReLU per
# level, 2x average pooling between levels; decoder: 2x upsampling of the coarser output,
# concatenation [upsampled, skip], two 3^3 conv+ReLU; head: 1^3 conv to the output channels.

def layer_shapes(chans, cin, cout):
    """(Co, Ci, k) of every convolution in execution order."""
    L = len(chans)
    shapes = []
    c = cin
    for l in range(L):
        shapes += [(chans[l], c, 3), (chans[l], chans[l], 3)]
        c = chans[l]
    for l in range(L - 2, -1, -1):
        shapes += [(chans[l], chans[l + 1] + chans[l], 3), (chans[l], chans[l], 3)]
    shapes.append((cout, chans[0], 1))
    return shapes


def net_forward(params, x, chans):
    """params: list of (w, b) per layer_shapes; returns (y, cache)."""
    L = len(chans)
    acts = {}
    h = np.asarray(x, np.float64)
    li = 0
    skips = []
    for l in range(L):
        for r in range(2):
            w, b = params[li]
            z = conv3d(h, w, b)
            acts[li] = (h, z)
            h = np.maximum(z, 0)
            li += 1
        skips.append(h)
        if l < L - 1:
            h = pool2(h)
    for l in range(L - 2, -1, -1):
        u = up2(h)
        h = np.concatenate([u, skips[l]], axis=1)
        for r in range(2):
            w, b = params[li]
            z = conv3d(h, w, b)
            acts[li] = (h, z)
            h = np.maximum(z, 0)
            li += 1
    w, b = params[li]
    y = conv3d(h, w, b)
    acts[li] = (h, y)
    return y, acts


def net_backward(params, acts, dy, chans):
    """Gradients of every (w, b) for output gradient dy (reverse of net_forward)."""
    L = len(chans)
    grads = [None] * len(params)
    li = len(params) - 1
    h_in, _ = acts[li]
    dw, db = conv3d_wgrad(h_in, dy, 1)
    grads[li] = (dw, db)
    g = conv3d_dgrad(dy, params[li][0])
    li -= 1
    dskips = [None] * L
    for l in range(0, L - 1):
        for r in range(2):
            h_in, z = acts[li]
            gz = g * (z > 0)
            grads[li] = conv3d_wgrad(h_in, gz, 3)
            g = conv3d_dgrad(gz, params[li][0])
            li -= 1
        cu = chans[l + 1]
        dskips[l] = g[:, cu:]
        g = up2_bwd(g[:, :cu])
    # bottom level's output feeds the first upsampling; walk the encoder back
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            g = pool2_bwd(g) + dskips[l]
        for r in range(2):
            h_in, z = acts[li]
            gz = g * (z > 0)
            grads[li] = conv3d_wgrad(h_in, gz, 3)
            g = conv3d_dgrad(gz, params[li][0])
            li -= 1
    return grads
