"""FP64 CPU oracle of the learned warm-start network (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this
module; the product path never does.

The network is the small 3D convolutional encoder-decoder that serves as the
learned warm start of the state solve: inputs are node fields (the physical
density averaged to the nodes and the three load components), the output is a
displacement direction field. This module states, plainly and slowly, what
every layer computes and its exact gradient:

* conv3d: zero padding 1, 3x3x3 taps, tap t = (dx+1)*9 + (dy+1)*3 + (dz+1),
  out[d, h, w, co] = b[co] + sum_t sum_ci x[d+dx, h+dy, w+dz, ci] W[t, ci, co];
* relu; 2x2x2 average pooling; nearest 2x upsampling; additive skips;
* mean squared error over a mask of valid voxels.

Architecture (levels L = 3, base channels c):
    e0 = relu(conv(relu(conv(x, 4->c)), c->c))
    e1 = relu(conv(relu(conv(pool(e0), c->2c)), 2c->2c))
    e2 = relu(conv(relu(conv(pool(e1), 2c->4c)), 4c->4c))
    d1 = relu(conv(relu(conv(up(e2), 4c->2c)) + e1, 2c->2c))
    d0 = relu(conv(relu(conv(up(d1), 2c->c)) + e0, c->c))
    y  = conv(d0, c->3)
Parameters are stored in this layer order, each layer as W[27, cin, cout]
followed by b[cout], flattened into one vector.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]


def layer_shapes(base=16, cin=4, cout=3):
    c = base
    return [(cin, c), (c, c), (c, 2 * c), (2 * c, 2 * c), (2 * c, 4 * c), (4 * c, 4 * c),
            (4 * c, 2 * c), (2 * c, 2 * c), (2 * c, c), (c, c), (c, cout)]


def n_params(base=16, cin=4, cout=3):
    return sum(27 * a * b + b for a, b in layer_shapes(base, cin, cout))


def unpack(theta, base=16, cin=4, cout=3):
    """Parameter vector -> list of (W[27, cin, cout], b[cout])."""
    out, k = [], 0
    for a, b in layer_shapes(base, cin, cout):
        W = theta[k:k + 27 * a * b].reshape(27, a, b)
        k += 27 * a * b
        out.append((W, theta[k:k + b]))
        k += b
    assert k == theta.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


# ------------------------------------------------------------------ layers

def conv3d(x, W, b):
    """Direct definition (zero padding): x[D, H, W, cin] -> [D, H, W, cout]."""
    D, H, Wd, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (D, H, Wd, b.size)).astype(float).copy()
    for t, (dx, dy, dz) in enumerate(TAPS):
        y += xp[1 + dx:1 + dx + D, 1 + dy:1 + dy + H, 1 + dz:1 + dz + Wd, :] @ W[t]
    return y


def conv3d_loops(x, W, b):
    """The same sum written as explicit loops (for pinning conv3d on tiny inputs)."""
    D, H, Wd, cin = x.shape
    cout = b.size
    y = np.zeros((D, H, Wd, cout))
    for d in range(D):
        for h in range(H):
            for w in range(Wd):
                for co in range(cout):
                    s = b[co]
                    for t, (dx, dy, dz) in enumerate(TAPS):
                        dd, hh, ww = d + dx, h + dy, w + dz
                        if 0 <= dd < D and 0 <= hh < H and 0 <= ww < Wd:
                            for ci in range(cin):
                                s += x[dd, hh, ww, ci] * W[t, ci, co]
                    y[d, h, w, co] = s
    return y


def conv3d_backward(x, W, gy):
    """Gradients of sum(gy * conv3d(x, W, b)) w.r.t. x, W and b."""
    D, H, Wd, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for t, (dx, dy, dz) in enumerate(TAPS):
        sl = (slice(1 + dx, 1 + dx + D), slice(1 + dy, 1 + dy + H), slice(1 + dz, 1 + dz + Wd))
        xs = xp[sl]
        gW[t] = np.einsum("dhwi,dhwo->io", xs, gy)
        gxp[sl] += gy @ W[t].T
    return gxp[1:-1, 1:-1, 1:-1], gW, gy.sum(axis=(0, 1, 2))


def pool(x):
    D, H, Wd, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, Wd // 2, 2, C).mean(axis=(1, 3, 5))


def pool_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_backward(gy):
    return pool(gy) * 8.0


def relu(x):
    return np.maximum(x, 0.0)


# ----------------------------------------------------------------- network

def forward(theta, x, base=16):
    """Returns the output and the cache of every pre-activation needed backward."""
    L = unpack(theta, base, x.shape[-1])
    cache = {}

    def cr(name, inp, k, act=True):
        z = conv3d(inp, *L[k])
        cache[name] = (inp, z)
        return relu(z) if act else z

    a = cr("c0", x, 0)
    e0 = cr("c1", a, 1)
    a = cr("c2", pool(e0), 2)
    e1 = cr("c3", a, 3)
    a = cr("c4", pool(e1), 4)
    e2 = cr("c5", a, 5)
    a = cr("c6", up(e2), 6)
    d1 = cr("c7", a + e1, 7)
    a = cr("c8", up(d1), 8)
    d0 = cr("c9", a + e0, 9)
    y = cr("c10", d0, 10, act=False)
    return y, cache


def loss(y, target, mask):
    """Mean squared error over the valid voxels (mask[D, H, W]) and channels."""
    m = mask[..., None].astype(float)
    n = m.sum() * y.shape[-1]
    return float(np.sum(m * (y - target) ** 2) / n)


def backward(theta, x, target, mask, base=16):
    """Loss and its gradient w.r.t. the parameter vector (chain rule by hand)."""
    L = unpack(theta, base, x.shape[-1])
    y, C = forward(theta, x, base)
    m = mask[..., None].astype(float)
    n = m.sum() * y.shape[-1]
    f = float(np.sum(m * (y - target) ** 2) / n)
    g = [None] * len(L)

    def back(name, k, gout, act=True):
        inp, z = C[name]
        gz = gout * (z > 0) if act else gout
        gx, gW, gb = conv3d_backward(inp, L[k][0], gz)
        g[k] = (gW, gb)
        return gx

    gy = 2.0 * m * (y - target) / n
    gd0 = back("c10", 10, gy, act=False)
    gs = back("c9", 9, gd0)        # gradient of (a + e0)
    ge0 = gs.copy()
    gd1 = up_backward(back("c8", 8, gs))
    gs = back("c7", 7, gd1)        # gradient of (a + e1)
    ge1 = gs.copy()
    ge2 = up_backward(back("c6", 6, gs))
    ga = back("c5", 5, ge2)
    ge1 += pool_backward(back("c4", 4, ga))
    ga = back("c3", 3, ge1)
    ge0 += pool_backward(back("c2", 2, ga))
    ga = back("c1", 1, ge0)
    back("c0", 0, ga)
    return f, pack(g)


def init_params(base=16, cin=4, cout=3, seed=0):
    """He-normal weights, zero biases (a reference initialisation for tests)."""
    rng = np.random.default_rng(seed)
    layers = []
    for a, b in layer_shapes(base, cin, cout):
        layers.append((rng.standard_normal((27, a, b)) * np.sqrt(2.0 / (27 * a)), np.zeros(b)))
    return pack(layers)
