"""FP64 CPU oracle of the learned warm start's 3-D U-Net (forward and backward).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module (and
``bench.py``'s CPU legs); the CUDA network never imports it and shares no
code with it.

The network is not in the paper: it maps a channel's solid-flag field and its
driving force to the steady (delta rho, u) that the lattice Boltzmann solver
reaches, so that the solver can start from that equilibrium instead of from
rest.  Three levels with 16 / 32 / 64 channels, 3x3x3 convolutions:

    e1 = relu(conv(relu(conv(x,  W1a)), W1b))          2 -> 16 -> 16  at n^3
    e2 = relu(conv(relu(conv(pool(e1), W2a)), W2b))   16 -> 32 -> 32  at (n/2)^3
    e3 = relu(conv(relu(conv(pool(e2), W3a)), W3b))   32 -> 64 -> 64  at (n/4)^3
    d2 = relu(conv(relu(conv([up(e3), e2], W4a)), W4b))  96 -> 32 -> 32 at (n/2)^3
    d1 = relu(conv(relu(conv([up(d2), e1], W5a)), W5b))  48 -> 16 -> 16 at n^3
    y  = d1 Wh^T + bh                                  16 -> 4  (1x1x1 head)

conv: 3x3x3 correlation with bias, periodic along x and z (the channel's
periodic axes) and zero padding along y (its walls).  pool: 2x2x2 average.
up: nearest-neighbour 2x upsampling.  [a, b]: channel concatenation.
Tensors are channels-last arrays of shape (nz, ny, nx, C); a weight W has
shape (Cout, 27, Cin) with tap t = 9 (dz+1) + 3 (dy+1) + (dx+1).
Loss: mean over voxels and channels of (y - target)^2.

Every function is written out directly (loops over the 27 taps, numpy
products per tap); pinned by ``tests/test_unet_oracle.py``.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]

# (name, Cin, Cout) of the ten 3x3x3 convolutions, in forward order
CONVS = [("W1a", 2, 16), ("W1b", 16, 16), ("W2a", 16, 32), ("W2b", 32, 32),
         ("W3a", 32, 64), ("W3b", 64, 64), ("W4a", 96, 32), ("W4b", 32, 32),
         ("W5a", 48, 16), ("W5b", 16, 16)]


def shift(x, dz, dy, dx):
    """s[z, y, x] = x[z + dz, y + dy, x + dx]: periodic in z and x, zero outside y."""
    s = np.roll(x, (-dz, -dx), axis=(0, 2))
    if dy == 0:
        return s
    out = np.zeros_like(s)
    if dy > 0:
        out[:, :-dy] = s[:, dy:]
    else:
        out[:, -dy:] = s[:, :dy]
    return out


def conv(x, W, b):
    """y[v, co] = b[co] + sum_t sum_ci x[v + off_t, ci] W[co, t, ci]."""
    y = np.broadcast_to(b, x.shape[:3] + (W.shape[0],)).astype(np.float64).copy()
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += shift(x, dz, dy, dx) @ W[:, t, :].T
    return y


def conv_backward(x, W, gy):
    """Gradients of conv for the output gradient gy: (gx, gW, gb)."""
    gx = np.zeros_like(x, dtype=np.float64)
    gW = np.zeros_like(W, dtype=np.float64)
    X = x.reshape(-1, x.shape[-1])
    for t, (dz, dy, dx) in enumerate(TAPS):
        # x[v + off] feeds y[v]: the adjoint of the shift moves gy back by -off
        gx += shift(gy, -dz, -dy, -dx) @ W[:, t, :]
        gW[:, t, :] = gy.reshape(-1, gy.shape[-1]).T @ shift(x, dz, dy, dx).reshape(-1, X.shape[1])
    gb = gy.reshape(-1, gy.shape[-1]).sum(axis=0)
    return gx, gW, gb


def relu(x):
    return np.maximum(x, 0.0)


def pool(x):
    nz, ny, nx, c = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(1, 3, 5))


def pool_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_backward(gy):
    nz, ny, nx, c = gy.shape
    return gy.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).sum(axis=(1, 3, 5))


def init_params(seed=0):
    """He-normal weights, zero biases; head small."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co in CONVS:
        p[name] = rng.normal(0.0, np.sqrt(2.0 / (27 * ci)), (co, 27, ci))
        p["b" + name[1:]] = np.zeros(co)
    p["Wh"] = rng.normal(0.0, np.sqrt(1.0 / 16), (4, 16))
    p["bh"] = np.zeros(4)
    return p


def forward(p, x):
    """Forward pass; returns the output and the activations the backward needs."""
    a = {"x": x}

    def block(name_a, name_b, inp, key):
        h = relu(conv(inp, p[name_a], p["b" + name_a[1:]]))
        o = relu(conv(h, p[name_b], p["b" + name_b[1:]]))
        a[key + "_in"], a[key + "_h"], a[key] = inp, h, o
        return o

    e1 = block("W1a", "W1b", x, "e1")
    e2 = block("W2a", "W2b", pool(e1), "e2")
    e3 = block("W3a", "W3b", pool(e2), "e3")
    d2 = block("W4a", "W4b", np.concatenate([up(e3), e2], axis=-1), "d2")
    d1 = block("W5a", "W5b", np.concatenate([up(d2), e1], axis=-1), "d1")
    y = d1 @ p["Wh"].T + p["bh"]
    return y, a


def loss(y, target):
    return float(np.mean((y - target) ** 2))


def backward(p, a, y, target):
    """Gradients of the loss with respect to every parameter (dict like p)."""
    g = {}
    gy = 2.0 * (y - target) / y.size
    d1 = a["d1"]
    g["Wh"] = gy.reshape(-1, 4).T @ d1.reshape(-1, 16)
    g["bh"] = gy.reshape(-1, 4).sum(axis=0)
    gd1 = gy @ p["Wh"]

    def block_back(name_a, name_b, key, gout):
        # relu(conv_b(relu(conv_a(in)))) -> gradient with respect to `in`
        go = gout * (a[key] > 0)
        gh, g[name_b], g["b" + name_b[1:]] = conv_backward(a[key + "_h"], p[name_b], go)
        gh = gh * (a[key + "_h"] > 0)
        gin, g[name_a], g["b" + name_a[1:]] = conv_backward(a[key + "_in"], p[name_a], gh)
        return gin

    gu1 = block_back("W5a", "W5b", "d1", gd1)
    c_d2 = a["d2"].shape[-1]
    gd2 = up_backward(gu1[..., :c_d2])
    ge1 = gu1[..., c_d2:]
    gu2 = block_back("W4a", "W4b", "d2", gd2)
    c_e3 = a["e3"].shape[-1]
    ge3 = up_backward(gu2[..., :c_e3])
    ge2 = gu2[..., c_e3:]
    gp2 = block_back("W3a", "W3b", "e3", ge3)
    ge2 = ge2 + pool_backward(gp2)
    gp1 = block_back("W2a", "W2b", "e2", ge2)
    ge1 = ge1 + pool_backward(gp1)
    block_back("W1a", "W1b", "e1", ge1)
    return g


def flops_forward(n):
    """Multiply-add FLOPs (2 per MAC) of one forward pass on an n^3 input."""
    v = [n**3, n**3, (n // 2) ** 3, (n // 2) ** 3, (n // 4) ** 3, (n // 4) ** 3,
         (n // 2) ** 3, (n // 2) ** 3, n**3, n**3]
    f = sum(2 * 27 * ci * co * vox for (_, ci, co), vox in zip(CONVS, v))
    return f + 2 * 16 * 4 * n**3
