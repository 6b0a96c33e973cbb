"""Pins of the U-Net oracle (CPU, FP64) against brute force, closed forms,
adjoint identities and central finite differences."""
import numpy as np
import pytest

from oracle import unet_oracle as U


def _brute_conv(x, W, b):
    """Direct loops over outputs, taps and channels (tiny inputs only)."""
    nz, ny, nx, ci = x.shape
    co = W.shape[0]
    y = np.zeros((nz, ny, nx, co))
    for z in range(nz):
        for yy in range(ny):
            for xx in range(nx):
                for o in range(co):
                    s = b[o]
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                sy = yy + dy
                                if sy < 0 or sy >= ny:
                                    continue  # wall: zero padding along y
                                sz, sx = (z + dz) % nz, (xx + dx) % nx
                                t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
                                for c in range(ci):
                                    s += x[sz, sy, sx, c] * W[o, t, c]
                    y[z, yy, xx, o] = s
    return y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 4, 5, 2))
    W = rng.normal(size=(3, 27, 2))
    b = rng.normal(size=3)
    assert np.allclose(U.conv(x, W, b), _brute_conv(x, W, b), atol=1e-12)


def test_conv_delta_kernel_is_a_shift():
    """A kernel with a single unit tap moves the field: periodic in z and x,
    zero-filled in y (closed form of the padding rule)."""
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 5, 6, 1))
    for (dz, dy, dx) in [(1, 0, 0), (0, 0, -1), (0, 1, 0), (0, -1, 1), (-1, 1, -1)]:
        W = np.zeros((1, 27, 1))
        W[0, (dz + 1) * 9 + (dy + 1) * 3 + dx + 1, 0] = 1.0
        y = U.conv(x, W, np.zeros(1))
        for z in range(4):
            for yy in range(5):
                for xx in range(6):
                    sy = yy + dy
                    ref = x[(z + dz) % 4, sy, (xx + dx) % 6, 0] if 0 <= sy < 5 else 0.0
                    assert y[z, yy, xx, 0] == ref


def test_adjoint_identities():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 6, 4, 3))
    W = rng.normal(size=(2, 27, 3))
    gy = rng.normal(size=(4, 6, 4, 2))
    gx, _, _ = U.conv_backward(x, W, gy)
    # <conv(x) - b, gy> = <x, conv^T gy>
    lhs = np.sum((U.conv(x, W, np.zeros(2))) * gy)
    assert abs(lhs - np.sum(x * gx)) <= 1e-10 * abs(lhs)
    p = rng.normal(size=(2, 3, 2, 3))
    assert abs(np.sum(U.pool(x) * p) - np.sum(x * U.pool_backward(p))) < 1e-12
    q = rng.normal(size=(8, 12, 8, 3))
    assert abs(np.sum(U.up(x) * q) - np.sum(x * U.up_backward(q))) < 1e-10
    # pool of a piecewise-constant field undoes up exactly
    assert np.allclose(U.pool(U.up(x)), x, rtol=0, atol=1e-15)


def test_conv_weight_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(3, 4, 3, 2))
    W = rng.normal(size=(2, 27, 2))
    b = rng.normal(size=2)
    gy = rng.normal(size=(3, 4, 3, 2))
    _, gW, gb = U.conv_backward(x, W, gy)
    f = lambda W_, b_: np.sum(U.conv(x, W_, b_) * gy)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 13, 1), (0, 26, 1), (1, 4, 0)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        assert abs((f(Wp, b) - f(Wm, b)) / (2 * h) - gW[idx]) < 1e-6 * max(1, abs(gW[idx]))
    bp = b.copy()
    bp[1] += h
    bm = b.copy()
    bm[1] -= h
    assert abs((f(W, bp) - f(W, bm)) / (2 * h) - gb[1]) < 1e-6 * max(1, abs(gb[1]))


@pytest.mark.slow
def test_network_gradient_by_central_differences():
    """Every parameter tensor of the whole network, sampled entries."""
    rng = np.random.default_rng(4)
    n = 8
    p = U.init_params(5)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(0, 0.05, p[k].shape)
    # continuous inputs keep pre-activations away from the ReLU kink with
    # probability one; h small enough that no kink is crossed
    x = rng.normal(size=(n, n, n, 2))
    target = rng.normal(size=(n, n, n, 4))
    y, a = U.forward(p, x)
    g = U.backward(p, a, y, target)
    h = 1e-7
    for k in sorted(p):
        flat = p[k].reshape(-1)
        for j in rng.choice(flat.size, size=3, replace=False):
            old = flat[j]
            flat[j] = old + h
            lp = U.loss(U.forward(p, x)[0], target)
            flat[j] = old - h
            lm = U.loss(U.forward(p, x)[0], target)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[j]
            assert abs(fd - an) <= 1e-5 * abs(an) + 1e-8, (k, j, fd, an)


def test_flop_count_of_the_64_cube_network():
    # 2 MAC-FLOPs per multiply-add: about 3e10 per 64^3 sample
    f = U.flops_forward(64)
    assert 2.9e10 < f < 3.1e10
