"""Pins of the surrogate network's FP64 oracle (oracle/unet_oracle.py).

The surrogate is not in the paper; its oracle is pinned by mathematics: a
periodic 3x3 convolution written as a brute-force sum, the adjoint identities
<A x, y> = <x, A^T y> of convolution, pooling and upsampling, BF16 rounding
against known bit patterns, and the whole backward pass against central
finite differences of the loss.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def U():
    from oracle import unet_oracle
    return unet_oracle


def test_conv_bruteforce(U):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    w = rng.standard_normal((9, 4, 3))
    b = rng.standard_normal(4)
    y = U.conv3x3(x, w, b)
    n, H, W, _ = x.shape
    for nn in range(n):
        for yy in range(H):
            for xx in range(W):
                for co in range(4):
                    acc = b[co]
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            tap = 3 * (dy + 1) + (dx + 1)
                            acc += w[tap, co] @ x[nn, (yy + dy) % H, (xx + dx) % W]
                    assert abs(y[nn, yy, xx, co] - acc) < 1e-12


def test_adjoints(U):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 8, 3))
    w = rng.standard_normal((9, 5, 3))
    dy = rng.standard_normal((2, 8, 8, 5))
    assert abs((U.conv3x3(x, w) * dy).sum() - (x * U.conv3x3_dgrad(dy, w)).sum()) < 1e-10
    # weight gradient: d/dw <conv(x, w), dy>
    dw = U.conv3x3_wgrad(x, dy)
    e = np.zeros_like(w)
    e[4, 2, 1] = 1e-6
    fd = ((U.conv3x3(x, w + e) - U.conv3x3(x, w - e)) * dy).sum() / 2e-6
    assert abs(fd - dw[4, 2, 1]) < 1e-7
    z = rng.standard_normal((2, 4, 4, 3))
    assert abs((U.pool(x) * z).sum() - (x * U.pool_bwd(z)).sum()) < 1e-12
    assert abs((U.up(z) * x).sum() - (z * U.up_bwd(x)).sum()) < 1e-12


def test_bf16_rounding(U):
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -9, -2.5, 3.14159265])
    r = U.bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == 1.0 + 2 ** -7
    assert r[4] == -2.5 and abs(r[5] - 3.140625) < 1e-12


def test_layer_list(U):
    """The default network's layers, written out, and the 4-level 32-channel
    one: encoder level by level, then the decoder from the deepest level up
    with the concatenated skip (upsampled deeper channels + this level's)."""
    assert U.layers() == [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16),
                          (16, 16)]
    assert U.layers((4, 32)) == [(16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256),
                                 (256, 256), (384, 128), (128, 128), (192, 64), (64, 64), (96, 32), (32, 32)]
    assert U.n_params((4, 32)) == sum(9 * a * b + b for a, b in U.layers((4, 32))) + 2 * 32 + 2


@pytest.mark.parametrize("arch,size", [((3, 16), 32), ((4, 16), 32), ((2, 16), 16)])
def test_backward_matches_finite_differences(U, arch, size):
    rng = np.random.default_rng(2)
    p = U.init_params(3, scale_head=0.3, arch=arch)
    p[p.size - 2:] = 0.1
    x = rng.standard_normal((1, size, size, 5))
    t = rng.standard_normal((1, size, size, 2))
    out, c = U.forward(p, x, arch=arch)
    g = U.backward(p, c, 2 * (out - t), arch=arch)
    loss = lambda q: ((U.forward(q, x, arch=arch)[0] - t) ** 2).sum()
    idx = rng.choice(p.size, 24, replace=False)
    for i in idx:
        h = 1e-5 * max(1.0, abs(p[i]))
        e = np.zeros_like(p)
        e[i] = h
        fd = (loss(p + e) - loss(p - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_weighted_mse_loops_and_gradient(U):
    """Weighted training loss: a plain loop over sites and channels, the plain
    mean squared error at alpha = 0, and its gradient by central differences."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 3, 4, 5))
    x[..., 0] = 1.2 * np.tanh(x[..., 0])  # some |phi| > 1: weight clipped at 1
    out = rng.standard_normal((2, 3, 4, 2))
    t = rng.standard_normal((2, 3, 4, 2))
    alpha = 7.0
    loss, dout = U.weighted_mse(out, t, x, alpha)
    acc = 0.0
    for n in range(2):
        for i in range(3):
            for j in range(4):
                ph = x[n, i, j, 0]
                w = 1.0 + alpha * max(0.0, 1.0 - ph * ph)
                for c in range(2):
                    acc += w * (out[n, i, j, c] - t[n, i, j, c]) ** 2
    assert abs(loss - acc / out.size) < 1e-12
    assert abs(U.weighted_mse(out, t, x, 0.0)[0] - ((out - t) ** 2).mean()) < 1e-12
    for k in rng.choice(out.size, 8, replace=False):
        e = np.zeros(out.size)
        e[k] = 1e-6
        e = e.reshape(out.shape)
        fd = (U.weighted_mse(out + e, t, x, alpha)[0] - U.weighted_mse(out - e, t, x, alpha)[0]) / 2e-6
        assert abs(fd - dout.ravel()[k]) < 1e-7
