"""FP64 NumPy oracle of the learned surrogate's U-Net (test infrastructure).

Same architecture and flat parameter layout as the CUDA network
(include/lbpf.h, "Learned surrogate"): a U-Net of `levels` levels with
base * 2^l channels at level l, two periodic 3x3 convolutions + ReLU per
level on the way down (2x2 average pooling between levels) and on the way up
(nearest 2x upsampling, concatenated with the level's skip), a 1x1 head to 2
channels whose phi channel is gated by (1 - phi^2); input (N, H, W, 5)
zero-padded to 16 channels.  The default (3 levels, base 16) has channels
16, 32, 64.  Layer order: the encoder's convolutions level by level, then the
decoder's from the deepest level up.  The
backward pass is written out layer by layer (plain chain rule).  With
emulate=True the operands of every 3x3 convolution
(weights, and the activations or gradients it reads) are rounded to BF16
first, as the tensor-core kernels do; accumulation stays FP64.

The surrogate is not part of the paper; nothing here is pinned by the paper.
The pins are mathematical: a brute-force periodic convolution, adjointness of
pooling and upsampling, and finite differences of the loss.
"""
from __future__ import annotations

import numpy as np

N_IN, N_IN_PAD, N_OUT = 5, 16, 2
ARCH = (3, 16)  # (levels, base channels) of the default network


def layers(arch=ARCH):
    """(cin, cout) of the 3x3 convolutions in order."""
    lv, base = arch
    c = [base << l for l in range(lv)]
    out = [(N_IN_PAD, c[0]), (c[0], c[0])]
    for l in range(1, lv):
        out += [(c[l - 1], c[l]), (c[l], c[l])]
    for l in range(lv - 2, -1, -1):
        out += [(c[l + 1] + c[l], c[l]), (c[l], c[l])]
    return out


LAYERS = layers()


def n_params(arch=ARCH):
    return sum(9 * ci * co + co for ci, co in layers(arch)) + N_OUT * arch[1] + N_OUT


def unpack(p, arch=ARCH):
    """Flat vector -> list of (W[tap][co][ci], b[co]) for the 3x3 layers, and
    the head (W[co][ci], b[co])."""
    p = np.asarray(p, dtype=np.float64)
    out, k = [], 0
    for ci, co in layers(arch):
        w = p[k:k + 9 * ci * co].reshape(9, co, ci)
        k += 9 * ci * co
        b = p[k:k + co]
        k += co
        out.append((w, b))
    c0 = arch[1]
    hw = p[k:k + N_OUT * c0].reshape(N_OUT, c0)
    k += N_OUT * c0
    hb = p[k:k + N_OUT]
    return out, (hw, hb)


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    r = ((bits + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(x, dy, dx):
    """x[n, (y + dy) mod H, (x + dx) mod W, c]."""
    return np.roll(np.roll(x, -dy, axis=1), -dx, axis=2)


def conv3x3(x, w, b=None, emulate=False):
    """Periodic 3x3 convolution y[p][co] = b[co] + sum_tap sum_ci w[tap][co][ci] x[p + tap][ci]."""
    if emulate:
        x, w = bf16(x), bf16(w)
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        y += shift(x, dy, dx) @ w[tap].T
    if b is not None:
        y += b
    return y


def conv3x3_dgrad(dy, w, emulate=False):
    """Adjoint of conv3x3 in its input: dx[p][ci] = sum_tap sum_co w[tap][co][ci] dy[p - tap][co]."""
    if emulate:
        dy, w = bf16(dy), bf16(w)
    dx = np.zeros(dy.shape[:3] + (w.shape[2],))
    for tap in range(9):
        ddy, ddx = tap // 3 - 1, tap % 3 - 1
        dx += shift(dy, -ddy, -ddx) @ w[tap]
    return dx


def conv3x3_wgrad(x, dy, emulate=False):
    """dw[tap][co][ci] = sum_p dy[p][co] x[p + tap][ci] (FP64; with emulate
    both operands rounded to BF16 first, as the tensor-core kernel does)."""
    if emulate:
        x, dy = bf16(x), bf16(dy)
    co, ci = dy.shape[-1], x.shape[-1]
    dw = np.zeros((9, co, ci))
    for tap in range(9):
        ddy, ddx = tap // 3 - 1, tap % 3 - 1
        dw[tap] = np.einsum("nhwo,nhwi->oi", dy, shift(x, ddy, ddx))
    return dw


def pool(x):
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(dy):
    n, h, w, c = dy.shape
    return dy.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def relu(x):
    return np.maximum(x, 0.0)


def forward(p, x, emulate=False, arch=ARCH):
    """Returns (out, cache).  Cache: the input, per encoder level l the
    convolution outputs ("ea", l), ("e", l) and the pooled input ("p", l)
    (l >= 1), per decoder level the concatenation ("u", l) and the outputs
    ("da", l), ("d", l)."""
    lv = arch[0]
    L, (hw, hb) = unpack(p, arch)
    xin = np.concatenate([x, np.zeros(x.shape[:3] + (N_IN_PAD - x.shape[3],))], axis=3)
    c = {"xin": xin}
    cv = lambda k, a: relu(conv3x3(a, L[k][0], L[k][1], emulate))
    k = 0
    a = xin
    for l in range(lv):
        if l > 0:
            a = c[("p", l)] = pool(c[("e", l - 1)])
        c[("ea", l)] = cv(k, a)
        c[("e", l)] = cv(k + 1, c[("ea", l)])
        k += 2
    prev = c[("e", lv - 1)]
    for l in range(lv - 2, -1, -1):
        c[("u", l)] = np.concatenate([up(prev), c[("e", l)]], axis=3)
        c[("da", l)] = cv(k, c[("u", l)])
        prev = c[("d", l)] = cv(k + 1, c[("da", l)])
        k += 2
    out = prev @ hw.T + hb
    out[..., 0] *= 1.0 - xin[..., 0] ** 2  # interface gate of the phi output
    c["top"] = prev
    return out, c


def backward(p, c, dout, emulate=False, arch=ARCH):
    """Gradient of sum(out * dout) with respect to the flat parameter vector."""
    lv, base = arch
    L, (hw, hb) = unpack(p, arch)
    grads = [None] * len(L)
    dout = dout.copy()
    dout[..., 0] *= 1.0 - c["xin"][..., 0] ** 2

    def cvb(k, a_in, y, dy, need_dx=True):
        dy = dy * (y > 0)
        grads[k] = (conv3x3_wgrad(a_in, dy, emulate), dy.sum(axis=(0, 1, 2)))
        return conv3x3_dgrad(dy, L[k][0], emulate) if need_dx else None

    ghw = np.einsum("nhwo,nhwi->oi", dout, c["top"])
    ghb = dout.sum(axis=(0, 1, 2))
    g = dout @ hw
    k = len(L)
    skip = {}
    for l in range(0, lv - 1):  # decoder, from the top level down
        k -= 2
        g = cvb(k + 1, c[("da", l)], c[("d", l)], g)
        g = cvb(k, c[("u", l)], c[("da", l)], g)
        cu = base << (l + 1)
        skip[l] = g[..., cu:]
        g = up_bwd(g[..., :cu])  # gradient of the level l + 1 output
    for l in range(lv - 1, -1, -1):  # encoder, from the deepest level up
        k -= 2
        if l < lv - 1:
            g = g + skip[l]
        g = cvb(k + 1, c[("ea", l)], c[("e", l)], g)
        g = cvb(k, c[("p", l)] if l > 0 else c["xin"], c[("ea", l)], g, need_dx=l > 0)
        if l > 0:
            g = pool_bwd(g)
    assert k == 0
    flat = []
    for dw, db in grads:
        flat += [dw.ravel(), db]
    flat += [ghw.ravel(), ghb]
    return np.concatenate(flat)


def weighted_mse(out, target, x, alpha=0.0):
    """Training loss and its gradient in out: mean over all values of
    w (out - target)^2, w = 1 + alpha max(0, 1 - phi^2) with phi = x[..., 0]
    the input phase field of the value's site."""
    w = 1.0 + alpha * np.maximum(0.0, 1.0 - np.asarray(x, np.float64)[..., :1] ** 2)
    d = np.asarray(out, np.float64) - target
    n = d.size
    return float((w * d * d).sum() / n), 2.0 * w * d / n


def init_params(seed, scale_head=1e-2, arch=ARCH):
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in layers(arch):
        a = np.sqrt(6.0 / (9 * ci))
        parts += [rng.uniform(-a, a, 9 * co * ci), np.zeros(co)]
    parts += [rng.uniform(-scale_head, scale_head, N_OUT * arch[1]), np.zeros(N_OUT)]
    return np.concatenate(parts)
