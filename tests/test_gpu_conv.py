"""The surrogate's 3x3 convolution on the tensor cores (tcgen05.mma, BF16
operands, FP32 accumulation in tensor memory) through the C ABI, element by
element against the oracle's periodic convolution with the same BF16 operand
rounding.  Products of two BF16 values are exact in FP32, so the two sides
differ only by the accumulation: FP32 over K = 9 cin terms in an order the
tensor core chooses, against FP64.  Bar per element: the recursive-summation
bound gamma_K = K u / (1 - K u), u = 2^-24, times the sum of the absolute
terms, and the exact sum where every term is an exact multiple of 2^-20
(sums of a few hundred such terms are exact in FP32 whatever the order).
Two kernels: 16 x 8 halo tiles where H and W allow them, pixel gathers
otherwise.  Shapes cover a partial last tile (pixels not a multiple of 128), several
channel blocks a tap (cin 384 in blocks of 64, 96 in blocks of 48), the
widest accumulator (cout 256), two output-channel tiles (cout 384, as in
the data gradient of the 4-level network's 384 -> 128 layer), odd image
sizes and both activations."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# H a multiple of 16 and W of 8: the halo-tile kernel; otherwise the gather kernel
SHAPES = [(1, 16, 24, 16, 16), (2, 32, 16, 32, 64), (1, 16, 8, 64, 256), (1, 48, 24, 96, 32), (1, 16, 16, 384, 128),
          (1, 16, 8, 128, 384), (2, 12, 20, 32, 64), (1, 8, 8, 96, 32), (1, 8, 16, 64, 256), (1, 8, 8, 64, 384),
          (3, 5, 7, 48, 16), (1, 1, 1, 16, 16)]


@pytest.fixture(scope="module")
def env():
    import torch

    from oracle import unet_oracle as U
    from paper_1606_09432_gb300 import build as B
    from paper_1606_09432_gb300 import lbpf as L
    B.build()
    L.load()
    return torch, U, L


def run(torch, L, x, wq, b, relu):
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    wt = torch.from_numpy(wq.astype(np.float32)).cuda().to(torch.bfloat16).contiguous()
    bt = torch.from_numpy(b.astype(np.float32)).cuda() if b is not None else None
    y = torch.full(x.shape[:3] + (wq.shape[1],), float("nan"), device="cuda")
    L.nn_conv3x3(xt, wt, bt, y, relu=relu)
    torch.cuda.synchronize()
    assert L.nn_conv_error() == 0
    return y.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("relu", [0, 1])
def test_conv_matches_oracle(env, shape, relu):
    torch, U, L = env
    n, H, W, cin, cout = shape
    rng = np.random.default_rng(hash(shape) % 2**32 + relu)
    x = rng.standard_normal((n, H, W, cin))
    wq = U.bf16(rng.standard_normal((9, cout, cin)) / np.sqrt(9 * cin))
    b = rng.standard_normal(cout) if relu else None
    y = run(torch, L, x, wq, b, relu)
    yo = U.conv3x3(x, wq, b, emulate=True)
    if relu:
        yo = np.maximum(yo, 0.0)
    absum = U.conv3x3(np.abs(U.bf16(x)), np.abs(wq)) + (np.abs(b) if b is not None else 0.0)
    K = 9 * cin + 1
    u = 2.0 ** -24
    bar = K * u / (1 - K * u) * absum
    err = np.abs(y - yo)
    print(f"{shape} relu={relu}: max |dy| {err.max():.2e}, max |dy| / bound {(err / np.maximum(bar, 1e-300)).max():.3f}")
    assert np.isfinite(y).all()
    assert np.all(err <= bar + 1e-30)


@pytest.mark.parametrize("shape", [(2, 9, 13, 64, 48), (2, 16, 16, 64, 48)])
def test_conv_exact_on_dyadic_inputs(env, shape):
    """Inputs and weights multiples of 1/8 and 1/16 with small numerators:
    every partial sum is exact in FP32, so the tensor-core result must equal
    the exact convolution bit for bit (gather and halo kernels)."""
    torch, U, L = env
    rng = np.random.default_rng(3)
    n, H, W, cin, cout = shape
    x = rng.integers(-8, 9, (n, H, W, cin)) / 8.0
    wq = rng.integers(-8, 9, (9, cout, cin)) / 16.0
    y = run(torch, L, x, wq, None, 0)
    yo = U.conv3x3(x, wq)
    assert np.array_equal(y, yo)


WG_SHAPES = [(2, 12, 20, 16, 32), (1, 16, 16, 384, 128), (1, 8, 16, 64, 256), (3, 5, 7, 48, 16), (4, 32, 32, 96, 32)]


@pytest.mark.parametrize("shape", WG_SHAPES)
def test_wgrad_matches_oracle(env, shape):
    """Weight gradient, element by element against the oracle's BF16-operand
    weight gradient: FP32 accumulation over K = n H W pixels (tensor core and
    atomics in an unknown order) within gamma_K times the sum of the absolute
    terms; the output starts from a non-zero dw (the call accumulates)."""
    torch, U, L = env
    n, H, W, cin, cout = shape
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal((n, H, W, cin))
    dy = rng.standard_normal((n, H, W, cout))
    d0 = rng.standard_normal((9, cout, cin))
    dw = torch.from_numpy(d0.astype(np.float32)).cuda()
    L.nn_conv3x3_wgrad(torch.from_numpy(x.astype(np.float32)).cuda(), torch.from_numpy(dy.astype(np.float32)).cuda(),
                       dw)
    torch.cuda.synchronize()
    assert L.nn_conv_error() == 0
    got = dw.cpu().numpy().astype(np.float64)
    want = d0.astype(np.float32).astype(np.float64) + U.conv3x3_wgrad(x, dy, emulate=True)
    absum = np.abs(d0) + U.conv3x3_wgrad(np.abs(x), np.abs(dy), emulate=True)
    K = n * H * W + 1
    u = 2.0 ** -24
    bar = K * u / (1 - K * u) * absum
    err = np.abs(got - want)
    print(f"wgrad {shape}: max |d dw| {err.max():.2e}, max / bound {(err / bar).max():.3f}")
    assert np.all(err <= bar)


def test_conv_rejects_bad_channels(env):
    torch, U, L = env
    x = torch.zeros((1, 8, 8, 24), device="cuda")
    y = torch.zeros((1, 8, 8, 16), device="cuda")
    w = torch.zeros((9, 16, 24), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(L.LbpfError):
        L.nn_conv3x3(x, w, None, y)
