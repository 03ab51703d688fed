"""The tcgen05 / TMA convolution kernels (forward and input gradient) against
the FP64 network oracle, and against the mma.sync kernels on the same
inputs.  Inputs are drawn in float and rounded to bfloat16 on the device;
the oracle runs in float64 on exactly those values, so outputs stored in
bfloat16 are compared at 5e-3 of their scale (2^-8 is the bfloat16 step)."""
import numpy as np
import pytest

from oracle import conv_oracle as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_02185_gb300 import nn  # noqa: E402

DEV = torch.device("cuda")


def bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV).to(torch.bfloat16)


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-30))


@pytest.fixture(autouse=True)
def impl_reset():
    nn.status(reset=True)
    yield
    nn.set_conv_impl(nn.IMPL_AUTO)
    assert nn.status(reset=True) == 0  # no bounded wait gave up


# (N, H, W, cin, cout): 32- and 64-channel chunks, every output tile width,
# rows shorter than one 128-pixel tile, ragged last tiles, one-row images,
# and an output split into two channel halves
TC_SHAPES = [(2, 5, 150, 32, 32), (1, 3, 300, 64, 64), (2, 4, 129, 128, 96), (1, 3, 70, 96, 192),
             (1, 2, 131, 384, 128), (1, 3, 45, 64, 384), (1, 2, 257, 256, 256), (3, 1, 20, 32, 64),
             (1, 6, 128, 192, 64)]


@pytest.mark.parametrize("N,H,W,cin,cout", TC_SHAPES)
@pytest.mark.parametrize("relu", [0, 1])
def test_tc_forward(N, H, W, cin, cout, relu):
    rng = np.random.default_rng(cin + 3 * cout + W)
    x = bf(rng.standard_normal((N, H, W, cin)))
    w = bf(rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin))
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).to(DEV)
    ref = C.conv3x3(f64(x), f64(w), b.cpu().numpy())
    if relu:
        ref = C.relu(ref)
    outs = {}
    for impl in (nn.IMPL_TCGEN05, nn.IMPL_MMA_SYNC):
        nn.set_conv_impl(impl)
        y = torch.full((N, H, W, cout), float("nan"), dtype=torch.bfloat16, device=DEV)
        nn.conv3x3_fwd(x, cin, w, b, y, cout, N, H, W, cin, cout, relu)
        torch.cuda.synchronize()
        outs[impl] = f64(y)
        assert rel_err(outs[impl], ref) <= 5e-3, impl
    # the two kernel families differ only in FP32 summation order
    assert rel_err(outs[nn.IMPL_TCGEN05], outs[nn.IMPL_MMA_SYNC]) <= 1e-2


def test_tc_forward_channel_slices():
    # read a slice of a wider buffer, write into the tail of another
    rng = np.random.default_rng(7)
    N, H, W = 1, 4, 140
    big = bf(rng.standard_normal((N, H, W, 96)))
    out = torch.zeros((N, H, W, 96), dtype=torch.bfloat16, device=DEV)
    w = bf(rng.standard_normal((32, 3, 3, 64)) / 24)
    nn.set_conv_impl(nn.IMPL_TCGEN05)
    nn.conv3x3_fwd(big[..., 32:], 96, w, None, out[..., 64:], 96, N, H, W, 64, 32, 0)
    torch.cuda.synchronize()
    assert rel_err(f64(out)[..., 64:], C.conv3x3(f64(big)[..., 32:], f64(w))) <= 5e-3
    assert np.all(f64(out)[..., :64] == 0)


@pytest.mark.parametrize("N,H,W,cin,cout", [(2, 5, 150, 32, 32), (1, 3, 130, 96, 32), (1, 2, 100, 384, 128),
                                            (1, 4, 70, 64, 256)])
def test_tc_input_gradient_with_relu_mask(N, H, W, cin, cout):
    rng = np.random.default_rng(1 + cin + cout)
    w = bf(rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin))
    gy = bf(rng.standard_normal((N, H, W, cout)))
    xmask = bf(rng.standard_normal((N, H, W, cin)))
    wf = torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device=DEV)
    nn.flip_weights(w, wf, cout, cin)
    gx = torch.empty((N, H, W, cin), dtype=torch.bfloat16, device=DEV)
    nn.set_conv_impl(nn.IMPL_TCGEN05)
    nn.conv3x3_dgrad(gy, cout, wf, gx, cin, N, H, W, cin, cout, mask=xmask, ms=cin)
    torch.cuda.synchronize()
    ref = C.relu_grad(f64(xmask), C.conv3x3_dgrad(f64(gy), f64(w)))
    assert rel_err(f64(gx), ref) <= 5e-3


def test_tc_required_but_shape_not_taken():
    x = torch.zeros((1, 2, 16, 16), dtype=torch.bfloat16, device=DEV)
    w = torch.zeros((32, 3, 3, 16), dtype=torch.bfloat16, device=DEV)
    y = torch.zeros((1, 2, 16, 32), dtype=torch.bfloat16, device=DEV)
    nn.set_conv_impl(nn.IMPL_TCGEN05)
    with pytest.raises(RuntimeError):
        nn.conv3x3_fwd(x, 16, w, None, y, 32, 1, 2, 16, 16, 32, 0)  # 16 input channels: mma.sync only
    nn.set_conv_impl(nn.IMPL_AUTO)
    nn.conv3x3_fwd(x, 16, w, None, y, 32, 1, 2, 16, 16, 32, 0)  # the automatic choice takes it
    torch.cuda.synchronize()


@pytest.mark.parametrize("N,H,W,cin,cout", [(2, 3, 150, 32, 32), (1, 4, 130, 96, 32), (1, 3, 70, 64, 128),
                                            (1, 2, 100, 128, 256), (2, 3, 45, 384, 128), (1, 5, 200, 192, 64),
                                            (1, 1, 20, 32, 96)])
@pytest.mark.parametrize("splits", [0, 3])
def test_tc_weight_gradient(N, H, W, cin, cout, splits):
    """gw[o, tap, c] = sum_p gy[p, o] x[p + shift(tap), c] and gb[o] = sum_p
    gy[p, o] on the tensor cores (split K, FP32 partial sums), at FP32
    precision of the oracle's scale."""
    rng = np.random.default_rng(2 + cin + 5 * cout)
    x = bf(rng.standard_normal((N, H, W, cin)))
    gy = bf(rng.standard_normal((N, H, W, cout)))
    gw = torch.zeros((cout, 3, 3, cin), dtype=torch.float32, device=DEV)
    gb = torch.zeros(cout, dtype=torch.float32, device=DEV)
    nn.set_conv_impl(nn.IMPL_TCGEN05)
    nn.conv3x3_wgrad(x, cin, gy, cout, gw, gb, N, H, W, cin, cout, splits=splits)
    torch.cuda.synchronize()
    rw, rb = C.conv3x3_wgrad(f64(x), f64(gy))
    assert rel_err(gw.cpu().numpy(), rw) <= 1e-4
    assert rel_err(gb.cpu().numpy(), rb) <= 1e-4


def test_tc_weight_gradient_of_channel_slices():
    rng = np.random.default_rng(11)
    N, H, W = 1, 3, 90
    xb = bf(rng.standard_normal((N, H, W, 96)))
    gyb = bf(rng.standard_normal((N, H, W, 192)))
    gw = torch.zeros((64, 3, 3, 32), dtype=torch.float32, device=DEV)
    nn.set_conv_impl(nn.IMPL_TCGEN05)
    nn.conv3x3_wgrad(xb[..., 64:], 96, gyb[..., 128:], 192, gw, None, N, H, W, 32, 64)
    torch.cuda.synchronize()
    rw, _ = C.conv3x3_wgrad(f64(xb)[..., 64:], f64(gyb)[..., 128:])
    assert rel_err(gw.cpu().numpy(), rw) <= 1e-4


# Network-sized shapes: many output tiles per persistent CTA (both
# tensor-memory accumulators in use, k-blocks streaming across tiles) and
# long split-K ranges.  The reference is the mma.sync kernel family, itself
# checked against the FP64 oracle above; the two differ only in FP32
# summation order and the last bfloat16 rounding.
LARGE = [(2, 100, 800, 32, 32), (1, 64, 400, 96, 32), (2, 50, 400, 64, 128), (1, 100, 200, 384, 128),
         (4, 25, 100, 128, 256), (1, 40, 1600, 192, 64)]


def both_impls(fn, first=nn.IMPL_TCGEN05):
    outs = {}
    for impl in (first, nn.IMPL_MMA_SYNC):
        nn.set_conv_impl(impl)
        outs[impl] = fn()
        torch.cuda.synchronize()
    nn.set_conv_impl(nn.IMPL_AUTO)
    return outs[first], outs[nn.IMPL_MMA_SYNC]


@pytest.mark.parametrize("N,H,W,cin,cout", LARGE)
def test_tc_network_sized_shapes_match_mma_sync(N, H, W, cin, cout):
    rng = np.random.default_rng(100 + cin + cout + W)
    x = bf(rng.standard_normal((N, H, W, cin)))
    w = bf(rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin))
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).to(DEV)
    gy = bf(rng.standard_normal((N, H, W, cout)))
    xm = bf(rng.standard_normal((N, H, W, cin)))
    wf = torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device=DEV)
    nn.flip_weights(w, wf, cout, cin)

    def fwd():
        y = torch.full((N, H, W, cout), float("nan"), dtype=torch.bfloat16, device=DEV)
        nn.conv3x3_fwd(x, cin, w, b, y, cout, N, H, W, cin, cout, 1)
        return f64(y)

    def dgrad():
        gx = torch.full((N, H, W, cin), float("nan"), dtype=torch.bfloat16, device=DEV)
        nn.conv3x3_dgrad(gy, cout, wf, gx, cin, N, H, W, cin, cout, mask=xm, ms=cin)
        return f64(gx)

    def wgrad():
        gw = torch.zeros((cout, 3, 3, cin), dtype=torch.float32, device=DEV)
        gb = torch.zeros(cout, dtype=torch.float32, device=DEV)
        nn.conv3x3_wgrad(x, cin, gy, cout, gw, gb, N, H, W, cin, cout)
        return np.concatenate([gw.cpu().numpy().ravel(), gb.cpu().numpy()]).astype(np.float64)

    for name, fn, tol in (("fwd", fwd, 1e-2), ("dgrad", dgrad, 1e-2), ("wgrad", wgrad, 1e-4)):
        a, ref = both_impls(fn)
        assert rel_err(a, ref) <= tol, name


def test_tc_whole_network_forward_matches_mma_sync():
    """The warm-start U-Net forward at a downsized training shape (every
    level, skip slices, ragged row tiles) with both kernel families."""
    net = nn.WarmStartNet(2, 96, 400, DEV, seed=4)
    rng = np.random.default_rng(8)
    net.x0.copy_(bf(rng.standard_normal(net.x0.shape)))
    for c in net.layers.values():  # non-trivial head weights
        c.w.copy_(torch.from_numpy(rng.standard_normal(tuple(c.w.shape)).astype(np.float32)
                                   * np.sqrt(2.0 / (9 * c.cin))).to(DEV))
        c.sync_bf16(None, t=0)

    def run():
        return f64(net.forward())[..., :3]

    # automatic choice: tcgen05 for every layer it takes (all but the first
    # layer, 8 input channels, and the head, 8 outputs)
    a, ref = both_impls(run, first=nn.IMPL_AUTO)
    assert rel_err(a, ref) <= 3e-2
