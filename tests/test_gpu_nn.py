"""Tensor-core network kernels against the FP64 network oracle.

Inputs are drawn in float, rounded to bfloat16 on the device, and the oracle
runs in float64 on exactly those rounded values, so the only differences are
FP32 accumulation order and the bfloat16 rounding of outputs: outputs stored
in bfloat16 are compared at 5e-3 of their scale (2^-8 is the bfloat16 step),
FP32 outputs (weight gradients) at 1e-4.
"""
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


def close(got, ref, tol):
    scale = max(np.max(np.abs(ref)), 1e-30)
    err = np.max(np.abs(got - ref)) / scale
    assert err <= tol, err


SHAPES = [(2, 6, 150, 16, 32), (1, 5, 130, 40, 48), (1, 4, 37, 8, 8), (2, 3, 129, 96, 64), (1, 4, 20, 64, 136)]


@pytest.mark.parametrize("N,H,W,cin,cout", SHAPES)
@pytest.mark.parametrize("relu", [0, 1])
def test_conv_forward(N, H, W, cin, cout, relu):
    rng = np.random.default_rng(cin + cout)
    x = bf(rng.standard_normal((N, H, W, cin)))
    w = bf(rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin))
    b = torch.from_numpy(rng.standard_normal(cout).astype(np.float32)).to(DEV)
    y = torch.empty((N, H, W, cout), dtype=torch.bfloat16, device=DEV)
    nn.conv3x3_fwd(x, cin, w, b, y, cout, N, H, W, cin, cout, relu)
    torch.cuda.synchronize()
    ref = C.conv3x3(f64(x), f64(w), b.cpu().numpy())
    if relu:
        ref = C.relu(ref)
    close(f64(y), ref, 5e-3)


def test_conv_forward_into_channel_slices():
    # read a slice of a wider buffer and write into the tail of another
    rng = np.random.default_rng(7)
    N, H, W = 1, 5, 70
    big = bf(rng.standard_normal((N, H, W, 48)))
    out = torch.zeros((N, H, W, 40), dtype=torch.bfloat16, device=DEV)
    w = bf(rng.standard_normal((16, 3, 3, 32)) / 17)
    nn.conv3x3_fwd(big[..., 16:], 48, w, None, out[..., 24:], 40, N, H, W, 32, 16, 0)
    torch.cuda.synchronize()
    ref = C.conv3x3(f64(big)[..., 16:], f64(w))
    close(f64(out)[..., 24:], ref, 5e-3)
    assert np.all(f64(out)[..., :24] == 0)


@pytest.mark.parametrize("N,H,W,cin,cout", SHAPES)
def test_conv_input_gradient(N, H, W, cin, cout):
    rng = np.random.default_rng(1 + cin)
    w = bf(rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin))
    gy = bf(rng.standard_normal((N, H, W, cout)))
    xmask = bf(rng.standard_normal((N, H, W, cin)))
    wf = torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device=DEV)
    nn.flip_weights(w, wf, cout, cin)
    gx = torch.empty((N, H, W, cin), dtype=torch.bfloat16, device=DEV)
    nn.conv3x3_dgrad(gy, cout, wf, gx, cin, N, H, W, cin, cout, mask=xmask, ms=cin)
    torch.cuda.synchronize()
    ref = C.relu_grad(f64(xmask), C.conv3x3_dgrad(f64(gy), f64(w)))
    close(f64(gx), ref, 5e-3)


@pytest.mark.parametrize("N,H,W,cin,cout", [(2, 6, 150, 16, 32), (1, 5, 130, 40, 48), (1, 4, 37, 8, 8),
                                            (2, 3, 129, 96, 64), (1, 4, 20, 64, 136)])
def test_conv_weight_gradient(N, H, W, cin, cout):
    rng = np.random.default_rng(2 + cout)
    x = bf(rng.standard_normal((N, H, W, cin)))
    gy = bf(rng.standard_normal((N, H, W, cout)))
    gw = torch.zeros((cout, 3, 3, cin), dtype=torch.float32, device=DEV)
    gb = torch.zeros(cout, dtype=torch.float32, device=DEV)
    nn.conv3x3_wgrad(x, cin, gy, cout, gw, gb, N, H, W, cin, cout, splits=7)
    torch.cuda.synchronize()
    rw, rb = C.conv3x3_wgrad(f64(x), f64(gy))
    close(gw.cpu().numpy(), rw, 1e-4)
    close(gb.cpu().numpy(), rb, 1e-4)


def test_pool_upsample_and_backward():
    rng = np.random.default_rng(3)
    N, H, W, Cc = 2, 6, 10, 16
    x = bf(rng.standard_normal((N, H, W, Cc)))
    y = torch.empty((N, H // 2, W // 2, Cc), dtype=torch.bfloat16, device=DEV)
    nn.avgpool2(x, Cc, y, Cc, N, H, W, Cc)
    gy = bf(rng.standard_normal((N, H // 2, W // 2, Cc)))
    gx = bf(rng.standard_normal((N, H, W, Cc)))
    gx0 = f64(gx)
    mask = bf(rng.standard_normal((N, H, W, Cc)))
    nn.avgpool2_bwd(gy, Cc, gx, Cc, N, H, W, Cc, accumulate=True, mask=mask, ms=Cc)
    u = torch.empty((N, 2 * H, 2 * W, Cc), dtype=torch.bfloat16, device=DEV)
    nn.upsample2(x, Cc, u, Cc, N, H, W, Cc)
    gu = bf(rng.standard_normal((N, 2 * H, 2 * W, Cc)))
    gxu = torch.empty((N, H, W, Cc), dtype=torch.bfloat16, device=DEV)
    nn.upsample2_bwd(gu, Cc, gxu, Cc, N, H, W, Cc)
    torch.cuda.synchronize()
    close(f64(y), C.avgpool2(f64(x)), 5e-3)
    close(f64(gx), gx0 + C.relu_grad(f64(mask), C.avgpool2_grad(f64(gy))), 5e-3)
    close(f64(u), C.upsample2(f64(x)), 0.0)
    close(f64(gxu), C.upsample2_grad(f64(gu)), 5e-3)


def test_mse_and_adam():
    rng = np.random.default_rng(4)
    P, Cc = 1000, 3
    pred = bf(rng.standard_normal((P, 8)))
    tgt = torch.from_numpy(rng.standard_normal((P, Cc)).astype(np.float32)).to(DEV)
    wgt = torch.from_numpy((rng.random(P) > 0.2).astype(np.float32)).to(DEV)
    grad = torch.zeros((P, 8), dtype=torch.bfloat16, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    nn.mse(pred, 8, tgt, wgt, grad, 8, P, Cc, 1.0 / (P * Cc), loss)
    torch.cuda.synchronize()
    L, g = C.mse(f64(pred)[:, :3], tgt.cpu().numpy(), wgt.cpu().numpy()[:, None])
    assert abs(loss.item() / (P * Cc) - L) <= 1e-5 * L
    close(f64(grad)[:, :3], g, 5e-3)
    assert np.all(f64(grad)[:, 3:] == 0)
    p = torch.from_numpy(rng.standard_normal(500).astype(np.float32)).to(DEV)
    gg = torch.from_numpy(rng.standard_normal(500).astype(np.float32)).to(DEV)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    p0 = p.cpu().numpy().astype(np.float64)
    p16 = torch.empty(500, dtype=torch.bfloat16, device=DEV)
    rp, rm, rv = p0, np.zeros(500), np.zeros(500)
    for t in (1, 2, 3):
        nn.adam(p, gg, m, v, p16, 500, 1e-2, t)
        rp, rm, rv = C.adam(rp, gg.cpu().numpy().astype(np.float64), rm, rv, t, 1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(p.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)
    close(f64(p16), rp, 5e-3)


def bf16_round(a):
    """Round float64 values to bfloat16 (nearest, ties to even) and back."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def oracle_network_grads(net, x0, target, weight, rnd=lambda a: a):
    """The same encoder-decoder in float64 from the oracle's layer functions,
    with the network's current bfloat16 weights; returns {layer: (gw, gb)}.
    rnd is applied wherever the device stores a bfloat16 tensor (identity:
    pure float64; bf16_round: the device's storage precision)."""
    W = {k: (f64(c.w16), c.b.cpu().numpy().astype(np.float64)) for k, c in net.layers.items()}
    cv = lambda k, x, relu=True: rnd((C.relu if relu else (lambda z: z))(C.conv3x3(x, *W[k])))  # noqa: E731
    a1 = cv("c1a", x0)
    s1 = cv("c1b", a1)
    p1 = rnd(C.avgpool2(s1))
    a2 = cv("c2a", p1)
    s2 = cv("c2b", a2)
    p2 = rnd(C.avgpool2(s2))
    a3 = cv("c3a", p2)
    s3 = cv("c3b", a3)
    p3 = rnd(C.avgpool2(s3))
    a4 = cv("c4a", p3)
    b4 = cv("c4b", a4)
    cat3 = np.concatenate([C.upsample2(b4), s3], -1)
    e3 = cv("d3a", cat3)
    d3 = cv("d3b", e3)
    cat2 = np.concatenate([C.upsample2(d3), s2], -1)
    e2 = cv("d2a", cat2)
    d2 = cv("d2b", e2)
    cat1 = np.concatenate([C.upsample2(d2), s1], -1)
    e1 = cv("d1a", cat1)
    d1 = cv("d1b", e1)
    out = cv("head", d1, relu=False)
    n = out[..., :3].size
    g_out = np.zeros_like(out)
    g_out[..., :3] = rnd(2 * weight[..., None] * (out[..., :3] - target) / n)
    grads = {}

    def back(k, x, g, mask):
        # g: gradient w.r.t. the layer's pre-activation; returns the input
        # gradient, masked by the ReLU derivative of the input if it is one
        grads[k] = C.conv3x3_wgrad(x, g)
        gx = C.conv3x3_dgrad(g, W[k][0])
        return rnd(C.relu_grad(mask, gx) if mask is not None else gx)

    g = back("head", d1, g_out, d1)
    g = back("d1b", e1, g, e1)
    g = back("d1a", cat1, g, cat1)
    g_up1, g_s1 = g[..., :64], g[..., 64:]
    g = back("d2b", e2, rnd(C.upsample2_grad(g_up1)), e2)
    g = back("d2a", cat2, g, cat2)
    g_up2, g_s2 = g[..., :128], g[..., 128:]
    g = back("d3b", e3, rnd(C.upsample2_grad(g_up2)), e3)
    g = back("d3a", cat3, g, cat3)
    g_up3, g_s3 = g[..., :256], g[..., 256:]
    g = back("c4b", a4, rnd(C.upsample2_grad(g_up3)), a4)
    g = back("c4a", p3, g, None)
    g = back("c3b", a3, rnd(g_s3 + C.relu_grad(s3, C.avgpool2_grad(g))), a3)
    g = back("c3a", p2, g, None)
    g = back("c2b", a2, rnd(g_s2 + C.relu_grad(s2, C.avgpool2_grad(g))), a2)
    g = back("c2a", p1, g, None)
    g = back("c1b", a1, rnd(g_s1 + C.relu_grad(s1, C.avgpool2_grad(g))), a1)
    grads["c1a"] = C.conv3x3_wgrad(x0, g)
    return grads


def test_network_gradients_match_oracle():
    N, H, W = 1, 16, 24
    net = nn.WarmStartNet(N, H, W, DEV, seed=3)
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal((N, H, W, 8)).astype(np.float32)
    net.x0.copy_(bf(x0))
    target = rng.standard_normal((N * H * W, 3)).astype(np.float32)
    weight = (rng.random(N * H * W) > 0.1).astype(np.float32)
    tg = torch.from_numpy(target).to(DEV)
    wg = torch.from_numpy(weight).to(DEV)
    net.forward()
    net.loss_and_grad(tg, wg)
    net.backward()
    torch.cuda.synchronize()
    x0r, tr, wr = f64(net.x0), target.reshape(N, H, W, 3), weight.reshape(N, H, W)
    exact = oracle_network_grads(net, x0r, tr, wr)
    emul = oracle_network_grads(net, x0r, tr, wr, rnd=bf16_round)
    errs = {}
    for k, c in net.layers.items():
        gw, gb = c.gw.cpu().numpy(), c.gb.cpu().numpy()
        for name, ref in (("exact", exact), ("bf16", emul)):
            rw, rb = ref[k]
            errs[(k, name)] = (np.linalg.norm(gw - rw) / max(np.linalg.norm(rw), 1e-30),
                               np.linalg.norm(gb - rb) / max(np.linalg.norm(rb), 1e-30))
    print({k: tuple(round(float(x), 5) for x in v) for k, v in errs.items()})
    for (k, name), (ew, eb) in errs.items():
        # against the oracle with the device's bfloat16 storage: FP32
        # accumulation order and rare ReLU-mask flips only
        if name == "bf16":
            assert ew < 0.02 and eb < 0.02, (k, ew, eb)
        # against pure float64: the bfloat16 storage along a 15-layer chain
        else:
            assert ew < 0.15 and eb < 0.15, (k, ew, eb)


def test_network_trains_on_a_fixed_target():
    N, H, W = 2, 32, 64
    net = nn.WarmStartNet(N, H, W, DEV, seed=1)
    rng = np.random.default_rng(6)
    net.x0.copy_(bf(rng.standard_normal((N, H, W, 8)) * 0.5))
    yy, xx = np.mgrid[0:H, 0:W]
    tgt = np.stack([np.sin(xx / 7.0), np.cos(yy / 5.0), 0.1 * np.ones_like(xx)], -1).astype(np.float32)
    tg = torch.from_numpy(np.broadcast_to(tgt, (N, H, W, 3)).reshape(-1, 3).copy()).to(DEV)
    wg = torch.ones(N * H * W, dtype=torch.float32, device=DEV)
    losses = []
    for it in range(150):
        net.forward()
        loss = net.loss_and_grad(tg, wg)
        net.backward()
        net.adam_step(2e-3)
        if it % 10 == 0:
            losses.append(loss.item() / (N * H * W * 3))
    assert losses[-1] < 0.2 * losses[0], losses


def test_encoders_and_decoder():
    """Network input channels; targets ((rho - 1)/s, (u - U)/q, v/q) with the
    fluid weight; the decoder inverts the target map of a bfloat16 output."""
    rng = np.random.default_rng(17)
    H, W, U, s, q = 7, 12, 0.05, 8 * 0.05 ** 2, 0.01
    P = H * W
    solid = np.zeros((H, W), np.uint8)
    solid[3, 4:7] = 1
    rho = (1 + 0.003 * rng.standard_normal((H, W))).astype(np.float32)
    u = (U * (1 + 0.2 * rng.standard_normal((H, W)))).astype(np.float32)
    v = (0.01 * rng.standard_normal((H, W))).astype(np.float32)
    t_solid = torch.from_numpy(solid).to(DEV)
    tr, tu, tv = (torch.from_numpy(a).to(DEV) for a in (rho, u, v))
    target = torch.empty((P, 3), dtype=torch.float32, device=DEV)
    weight = torch.empty(P, dtype=torch.float32, device=DEV)
    nn.encode_target(tr, tu, tv, t_solid, P, U, q, s, target, weight)
    want = np.stack([(rho - np.float32(1)) / np.float32(s), (u - np.float32(U)) / np.float32(q), v / np.float32(q)],
                    -1).reshape(P, 3)
    np.testing.assert_allclose(target.cpu().numpy(), want, rtol=1e-6, atol=1e-6)
    assert np.array_equal(weight.cpu().numpy(), 1.0 - solid.reshape(-1))
    out = torch.zeros((P, 8), dtype=torch.bfloat16, device=DEV)
    out[:, :3] = target.to(torch.bfloat16)
    r2, u2, v2 = (torch.empty((H, W), dtype=torch.float32, device=DEV) for _ in range(3))
    nn.decode_output(out, 8, t_solid, P, U, q, s, r2, u2, v2)
    o = out[:, :3].float().cpu().numpy().reshape(H, W, 3)
    fl = solid == 0
    np.testing.assert_allclose(r2.cpu().numpy()[fl], (1 + s * o[..., 0])[fl], rtol=1e-6)
    np.testing.assert_allclose(u2.cpu().numpy()[fl], (U + q * o[..., 1])[fl], rtol=1e-6)
    np.testing.assert_allclose(v2.cpu().numpy()[fl], (q * o[..., 2])[fl], rtol=1e-6, atol=1e-9)
    assert np.all(r2.cpu().numpy()[~fl] == 1) and np.all(u2.cpu().numpy()[~fl] == 0)
    x = torch.empty((H, W, 8), dtype=torch.bfloat16, device=DEV)
    nn.encode_input(t_solid, 0.25, 1.0, H, W, x, wave_k=0.3, wave_x0=2.0)
    xs = x.float().cpu().numpy()
    assert np.array_equal(xs[..., 0], solid.astype(np.float32))
    np.testing.assert_allclose(xs[..., 1], 0.25)
    np.testing.assert_allclose(xs[..., 2], np.sin(1.0), rtol=4e-3)
    np.testing.assert_allclose(xs[..., 3], np.cos(1.0), rtol=4e-3)
    np.testing.assert_allclose(xs[..., 4], np.arange(W)[None, :] / W * np.ones((H, 1)), rtol=4e-3, atol=1e-6)
    np.testing.assert_allclose(xs[..., 5], np.arange(H)[:, None] / H * np.ones((1, W)), rtol=4e-3, atol=1e-6)
    arg = 0.3 * (np.arange(W)[None, :] - 2.0) - 1.0 + np.zeros((H, 1))
    np.testing.assert_allclose(xs[..., 6], np.cos(arg), atol=4e-3)
    np.testing.assert_allclose(xs[..., 7], np.sin(arg), atol=4e-3)
