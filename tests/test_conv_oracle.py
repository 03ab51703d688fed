"""Pins of the FP64 network oracle: closed forms, brute force, adjoint
identities and finite differences."""
import numpy as np
import pytest

from oracle import conv_oracle as C


def brute_conv(x, w, b):
    n, H, W, cin = x.shape
    cout = w.shape[0]
    y = np.zeros((n, H, W, cout))
    for i in range(n):
        for h in range(H):
            for q in range(W):
                for o in range(cout):
                    s = b[o]
                    for dy in range(3):
                        for dx in range(3):
                            hh, qq = h + dy - 1, q + dx - 1
                            if 0 <= hh < H and 0 <= qq < W:
                                for c in range(cin):
                                    s += x[i, hh, qq, c] * w[o, dy, dx, c]
                    y[i, h, q, o] = s
    return y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(C.conv3x3(x, w, b), brute_conv(x, w, b), rtol=1e-13, atol=1e-13)


def test_conv_delta_kernels_are_identity_and_shift():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 6, 7, 2))
    w = np.zeros((2, 3, 3, 2))
    w[0, 1, 1, 0] = w[1, 1, 1, 1] = 1.0
    np.testing.assert_array_equal(C.conv3x3(x, w), x)
    w = np.zeros((2, 3, 3, 2))
    w[0, 0, 1, 0] = w[1, 0, 1, 1] = 1.0  # y[h] = x[h - 1]
    y = C.conv3x3(x, w)
    np.testing.assert_array_equal(y[:, 1:], x[:, :-1])
    np.testing.assert_array_equal(y[:, 0], 0.0)


def test_conv_gradients_adjoint_and_finite_difference():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 6, 5, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    gy = rng.standard_normal((2, 6, 5, 4))
    y = C.conv3x3(x, w)
    gx = C.conv3x3_dgrad(gy, w)
    gw, gb = C.conv3x3_wgrad(x, gy)
    # <conv(x), gy> = <x, dgrad(gy)> = <w, wgrad(x, gy)>
    s = (y * gy).sum()
    assert abs(s - (x * gx).sum()) <= 1e-12 * abs(s)
    assert abs(s - (w * gw).sum()) <= 1e-12 * abs(s)
    # central finite differences of L = <conv(x, w) + b, gy>
    h = 1e-6
    for idx in [(0, 2, 3, 1), (1, 0, 4, 2), (1, 5, 0, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = ((C.conv3x3(xp, w) * gy).sum() - (C.conv3x3(xm, w) * gy).sum()) / (2 * h)
        assert abs(fd - gx[idx]) <= 1e-6 * max(1.0, abs(gx[idx]))
    for idx in [(0, 0, 0, 0), (3, 2, 1, 2), (2, 1, 1, 1)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = ((C.conv3x3(x, wp) * gy).sum() - (C.conv3x3(x, wm) * gy).sum()) / (2 * h)
        assert abs(fd - gw[idx]) <= 1e-6 * max(1.0, abs(gw[idx]))
    b = rng.standard_normal(4)
    fd = ((C.conv3x3(x, w, b + h * np.eye(4)[1]) * gy).sum() - (C.conv3x3(x, w, b - h * np.eye(4)[1]) * gy).sum()) / (2 * h)
    assert abs(fd - gb[1]) <= 1e-6 * max(1.0, abs(gb[1]))


def test_pool_upsample_adjoints():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 8, 6, 3))
    g = rng.standard_normal((2, 4, 3, 3))
    assert abs((C.avgpool2(x) * g).sum() - (x * C.avgpool2_grad(g)).sum()) < 1e-12
    u = rng.standard_normal((2, 4, 3, 3))
    gu = rng.standard_normal((2, 8, 6, 3))
    assert abs((C.upsample2(u) * gu).sum() - (u * C.upsample2_grad(gu)).sum()) < 1e-12
    # avgpool of a constant is the constant; upsample repeats
    np.testing.assert_allclose(C.avgpool2(np.full((1, 4, 4, 1), 3.0)), 3.0)
    assert C.upsample2(np.arange(4.0).reshape(1, 2, 2, 1))[0, :, :, 0].tolist() == \
        [[0, 0, 1, 1], [0, 0, 1, 1], [2, 2, 3, 3], [2, 2, 3, 3]]


def test_mse_and_relu_gradients():
    rng = np.random.default_rng(4)
    p = rng.standard_normal((3, 4))
    t = rng.standard_normal((3, 4))
    L, g = C.mse(p, t)
    assert L == pytest.approx(((p - t) ** 2).mean())
    h = 1e-7
    p2 = p.copy()
    p2[1, 2] += h
    assert (C.mse(p2, t)[0] - L) / h == pytest.approx(g[1, 2], rel=1e-5)
    y = C.relu(p)
    assert np.all(C.relu_grad(y, np.ones_like(p)) == (p > 0))


def test_adam_first_step_closed_form():
    # at t = 1 the bias-corrected moments are g and g^2: step = lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = C.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_noneq_moments_for_linear_shear():
    # u = a y + b x, v = c x + d y: central differences are exact in the interior
    ny, nx = 9, 11
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    a, b, c, d = 1e-3, -2e-3, 5e-4, 2e-3
    u = 0.05 + a * yy + b * xx
    v = c * xx + d * yy
    rho = np.full((ny, nx), 1.02)
    tau = 0.7
    fn = C.noneq_populations(rho, u, v, tau)
    inner = (slice(None), slice(1, -1), slice(1, -1))
    f = fn[inner]
    np.testing.assert_allclose(f.sum(axis=0), 0.0, atol=1e-18)
    np.testing.assert_allclose((f * C.CX[:, None, None]).sum(axis=0), 0.0, atol=1e-18)
    np.testing.assert_allclose((f * C.CY[:, None, None]).sum(axis=0), 0.0, atol=1e-18)
    cs2 = 1 / 3
    r = 1.02
    pxx = (f * (C.CX ** 2)[:, None, None]).sum(axis=0)
    pyy = (f * (C.CY ** 2)[:, None, None]).sum(axis=0)
    pxy = (f * (C.CX * C.CY)[:, None, None]).sum(axis=0)
    np.testing.assert_allclose(pxx, -tau * r * cs2 * 2 * b, rtol=1e-12)
    np.testing.assert_allclose(pyy, -tau * r * cs2 * 2 * d, rtol=1e-12)
    np.testing.assert_allclose(pxy, -tau * r * cs2 * (a + c), rtol=1e-12)


def test_velocity_gradient_one_sided_at_edges_and_solid():
    ny, nx = 5, 6
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    u = 2.0 * xx + 3.0 * yy
    v = np.zeros_like(u)
    solid = np.zeros((ny, nx), bool)
    solid[2, 3] = True
    dudx, dudy, _, _ = C.velocity_gradient(u, v, solid)
    assert np.allclose(dudx[~solid], 2.0) and np.allclose(dudy[~solid], 3.0)
