"""Plain FP64 CPU oracle of the warm-start network's arithmetic.

TEST INFRASTRUCTURE ONLY: imported by the tests (and nothing in the product
path).  Every function is the textbook definition written with numpy in
float64, with no blocking or fusion: 3x3 convolution with zero padding 1
(cross-correlation, NHWC activations, weights [Cout][3][3][Cin]), its two
gradients, ReLU, 2x2 average pooling, 2x nearest upsampling, mean squared
error, one Adam update (Kingma and Ba 2015, with bias correction), and the
first-order Chapman-Enskog non-equilibrium populations used to start the
lattice from predicted macroscopic fields.
"""
from __future__ import annotations

import numpy as np

# D2Q9, Table 1 of the paper (k = i - 1)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], np.float64)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], np.float64)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, np.float64)


def conv3x3(x, w, b=None):
    """y[n,h,w,o] = b[o] + sum_{dy,dx,c} x[n,h+dy-1,w+dx-1,c] w[o,dy,dx,c]."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    n, H, Wd, cin = x.shape
    cout = w.shape[0]
    xp = np.zeros((n, H + 2, Wd + 2, cin))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((n, H, Wd, cout))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + Wd, :]
            y += patch @ w[:, dy, dx, :].T
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3x3_dgrad(gy, w):
    """dL/dx for y = conv3x3(x, w): gx[n,h,w,c] = sum gy[n,h-dy+1,w-dx+1,o] w[o,dy,dx,c]."""
    gy = np.asarray(gy, np.float64)
    w = np.asarray(w, np.float64)
    n, H, Wd, cout = gy.shape
    cin = w.shape[3]
    gp = np.zeros((n, H + 2, Wd + 2, cout))
    gp[:, 1:-1, 1:-1, :] = gy
    gx = np.zeros((n, H, Wd, cin))
    for dy in range(3):
        for dx in range(3):
            # x[h + dy - 1] feeds y[h]; so x[h] feeds y[h - dy + 1]
            patch = gp[:, 2 - dy:2 - dy + H, 2 - dx:2 - dx + Wd, :]
            gx += patch @ w[:, dy, dx, :]
    return gx


def conv3x3_wgrad(x, gy):
    """dL/dw[o,dy,dx,c] = sum_{n,h,w} gy[n,h,w,o] x[n,h+dy-1,w+dx-1,c]; dL/db = sum gy."""
    x = np.asarray(x, np.float64)
    gy = np.asarray(gy, np.float64)
    n, H, Wd, cin = x.shape
    cout = gy.shape[3]
    xp = np.zeros((n, H + 2, Wd + 2, cin))
    xp[:, 1:-1, 1:-1, :] = x
    gw = np.zeros((cout, 3, 3, cin))
    g2 = gy.reshape(-1, cout)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + Wd, :].reshape(-1, cin)
            gw[:, dy, dx, :] = g2.T @ patch
    return gw, g2.sum(axis=0)


def relu(x):
    return np.maximum(x, 0.0)


def relu_grad(y, gy):
    """Gradient through ReLU given its output y."""
    return np.where(y > 0.0, gy, 0.0)


def avgpool2(x):
    n, H, Wd, c = x.shape
    return x.reshape(n, H // 2, 2, Wd // 2, 2, c).mean(axis=(2, 4))


def avgpool2_grad(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_grad(gy):
    n, H, Wd, c = gy.shape
    return gy.reshape(n, H // 2, 2, Wd // 2, 2, c).sum(axis=(2, 4))


def mse(pred, target, weight=None):
    """L = mean over elements of weight * (pred - target)^2 and dL/dpred."""
    d = np.asarray(pred, np.float64) - np.asarray(target, np.float64)
    wgt = np.ones_like(d) if weight is None else np.broadcast_to(weight, d.shape)
    n = d.size
    return float((wgt * d * d).sum() / n), 2.0 * wgt * d / n


def adam(param, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (param, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def velocity_gradient(u, v, solid=None):
    """du_a/dx_b on the lattice: central differences, one-sided next to the
    lattice edge or a solid node (then the difference uses the fluid side
    only), zero where both neighbours are unavailable.  Returns
    (dudx, dudy, dvdx, dvdy) as [ny, nx] arrays."""
    ny, nx = u.shape
    fluid = np.ones((ny, nx), bool) if solid is None else ~np.asarray(solid, bool)

    def deriv(f, axis):
        out = np.zeros_like(f)
        n = f.shape[axis]
        for i in range(n):
            sl = [slice(None)] * 2
            sl[axis] = i
            lo = [slice(None)] * 2
            hi = [slice(None)] * 2
            ok_lo = np.zeros(f.shape[1 - axis], bool)
            ok_hi = np.zeros(f.shape[1 - axis], bool)
            if i - 1 >= 0:
                lo[axis] = i - 1
                ok_lo = fluid[tuple(lo)]
            if i + 1 < n:
                hi[axis] = i + 1
                ok_hi = fluid[tuple(hi)]
            fc = f[tuple(sl)]
            flo = f[tuple(lo)] if i - 1 >= 0 else fc
            fhi = f[tuple(hi)] if i + 1 < n else fc
            d = np.where(ok_lo & ok_hi, 0.5 * (fhi - flo),
                         np.where(ok_hi, fhi - fc, np.where(ok_lo, fc - flo, 0.0)))
            out[tuple(sl)] = d
        return out

    return deriv(u, 1), deriv(u, 0), deriv(v, 1), deriv(v, 0)


def noneq_populations(rho, u, v, tau, solid=None):
    """First-order Chapman-Enskog non-equilibrium part of f for BGK:
    f_neq_i = -(tau w_i rho / c_s^2) Q_i:grad(u), Q_i = c_i c_i - c_s^2 I,
    c_s^2 = 1/3.  Returns [9, ny, nx]; zero on solid nodes."""
    dudx, dudy, dvdx, dvdy = velocity_gradient(u, v, solid)
    cs2 = 1.0 / 3.0
    out = np.zeros((9,) + u.shape)
    for k in range(9):
        qxx = CX[k] * CX[k] - cs2
        qyy = CY[k] * CY[k] - cs2
        qxy = CX[k] * CY[k]
        contr = qxx * dudx + qyy * dvdy + qxy * (dudy + dvdx)
        out[k] = -(tau * W9[k] * rho / cs2) * contr
    if solid is not None:
        out[:, np.asarray(solid, bool)] = 0.0
    return out
