"""Pins of the oracle's interpolated bounce-back (Bouzidi-Firdaouss-Lallemand,
linear) and of its momentum exchange, against what the mathematics fixes:
q = 1/2 is the half-way rule bit for bit, a force-driven channel whose walls
sit a fraction q of a link from the last fluid row converges to the parabola
through the true wall positions at second order, and the wall force balances
the body force at steady state."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_02185_gb300 import workloads as W


def channel_q(H, q, tau=0.8, lib=None, nx=3, umax=0.01, tol=1e-14, max_steps=400_000):
    """Fluid rows 1..H between solid rows 0 and H+1; every link into a wall
    has fraction q, so the walls are at y = 1 - q and y = H + q.  Returns
    (max error of u / umax against the parabola through the walls, wall
    force Fx, total body force)."""
    nu = (tau - 0.5) / 3.0
    y0, y1 = 1.0 - q, H + q
    g = 8.0 * nu * umax / (y1 - y0) ** 2
    ny = H + 2
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = mask[-1, :] = 1
    o = O.Oracle(nx, ny, tau, 0.0, bc_y=O.Y_WALLS, bc_x=O.X_PERIODIC, mask=mask, lib=lib)
    qa = np.zeros((9, ny, nx))
    cx, cy, _, _ = O.constants(lib)
    for i in range(1, 9):
        if cy[i] == -1:
            qa[i, 1, :] = q
        if cy[i] == 1:
            qa[i, H, :] = q
    o.set_link_q(qa)
    o.set_body_force(g, 0.0)
    y = np.arange(ny, dtype=np.float64)
    exact = g / (2 * nu) * (y - y0) * (y1 - y)
    o.init_equilibrium(1.0, np.where(mask[:, 0:1] == 1, 0.0, exact[:, None]) * np.ones((1, nx)), 0.0)
    prev, steps = None, 0
    while steps < max_steps:
        F = o.run(2000)
        steps += 2000
        _, u, _ = o.fields()
        prof = u[1:-1, 0].copy()
        if prev is not None and np.max(np.abs(prof - prev)) <= tol * umax:
            break
        prev = prof
    err = np.max(np.abs(prof - exact[1:-1])) / umax
    return err, F[-1, 0], g * nx * H


@pytest.mark.parametrize("q", [0.25, 0.7])
def test_channel_with_offset_walls_second_order(orc, q):
    errs = [channel_q(H, q)[0] for H in (8, 16, 32)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs
    assert errs[2] < 3e-3, errs


def test_halfway_rule_misplaces_offset_walls(orc):
    # the same parabola (walls at 1 - q, H + q) is not reached by the
    # half-way rule, whose walls sit at 1/2 and H + 1/2: the interpolation
    # is what moves the wall
    H, q = 16, 0.25
    err_interp = channel_q(H, q)[0]
    err_halfway = channel_q(H, 0.5)[0]  # exact parabola of the half-way walls
    shift = abs((H - 1 + 2 * q) ** 2 - H ** 2) / H ** 2  # size of the wall displacement effect
    assert err_interp < 0.1 * shift and err_halfway < 0.1 * shift, (err_interp, err_halfway, shift)


@pytest.mark.parametrize("q", [0.25, 0.7])
def test_wall_force_balances_body_force(orc, q):
    _, fx, total = channel_q(16, q)
    assert abs(fx - total) <= 1e-9 * total


def test_half_link_fraction_is_the_halfway_rule(orc):
    wl = W.random_case(41, 23, seed=5, bc=W.BC_FREESLIP, D=8)
    a = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
    b = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
    b.set_link_q(np.full((9, wl.ny, wl.nx), 0.5))
    for o in (a, b):
        o.init_equilibrium(*wl.initial_fields())
    Fa, Fb = a.run(30), b.run(30)
    assert np.array_equal(a.get_f(), b.get_f())
    assert np.array_equal(Fa, Fb)


def test_circle_fractions_lie_on_the_circle(orc):
    # every link fraction q places x + q c_i on the circle |p - c| = D/2
    wl = W.random_case(61, 41, seed=3, bc=W.BC_FREESLIP, D=12)
    o = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
    o.set_circle_q(wl.xc, wl.yc, wl.D / 2)
    links = o.links()
    cx, cy, _, _ = O.constants()
    assert len(links) > 0
    qa = o.link_q()
    for (x, y, i) in links:
        t = qa[i, y, x]
        assert 0.0 < t <= 1.0
        px, py = x + t * cx[i] - wl.xc, y + t * cy[i] - wl.yc
        assert abs(np.hypot(px, py) - wl.D / 2) <= 1e-12


def test_symmetric_body_at_rest_feels_no_force(orc):
    # fluid at rest around a mirror-symmetric staircased circle with its
    # link fractions: every step's two-sided momentum exchange cancels
    nx, ny, D = 41, 41, 14
    yy, xx = np.mgrid[0:ny, 0:nx]
    mask = (4 * ((xx - 20) ** 2 + (yy - 20) ** 2) <= D * D).astype(np.uint8)
    o = O.Oracle(nx, ny, 0.7, 0.0, bc_y=O.Y_PERIODIC, bc_x=O.X_PERIODIC, mask=mask)
    o.set_circle_q(20.0, 20.0, D / 2)
    o.init_equilibrium(1.0, 0.0, 0.0)
    F = o.run(20)
    assert np.max(np.abs(F)) <= 1e-13
    r, u, v = o.fields()
    fluid = mask == 0
    assert np.max(np.abs(u[fluid])) <= 1e-15 and np.max(np.abs(v[fluid])) <= 1e-15
