"""Pins of the oracle's MRT collision (Eq. 6)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def eq6_fixture():
    M, S = [], None
    with open(os.path.join(GOLDEN, "mrt_eq6.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] == "M":
                M.append([float(v) for v in line[1:]])
            elif line[0] == "S":
                S = line[1:]
    return np.array(M), S


def rates(tau, s=(1.1, 1.1, 1.1)):
    return np.array([1.0, s[0], s[1], 1.0, s[2], 1.0, s[2], 1 / tau, 1 / tau])


def test_matrix_matches_paper_and_rows_are_orthogonal(orc):
    M, S = eq6_fixture()
    assert np.array_equal(O.mrt_matrix(), M)
    G = M @ M.T
    assert np.array_equal(G, np.diag(np.diag(G)))
    # the rows are the moments rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy
    cx, cy, _, _ = O.constants()
    assert np.array_equal(M[0], np.ones(9)) and np.array_equal(M[3], cx) and np.array_equal(M[5], cy)
    assert np.array_equal(M[7], cx * cx - cy * cy) and np.array_equal(M[8], cx * cy)
    assert S[:7] == ["1", "1.1", "1.1", "1", "1.1", "1", "1.1"] and S[7:] == ["tau", "tau"]


def test_equilibrium_moments_equal_M_times_feq(orc):
    M, _ = eq6_fixture()
    rng = np.random.default_rng(1)
    for _ in range(50):
        r = rng.uniform(0.8, 1.2)
        u, v = rng.uniform(-0.15, 0.15, 2)
        feq = O.feq(r, u, v)
        # Eq. 6 collision of an equilibrium is the identity for any rates
        out = O.collide_node_mrt(feq, rates(0.7, (0.3, 1.7, 1.9)))
        np.testing.assert_allclose(out, feq, atol=2e-16)


def test_single_rate_reduces_to_bgk(orc):
    rng = np.random.default_rng(2)
    for tau in (0.53, 0.8, 1.3):
        f = rng.uniform(0.02, 0.4, 9)
        s = np.full(9, 1 / tau)
        np.testing.assert_allclose(O.collide_node_mrt(f, s), O.collide_node(f, tau), atol=5e-16)


def test_mrt_conserves_and_relaxes_each_moment(orc):
    M, _ = eq6_fixture()
    cx, cy, _, _ = O.constants()
    rng = np.random.default_rng(3)
    r, u, v = 1.01, 0.05, -0.02
    feq = O.feq(r, u, v)
    s = rates(0.6, (1.2, 1.4, 1.6))
    for k in (1, 2, 4, 6, 7, 8):  # non-conserved moments
        e = np.zeros(9)
        e[k] = 1e-3
        f = feq + np.linalg.solve(M, e)  # perturb one moment only
        out = O.collide_node_mrt(f, s)
        dm = M @ (out - feq)
        want = np.zeros(9)
        want[k] = (1 - s[k]) * 1e-3
        np.testing.assert_allclose(dm, want, atol=1e-15)
    f = rng.uniform(0.02, 0.4, 9)
    out = O.collide_node_mrt(f, s)
    assert abs(out.sum() - f.sum()) < 1e-15
    assert abs((out * cx).sum() - (f * cx).sum()) < 1e-15
    assert abs((out * cy).sum() - (f * cy).sum()) < 1e-15


def test_mrt_taylor_green_viscosity():
    # the shear rate 1/tau of Eq. 6 sets nu = (tau - 1/2)/3
    N, tau, U0 = 48, 0.8, 0.01
    k = 2 * math.pi / N
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    u = -U0 * np.cos(k * x) * np.sin(k * y)
    v = U0 * np.sin(k * x) * np.cos(k * y)
    rho = 1.0 - 0.75 * U0 ** 2 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    o = O.Oracle(N, N, tau, 0.0, bc_y=O.Y_PERIODIC, bc_x=O.X_PERIODIC)
    o.set_collision(O.MRT)
    o.init_equilibrium(rho, u, v)
    nu = (tau - 0.5) / 3
    t1, t2 = 200, 1200

    def energy():
        r, uu, vv = o.fields()
        return float((r * (uu * uu + vv * vv)).sum())

    o.run(t1)
    e1 = energy()
    o.run(t2 - t1)
    e2 = energy()
    nu_eff = math.log(e1 / e2) / (t2 - t1) / (4 * k * k)
    assert abs(nu_eff - nu) / nu < 2e-3


@pytest.mark.parametrize("bc", [O.Y_FREESLIP, O.Y_PERIODIC, O.Y_ZOUHE])
def test_mrt_uniform_stream_stays_uniform(orc, bc):
    nx, ny, U = 24, 12, 0.08
    o = O.Oracle(nx, ny, 0.7, U, bc_y=bc, bc_x=O.X_INOUT)
    o.set_collision(O.MRT)
    o.init_equilibrium(1.0, U, 0.0)
    o.run(5000)
    r, u, v = o.fields()
    assert np.max(np.abs(r - 1.0)) <= 1e-13 and np.max(np.abs(u - U)) <= 1e-13 and np.max(np.abs(v)) <= 1e-13
