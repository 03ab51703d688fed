"""Seeded workload inputs: generator definition, geometry, parameters."""
import math

import numpy as np

from paper_2605_02185_gb300 import workloads as W


def test_splitmix64_reference_outputs():
    # first outputs of splitmix64 seeded with 0, as published with the generator
    assert [int(z) for z in W.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # draws are addressable: start=k gives the k-th draw onwards
    assert np.array_equal(W.splitmix64(7, 5, start=3), W.splitmix64(7, 8)[3:])


def test_uniform01_range_and_mean():
    r = W.uniform01(123, 200_000)
    assert r.min() >= 0.0 and r.max() < 1.0
    assert abs(r.mean() - 0.5) < 5e-3


def test_relaxation_time_eq17():
    assert W.relaxation_time(0.1, 10, 100) == 0.53
    assert abs(W.PRODUCTION_D80.tau - 0.62) < 1e-15
    assert abs(W.THROUGHPUT_D400.tau - 0.98) < 1e-15
    assert abs(W.PARITY_D10.tau - 0.53) < 1e-15


def test_paper_box_geometry():
    for wl in (W.PARITY_D10, W.PRODUCTION_D80):
        D = wl.D
        assert (wl.nx, wl.ny, wl.xc, wl.yc) == (40 * D, 20 * D, 10 * D, 10 * D)
    m = W.PARITY_D10.mask()
    ys, xs = np.nonzero(m)
    assert ys.max() - ys.min() == 10 and xs.max() - xs.min() == 10  # D + 1 nodes across
    sub = m[90:111, 90:111]
    assert np.array_equal(sub, sub[::-1, :]) and np.array_equal(sub, sub[:, ::-1]) and np.array_equal(sub, sub.T)
    big = W.cylinder_mask(400, 400, 200, 200, 200)
    assert abs(big.sum() / (math.pi * 100 ** 2) - 1) < 5e-3


def test_initial_fields():
    wl = W.PARITY_D10
    r, u, v = wl.initial_fields()
    solid = wl.mask() == 1
    assert np.all(r == 1.0)
    assert np.all(u[solid] == 0) and np.all(v[solid] == 0)
    a = wl.perturb * wl.U
    assert np.max(np.abs(u[~solid] - wl.U)) <= a and np.max(np.abs(v[~solid])) <= a
    assert np.max(np.abs(v)) > 0.9 * a


def test_batched_cases_are_seeded():
    a = W.batched_cases(64, seed=4)
    b = W.batched_cases(64, seed=4)
    assert [c.name for c in a] == [c.name for c in b]
    assert {c.D for c in a} <= {20, 30, 40, 60}
    assert all(60 <= c.Re <= 200 for c in a)
    for c in a:
        assert abs(c.tau - (0.5 + 3 * c.U * c.D / c.Re)) < 1e-15
