"""Post-processing on synthetic signals with known answers."""
import math

import numpy as np

from paper_2605_02185_gb300 import postprocess as PP


def test_period_of_a_sinusoid():
    T = 612.7
    n = np.arange(20000)
    cl = 0.31 * np.sin(2 * math.pi * n / T + 0.3)
    assert abs(PP.period_from_crossings(cl) - T) < 0.05
    assert abs(PP.period_from_spectrum(cl) - T) / T < 2e-3
    st = PP.statistics(1.4 + 0.01 * np.sin(4 * math.pi * n / T), cl, D=10, U=0.1, periods=10)
    assert abs(st["st_zc"] - 10 / (0.1 * T)) / (10 / (0.1 * T)) < 1e-3
    assert abs(st["cl_amp"] - 0.31) < 1e-3 and abs(st["cd_mean"] - 1.4) < 1e-3


def test_periodicity_detector():
    T = 400.0
    n = np.arange(30000)
    amp = 0.3 * (1 - np.exp(-n / 3000.0))  # growing, then saturating
    cl = amp * np.sin(2 * math.pi * n / T)
    i = PP.periodic_index(cl)
    assert i is not None
    # per-period growth 0.3 e^{-n/3000} (1 - e^{-T/3000}) / amp falls below
    # 0.5 % near n ~ 9.4k; two such periods later the detector fires
    assert 9000 < i < 12000
    assert PP.periodic_index(1e-3 * np.sin(2 * math.pi * n / T)) is None  # below the amplitude floor


def test_limit_cycle_separates_clean_from_modulated_lift():
    n = np.arange(60000)
    T = 2500.0
    clean = 0.3 * np.sin(2 * math.pi * n / T)
    beat = 0.3 * (1 + 0.03 * np.sin(2 * math.pi * n / (6.3 * T))) * np.sin(2 * math.pi * n / T)
    assert PP.limit_cycle(clean)
    assert not PP.limit_cycle(beat)
    assert not PP.limit_cycle(clean[:int(3 * T)])        # too few periods
    assert not PP.limit_cycle(0.01 * clean)              # below the amplitude floor


def test_periodicity_ignores_periods_outside_the_shedding_range():
    # a clean short ringing (period 60 steps) passes the amplitude test but is
    # no shedding for D = 20, U = 0.05 (St 0.08-0.4: periods 1000-5000 steps)
    n = np.arange(6000)
    ring = 0.3 * np.sin(2 * math.pi * n / 60.0)
    rng = PP.shedding_periods(20, 0.05)
    assert abs(rng[0] - 1000) < 1e-9 and abs(rng[1] - 5000) < 1e-9
    assert PP.periodic_index(ring) is not None
    assert PP.periodic_index(ring, period_range=rng) is None
    shed = 0.3 * np.sin(2 * math.pi * np.arange(20000) / 1900.0)
    assert PP.periodic_index(shed, period_range=rng) is not None


def test_first_harmonic_amplitude_ignores_noise():
    n = np.arange(40000)
    rng = np.random.default_rng(1)
    cl = 0.3 * np.sin(2 * math.pi * n / 2000.0 + 0.4) + 0.005 * rng.standard_normal(n.size)
    cd = 1.4 + 0.01 * np.cos(4 * math.pi * n / 2000.0)
    st = PP.statistics(cd, cl, 20, 0.05, periods=10)
    assert abs(st["cl_amp_h1"] - 0.3) < 0.003       # the fundamental
    assert st["cl_amp"] > 0.31                       # (max - min) / 2 picks up the noise peaks
    assert abs(st["st"] - 20 / (0.05 * 2000)) < 1e-3
