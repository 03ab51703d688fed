"""Force-coefficient post-processing: mean drag, lift amplitude, Strouhal
number and a periodicity detector (host side, numpy).

Cd and Cl histories come from the solver one entry per step (Eq. 15).  The
Strouhal number is St = f D / U with f the shedding frequency in steps^-1,
which equals the paper's physical definition with Delta t from Eq. 18 (the
conversion factors cancel).  The shedding period T is taken from the lift
spectrum (Hann window, zero-padded FFT, parabolic interpolation of the peak)
and cross-checked against the mean spacing of upward zero crossings of Cl.
"""
from __future__ import annotations

import math

import numpy as np


# Hysteresis of the zero-crossing detector, as a fraction of max |Cl|: a
# crossing counts only after the lift has been below -HYST max |Cl| since the
# previous one, so noise on the history (16-bit storage with stochastic
# rounding) does not split one crossing into several.
HYST = 0.05


def upward_crossings(cl, hysteresis: float | None = None) -> np.ndarray:
    """Fractional indices where cl crosses zero from below (linear
    interpolation), each after cl went below -hysteresis (default HYST max |cl|)."""
    c = np.asarray(cl, np.float64)
    if len(c) < 2:
        return np.zeros(0)
    eps = HYST * float(np.max(np.abs(c))) if hysteresis is None else hysteresis
    i = np.nonzero((c[:-1] < 0.0) & (c[1:] >= 0.0))[0]
    if eps > 0.0 and len(i):
        below = np.nonzero(c <= -eps)[0]
        # keep crossing i if some sample in (previous kept crossing, i] is <= -eps
        keep, last = [], -1
        for j in i:
            k = np.searchsorted(below, last + 1)
            if k < len(below) and below[k] <= j:
                keep.append(j)
                last = j
        i = np.asarray(keep, dtype=np.int64)
    return i + (-c[i]) / (c[i + 1] - c[i])


def period_from_crossings(cl) -> float:
    z = upward_crossings(cl)
    if len(z) < 2:
        return math.nan
    return float(np.mean(np.diff(z)))


def period_from_spectrum(cl, pad: int = 16) -> float:
    """Dominant period of cl (in entries) from a Hann-windowed, zero-padded
    FFT with a parabolic fit through the peak bin and its neighbours."""
    c = np.asarray(cl, np.float64)
    c = c - c.mean()
    n = len(c)
    if n < 8:
        return math.nan
    spec = np.abs(np.fft.rfft(c * np.hanning(n), n * pad))
    spec[0] = 0.0
    k = int(np.argmax(spec))
    if 0 < k < len(spec) - 1:
        a, b, g = spec[k - 1], spec[k], spec[k + 1]
        den = a - 2 * b + g
        k = k + (0.5 * (a - g) / den if den != 0 else 0.0)
    f = k / (n * pad)
    return 1.0 / f if f > 0 else math.nan


def period_amplitudes(cl) -> np.ndarray:
    """(max - min)/2 of cl over each complete period between upward crossings."""
    c = np.asarray(cl, np.float64)
    z = upward_crossings(c)
    out = []
    for a, b in zip(z[:-1], z[1:]):
        seg = c[int(math.ceil(a)):int(math.floor(b)) + 1]
        if len(seg):
            out.append(0.5 * (seg.max() - seg.min()))
    return np.array(out)


def shedding_periods(D: float, U: float, st_lo: float = 0.08, st_hi: float = 0.4):
    """Range of lift periods (in steps) that belong to vortex shedding: a
    Strouhal number D / (U T) between st_lo and st_hi."""
    return D / (st_hi * U), D / (st_lo * U)


def periodic_index(cl, amp_min: float = 0.05, tol: float = 0.005, consecutive: int = 2, period_range=None):
    """First entry index at which shedding counts as periodic: each of the
    last `consecutive` complete periods has amplitude >= amp_min and differs
    from the period before it by less than tol (relative), and -- if
    period_range = (T_min, T_max) is given -- lasts between T_min and T_max
    steps (so that a short acoustic ringing of the start is not taken for
    shedding).  None if never."""
    c = np.asarray(cl, np.float64)
    z = upward_crossings(c)
    amps = period_amplitudes(c)
    lens = np.diff(z) if len(z) > 1 else np.zeros(0)
    run = 0
    for k in range(1, len(amps)):
        ok = amps[k] >= amp_min and amps[k - 1] >= amp_min and abs(amps[k] - amps[k - 1]) < tol * amps[k]
        if ok and period_range is not None:
            ok = all(period_range[0] <= lens[j] <= period_range[1] for j in (k - 1, k))
        run = run + 1 if ok else 0
        if run >= consecutive:
            return int(math.ceil(z[k + 1]))
    return None


def limit_cycle(cl, periods: int = 6, tol: float = 0.01, amp_min: float = 0.05) -> bool:
    """True when the last `periods` complete lift periods all have amplitude
    >= amp_min and spread by less than tol (relative to their mean): a clean
    limit cycle, as opposed to a modulated or chaotic lift that passes the
    period-to-period test by chance."""
    a = period_amplitudes(cl)
    if len(a) < periods:
        return False
    a = a[-periods:]
    return bool(a.min() >= amp_min and (a.max() - a.min()) < tol * a.mean())


def statistics(cd, cl, D: float, U: float, periods: int | None = None) -> dict:
    """Mean Cd, Cl amplitude and Strouhal number over the window: the last
    `periods` complete lift periods (all of them if None)."""
    cd = np.asarray(cd, np.float64)
    cl = np.asarray(cl, np.float64)
    z = upward_crossings(cl)
    if periods is not None and len(z) > periods:
        a, b = int(math.ceil(z[-periods - 1])), int(math.floor(z[-1]))
    elif len(z) >= 2:
        a, b = int(math.ceil(z[0])), int(math.floor(z[-1]))
    else:
        a, b = 0, len(cl) - 1
    w_cd, w_cl = cd[a:b + 1], cl[a:b + 1]
    T_zc = period_from_crossings(cl[a:b + 1]) if b > a else math.nan
    T_fft = period_from_spectrum(cl[a:b + 1]) if b > a else math.nan
    # amplitude of the lift's fundamental over the window (least-squares fit
    # of one harmonic at the spectral period): unlike (max - min) / 2 it does
    # not grow with noise on the history
    h1 = math.nan
    if len(w_cl) > 8 and T_fft == T_fft:
        t = np.arange(len(w_cl), dtype=np.float64)
        basis = np.stack([np.cos(2 * math.pi * t / T_fft), np.sin(2 * math.pi * t / T_fft), np.ones_like(t)], 1)
        coef, *_ = np.linalg.lstsq(basis, w_cl, rcond=None)
        h1 = float(math.hypot(coef[0], coef[1]))
    return {"cd_mean": float(w_cd.mean()) if len(w_cd) else math.nan,
            "cl_amp": float(0.5 * (w_cl.max() - w_cl.min())) if len(w_cl) else math.nan,
            "cl_amp_h1": h1,
            "st": D / (U * T_fft) if T_fft == T_fft else math.nan,
            "st_zc": D / (U * T_zc) if T_zc == T_zc else math.nan,
            "window": (a, b)}
