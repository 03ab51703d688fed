"""Plant plausible mistakes in a copy of the oracle and check that a pin fails.

Each mutant is a one-token change of ``oracle/lbm_oracle.c`` compiled into a
temporary library on the CPU.  The pins are the closed forms and algebraic
properties of ``test_oracle_pins.py``; a pin that still passes on a mutant
would not be pinning that part of the oracle.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import oracle as O

import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "lbm_oracle.c")


def _mutant(old, new, count=1):
    src = open(SRC).read()
    assert src.count(old) >= 1, old
    src = src.replace(old, new, count)
    d = tempfile.mkdtemp(prefix="orc_mut_")
    c = os.path.join(d, "m.c")
    so = os.path.join(d, "m.so")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    c, "-o", so, "-lm"], check=True)
    return O.load(so)


def uniform_stream_error(lib, bc, steps=2000):
    nx, ny, U = 24, 12, 0.08
    o = O.Oracle(nx, ny, 0.7, U, bc_y=bc, bc_x=O.X_INOUT, lib=lib)
    o.init_equilibrium(1.0, U, 0.0)
    o.run(steps)
    r, u, v = o.fields()
    return max(np.max(np.abs(r - 1)), np.max(np.abs(u - U)), np.max(np.abs(v)))


def flat_wall_force(lib):
    nx, ny = 6, 5
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = 1
    o = O.Oracle(nx, ny, 0.7, 0.0, bc_y=O.Y_FREESLIP, bc_x=O.X_PERIODIC, mask=mask, lib=lib)
    o.init_equilibrium(1.0, 0.0, 0.0)
    return o.run(1)[0]


def freeslip_normal_velocity(lib):
    nx, ny, U = 31, 17, 0.08
    o = O.Oracle(nx, ny, 0.65, U, bc_y=O.Y_FREESLIP, bc_x=O.X_INOUT, lib=lib)
    rng = np.random.default_rng(9)
    o.init_equilibrium(1 + 0.01 * rng.standard_normal((ny, nx)),
                       U + 0.02 * rng.standard_normal((ny, nx)), 0.02 * rng.standard_normal((ny, nx)))
    o.run(10)
    _, _, v = o.fields()
    return max(np.max(np.abs(v[0])), np.max(np.abs(v[-1])))


def outlet_copies(lib):
    nx, ny, U = 31, 17, 0.08
    o = O.Oracle(nx, ny, 0.65, U, bc_y=O.Y_PERIODIC, bc_x=O.X_INOUT, lib=lib)
    rng = np.random.default_rng(9)
    o.init_equilibrium(1.0, U + 0.02 * rng.standard_normal((ny, nx)), 0.02 * rng.standard_normal((ny, nx)))
    o.run(10)
    f = o.get_f()
    return np.array_equal(f[:, :, -1], f[:, :, -2])


def equilibrium_second_moment_ok(lib):
    cx, cy, _, _ = O.constants(lib)
    rho, ux, uy = 1.1, 0.07, -0.04
    f = O.feq(rho, ux, uy, lib=lib)
    return (abs((f * cx * cx).sum() - rho * (1 / 3 + ux * ux)) <= 4e-16
            and abs((f * cx * cy).sum() - rho * ux * uy) <= 4e-16)


def channel_q_converges(lib, q=0.25):
    import test_oracle_interpolated as I
    e1, e2 = I.channel_q(8, q, lib=lib, max_steps=60_000)[0], I.channel_q(16, q, lib=lib, max_steps=120_000)[0]
    return 3.3 < e1 / e2 < 4.7


def channel_q_force_balance(lib, q=0.25):
    import test_oracle_interpolated as I
    _, fx, total = I.channel_q(12, q, lib=lib, max_steps=120_000)
    return abs(fx - total) <= 1e-9 * total


def couette_exact(lib, rho0=1.0):
    ny, ut, ub = 16, 0.05, -0.02
    _, u, _ = P.couette(ny, ut, ub, rho0, steps=12_000, lib=lib)
    y = np.arange(ny)[:, None]
    return np.max(np.abs(u - (ub + (ut - ub) * (y + 0.5) / ny))) <= 1e-10


def single_population_moves_by_c(lib):
    cx, cy, _, _ = O.constants(lib)
    nx, ny = 5, 4
    o = O.Oracle(nx, ny, 0.8, 0.0, bc_y=O.Y_PERIODIC, bc_x=O.X_PERIODIC, lib=lib)
    for k in range(9):
        fs = np.zeros((9, ny, nx))
        fs[k, 1, 2] = 1.0
        o.set_fs(fs)
        o.stream()
        if o.get_f()[k, (1 + cy[k]) % ny, (2 + cx[k]) % nx] != 1.0:
            return False
    return True


MUTANTS = [
    # (name, old, new, check returning True when the pin still passes)
    ("zouhe_top_sign", "- 0.5 * rho * U;  /* f8 */", "+ 0.5 * rho * U;  /* f8 */",
     lambda lib: uniform_stream_error(lib, O.Y_ZOUHE) <= 1e-13),
    ("inlet_coefficient", "(2.0 / 3.0) * rho * U", "(1.0 / 3.0) * rho * U",
     lambda lib: uniform_stream_error(lib, O.Y_FREESLIP) <= 1e-13),
    ("bounce_back_not_reversed", "interpolated_bounce(o, x, y, k) : o->fs[IDX(o, opposite(k), x, y)];",
     "interpolated_bounce(o, x, y, k) : o->fs[IDX(o, k, x, y)];",
     lambda lib: P.poiseuille(8, 0.8, lib=lib, max_steps=40_000)[0] < 0.009),
    ("force_factor", "double v = 2.0 * o->fs", "double v = 1.0 * o->fs",
     lambda lib: abs(flat_wall_force(lib)[1] + 2.0) <= 1e-12),
    ("equilibrium_quadratic", "4.5 * cu * cu", "3.0 * cu * cu", equilibrium_second_moment_ok),
    ("relaxation_inverted", "- (f9[k] - feq[k]) / tau;", "- (f9[k] - feq[k]) * (tau - 0.3);",
     lambda lib: abs(P.taylor_green_nu(32, 0.8, lib=lib)[0] - 0.1) / 0.1 < 2e-3),
    ("freeslip_transposed", "f[8] = f[5]; /* f9 = f6 */", "f[8] = f[6]; /* f9 = f6 */",
     lambda lib: freeslip_normal_velocity(lib) <= 1e-16),
    ("outlet_wrong_column", "load9(o, nx - 2, y, f);", "load9(o, nx - 3, y, f);",
     outlet_copies),
    ("stream_wrong_sign", "neighbour(o, x, y, k, -1, &sx, &sy)", "neighbour(o, x, y, k, +1, &sx, &sy)",
     single_population_moves_by_c),
    ("moving_wall_factor", "fs[k] - 2.0 * WT[k] * rho", "fs[k] - 1.0 * WT[k] * rho", couette_exact),
    ("moving_wall_sign", "fs[k] - 2.0 * WT[k] * rho", "fs[k] + 2.0 * WT[k] * rho", couette_exact),
    ("moving_wall_unit_density", "WT[k] * rho * (CX[k] * uw)", "WT[k] * 1.0 * (CX[k] * uw)",
     lambda lib: couette_exact(lib, rho0=1.5)),
    ("interp_drops_behind_node", "+ (1.0 - 2.0 * q) * o->fs[IDX(o, i, bx, by)]", "+ 0.0 * o->fs[IDX(o, i, bx, by)]",
     channel_q_converges),
    ("interp_far_branch_weight", "o->fs[IDX(o, i, x, y)] / (2.0 * q) +", "o->fs[IDX(o, i, x, y)] / (2.0 * 0.5) +",
     lambda lib: channel_q_converges(lib, q=0.7)),
    ("interp_force_one_sided", "double v = o->fs[IDX(o, k, x, y)] + o->f[IDX(o, opposite(k), x, y)];",
     "double v = 2.0 * o->fs[IDX(o, k, x, y)];", channel_q_force_balance),
    ("moving_wall_not_reversed", "if (CY[k] == into) f[opposite(k)] = fs[k]", "if (CY[k] == into) f[k] = fs[k]",
     couette_exact),
]


@pytest.mark.parametrize("name,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(orc, name, old, new, check):
    # the unmutated oracle passes the same check ...
    assert check(O.load())
    # ... and the mutant does not
    with np.errstate(all="ignore"):
        try:
            ok = check(_mutant(old, new))
        except (ValueError, FloatingPointError, ZeroDivisionError):
            ok = False
    assert not ok, f"mutant {name} passed its pin"
