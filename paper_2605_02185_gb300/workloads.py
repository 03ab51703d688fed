"""Seeded synthetic inputs for the cylinder-flow workloads.

This module holds no arithmetic of the lattice Boltzmann method.  It only
describes workloads (lattice size, cylinder, inlet speed, relaxation time,
boundary mode, step count) and generates their inputs: the solid mask and the
initial macroscopic fields.  Both the CUDA path and the test oracle receive
the same arrays from here; neither side regenerates them.

Geometry follows Section 3.1 of the paper: a circular cylinder of diameter D
with its centre 10D behind the inlet and 10D from the bottom wall, in a
40D x 20D box.  The staircased solid set is
{(x, y) : 4 ((x - xc)^2 + (y - yc)^2) <= D^2} on integer node coordinates.
The relaxation time is tau = 0.5 + 3 U D / Re (Eqs. 16-17).

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the n-th draw (n = 0, 1, ...)
mixes the state seed + (n + 1) * 0x9E3779B97F4A7C15; a double in [0, 1) is
(z >> 11) * 2^-53.  Draws are taken in row-major order, all du first, then all
dv.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_FREESLIP, BC_PERIODIC, BC_ZOUHE, BC_MOVINGWALL = 0, 1, 2, 3
BC_NAMES = {BC_FREESLIP: "freeslip", BC_PERIODIC: "periodic", BC_ZOUHE: "zouhe", BC_MOVINGWALL: "movingwall"}

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Draws start .. start+n-1 of the splitmix64 sequence for ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from splitmix64: (z >> 11) * 2^-53."""
    z = splitmix64(seed, n, start)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def relaxation_time(U: float, D: float, Re: float) -> float:
    """Eqs. 16-17: nu = U D / Re, tau = 3 nu + 1/2 (lattice units)."""
    return 3.0 * U * D / Re + 0.5


def cylinder_mask(nx: int, ny: int, xc: int, yc: int, D: int) -> np.ndarray:
    """uint8 [ny, nx], 1 on nodes with 4((x-xc)^2 + (y-yc)^2) <= D^2."""
    y, x = np.mgrid[0:ny, 0:nx]
    d2 = 4 * ((x - xc).astype(np.int64) ** 2 + (y - yc).astype(np.int64) ** 2)
    return (d2 <= int(D) * int(D)).astype(np.uint8)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One cylinder-flow case in lattice units."""

    name: str
    nx: int
    ny: int
    D: int
    xc: int
    yc: int
    U: float
    tau: float
    bc: int = BC_FREESLIP
    steps: int = 0
    seed: int = 0
    perturb: float = 0.0  # amplitude of the uniform velocity perturbation, as a fraction of U
    Re: float = 100.0

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def mask(self) -> np.ndarray:
        return cylinder_mask(self.nx, self.ny, self.xc, self.yc, self.D)

    def initial_fields(self):
        """rho = 1, u = (U + du, dv) on fluid nodes; rho = 1, u = 0 on solid nodes.

        du, dv ~ uniform(-a, a) with a = perturb * U, drawn from splitmix64.
        Returns float64 arrays [ny, nx].
        """
        n = self.cells
        rho = np.ones((self.ny, self.nx), np.float64)
        u = np.full((self.ny, self.nx), self.U, np.float64)
        v = np.zeros((self.ny, self.nx), np.float64)
        if self.perturb > 0.0:
            a = self.perturb * self.U
            uf, vf = u.reshape(-1), v.reshape(-1)
            chunk = 1 << 24
            for s in range(0, n, chunk):
                m = min(chunk, n - s)
                uf[s:s + m] += a * (2.0 * uniform01(self.seed, m, start=s) - 1.0)
                vf[s:s + m] += a * (2.0 * uniform01(self.seed, m, start=n + s) - 1.0)
        solid = self.mask().astype(bool)
        u[solid] = 0.0
        v[solid] = 0.0
        return rho, u, v

    def with_bc(self, bc: int) -> "Workload":
        return dataclasses.replace(self, bc=bc, name=f"{self.name}_{BC_NAMES[bc]}")


def cylinder_case(D: int, U: float, Re: float, bc: int = BC_FREESLIP, seed: int = 0,
                  perturb: float = 0.0, steps: int = 0, name: str | None = None,
                  tau: float | None = None) -> Workload:
    """The paper's box (Section 3.1): 40D x 20D, centre (10D, 10D)."""
    t = relaxation_time(U, D, Re) if tau is None else tau
    return Workload(name=name or f"cyl_D{D}_{40 * D}x{20 * D}", nx=40 * D, ny=20 * D, D=D,
                    xc=10 * D, yc=10 * D, U=U, tau=t, bc=bc, steps=steps, seed=seed,
                    perturb=perturb, Re=Re)


# Small parity case: Re = 100, D = 10, U = 0.1, tau = 0.53, 2000 steps, perturbed (seed 1).
PARITY_D10 = cylinder_case(10, 0.1, 100.0, seed=1, perturb=1e-3, steps=2000,
                           name="cyl_Re100_D10_400x200")
# Production case: Re = 100, D = 80, U = 0.05, tau = 0.62, 300k steps, perturbed (seed 2).
PRODUCTION_D80 = cylinder_case(80, 0.05, 100.0, seed=2, perturb=1e-3, steps=300_000,
                               name="cyl_Re100_D80_3200x1600")
# Throughput case: 128M cells, Re = 100, D = 400, U = 0.04 (Eq. 17 gives tau = 0.98).
THROUGHPUT_D400 = cylinder_case(400, 0.04, 100.0, seed=3, perturb=1e-3, steps=50_000,
                                name="cyl_Re100_D400_16000x8000")
# The throughput geometry at half the size (32M cells, 2.3 GB of FP32
# populations): small enough for counter captures, far above L2.
THROUGHPUT_D200 = cylinder_case(200, 0.04, 100.0, seed=3, perturb=1e-3, steps=50_000,
                                name="cyl_Re100_D200_8000x4000")
# Warm-start grid: D = 40, U = 0.05, 1600 x 800.
WARMSTART_D40 = cylinder_case(40, 0.05, 100.0, seed=5, perturb=1e-3,
                              name="cyl_D40_1600x800")


def batched_cases(n: int = 64, seed: int = 4, U: float = 0.05,
                  diameters=(20, 30, 40, 60), re_range=(60.0, 200.0)):
    """Independent cylinder cases of uneven size and Re (free-slip, FP32).

    Re = exp(uniform(ln 60, ln 200)), D uniform over ``diameters``; draws
    interleaved as (Re, D) per case from one splitmix64 stream.
    """
    r = uniform01(seed, 2 * n)
    lo, hi = math.log(re_range[0]), math.log(re_range[1])
    out = []
    for c in range(n):
        Re = math.exp(lo + (hi - lo) * r[2 * c])
        D = int(diameters[min(int(r[2 * c + 1] * len(diameters)), len(diameters) - 1)])
        out.append(cylinder_case(D, U, Re, seed=seed * 1000 + c, perturb=1e-3,
                                 name=f"case{c:02d}_D{D}_Re{Re:.1f}"))
    return out


def random_case(nx: int, ny: int, seed: int, bc: int, D: int | None = None,
                U: float = 0.08, tau: float = 0.6, perturb: float = 0.05) -> Workload:
    """A small odd-sized lattice with an off-centre cylinder, for parity tests.

    The cylinder keeps a margin of at least two nodes from every edge.
    """
    r = uniform01(seed, 3)
    if D is None:
        D = max(2, min(nx, ny) // 4)
    rad = (D + 1) // 2
    lo_x, hi_x = 2 + rad, nx - 3 - rad
    lo_y, hi_y = 2 + rad, ny - 3 - rad
    xc = lo_x + int(r[0] * max(hi_x - lo_x + 1, 1))
    yc = lo_y + int(r[1] * max(hi_y - lo_y + 1, 1))
    return Workload(name=f"rand{nx}x{ny}_s{seed}_{BC_NAMES[bc]}", nx=nx, ny=ny, D=D, xc=xc, yc=yc,
                    U=U, tau=tau, bc=bc, seed=seed, perturb=perturb)
