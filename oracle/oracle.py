"""ctypes wrapper around the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product path
(the ``paper_2605_02185_gb300`` package) never imports it, and this module
imports nothing from the package.

The oracle follows the paper's step order (Section 2.1): collide (Eq. 2,
Eq. 3, Eq. 4), momentum exchange (Eq. 14), pull-stream with half-way
bounce-back (Section 2.4), then the top/bottom rules (Eqs. 7-10), the Zou-He
inlet (Section 3.1) and the zero-gradient outlet (Eq. 13).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(BUILD_DIR, "liblbm_oracle.so")

Y_FREESLIP, Y_PERIODIC, Y_ZOUHE, Y_MOVING, Y_WALLS = 0, 1, 2, 3, 4
X_INOUT, X_PERIODIC = 0, 1

_lib = None


def build(force: bool = False, extra_flags=(), out: str | None = None) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    out = out or LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           *extra_flags, SRC, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _bind(lib):
    d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    lib.orc_create.restype = p
    lib.orc_create.argtypes = [i, i, d, d, i, i, p]
    lib.orc_destroy.argtypes = [p]
    lib.orc_set_body_force.argtypes = [p, d, d]
    lib.orc_set_wall_velocity.argtypes = [p, d, d]
    lib.orc_set_link_q.argtypes = [p, p]
    lib.orc_set_circle_q.argtypes = [p, d, d, d]
    lib.orc_force_interpolated.argtypes = [p, p]
    lib.orc_get_link_q.argtypes = [p, p]
    lib.orc_init_equilibrium.argtypes = [p, p, p, p]
    for name in ("orc_set_f", "orc_get_f", "orc_set_fs", "orc_get_fs"):
        getattr(lib, name).argtypes = [p, p]
    lib.orc_collide.argtypes = [p]
    lib.orc_force.argtypes = [p, p]
    lib.orc_stream.argtypes = [p]
    lib.orc_boundaries.argtypes = [p]
    lib.orc_run.argtypes = [p, ctypes.c_long, p]
    lib.orc_fields.argtypes = [p, p, p, p]
    lib.orc_links.restype = ctypes.c_long
    lib.orc_links.argtypes = [p, p, ctypes.c_long]
    lib.orc_feq.argtypes = [d, d, d, p]
    lib.orc_moments.argtypes = [p, p, p, p]
    lib.orc_collide_node.argtypes = [p, d, d, d, p]
    lib.orc_constants.argtypes = [p, p, p, p]
    lib.orc_set_threads.argtypes = [i]
    lib.orc_set_collision.argtypes = [p, i, d, d, d]
    lib.orc_collide_node_mrt.argtypes = [p, p, p]
    lib.orc_mrt_matrix.argtypes = [p]
    lib.orc_max_threads.restype = i
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def constants(lib=None):
    """Table 1 as seen by the oracle: (cx, cy, w, opposite)."""
    lib = lib or load()
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    w = np.zeros(9, np.float64)
    opp = np.zeros(9, np.int32)
    lib.orc_constants(_ptr(cx), _ptr(cy), _ptr(w), _ptr(opp))
    return cx, cy, w, opp


def feq(rho: float, ux: float, uy: float, lib=None) -> np.ndarray:
    """Eq. 3 for one node."""
    lib = lib or load()
    out = np.zeros(9, np.float64)
    lib.orc_feq(rho, ux, uy, _ptr(out))
    return out


def moments(f9, lib=None):
    """Eq. 4 for one node: (rho, ux, uy)."""
    lib = lib or load()
    f9 = np.ascontiguousarray(f9, np.float64)
    r, u, v = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib.orc_moments(_ptr(f9), ctypes.byref(r), ctypes.byref(u), ctypes.byref(v))
    return r.value, u.value, v.value


def collide_node(f9, tau: float, gx: float = 0.0, gy: float = 0.0, lib=None) -> np.ndarray:
    """Eq. 2 right-hand side for one node (BGK, optional test-only Guo force)."""
    lib = lib or load()
    f9 = np.ascontiguousarray(f9, np.float64)
    out = np.zeros(9, np.float64)
    lib.orc_collide_node(_ptr(f9), tau, gx, gy, _ptr(out))
    return out


BGK, MRT = 0, 1
MRT_PAPER_RATES = (1.1, 1.1, 1.1)  # s_e, s_epsilon, s_q of the paper's S (Eq. 6)


def mrt_matrix(lib=None) -> np.ndarray:
    """M of Eq. 6 as the oracle holds it."""
    lib = lib or load()
    m = np.zeros(81, np.float64)
    lib.orc_mrt_matrix(_ptr(m))
    return m.reshape(9, 9)


def collide_node_mrt(f9, s, lib=None) -> np.ndarray:
    """Eq. 6 for one node with the rate vector s (diagonal of S)."""
    lib = lib or load()
    f9 = np.ascontiguousarray(f9, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    out = np.zeros(9, np.float64)
    lib.orc_collide_node_mrt(_ptr(f9), _ptr(s), _ptr(out))
    return out


def set_threads(n: int, lib=None):
    (lib or load()).orc_set_threads(int(n))


def max_threads(lib=None) -> int:
    return int((lib or load()).orc_max_threads())


class Oracle:
    """One FP64 lattice.  Arrays are numpy float64, populations [9, ny, nx]."""

    def __init__(self, nx, ny, tau, U, bc_y=Y_FREESLIP, bc_x=X_INOUT, mask=None, lib=None):
        self.lib = lib or load()
        self.nx, self.ny = int(nx), int(ny)
        self.tau, self.U = float(tau), float(U)
        m = None
        if mask is not None:
            m = np.ascontiguousarray(mask, np.uint8)
            assert m.shape == (self.ny, self.nx)
            self._mask = m
        self.h = self.lib.orc_create(self.nx, self.ny, self.tau, self.U, int(bc_y), int(bc_x),
                                     _ptr(m) if m is not None else None)
        if not self.h:
            raise ValueError("orc_create rejected the arguments")
        self.steps = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_collision(self, model, s_e=1.1, s_eps=1.1, s_q=1.1):
        self.lib.orc_set_collision(self.h, int(model), float(s_e), float(s_eps), float(s_q))

    def set_link_q(self, q):
        """Interpolated bounce-back with link fractions q[9, ny, nx] (None: half-way)."""
        if q is None:
            self.lib.orc_set_link_q(self.h, None)
            return
        q = np.ascontiguousarray(q, np.float64)
        assert q.shape == (9, self.ny, self.nx)
        self.lib.orc_set_link_q(self.h, q.ctypes.data)

    def set_circle_q(self, xc, yc, r):
        """Interpolated bounce-back on a circle of centre (xc, yc), radius r."""
        self.lib.orc_set_circle_q(self.h, float(xc), float(yc), float(r))

    def link_q(self) -> np.ndarray:
        """Link fractions [9, ny, nx] (zeros under the half-way rule)."""
        out = np.zeros((9, self.ny, self.nx))
        self.lib.orc_get_link_q(self.h, out.ctypes.data)
        return out

    def set_wall_velocity(self, uw_top, uw_bot):
        """Wall speeds of the constant-velocity bounce-back (Y_MOVING); both U by default."""
        self.lib.orc_set_wall_velocity(self.h, float(uw_top), float(uw_bot))

    def set_body_force(self, gx, gy):
        self.lib.orc_set_body_force(self.h, float(gx), float(gy))

    def init_equilibrium(self, rho, ux, uy):
        shp = (self.ny, self.nx)
        r = np.ascontiguousarray(np.broadcast_to(rho, shp), np.float64)
        u = np.ascontiguousarray(np.broadcast_to(ux, shp), np.float64)
        v = np.ascontiguousarray(np.broadcast_to(uy, shp), np.float64)
        self.lib.orc_init_equilibrium(self.h, _ptr(r), _ptr(u), _ptr(v))

    def _get(self, fn):
        a = np.empty((9, self.ny, self.nx), np.float64)
        fn(self.h, _ptr(a))
        return a

    def _set(self, fn, a):
        a = np.ascontiguousarray(a, np.float64)
        assert a.shape == (9, self.ny, self.nx)
        fn(self.h, _ptr(a))

    def get_f(self):
        return self._get(self.lib.orc_get_f)

    def set_f(self, a):
        self._set(self.lib.orc_set_f, a)

    def get_fs(self):
        return self._get(self.lib.orc_get_fs)

    def set_fs(self, a):
        self._set(self.lib.orc_set_fs, a)

    def collide(self):
        self.lib.orc_collide(self.h)

    def force(self):
        F = np.zeros(2, np.float64)
        self.lib.orc_force(self.h, _ptr(F))
        return F

    def stream(self):
        self.lib.orc_stream(self.h)

    def boundaries(self):
        self.lib.orc_boundaries(self.h)

    def run(self, nsteps: int) -> np.ndarray:
        """Advance nsteps; returns the (Fx, Fy) history, shape [nsteps, 2]."""
        F = np.zeros((max(int(nsteps), 0), 2), np.float64)
        if nsteps > 0:
            self.lib.orc_run(self.h, int(nsteps), _ptr(F))
        self.steps += int(nsteps)
        return F

    def fields(self):
        r = np.empty((self.ny, self.nx), np.float64)
        u = np.empty_like(r)
        v = np.empty_like(r)
        self.lib.orc_fields(self.h, _ptr(r), _ptr(u), _ptr(v))
        return r, u, v

    def links(self) -> np.ndarray:
        n = self.lib.orc_links(self.h, None, 0)
        out = np.zeros((max(n, 1), 3), np.int32)
        self.lib.orc_links(self.h, _ptr(out), n)
        return out[:n]


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
