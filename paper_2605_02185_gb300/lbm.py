"""Python binding of the C ABI in ``include/gblbm.h`` (argument marshalling only).

Every function here has the name of the C entry point it wraps and raises
``LBMError`` on a negative return code.  All lattice work runs in the CUDA
library ``_lib/libgblbm.so``; there is no Python or CPU fallback: if the
library is missing, importing the binding's loader raises.

``Lattice`` is a thin convenience wrapper: it allocates the device workspace
as a torch tensor and runs the context on a torch stream, so PyTorch supplies
device memory and streams while the library does all the computing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgblbm.so")

LBM_OK = 0
LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT = -1, -2, -3, -4
LBM_ERR_OOM, LBM_ERR_RANGE, LBM_ERR_STATE = -5, -6, -7
LBM_BC_FREESLIP, LBM_BC_PERIODIC, LBM_BC_ZOUHE, LBM_BC_MOVINGWALL = 0, 1, 2, 3
LBM_F32, LBM_F16_OFS, LBM_BF16_OFS, LBM_F64, LBM_F16_SR, LBM_BF16_SR = 0, 1, 2, 3, 4, 5
LBM_KERNEL_AUTO, LBM_KERNEL_DIRECT, LBM_KERNEL_TMA, LBM_KERNEL_TMA_BULK, LBM_KERNEL_TMA_WAVE = 0, 1, 2, 3, 4
LBM_COLLIDE_BGK, LBM_COLLIDE_MRT = 0, 1
LBM_BOUNCE_HALFWAY, LBM_BOUNCE_INTERPOLATED = 0, 1
ELEM_BYTES = {LBM_F32: 4, LBM_F16_OFS: 2, LBM_BF16_OFS: 2, LBM_F64: 8, LBM_F16_SR: 2, LBM_BF16_SR: 2}
ELEM_NUMPY = {LBM_F32: np.float32, LBM_F16_OFS: np.float16, LBM_BF16_OFS: np.uint16, LBM_F64: np.float64,
              LBM_F16_SR: np.float16, LBM_BF16_SR: np.uint16}


class LBMError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lbm_error_string(code)} ({code})")


class lbm_opts(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau", ctypes.c_double), ("U", ctypes.c_double),
        ("bc_top_bottom", ctypes.c_int), ("storage", ctypes.c_int),
        ("D_ref", ctypes.c_double), ("rho_in", ctypes.c_double),
        ("history_capacity", ctypes.c_int64),
        ("kernel", ctypes.c_int), ("consumer_warps", ctypes.c_int),
        ("cells_per_thread", ctypes.c_int), ("stages", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int), ("graph_steps", ctypes.c_int),
        ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("collision", ctypes.c_int),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("bounce", ctypes.c_int),
        ("body_xc", ctypes.c_double), ("body_yc", ctypes.c_double), ("body_r", ctypes.c_double),
    ]


class lbm_case(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau", ctypes.c_double), ("U", ctypes.c_double),
        ("bc_top_bottom", ctypes.c_int), ("mask", ctypes.c_void_p),
        ("D_ref", ctypes.c_double), ("rho_in", ctypes.c_double),
    ]


_lib = None


def load_library(path: str | None = None):
    """Load libgblbm.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CUDA library {p} is missing: run __graft_entry__.build() "
                          "(nvcc for sm_103a) first; there is no CPU fallback")
    lib = ctypes.CDLL(p)
    vp, i, i64, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    sig = {
        "lbm_opts_default": (i, [ctypes.POINTER(lbm_opts)]),
        "lbm_workspace_bytes": (i, [ctypes.POINTER(lbm_opts), vp, ctypes.POINTER(sz)]),
        "lbm_create": (i, [i, i, d, d, vp, i, ctypes.POINTER(vp)]),
        "lbm_create_ex": (i, [ctypes.POINTER(lbm_opts), vp, ctypes.POINTER(vp)]),
        "lbm_destroy": (None, [vp]),
        "lbm_init_fields": (i, [vp, vp, vp, vp]),
        "lbm_init_fields_device": (i, [vp, vp, vp, vp, i]),
        "lbm_step": (i, [vp, i64]),
        "lbm_sync": (i, [vp]),
        "lbm_force_count": (i, [vp, ctypes.POINTER(i64)]),
        "lbm_forces": (i, [vp, i64, i64, vp, vp]),
        "lbm_forces_raw": (i, [vp, i64, i64, vp]),
        "lbm_set_reference": (i, [vp, d, d]),
        "lbm_fields": (i, [vp, i, vp, vp, vp]),
        "lbm_fields_device": (i, [vp, vp, vp, vp]),
        "lbm_mass": (i, [vp, ctypes.POINTER(d)]),
        "lbm_get_populations": (i, [vp, vp, sz]),
        "lbm_set_populations": (i, [vp, vp, sz, i64]),
        "lbm_get_window": (i, [vp, i, i, i, i, vp]),
        "lbm_set_kernel": (i, [vp, i, i, i, i, i]),
        "lbm_get_kernel": (i, [vp, vp]),
        "lbm_default_kernel": (i, [ctypes.POINTER(lbm_opts), vp]),
        "lbm_kernel_shapes": (i, [vp, i, ctypes.POINTER(i)]),
        "lbm_kernel_shapes_for": (i, [i, vp, i, ctypes.POINTER(i)]),
        "lbm_get_stream": (i, [vp, ctypes.POINTER(vp)]),
        "lbm_launch_count": (i, [vp, ctypes.POINTER(i64)]),
        "lbm_bytes_per_step": (i, [vp, ctypes.POINTER(d)]),
        "lbm_step_noalloc": (i, [vp, vp, vp, vp]),
        "lbm_set_fault_injection": (i, [vp, i64, d]),
        "lbm_checkpoint_bytes": (i, [vp, ctypes.POINTER(sz)]),
        "lbm_checkpoint_save": (i, [vp, vp, sz]),
        "lbm_checkpoint_load": (i, [vp, vp, sz]),
        "lbm_probe_neg_recip": (i, [vp, vp, vp, i64, vp]),
        "lbm_probe_stochastic_round": (i, [i, vp, vp, vp, i64, vp]),
        "lbm_batch_workspace_bytes": (i, [i, vp, ctypes.POINTER(lbm_opts), ctypes.POINTER(sz)]),
        "lbm_batch_create": (i, [i, vp, ctypes.POINTER(lbm_opts), ctypes.POINTER(vp)]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_batch_case": (i, [vp, i, ctypes.POINTER(vp)]),
        "lbm_batch_init_fields": (i, [vp, i, vp, vp, vp]),
        "lbm_batch_step": (i, [vp, i64]),
        "lbm_batch_sync": (i, [vp]),
        "lbm_batch_set_kernel": (i, [vp, i, i, i, i, i]),
        "lbm_batch_get_kernel": (i, [vp, vp]),
        "lbm_batch_get_stream": (i, [vp, ctypes.POINTER(vp)]),
        "lbm_batch_launch_count": (i, [vp, ctypes.POINTER(i64)]),
        "lbm_batch_nodes": (i, [vp, ctypes.POINTER(i64), ctypes.POINTER(d)]),
        "lbm_error_string": (ctypes.c_char_p, [i]),
        "lbm_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc < 0:
        raise LBMError(rc, where)
    return rc


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def lbm_error_string(code: int) -> str:
    return load_library().lbm_error_string(int(code)).decode()


def lbm_version() -> str:
    return load_library().lbm_version().decode()


def lbm_opts_default() -> lbm_opts:
    o = lbm_opts()
    _check(load_library().lbm_opts_default(ctypes.byref(o)), "lbm_opts_default")
    return o


def _mask_arg(mask, nx, ny):
    if mask is None:
        return None, None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.shape != (ny, nx):
        raise ValueError(f"mask shape {m.shape} != ({ny}, {nx})")
    return m, _p(m)


def lbm_workspace_bytes(opts: lbm_opts, mask=None) -> int:
    _, mp = _mask_arg(mask, opts.nx, opts.ny)
    out = ctypes.c_size_t()
    _check(load_library().lbm_workspace_bytes(ctypes.byref(opts), mp, ctypes.byref(out)), "lbm_workspace_bytes")
    return int(out.value)


def lbm_create(nx, ny, tau, U, mask, bc_top_bottom) -> ctypes.c_void_p:
    _, mp = _mask_arg(mask, nx, ny)
    h = ctypes.c_void_p()
    _check(load_library().lbm_create(int(nx), int(ny), float(tau), float(U), mp, int(bc_top_bottom),
                                     ctypes.byref(h)), "lbm_create")
    return h


def lbm_create_ex(opts: lbm_opts, mask=None) -> ctypes.c_void_p:
    _, mp = _mask_arg(mask, opts.nx, opts.ny)
    h = ctypes.c_void_p()
    _check(load_library().lbm_create_ex(ctypes.byref(opts), mp, ctypes.byref(h)), "lbm_create_ex")
    return h


def lbm_destroy(h):
    if h:
        load_library().lbm_destroy(h)


def lbm_init_fields(h, rho, u, v):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, u, v)]
    _check(load_library().lbm_init_fields(h, *[_p(a) for a in arrs]), "lbm_init_fields")


def lbm_init_fields_ptr(h, rho_ptr: int, u_ptr: int, v_ptr: int):
    """Same as lbm_init_fields from raw host pointers (e.g. pinned tensors)."""
    _check(load_library().lbm_init_fields(h, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr),
                                          ctypes.c_void_p(v_ptr)), "lbm_init_fields")


def lbm_init_fields_device(h, rho_ptr: int, u_ptr: int, v_ptr: int, with_noneq: bool):
    _check(load_library().lbm_init_fields_device(h, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr),
                                                 ctypes.c_void_p(v_ptr), int(bool(with_noneq))),
           "lbm_init_fields_device")


def lbm_step(h, n: int):
    _check(load_library().lbm_step(h, int(n)), "lbm_step")


def lbm_sync(h):
    _check(load_library().lbm_sync(h), "lbm_sync")


def lbm_force_count(h) -> int:
    c = ctypes.c_int64()
    _check(load_library().lbm_force_count(h, ctypes.byref(c)), "lbm_force_count")
    return int(c.value)


def lbm_forces(h, first: int, n: int):
    cd = np.zeros(max(int(n), 0), np.float64)
    cl = np.zeros_like(cd)
    _check(load_library().lbm_forces(h, int(first), int(n), _p(cd), _p(cl)), "lbm_forces")
    return cd, cl


def lbm_forces_ptr(h, first: int, n: int, cd_ptr: int, cl_ptr: int):
    _check(load_library().lbm_forces(h, int(first), int(n), ctypes.c_void_p(cd_ptr), ctypes.c_void_p(cl_ptr)),
           "lbm_forces")


def lbm_forces_raw(h, first: int, n: int) -> np.ndarray:
    out = np.zeros((max(int(n), 0), 2), np.float64)
    _check(load_library().lbm_forces_raw(h, int(first), int(n), _p(out)), "lbm_forces_raw")
    return out


def lbm_set_reference(h, D_ref: float, rho_in: float = 1.0):
    _check(load_library().lbm_set_reference(h, float(D_ref), float(rho_in)), "lbm_set_reference")


def lbm_fields(h, nx: int, ny: int, dtype=np.float64):
    dt = np.dtype(dtype)
    flag = 1 if dt == np.float64 else 0
    if dt not in (np.dtype(np.float64), np.dtype(np.float32)):
        raise ValueError("dtype must be float32 or float64")
    out = [np.empty((ny, nx), dt) for _ in range(3)]
    _check(load_library().lbm_fields(h, flag, *[_p(a) for a in out]), "lbm_fields")
    return tuple(out)


def lbm_fields_ptr(h, dtype_flag: int, rho_ptr: int, u_ptr: int, v_ptr: int):
    _check(load_library().lbm_fields(h, int(dtype_flag), ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr),
                                     ctypes.c_void_p(v_ptr)), "lbm_fields")


def lbm_fields_device(h, rho_ptr: int, u_ptr: int, v_ptr: int):
    _check(load_library().lbm_fields_device(h, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr),
                                            ctypes.c_void_p(v_ptr)), "lbm_fields_device")


def lbm_mass(h) -> float:
    m = ctypes.c_double()
    _check(load_library().lbm_mass(h, ctypes.byref(m)), "lbm_mass")
    return float(m.value)


def lbm_get_populations(h, nx: int, ny: int, storage: int) -> np.ndarray:
    out = np.empty((9, ny, nx), ELEM_NUMPY[storage])
    _check(load_library().lbm_get_populations(h, _p(out), out.nbytes), "lbm_get_populations")
    return out


def lbm_set_populations(h, pops: np.ndarray, history_count: int):
    a = np.ascontiguousarray(pops)
    _check(load_library().lbm_set_populations(h, _p(a), a.nbytes, int(history_count)), "lbm_set_populations")


def lbm_get_window(h, x0: int, y0: int, w: int, hh: int, storage: int) -> np.ndarray:
    out = np.empty((9, hh, w), ELEM_NUMPY[storage])
    _check(load_library().lbm_get_window(h, int(x0), int(y0), int(w), int(hh), _p(out)), "lbm_get_window")
    return out


def lbm_step_noalloc(h, f_in_ptr: int, f_out_ptr: int, force_out_ptr: int):
    """One step from caller-owned device buffers, with no allocation (see gblbm.h)."""
    _check(load_library().lbm_step_noalloc(h, ctypes.c_void_p(f_in_ptr), ctypes.c_void_p(f_out_ptr),
                                           ctypes.c_void_p(force_out_ptr)), "lbm_step_noalloc")


def lbm_set_fault_injection(h, tile: int, wait_seconds: float):
    """Failure-path test control (see gblbm.h): bounded-wait limit and a row
    tile whose copies are announced but never issued (tile < 0: none)."""
    _check(load_library().lbm_set_fault_injection(h, int(tile), float(wait_seconds)), "lbm_set_fault_injection")


def lbm_checkpoint_save(h) -> bytes:
    """The self-describing checkpoint image of the current state."""
    lib = load_library()
    n = ctypes.c_size_t()
    _check(lib.lbm_checkpoint_bytes(h, ctypes.byref(n)), "lbm_checkpoint_bytes")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.lbm_checkpoint_save(h, buf, n.value), "lbm_checkpoint_save")
    return buf.raw


def lbm_checkpoint_load(h, image: bytes):
    buf = ctypes.create_string_buffer(bytes(image), len(image))
    _check(load_library().lbm_checkpoint_load(h, buf, len(image)), "lbm_checkpoint_load")


def lbm_probe_neg_recip(x_ptr: int, y_single_ptr: int, y_pair_ptr: int, n: int, stream_ptr: int = 0):
    _check(load_library().lbm_probe_neg_recip(ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_single_ptr),
                                              ctypes.c_void_p(y_pair_ptr), int(n), ctypes.c_void_p(stream_ptr)),
           "lbm_probe_neg_recip")


def lbm_probe_stochastic_round(storage: int, x_ptr: int, salt_ptr: int, out_ptr: int, n: int, stream_ptr: int = 0):
    _check(load_library().lbm_probe_stochastic_round(int(storage), ctypes.c_void_p(x_ptr), ctypes.c_void_p(salt_ptr),
                                                     ctypes.c_void_p(out_ptr), int(n), ctypes.c_void_p(stream_ptr)),
           "lbm_probe_stochastic_round")


def lbm_set_kernel(h, kernel: int, consumer_warps=0, cells_per_thread=0, stages=0, ctas_per_sm=1):
    _check(load_library().lbm_set_kernel(h, int(kernel), int(consumer_warps), int(cells_per_thread), int(stages),
                                         int(ctas_per_sm)), "lbm_set_kernel")


def lbm_get_kernel(h) -> dict:
    out = np.zeros(6, np.int32)
    _check(load_library().lbm_get_kernel(h, _p(out)), "lbm_get_kernel")
    keys = ("kernel", "consumer_warps", "cells_per_thread", "stages", "ctas_per_sm", "grid")
    return dict(zip(keys, (int(v) for v in out)))


def lbm_default_kernel(opts: lbm_opts) -> dict:
    out = np.zeros(5, np.int32)
    _check(load_library().lbm_default_kernel(ctypes.byref(opts), _p(out)), "lbm_default_kernel")
    keys = ("kernel", "consumer_warps", "cells_per_thread", "stages", "ctas_per_sm")
    return dict(zip(keys, (int(v) for v in out)))


def lbm_kernel_shapes(kernel: int = LBM_KERNEL_TMA) -> list:
    n = ctypes.c_int()
    _check(load_library().lbm_kernel_shapes_for(int(kernel), None, 0, ctypes.byref(n)), "lbm_kernel_shapes_for")
    out = np.zeros(3 * n.value, np.int32)
    _check(load_library().lbm_kernel_shapes_for(int(kernel), _p(out), n.value, ctypes.byref(n)),
           "lbm_kernel_shapes_for")
    return [tuple(int(v) for v in out[3 * i:3 * i + 3]) for i in range(n.value)]


def lbm_get_stream(h) -> int:
    s = ctypes.c_void_p()
    _check(load_library().lbm_get_stream(h, ctypes.byref(s)), "lbm_get_stream")
    return int(s.value or 0)


def lbm_launch_count(h) -> int:
    c = ctypes.c_int64()
    _check(load_library().lbm_launch_count(h, ctypes.byref(c)), "lbm_launch_count")
    return int(c.value)


def lbm_bytes_per_step(h) -> float:
    b = ctypes.c_double()
    _check(load_library().lbm_bytes_per_step(h, ctypes.byref(b)), "lbm_bytes_per_step")
    return float(b.value)


class Lattice:
    """One cylinder-flow lattice on the GPU.

    Device memory is a torch uint8 tensor handed to the library as its
    workspace; the context runs on ``stream`` (a torch.cuda.Stream, created
    if not given).  All computation happens in libgblbm.
    """

    def __init__(self, nx, ny, tau, U, mask=None, bc=LBM_BC_FREESLIP, storage=LBM_F32, D_ref=0.0,
                 rho_in=1.0, kernel=LBM_KERNEL_AUTO, shape=None, ctas_per_sm=0, graph_steps=0,
                 history_capacity=1 << 20, stream=None, device=None, collision=LBM_COLLIDE_BGK,
                 mrt_rates=(1.1, 1.1, 1.1), bounce=LBM_BOUNCE_HALFWAY, body=None):
        import torch

        load_library()
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        o = lbm_opts_default()
        o.nx, o.ny, o.tau, o.U = int(nx), int(ny), float(tau), float(U)
        o.bc_top_bottom, o.storage = int(bc), int(storage)
        o.D_ref, o.rho_in = float(D_ref), float(rho_in)
        o.history_capacity = int(history_capacity)
        o.kernel = int(kernel)
        if shape is not None:
            o.consumer_warps, o.cells_per_thread, o.stages = (int(v) for v in shape)
        o.ctas_per_sm = int(ctas_per_sm)
        o.graph_steps = int(graph_steps)
        o.collision = int(collision)
        o.s_e, o.s_eps, o.s_q = (float(v) for v in mrt_rates)
        o.bounce = int(bounce)
        if body is not None:
            o.body_xc, o.body_yc, o.body_r = (float(v) for v in body)
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        nbytes = lbm_workspace_bytes(o, mask)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        o.workspace = ctypes.c_void_p(self.workspace.data_ptr())
        o.workspace_bytes = nbytes
        self.opts = o
        self.nx, self.ny, self.storage = int(nx), int(ny), int(storage)
        self.U, self.tau = float(U), float(tau)
        with torch.cuda.device(self.device):
            self.h = lbm_create_ex(o, mask)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_fields(self, rho, u, v):
        lbm_init_fields(self.h, rho, u, v)

    def step(self, n: int):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def force_count(self) -> int:
        return lbm_force_count(self.h)

    def forces(self, first: int = 0, n: int | None = None):
        if n is None:
            n = self.force_count() - first
        return lbm_forces(self.h, first, n)

    def forces_raw(self, first: int = 0, n: int | None = None):
        if n is None:
            n = self.force_count() - first
        return lbm_forces_raw(self.h, first, n)

    def fields(self, dtype=np.float64):
        return lbm_fields(self.h, self.nx, self.ny, dtype)

    def mass(self) -> float:
        return lbm_mass(self.h)

    def get_populations(self) -> np.ndarray:
        return lbm_get_populations(self.h, self.nx, self.ny, self.storage)

    def set_populations(self, pops, history_count: int):
        lbm_set_populations(self.h, pops, history_count)

    def checkpoint(self) -> bytes:
        return lbm_checkpoint_save(self.h)

    def restore(self, image: bytes):
        lbm_checkpoint_load(self.h, image)

    def get_window(self, x0, y0, w, h) -> np.ndarray:
        return lbm_get_window(self.h, x0, y0, w, h, self.storage)

    def set_kernel(self, kernel, consumer_warps=0, cells_per_thread=0, stages=0, ctas_per_sm=0):
        lbm_set_kernel(self.h, kernel, consumer_warps, cells_per_thread, stages, ctas_per_sm)

    def kernel_info(self) -> dict:
        return lbm_get_kernel(self.h)

    def launch_count(self) -> int:
        return lbm_launch_count(self.h)

    def bytes_per_step(self) -> float:
        return lbm_bytes_per_step(self.h)


def lattice_for(workload, **kw) -> Lattice:
    """A Lattice for a ``workloads.Workload`` (its mask, tau, U, bc, D; with
    interpolated bounce-back its circle)."""
    kw.setdefault("bc", workload.bc)
    kw.setdefault("D_ref", float(workload.D))
    if kw.get("bounce", LBM_BOUNCE_HALFWAY) == LBM_BOUNCE_INTERPOLATED:
        kw.setdefault("body", (float(workload.xc), float(workload.yc), 0.5 * float(workload.D)))
    return Lattice(workload.nx, workload.ny, workload.tau, workload.U, mask=workload.mask(), **kw)


def _case_array(cases, masks):
    arr = (lbm_case * len(cases))()
    for i, c in enumerate(cases):
        arr[i].nx, arr[i].ny = int(c["nx"]), int(c["ny"])
        arr[i].tau, arr[i].U = float(c["tau"]), float(c["U"])
        arr[i].bc_top_bottom = int(c.get("bc", LBM_BC_FREESLIP))
        arr[i].mask = masks[i].ctypes.data if masks[i] is not None else None
        arr[i].D_ref = float(c.get("D_ref", 0.0))
        arr[i].rho_in = float(c.get("rho_in", 1.0))
    return arr


def lbm_batch_workspace_bytes(cases, masks, opts: lbm_opts) -> int:
    arr = _case_array(cases, masks)
    out = ctypes.c_size_t()
    _check(load_library().lbm_batch_workspace_bytes(len(cases), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(opts),
                                                    ctypes.byref(out)), "lbm_batch_workspace_bytes")
    return int(out.value)


def lbm_batch_create(cases, masks, opts: lbm_opts):
    arr = _case_array(cases, masks)
    h = ctypes.c_void_p()
    _check(load_library().lbm_batch_create(len(cases), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(opts),
                                           ctypes.byref(h)), "lbm_batch_create")
    return h


def lbm_batch_destroy(h):
    if h:
        load_library().lbm_batch_destroy(h)


def lbm_batch_case(h, c: int):
    ctx = ctypes.c_void_p()
    _check(load_library().lbm_batch_case(h, int(c), ctypes.byref(ctx)), "lbm_batch_case")
    return ctx


def lbm_batch_init_fields(h, c: int, rho, u, v):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, u, v)]
    _check(load_library().lbm_batch_init_fields(h, int(c), *[_p(a) for a in arrs]), "lbm_batch_init_fields")


def lbm_batch_step(h, n: int):
    _check(load_library().lbm_batch_step(h, int(n)), "lbm_batch_step")


def lbm_batch_sync(h):
    _check(load_library().lbm_batch_sync(h), "lbm_batch_sync")


def lbm_batch_set_kernel(h, kernel: int, consumer_warps=0, cells_per_thread=0, stages=0, ctas_per_sm=0):
    _check(load_library().lbm_batch_set_kernel(h, int(kernel), int(consumer_warps), int(cells_per_thread),
                                               int(stages), int(ctas_per_sm)), "lbm_batch_set_kernel")


def lbm_batch_get_kernel(h) -> dict:
    out = np.zeros(6, np.int32)
    _check(load_library().lbm_batch_get_kernel(h, _p(out)), "lbm_batch_get_kernel")
    keys = ("kernel", "consumer_warps", "cells_per_thread", "stages", "ctas_per_sm", "grid")
    return dict(zip(keys, (int(v) for v in out)))


def lbm_batch_launch_count(h) -> int:
    c = ctypes.c_int64()
    _check(load_library().lbm_batch_launch_count(h, ctypes.byref(c)), "lbm_batch_launch_count")
    return int(c.value)


def lbm_batch_nodes(h):
    n = ctypes.c_int64()
    b = ctypes.c_double()
    _check(load_library().lbm_batch_nodes(h, ctypes.byref(n), ctypes.byref(b)), "lbm_batch_nodes")
    return int(n.value), float(b.value)


class Batch:
    """Independent cylinder lattices advanced by one kernel launch per step.

    ``cases`` is a list of ``workloads.Workload``.  Device memory is one
    torch uint8 tensor; all cases run on one torch stream.
    """

    def __init__(self, cases, storage=LBM_F32, kernel=LBM_KERNEL_AUTO, shape=None, ctas_per_sm=0,
                 graph_steps=0, history_capacity=1 << 16, stream=None, device=None, collision=LBM_COLLIDE_BGK,
                 mrt_rates=(1.1, 1.1, 1.1)):
        import torch

        load_library()
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.workloads = list(cases)
        self.masks = [np.ascontiguousarray(w.mask(), np.uint8) for w in self.workloads]
        self.cases = [dict(nx=w.nx, ny=w.ny, tau=w.tau, U=w.U, bc=w.bc, D_ref=float(w.D)) for w in self.workloads]
        o = lbm_opts_default()
        o.storage = int(storage)
        o.kernel = int(kernel)
        if shape is not None:
            o.consumer_warps, o.cells_per_thread, o.stages = (int(v) for v in shape)
        o.ctas_per_sm = int(ctas_per_sm)
        o.graph_steps = int(graph_steps)
        o.history_capacity = int(history_capacity)
        o.collision = int(collision)
        o.s_e, o.s_eps, o.s_q = (float(v) for v in mrt_rates)
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        nbytes = lbm_batch_workspace_bytes(self.cases, self.masks, o)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        o.workspace = ctypes.c_void_p(self.workspace.data_ptr())
        o.workspace_bytes = nbytes
        self.opts = o
        self.storage = int(storage)
        with torch.cuda.device(self.device):
            self.h = lbm_batch_create(self.cases, self.masks, o)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.cases)

    def init_fields(self, c, rho, u, v):
        lbm_batch_init_fields(self.h, c, rho, u, v)

    def init_all(self):
        for c, w in enumerate(self.workloads):
            self.init_fields(c, *w.initial_fields())

    def step(self, n: int):
        lbm_batch_step(self.h, n)

    def sync(self):
        lbm_batch_sync(self.h)

    def case(self, c):
        return lbm_batch_case(self.h, c)

    def case_status(self, c) -> int:
        """0, or the LBM_ERR_* code (e.g. LBM_ERR_UNSTABLE) case c reported."""
        return int(load_library().lbm_sync(self.case(c)))

    def forces_raw(self, c, first=0, n=None):
        ctx = self.case(c)
        if n is None:
            n = lbm_force_count(ctx) - first
        return lbm_forces_raw(ctx, first, n)

    def forces(self, c, first=0, n=None):
        ctx = self.case(c)
        if n is None:
            n = lbm_force_count(ctx) - first
        return lbm_forces(ctx, first, n)

    def fields(self, c, dtype=np.float64):
        w = self.cases[c]
        return lbm_fields(self.case(c), w["nx"], w["ny"], dtype)

    def get_populations(self, c):
        w = self.cases[c]
        return lbm_get_populations(self.case(c), w["nx"], w["ny"], self.storage)

    def set_kernel(self, kernel, consumer_warps=0, cells_per_thread=0, stages=0, ctas_per_sm=0):
        lbm_batch_set_kernel(self.h, kernel, consumer_warps, cells_per_thread, stages, ctas_per_sm)

    def kernel_info(self) -> dict:
        return lbm_batch_get_kernel(self.h)

    def launch_count(self) -> int:
        return lbm_batch_launch_count(self.h)

    def nodes(self):
        return lbm_batch_nodes(self.h)
