"""C ABI: the library loads and exports every entry point its header declares.

These run without a GPU: only host-side entry points (defaults, workspace
sizing, argument validation, strings) are called.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gblbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2605_02185_gb300 import _build, lbm
    _build.build()
    return lbm.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(lbm_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lbm_create", "lbm_step", "lbm_forces", "lbm_fields", "lbm_init_fields", "lbm_destroy"):
        assert n in names
    assert len(names) >= 20


def test_every_declared_symbol_is_exported(lib):
    from paper_2605_02185_gb300 import lbm
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_host_only_entry_points(lib):
    from paper_2605_02185_gb300 import lbm
    assert "sm_103a" in lbm.lbm_version()
    assert lbm.lbm_error_string(lbm.LBM_ERR_ARG) == "invalid argument or geometry"
    o = lbm.lbm_opts_default()
    assert o.storage == lbm.LBM_F32 and o.history_capacity == 1 << 20
    assert o.kernel == lbm.LBM_KERNEL_AUTO and o.ctas_per_sm == 0
    o.nx, o.ny, o.tau, o.U = 400, 200, 0.53, 0.1
    mask = np.zeros((200, 400), np.uint8)
    mask[95:106, 95:106] = 1
    b = lbm.lbm_workspace_bytes(o, mask)
    # two population buffers of 9 planes, rows padded to 64 nodes, float
    assert b >= 2 * 9 * 200 * 448 * 4
    o.storage = lbm.LBM_F16_OFS
    assert lbm.lbm_workspace_bytes(o, mask) < b
    # default kernel and shape by lattice size (host only)
    def default(nx, ny, **kw):
        q = lbm.lbm_opts_default()
        q.nx, q.ny, q.tau, q.U = nx, ny, 0.6, 0.05
        for k, v in kw.items():
            setattr(q, k, v)
        d = lbm.lbm_default_kernel(q)
        return d["kernel"], (d["consumer_warps"], d["cells_per_thread"], d["stages"]), d["ctas_per_sm"]
    T = lbm.LBM_KERNEL_TMA
    assert default(16000, 8000) == (T, (12, 2, 4), 1)
    assert default(8000, 4000) == (T, (12, 2, 4), 1)
    assert default(3200, 1600) == (T, (16, 1, 4), 2)
    assert default(1600, 800) == (T, (10, 2, 4), 2)
    assert default(3200, 1600, bounce=lbm.LBM_BOUNCE_INTERPOLATED, body_r=10.0, body_xc=400, body_yc=800) \
        == (T, (10, 2, 4), 1)
    assert default(3200, 1600, kernel=lbm.LBM_KERNEL_TMA_WAVE) == (lbm.LBM_KERNEL_TMA_WAVE, (10, 2, 4), 1)
    assert default(3200, 1600, storage=lbm.LBM_BF16_SR) == (T, (12, 2, 4), 2)
    assert default(3200, 1600, storage=lbm.LBM_F64)[0] == lbm.LBM_KERNEL_DIRECT
    assert default(3200, 1600, consumer_warps=13, cells_per_thread=2, stages=3) == (T, (13, 2, 3), 1)
    assert default(3200, 1600, ctas_per_sm=1) == (T, (16, 1, 4), 1)
    with pytest.raises(lbm.LBMError):
        default(3200, 1600, kernel=lbm.LBM_KERNEL_TMA_WAVE, consumer_warps=16, cells_per_thread=1, stages=6)
    # the multi-step kernel is built for four of the TMA kernel's shapes
    wave = lbm.lbm_kernel_shapes(lbm.LBM_KERNEL_TMA_WAVE)
    assert wave == [(8, 2, 4), (12, 2, 4), (10, 2, 4), (13, 2, 3)]
    assert set(wave) <= set(lbm.lbm_kernel_shapes(lbm.LBM_KERNEL_TMA))


@pytest.mark.parametrize("bad", [
    dict(nx=4), dict(ny=3), dict(tau=0.5), dict(tau=0.4), dict(U=0.35), dict(U=-0.1),
    dict(bc_top_bottom=4), dict(storage=7), dict(kernel=9), dict(bounce=2), dict(bounce=1, body_r=0.0),
])
def test_argument_validation(lib, bad):
    from paper_2605_02185_gb300 import lbm
    o = lbm.lbm_opts_default()
    o.nx, o.ny, o.tau, o.U = 40, 20, 0.6, 0.05
    for k, v in bad.items():
        setattr(o, k, v)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_workspace_bytes(o, None)
    assert e.value.code == lbm.LBM_ERR_ARG


@pytest.mark.parametrize("where", [(0, 10), (1, 10), (38, 10), (39, 10), (20, 0), (20, 1), (20, 18), (20, 19)])
def test_solid_margin_is_enforced(lib, where):
    from paper_2605_02185_gb300 import lbm
    o = lbm.lbm_opts_default()
    o.nx, o.ny, o.tau, o.U = 40, 20, 0.6, 0.05
    mask = np.zeros((20, 40), np.uint8)
    mask[where[1], where[0]] = 1
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_workspace_bytes(o, mask)
    assert e.value.code == lbm.LBM_ERR_ARG
    mask[:] = 0
    mask[2, 2] = mask[17, 37] = 1  # the allowed extremes
    assert lbm.lbm_workspace_bytes(o, mask) > 0


def test_missing_library_fails_loudly(tmp_path):
    from paper_2605_02185_gb300 import lbm
    with pytest.raises(ImportError):
        lbm.load_library(str(tmp_path / "nope.so"))


def test_every_network_symbol_is_exported(lib):
    from paper_2605_02185_gb300 import lbm
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "gbnn.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"^\s*int\s+(gbnn_\w+)\s*\(", src, flags=re.M)))
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(gbnn_\w+)", out))
    assert not [n for n in names if n not in exported]
