"""lbm_step_noalloc: one step on caller-owned device buffers, no allocation.

Some callers cannot allocate device memory (their memory comes from a pool
or arena they manage, or another runtime owns the allocator); this entry
point takes their input and output buffers and keeps its own scratch in a
fixed device array inside the library.  Its populations and forces must be
bit-identical to the ordinary entry point, lbm_step, on two calls in a row
(the second call reuses the scratch the first left behind): every step
kernel of the library runs the same per-node arithmetic and the same
fixed-order force reduction.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2605_02185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_02185_gb300 import lbm  # noqa: E402


def two_steps(wl, **kw):
    """f*(n0), f*(n0+1), f*(n0+2) and the forces of the last two, via lbm_step."""
    lat = lbm.lattice_for(wl, **kw)
    lat.init_fields(*wl.initial_fields())
    lat.step(3)
    lat.sync()
    h0 = lat.get_populations()
    n0 = lat.force_count()
    lat.step(1)
    lat.sync()
    h1 = lat.get_populations()
    lat.step(1)
    lat.sync()
    h2 = lat.get_populations()
    F = lat.forces_raw(n0, 2)
    return lat, h0, h1, h2, F


def noalloc_twice(lat, h0):
    dev = torch.device("cuda")
    a = torch.from_numpy(h0).to(dev)
    b = torch.empty_like(a)
    force = torch.zeros(2, 2, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    lbm.lbm_step_noalloc(lat.h, a.data_ptr(), b.data_ptr(), force[0].data_ptr())
    lbm.lbm_step_noalloc(lat.h, b.data_ptr(), a.data_ptr(), force[1].data_ptr())
    lat.sync()
    return b.cpu().numpy(), a.cpu().numpy(), force.cpu().numpy()


@pytest.mark.parametrize("kernel", [lbm.LBM_KERNEL_DIRECT, lbm.LBM_KERNEL_TMA], ids=["direct", "tma"])
def test_noalloc_step_matches_lbm_step_twice(kernel):
    wl = W.random_case(613, 57, seed=21, bc=W.BC_ZOUHE, D=10)
    lat, h0, h1, h2, F = two_steps(wl, kernel=kernel)
    try:
        got1, got2, got_force = noalloc_twice(lat, h0)
    finally:
        lat.close()
    assert np.array_equal(got1.view(np.uint8), h1.view(np.uint8))
    assert np.array_equal(got2.view(np.uint8), h2.view(np.uint8))
    assert np.array_equal(got_force, F)


def test_noalloc_16bit_and_mrt_bitwise():
    wl = W.random_case(300, 41, seed=22, bc=W.BC_MOVINGWALL, D=8, tau=0.56)
    lat, h0, h1, h2, F = two_steps(wl, storage=lbm.LBM_F16_OFS, collision=lbm.LBM_COLLIDE_MRT)
    try:
        got1, got2, got_force = noalloc_twice(lat, h0)
    finally:
        lat.close()
    assert np.array_equal(got1.view(np.uint8), h1.view(np.uint8))
    assert np.array_equal(got2.view(np.uint8), h2.view(np.uint8))
    assert np.array_equal(got_force, F)


def test_noalloc_rejections():
    dev = torch.device("cuda")
    wl = W.random_case(97, 33, seed=3, bc=W.BC_FREESLIP, D=8)
    lat = lbm.lattice_for(wl)
    try:
        a = torch.zeros(9 * wl.nx * wl.ny, dtype=torch.float32, device=dev)
        b = torch.zeros_like(a)
        force = torch.zeros(2, dtype=torch.float64, device=dev)
        for args in ((a.data_ptr(), a.data_ptr(), force.data_ptr()),   # in place
                     (0, b.data_ptr(), force.data_ptr()), (a.data_ptr(), 0, force.data_ptr()),
                     (a.data_ptr(), b.data_ptr(), 0)):
            with pytest.raises(lbm.LBMError) as e:
                lbm.lbm_step_noalloc(lat.h, *args)
            assert e.value.code == lbm.LBM_ERR_ARG
    finally:
        lat.close()
    # interpolated bounce-back: the step's force needs the next step
    lat = lbm.lattice_for(wl, bounce=lbm.LBM_BOUNCE_INTERPOLATED)
    try:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_step_noalloc(lat.h, a.data_ptr(), b.data_ptr(), force.data_ptr())
        assert e.value.code == lbm.LBM_ERR_ARG
    finally:
        lat.close()


def test_noalloc_rejects_a_body_beyond_the_fixed_scratch():
    # two small bodies at opposite corners: the link-owning bounding box
    # spans 226 rows x 300 tiles of 256 nodes = 67,800 > 65,520 force slots
    nx, ny = 300 * 256, 240
    mask = np.zeros((ny, nx), np.uint8)
    mask[8:12, 8:12] = 1
    mask[ny - 12:ny - 8, nx - 12:nx - 8] = 1
    lat = lbm.Lattice(nx, ny, 0.6, 0.05, mask=mask, bc=lbm.LBM_BC_FREESLIP, D_ref=4.0)
    try:
        # buffers of the full size, so that nothing is out of bounds even if
        # the size check let the call through
        a = torch.zeros(9 * nx * ny, dtype=torch.float32, device="cuda")
        b = torch.zeros_like(a)
        force = torch.zeros(2, dtype=torch.float64, device="cuda")
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_step_noalloc(lat.h, a.data_ptr(), b.data_ptr(), force.data_ptr())
        assert e.value.code == lbm.LBM_ERR_ARG
    finally:
        lat.close()
