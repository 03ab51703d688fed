"""The multi-step kernel (LBM_KERNEL_TMA_WAVE) against the one-step TMA
kernel: the same bits in populations and force histories, whatever the
storage form, boundary rule, collision model, tiling (fewer tiles than CTAs,
a few more, many more; rows of one tile or several) or split of the steps
into launches; one run against the FP64 oracle; its failure path and its
argument checks."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_02185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_02185_gb300 import lbm  # noqa: E402

STORAGES = [lbm.LBM_F32, lbm.LBM_F16_OFS, lbm.LBM_BF16_OFS, lbm.LBM_F16_SR, lbm.LBM_BF16_SR, lbm.LBM_F64]
BCS = [W.BC_FREESLIP, W.BC_PERIODIC, W.BC_ZOUHE, W.BC_MOVINGWALL]


def run(wl, chunks, kernel, storage=lbm.LBM_F32, mrt=False, ctas=0):
    kw = dict(kernel=kernel, storage=storage, ctas_per_sm=ctas)
    if mrt:
        kw["collision"] = lbm.LBM_COLLIDE_MRT
    lat = lbm.lattice_for(wl, **kw)
    try:
        lat.init_fields(*wl.initial_fields())
        for n in chunks:
            lat.step(n)
        lat.sync()
        steps = sum(chunks)
        return lat.get_populations(), lat.forces_raw(0, steps + 1), lat.kernel_info(), lat.launch_count()
    finally:
        lat.close()


def same(a, b):
    assert a[0].shape == b[0].shape
    assert np.array_equal(a[0].view(np.uint8), b[0].view(np.uint8)), "populations differ"
    assert np.array_equal(a[1].view(np.uint8), b[1].view(np.uint8)), "force histories differ"


@pytest.mark.parametrize("storage", STORAGES, ids=["f32", "f16", "bf16", "f16sr", "bf16sr", "f64"])
@pytest.mark.parametrize("bc", BCS, ids=["freeslip", "periodic", "zouhe", "movingwall"])
def test_wave_bitwise_equals_one_step_kernel(storage, bc):
    # 401 x 77: 512-node (float, double) or 768-node (16-bit) tiles, one per
    # row: 77 CTAs of one tile each, so a tile of step s waits for tiles of
    # step s - 1 on other CTAs; 150 steps = launches of 64, 64, 22
    wl = W.random_case(401, 77, seed=3 + bc, bc=bc, D=12)
    mrt = (bc + storage) % 2 == 1
    ctas = 2 if lbm.ELEM_BYTES[storage] == 2 else 1
    ref = run(wl, [150], lbm.LBM_KERNEL_TMA, storage, mrt, ctas)
    got = run(wl, [150], lbm.LBM_KERNEL_TMA_WAVE, storage, mrt, ctas)
    assert got[2]["kernel"] == lbm.LBM_KERNEL_TMA_WAVE
    same(ref, got)


@pytest.mark.parametrize("bc", [W.BC_PERIODIC, W.BC_FREESLIP], ids=["periodic", "freeslip"])
def test_wave_uneven_tiling(bc):
    # 3000 x 50 with 768-node tiles: 4 tiles a row, 200 tiles on 152 CTAs, so
    # some CTAs run two tiles a step and others one, and a row's tiles sit on
    # several CTAs (periodic: rows 0 and 49 depend on each other); launches of
    # 1, 63, 64, 65 (= 64 + 1) and 7 steps
    wl = W.random_case(3000, 50, seed=11, bc=bc, D=14)
    chunks = [1, 63, 64, 65, 7]
    ref = run(wl, chunks, lbm.LBM_KERNEL_TMA)
    got = run(wl, chunks, lbm.LBM_KERNEL_TMA_WAVE)
    assert got[2]["grid"] == min(200, torch.cuda.get_device_properties(0).multi_processor_count)
    same(ref, got)


@pytest.mark.parametrize("shape", [(8, 2, 4), (12, 2, 4), (10, 2, 4), (13, 2, 3)])
def test_wave_many_tiles_per_cta_every_shape(shape):
    # 1601 x 900 (ragged last tile): thousands of tiles a step on 152 CTAs
    wl = W.random_case(1601, 900, seed=17, bc=W.BC_ZOUHE, D=40)
    ncw, cpt, st = shape
    a = lbm.lattice_for(wl, kernel=lbm.LBM_KERNEL_TMA)
    b = lbm.lattice_for(wl, kernel=lbm.LBM_KERNEL_TMA_WAVE, shape=shape, ctas_per_sm=1)
    try:
        for lat in (a, b):
            lat.init_fields(*wl.initial_fields())
            lat.step(97)
            lat.sync()
        info = b.kernel_info()
        assert (info["consumer_warps"], info["cells_per_thread"], info["stages"]) == shape
        same((a.get_populations(), a.forces_raw(0, 98)), (b.get_populations(), b.forces_raw(0, 98)))
    finally:
        a.close()
        b.close()


def test_wave_matches_oracle():
    wl = W.random_case(333, 61, seed=29, bc=W.BC_ZOUHE, D=10)
    steps = 200
    o = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
    o.init_equilibrium(*wl.initial_fields())
    Fo = o.run(steps)  # F(0 .. steps - 1)
    o.collide()
    Fo = np.vstack([Fo, o.force()[None, :]])
    fs_o = o.get_fs()  # f*(steps)
    pops, F, info, _ = run(wl, [steps], lbm.LBM_KERNEL_TMA_WAVE)
    f = pops.astype(np.float64) + O.feq(1.0, wl.U, 0.0)[:, None, None]
    fluid = wl.mask() == 0
    assert np.max(np.abs(f - fs_o)[:, fluid]) <= 1e-5 * wl.U
    for k in (0, 1):
        scale = np.max(np.abs(Fo[:, k]))
        assert np.max(np.abs(F[:, k] - Fo[:, k])) <= 1e-4 * scale


def test_wave_launch_count():
    wl = W.random_case(401, 77, seed=1, bc=W.BC_FREESLIP, D=12)
    n0 = run(wl, [0], lbm.LBM_KERNEL_TMA_WAVE)[3]
    n1 = run(wl, [150], lbm.LBM_KERNEL_TMA_WAVE)[3]
    assert n1 - n0 == 2 * 3  # three launches of the step kernel and its force reduction


def test_wave_timeout_then_recovers():
    wl = W.random_case(613, 57, seed=21, bc=W.BC_FREESLIP, D=10)
    want = run(wl, [70], lbm.LBM_KERNEL_TMA)[0]
    lat = lbm.lattice_for(wl, kernel=lbm.LBM_KERNEL_TMA_WAVE)
    try:
        lat.init_fields(*wl.initial_fields())
        lbm.lbm_set_fault_injection(lat.h, 7, 0.05)  # tile 7: announced, never copied; 50 ms waits
        lat.step(3)
        with pytest.raises(lbm.LBMError) as e:
            lat.sync()
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
        lbm.lbm_set_fault_injection(lat.h, -1, 0.0)
        lat.init_fields(*wl.initial_fields())
        lat.step(70)
        lat.sync()
        assert np.array_equal(lat.get_populations(), want)
    finally:
        lat.close()


def test_wave_rejects_shapes_it_is_not_built_for():
    wl = W.random_case(401, 77, seed=1, bc=W.BC_FREESLIP, D=12)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lattice_for(wl, kernel=lbm.LBM_KERNEL_TMA_WAVE, shape=(16, 2, 3))
    assert e.value.code == lbm.LBM_ERR_ARG
    lat = lbm.lattice_for(wl)
    try:
        with pytest.raises(lbm.LBMError):
            lat.set_kernel(lbm.LBM_KERNEL_TMA_WAVE, 16, 1, 6, 1)
        lat.set_kernel(lbm.LBM_KERNEL_TMA_WAVE, 13, 2, 3, 1)
        assert lat.kernel_info()["kernel"] == lbm.LBM_KERNEL_TMA_WAVE
    finally:
        lat.close()
