"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances.  The CUDA path stores post-collision offsets g = f - w and does
float arithmetic (FP32 storage); the oracle is double.  One step rounds each
stored offset (|g| <~ 0.05) to float, a relative 2^-24, i.e. <~ 3e-9 absolute,
and the collision adds a few such roundings.  Over n steps these errors
accumulate roughly like a random walk and are carried by the flow, so after
n <= 2000 steps velocity errors stay well below 1e-5 U, the tolerance the
small cylinder case is held to (max |u - u_ref| <= 1e-5 U after 2000 steps).
Populations are compared with the same absolute bound; force histories with
a relative bound of 1e-4 per entry.
"""
import functools
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_02185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_02185_gb300 import lbm  # noqa: E402



def reference_pops(U):
    """r_i = f_eq_i(1, (U, 0)): the library stores f* - r."""
    return O.feq(1.0, U, 0.0)


@functools.lru_cache(maxsize=64)
def oracle_run(wl: W.Workload, steps: int, mrt: bool = False):
    """Oracle after `steps` steps: f*(steps), forces F(0..steps), fields of f(steps)."""
    o = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
    if mrt:
        o.set_collision(O.MRT, *O.MRT_PAPER_RATES)
    o.init_equilibrium(*wl.initial_fields())
    F = o.run(steps)
    fields = o.fields()
    o.collide()
    Fn = o.force()
    fs = o.get_fs()
    return fs, np.vstack([F, Fn[None, :]]), fields


def gpu_run(wl, steps, **kw):
    lat = lbm.lattice_for(wl, **kw)
    try:
        lat.init_fields(*wl.initial_fields())
        lat.step(steps)
        lat.sync()
        pops = lat.get_populations()
        F = lat.forces_raw(0, steps + 1)
        fields = lat.fields()
        info = lat.kernel_info()
    finally:
        lat.close()
    return pops, F, fields, info


def offsets_to_f(pops, U, storage=lbm.LBM_F32):
    if storage in (lbm.LBM_BF16_OFS, lbm.LBM_BF16_SR):
        g = (pops.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    elif storage in (lbm.LBM_F16_OFS, lbm.LBM_F16_SR):
        g = pops.astype(np.float64) / 4096.0  # IEEE half holds 2^12 x the offset
    else:
        g = pops.astype(np.float64)
    return g + reference_pops(U)[:, None, None]


def force_errors(F, Fo):
    """Drag and lift checked each in its own terms: max over the history of
    |F_k(n) - Fo_k(n)| relative to max |Fo_k| of that component (k = x, y)."""
    return tuple(float(np.max(np.abs(F[:, k] - Fo[:, k])) / max(np.max(np.abs(Fo[:, k])), 1e-300)) for k in (0, 1))


def compare(wl, steps, pops, F, fields, tol_f, tol_F, storage=lbm.LBM_F32, mrt=False, tol_Fy=None):
    """Every fluid node's populations, velocity and density, and every force
    entry (drag to tol_F of the drag scale, lift to tol_Fy -- default tol_F --
    of the lift scale), against the oracle."""
    fs, Fo, (ro, uo, vo) = oracle_run(wl, steps, mrt)
    f = offsets_to_f(pops, wl.U, storage)
    fluid = wl.mask() == 0
    df = np.max(np.abs(f - fs)[:, fluid])
    r, u, v = fields
    du = max(np.max(np.abs(u - uo)[fluid]), np.max(np.abs(v - vo)[fluid]))
    dr = np.max(np.abs(r - ro)[fluid])
    dFx, dFy = force_errors(F, Fo)
    tol_Fy = tol_F if tol_Fy is None else tol_Fy
    assert df <= tol_f, f"populations differ by {df:.3e}"
    assert du <= tol_f, f"velocity differs by {du:.3e}"
    assert dr <= 3 * tol_f, f"density differs by {dr:.3e}"
    assert dFx <= tol_F, f"drag differs by {dFx:.3e} of its scale"
    assert dFy <= tol_Fy, f"lift differs by {dFy:.3e} of its scale (max |Fy| = {np.max(np.abs(Fo[:, 1])):.3e})"
    return df, du, dFx, dFy


KERNELS = [("direct", dict(kernel=lbm.LBM_KERNEL_DIRECT)), ("tma", dict(kernel=lbm.LBM_KERNEL_TMA))]
BCS = [W.BC_FREESLIP, W.BC_PERIODIC, W.BC_ZOUHE, W.BC_MOVINGWALL]


@pytest.mark.parametrize("kname,kw", KERNELS, ids=[k[0] for k in KERNELS])
@pytest.mark.parametrize("bc", BCS, ids=[W.BC_NAMES[b] for b in BCS])
@pytest.mark.parametrize("size", [(37, 23), (300, 41)], ids=["37x23", "300x41"])
def test_small_lattices_match_oracle(kname, kw, bc, size):
    wl = W.random_case(size[0], size[1], seed=100 + size[0] + bc, bc=bc, D=6)
    pops, F, fields, _ = gpu_run(wl, 60, **kw)
    compare(wl, 60, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4)


@pytest.mark.parametrize("nx", [257, 513, 1025])
@pytest.mark.parametrize("shape", [(8, 1, 8), (8, 2, 6), (8, 4, 4)], ids=["w256", "w512", "w1024"])
def test_outlet_alone_at_tile_start(nx, shape):
    # nx - 1 is a multiple of the tile width: the outlet column starts a tile
    wl = W.random_case(nx, 31, seed=7, bc=W.BC_ZOUHE, D=8)
    pops, F, fields, info = gpu_run(wl, 40, kernel=lbm.LBM_KERNEL_TMA, shape=shape)
    assert (info["consumer_warps"], info["cells_per_thread"], info["stages"]) == shape
    compare(wl, 40, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4)


PARITY_HORIZON = 1000


def test_parity_small_cylinder():
    """Re = 100, D = 10, 400 x 200, U = 0.1, tau = 0.53, free-slip.

    With BGK at tau = 0.53 and the Zou-He inlet this case is not stable: the
    FP64 oracle itself leaves the physical range near step 1900 and
    overflows by step 2000 (an inlet-column mode seeded by the velocity
    perturbation; the paper warns about tau near 1/2 with U near 0.1 and
    switches to MRT, Section 3.1).  Parity is therefore checked at step
    1000, before the mode has grown, with the 1e-5 U tolerance.
    """
    wl = W.PARITY_D10
    n = PARITY_HORIZON
    pops, F, fields, _ = gpu_run(wl, n)
    compare(wl, n, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4)
    q = 0.5 * wl.U ** 2 * wl.D  # Eq. 15 denominator
    _, Fo, _ = oracle_run(wl, n)
    cd, cdo = F[:, 0] / q, Fo[:, 0] / q
    assert np.max(np.abs(cd - cdo)) <= 1e-4 * np.max(np.abs(cdo))


def test_parity_small_cylinder_stable_tau_2000_steps():
    """The same geometry and inlet speed at tau = 0.55, where the run stays
    bounded: 2000 steps within max |u - u_ref| <= 1e-5 U."""
    import dataclasses
    wl = dataclasses.replace(W.PARITY_D10, tau=0.55, name="cyl_D10_400x200_tau055")
    pops, F, fields, _ = gpu_run(wl, 2000)
    compare(wl, 2000, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4)


# Steps of the production-case trajectory check; the full 20k-step record
# is taken with GBLBM_PRODUCTION_STEPS=20000 (about 10 minutes of oracle time
# per top/bottom rule on 16 host cores).
PRODUCTION_STEPS = int(os.environ.get("GBLBM_PRODUCTION_STEPS", "3000"))
# Before shedding the lift is the small response to the seeded perturbation;
# it is held to the same relative bound as the drag.
PRODUCTION_TOL_FY = {lbm.LBM_F32: 1e-4, lbm.LBM_F64: 1e-10}


# FP64 storage: the GPU's double arithmetic on offsets and the oracle's on
# the populations themselves (|f| up to 0.44, so its own rounding steps are
# ~10x larger) drift apart like two double-precision runs of the same
# unstable wake; measured 2.4e-12 U after 3000 steps.
@pytest.mark.slow
@pytest.mark.parametrize("storage,tol,tol_F", [(lbm.LBM_F32, 1e-5, 1e-4), (lbm.LBM_F64, 1e-11, 1e-10)],
                         ids=["f32", "f64"])
@pytest.mark.parametrize("bc", [W.BC_FREESLIP, W.BC_ZOUHE], ids=["freeslip", "zouhe"])
def test_production_case_matches_oracle_every_node(bc, storage, tol, tol_F):
    """The 3200 x 1600 production case (Re = 100, D = 80, U = 0.05,
    tau = 0.62, seeded perturbation) with free-slip and with Zou-He
    top/bottom walls: after PRODUCTION_STEPS steps every node within
    1e-5 U (FP32) or 1e-12 U (FP64 storage) of the oracle, and every drag and
    lift entry within its tolerance of the oracle's."""
    wl = W.PRODUCTION_D80.with_bc(bc)
    n = PRODUCTION_STEPS
    pops, F, fields, _ = gpu_run(wl, n, storage=storage)
    fs, Fo, (ro, uo, vo) = oracle_run(wl, n, False)
    fluid = wl.mask() == 0
    r, u, v = fields
    df = np.max(np.abs(offsets_to_f(pops, wl.U, storage) - fs)[:, fluid])
    du = max(np.max(np.abs(u - uo)[fluid]), np.max(np.abs(v - vo)[fluid]))
    dFx, dFy = force_errors(F, Fo)
    print(f"production {W.BC_NAMES[bc]} storage {storage} {n} steps: max|f-f_ref| {df / wl.U:.2e} U, "
          f"max|u-u_ref| {du / wl.U:.2e} U, drag {dFx:.2e}, lift {dFy:.2e} of their scales")
    compare(wl, n, pops, F, fields, tol_f=tol * wl.U, tol_F=tol_F, storage=storage,
            tol_Fy=PRODUCTION_TOL_FY[storage])


@pytest.mark.parametrize("with_noneq", [False, True], ids=["equilibrium", "with_noneq"])
def test_device_init_matches_oracle(with_noneq):
    """lbm_init_fields_device: f(0) = f_eq(rho, u) [+ the Chapman-Enskog
    f_neq(grad u) of the oracle], stored as its collision
    f*(0) = f_eq + (1 - 1/tau) f_neq; FP64 storage, fluid nodes."""
    from oracle import conv_oracle as C
    wl = W.random_case(67, 37, seed=13, bc=W.BC_FREESLIP, D=8, tau=0.56)
    yy, xx = np.mgrid[0:wl.ny, 0:wl.nx].astype(np.float64)
    rho = (1.0 + 0.01 * np.sin(0.21 * xx) * np.cos(0.17 * yy)).astype(np.float32)
    u = (wl.U * (1.0 + 0.3 * np.sin(0.13 * yy + 0.05 * xx))).astype(np.float32)
    v = (0.02 * np.cos(0.11 * xx - 0.07 * yy)).astype(np.float32)
    solid = wl.mask().astype(bool)
    u[solid] = 0.0
    v[solid] = 0.0
    lat = lbm.lattice_for(wl, storage=lbm.LBM_F64)
    try:
        dev = [torch.from_numpy(a).cuda() for a in (rho, u, v)]
        lbm.lbm_init_fields_device(lat.h, *(t.data_ptr() for t in dev), with_noneq)
        lat.sync()
        pops = lat.get_populations()
    finally:
        lat.close()
    o = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
    o.init_equilibrium(rho.astype(np.float64), u.astype(np.float64), v.astype(np.float64))
    want = o.get_f()
    if with_noneq:
        want = want + (1.0 - 1.0 / wl.tau) * C.noneq_populations(rho.astype(np.float64), u.astype(np.float64),
                                                                  v.astype(np.float64), wl.tau, solid)
    got = offsets_to_f(pops, wl.U, lbm.LBM_F64)
    assert np.max(np.abs(got - want)[:, ~solid]) <= 1e-13


def test_unstable_case_is_flagged_like_the_oracle():
    """Past its stable span the small cylinder case diverges on both sides;
    the GPU path reports it through lbm_sync instead of returning garbage."""
    wl = W.PARITY_D10
    lat = lbm.lattice_for(wl)
    lat.init_fields(*wl.initial_fields())
    lat.step(2000)
    with pytest.raises(lbm.LBMError) as e:
        lat.sync()
    assert e.value.code == lbm.LBM_ERR_UNSTABLE
    lat.close()
    o = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
    o.init_equilibrium(*wl.initial_fields())
    o.run(2000)
    _, u, v = o.fields()
    with np.errstate(invalid="ignore", over="ignore"):
        assert not np.all(np.sqrt(u * u + v * v) <= 0.3)


MRT = dict(collision=lbm.LBM_COLLIDE_MRT, mrt_rates=O.MRT_PAPER_RATES)


@pytest.mark.parametrize("kname,kw", KERNELS, ids=[k[0] for k in KERNELS])
@pytest.mark.parametrize("bc", BCS, ids=[W.BC_NAMES[b] for b in BCS])
def test_mrt_small_lattices_match_oracle(kname, kw, bc):
    """The paper's MRT collision (Eq. 6, S = diag[1, 1.1, 1.1, 1, 1.1, 1, 1.1, 1/tau, 1/tau])."""
    wl = W.random_case(300, 41, seed=500 + bc, bc=bc, D=8, tau=0.56)
    pops, F, fields, _ = gpu_run(wl, 60, **kw, **MRT)
    compare(wl, 60, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4, mrt=True)


def test_mrt_parity_small_cylinder_2000_steps():
    """Re = 100, D = 10, 400 x 200, U = 0.1, tau = 0.53, free-slip, 2000 steps
    with the paper's MRT collision, which keeps this case stable: max |u - u_ref|
    <= 1e-5 U and Cd within 1e-4 of the oracle at every step."""
    wl = W.PARITY_D10
    pops, F, fields, _ = gpu_run(wl, wl.steps, **MRT)
    compare(wl, wl.steps, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4, mrt=True)
    q = 0.5 * wl.U ** 2 * wl.D
    _, Fo, _ = oracle_run(wl, wl.steps, True)
    assert np.max(np.abs(F[:, 0] - Fo[:, 0]) / q) <= 1e-4 * np.max(np.abs(Fo[:, 0]) / q)


def test_moving_walls_small_cylinder_mrt():
    """The C1 geometry (Re = 100, D = 10, 400 x 200, U = 0.1, tau = 0.53) with
    constant-velocity bounce-back top and bottom (Eq. 11) and the paper's MRT
    collision: 1000 steps within max |u - u_ref| <= 1e-5 U."""
    import dataclasses
    wl = dataclasses.replace(W.PARITY_D10, bc=W.BC_MOVINGWALL, name="cyl_D10_400x200_movingwall")
    pops, F, fields, _ = gpu_run(wl, 1000, **MRT)
    compare(wl, 1000, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4, mrt=True)


def test_paper_setup_mrt_tau_0512_matches_oracle():
    """The paper's own setup (Section 3.1): D = 20, 800 x 400, U = 0.02,
    Re = 100, so tau = 0.512 (Eqs. 16-17), with its MRT collision (Eq. 6),
    free-slip walls; 2000 steps, every node within 1e-5 U."""
    wl = W.cylinder_case(20, 0.02, 100.0, seed=6, perturb=1e-3, name="cyl_Re100_D20_paper")
    assert abs(wl.tau - 0.512) < 1e-12
    pops, F, fields, _ = gpu_run(wl, 2000, **MRT)
    compare(wl, 2000, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4, mrt=True)


# A case that sheds within a few ten thousand steps, cheap enough for the
# oracle: D = 10, 400 x 200, U = 0.05, Re = 80 (tau = 0.51875), MRT, started
# with a +-0.1 U kick; the lift reaches a limit cycle of amplitude ~0.34
# with a period of ~1300 steps.
SHEDDING_D10 = W.cylinder_case(10, 0.05, 80.0, seed=31, perturb=0.1, name="cyl_Re80_D10_shedding")
SHEDDING_STEPS = 30000
SHEDDING_TOL_F = 1e-3  # per entry, relative to each component's scale


def test_shedding_lift_and_statistics_match_oracle():
    """Drag and lift of a shedding cylinder, each entry against the oracle's
    in its own scale, and mean Cd, Cl amplitude and Strouhal number over the
    last four periods within 0.5 % of the oracle's (the criterion for the
    production statistics)."""
    from paper_2605_02185_gb300 import postprocess
    wl = SHEDDING_D10
    n = SHEDDING_STEPS
    pops, F, fields, _ = gpu_run(wl, n, **MRT)
    _, Fo, _ = oracle_run(wl, n, True)
    q = 0.5 * wl.U ** 2 * wl.D
    cl_amp = 0.5 * (np.max(Fo[-5000:, 1]) - np.min(Fo[-5000:, 1])) / q
    assert cl_amp > 0.2, cl_amp  # the oracle run does shed
    dFx, dFy = force_errors(F, Fo)
    st, sto = (postprocess.statistics(X[:, 0] / q, X[:, 1] / q, wl.D, wl.U, periods=4) for X in (F, Fo))
    rel = {k: abs(st[k] - sto[k]) / abs(sto[k]) for k in ("cd_mean", "cl_amp", "st")}
    print(f"shedding: drag {dFx:.2e}, lift {dFy:.2e} of scale; statistics {rel}")
    assert dFx <= SHEDDING_TOL_F and dFy <= SHEDDING_TOL_F, (dFx, dFy)
    assert all(v <= 0.005 for v in rel.values()), rel


@pytest.mark.parametrize("storage", [lbm.LBM_F16_OFS, lbm.LBM_BF16_OFS, lbm.LBM_F16_SR, lbm.LBM_BF16_SR],
                         ids=["f16", "bf16", "f16sr", "bf16sr"])
@pytest.mark.parametrize("mrt", [False, True], ids=["bgk", "mrt"])
def test_paired_16bit_tma_matches_direct(storage, mrt):
    """The 16-bit TMA kernel updates plain spans two adjacent nodes at a time
    with packed FP32 instructions and 32-bit loads and stores; every node must
    still get the bits of the one-node path of the direct kernel."""
    wl = W.random_case(613, 57, seed=23, bc=W.BC_MOVINGWALL if mrt else W.BC_FREESLIP, D=10)
    kw = dict(storage=storage, **(MRT if mrt else {}))
    ref, Fr, _, _ = gpu_run(wl, 30, kernel=lbm.LBM_KERNEL_DIRECT, **kw)
    for shape in lbm.lbm_kernel_shapes():
        pops, F, _, info = gpu_run(wl, 30, kernel=lbm.LBM_KERNEL_TMA, shape=shape, **kw)
        assert (info["consumer_warps"], info["cells_per_thread"], info["stages"]) == shape
        assert np.array_equal(pops, ref), shape
        assert np.array_equal(F, Fr), shape


# ------------------------------------------------ interpolated bounce-back

INTERP = dict(bounce=lbm.LBM_BOUNCE_INTERPOLATED)


@functools.lru_cache(maxsize=16)
def oracle_run_interpolated(wl: W.Workload, steps: int, mrt: bool = False):
    """Oracle with interpolated bounce-back on the workload's circle: f*(steps),
    forces F(0..steps-1) (each needs the next step's returning populations),
    fields of f(steps)."""
    o = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
    if mrt:
        o.set_collision(O.MRT, *O.MRT_PAPER_RATES)
    o.set_circle_q(wl.xc, wl.yc, wl.D / 2)
    o.init_equilibrium(*wl.initial_fields())
    F = o.run(steps)
    fields = o.fields()
    o.collide()
    return o.get_fs(), F, fields


def gpu_run_interpolated(wl, steps, **kw):
    lat = lbm.lattice_for(wl, **INTERP, **kw)
    try:
        lat.init_fields(*wl.initial_fields())
        assert lat.force_count() == 0
        lat.step(steps)
        lat.sync()
        assert lat.force_count() == steps
        pops, F, fields = lat.get_populations(), lat.forces_raw(0, steps), lat.fields()
    finally:
        lat.close()
    return pops, F, fields


def compare_interpolated(wl, steps, pops, F, fields, tol_f, tol_F, storage=lbm.LBM_F32, mrt=False):
    fs, Fo, (ro, uo, vo) = oracle_run_interpolated(wl, steps, mrt)
    fluid = wl.mask() == 0
    f = offsets_to_f(pops, wl.U, storage)
    r, u, v = fields
    assert np.max(np.abs(f - fs)[:, fluid]) <= tol_f
    assert max(np.max(np.abs(u - uo)[fluid]), np.max(np.abs(v - vo)[fluid])) <= tol_f
    assert np.max(np.abs(r - ro)[fluid]) <= 3 * tol_f
    dFx, dFy = force_errors(F, Fo)
    assert dFx <= tol_F and dFy <= tol_F, (dFx, dFy)


@pytest.mark.parametrize("size", [(37, 23), (300, 41)], ids=["37x23", "300x41"])
def test_interpolated_bounce_back_matches_oracle(size):
    """Bouzidi linear bounce-back with the circle's link fractions, and its
    two-sided momentum exchange (history entry n written by step n + 1)."""
    wl = W.random_case(size[0], size[1], seed=700 + size[0], bc=W.BC_FREESLIP, D=8)
    pops, F, fields = gpu_run_interpolated(wl, 60)
    compare_interpolated(wl, 60, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4)


def test_interpolated_bounce_back_16bit_and_mrt():
    wl = W.random_case(300, 41, seed=711, bc=W.BC_ZOUHE, D=8, tau=0.56)
    pops, F, fields = gpu_run_interpolated(wl, 60, **MRT)
    compare_interpolated(wl, 60, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4, mrt=True)
    pops, F, fields = gpu_run_interpolated(wl, 60, storage=lbm.LBM_F16_OFS, **MRT)
    compare_interpolated(wl, 60, pops, F, fields, tol_f=2e-3 * wl.U, tol_F=2e-2, storage=lbm.LBM_F16_OFS,
                         mrt=True)


def test_interpolated_small_cylinder_mrt():
    """The C1 geometry with interpolated bounce-back and the paper's MRT:
    1000 steps within max |u - u_ref| <= 1e-5 U, every force entry within
    1e-4 of the oracle's."""
    wl = W.PARITY_D10
    pops, F, fields = gpu_run_interpolated(wl, 1000, **MRT)
    compare_interpolated(wl, 1000, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4, mrt=True)


def test_interpolated_bounce_back_kernel_choice():
    """Float storage: the TMA kernel in its default shapes; 16-bit storage
    and other shapes: the direct kernel."""
    wl = W.random_case(97, 33, seed=3, bc=W.BC_FREESLIP, D=8)
    for kw, want in ((dict(kernel=lbm.LBM_KERNEL_TMA), lbm.LBM_KERNEL_TMA),
                     (dict(kernel=lbm.LBM_KERNEL_TMA, storage=lbm.LBM_F16_OFS), lbm.LBM_KERNEL_DIRECT),
                     (dict(kernel=lbm.LBM_KERNEL_TMA, shape=(16, 2, 2)), lbm.LBM_KERNEL_DIRECT)):
        lat = lbm.lattice_for(wl, **INTERP, **kw)
        try:
            assert lat.kernel_info()["kernel"] == want, kw
        finally:
            lat.close()


@pytest.mark.parametrize("mrt", [False, True], ids=["bgk", "mrt"])
def test_interpolated_tma_kernel_matches_direct(mrt):
    """Interpolated bounce-back on the TMA kernel: the same per-node
    arithmetic as the direct kernel, identical bits, in each shape it is
    built for, with the link-owning rows spread over several row tiles."""
    wl = W.random_case(1025, 61, seed=12, bc=W.BC_ZOUHE, D=24)
    coll = MRT if mrt else {}
    kw = dict(**INTERP, **coll)
    ref, Fr, _ = gpu_run_interpolated(wl, 30, kernel=lbm.LBM_KERNEL_DIRECT, **coll)
    for shape in [(12, 2, 4), (10, 2, 4), (8, 2, 4)]:
        lat = lbm.lattice_for(wl, kernel=lbm.LBM_KERNEL_TMA, shape=shape, **kw)
        try:
            assert lat.kernel_info()["kernel"] == lbm.LBM_KERNEL_TMA
            lat.init_fields(*wl.initial_fields())
            lat.step(30)
            lat.sync()
            assert np.array_equal(lat.get_populations(), ref), shape
            assert np.array_equal(lat.forces_raw(0, 30), Fr), shape
        finally:
            lat.close()


def test_every_tma_shape_matches_direct():
    wl = W.random_case(613, 57, seed=21, bc=W.BC_FREESLIP, D=10)
    ref, Fr, _, _ = gpu_run(wl, 30, kernel=lbm.LBM_KERNEL_DIRECT)
    shapes = lbm.lbm_kernel_shapes()
    assert len(shapes) >= 10
    for shape in shapes:
        for ctas in (1, 2):
            pops, F, _, info = gpu_run(wl, 30, kernel=lbm.LBM_KERNEL_TMA, shape=shape, ctas_per_sm=ctas)
            assert (info["consumer_warps"], info["cells_per_thread"], info["stages"]) == shape
            # same per-node arithmetic, different staging: identical bits
            assert np.array_equal(pops, ref), (shape, ctas)
            assert np.array_equal(F, Fr), (shape, ctas)


def test_bitwise_deterministic_and_graph_independent():
    wl = W.random_case(401, 77, seed=5, bc=W.BC_PERIODIC, D=12)
    a = gpu_run(wl, 50, graph_steps=0)
    b = gpu_run(wl, 50, graph_steps=-1)
    c = gpu_run(wl, 50, graph_steps=8)
    for x in (b, c):
        assert np.array_equal(a[0], x[0])
        assert np.array_equal(a[1], x[1])


def test_checkpoint_resume_is_bitwise():
    wl = W.random_case(301, 61, seed=9, bc=W.BC_ZOUHE, D=10)
    full = gpu_run(wl, 40)
    lat = lbm.lattice_for(wl)
    lat.init_fields(*wl.initial_fields())
    lat.step(17)
    ck = lat.get_populations()
    n = lat.force_count()
    lat.close()
    lat2 = lbm.lattice_for(wl)
    lat2.set_populations(ck, n)
    lat2.step(23)
    lat2.sync()
    assert np.array_equal(lat2.get_populations(), full[0])
    assert np.array_equal(lat2.forces_raw(n, 23), full[1][n:])
    lat2.close()


def test_window_readback_matches_full():
    wl = W.random_case(333, 45, seed=2, bc=W.BC_FREESLIP, D=8)
    lat = lbm.lattice_for(wl)
    lat.init_fields(*wl.initial_fields())
    lat.step(5)
    full = lat.get_populations()
    win = lat.get_window(100, 7, 70, 20)
    lat.close()
    assert np.array_equal(win, full[:, 7:27, 100:170])


def test_mass_matches_oracle():
    wl = W.random_case(121, 47, seed=4, bc=W.BC_PERIODIC, D=8)
    lat = lbm.lattice_for(wl)
    lat.init_fields(*wl.initial_fields())
    lat.step(25)
    m = lat.mass()
    lat.close()
    fs, _, _ = oracle_run(wl, 25)
    fluid = wl.mask() == 0
    assert abs(m - fs[:, fluid].sum()) <= 1e-7 * fluid.sum()


def test_uniform_stream_stays_uniform_on_gpu():
    for bc in BCS:
        lat = lbm.Lattice(130, 40, 0.7, 0.08, mask=None, bc=bc, D_ref=10.0)
        lat.init_fields(np.ones((40, 130)), np.full((40, 130), 0.08), np.zeros((40, 130)))
        lat.step(500)
        lat.sync()
        r, u, v = lat.fields()
        F = lat.forces_raw()
        lat.close()
        assert np.max(np.abs(u - 0.08)) < 1e-6 and np.max(np.abs(v)) < 1e-6 and np.max(np.abs(r - 1)) < 1e-6
        assert np.all(F == 0.0) and len(F) == 501


def test_force_history_ring():
    wl = W.random_case(97, 33, seed=3, bc=W.BC_FREESLIP, D=8)
    big = gpu_run(wl, 40)[1]
    lat = lbm.lattice_for(wl, history_capacity=16)
    lat.init_fields(*wl.initial_fields())
    lat.step(40)
    assert lat.force_count() == 41
    assert np.array_equal(lat.forces_raw(25, 16), big[25:41])
    with pytest.raises(lbm.LBMError) as e:
        lat.forces_raw(24, 2)
    assert e.value.code == lbm.LBM_ERR_RANGE
    with pytest.raises(lbm.LBMError) as e:
        lat.forces_raw(40, 2)
    assert e.value.code == lbm.LBM_ERR_RANGE
    cd, cl = lat.forces(30, 5)
    q = 0.5 * wl.U ** 2 * wl.D
    np.testing.assert_allclose(cd, big[30:35, 0] / q, rtol=1e-15)
    np.testing.assert_allclose(cl, big[30:35, 1] / q, rtol=1e-15)
    lat.close()


def test_step_before_init_is_refused():
    wl = W.random_case(40, 20, seed=1, bc=W.BC_FREESLIP, D=4)
    lat = lbm.lattice_for(wl)
    with pytest.raises(lbm.LBMError) as e:
        lat.step(1)
    assert e.value.code == lbm.LBM_ERR_STATE
    lat.close()


def test_instability_is_reported():
    # a node started at |u| = 0.35 trips the |u| > 0.3 check of the first step
    wl = W.random_case(64, 32, seed=1, bc=W.BC_FREESLIP, D=6)
    lat = lbm.lattice_for(wl)
    r, u, v = wl.initial_fields()
    u[5:12, 5:12] = 0.35
    lat.init_fields(r, u, v)
    lat.step(1)
    with pytest.raises(lbm.LBMError) as e:
        lat.sync()
    assert e.value.code == lbm.LBM_ERR_UNSTABLE
    lat.close()


# measured on 300 x 41, 60 steps: populations f16 8.5e-4 U, bf16 8.2e-3 U,
# f64 1.4e-14 U; drag 1e-4 / 1e-3 of its scale; lift (max |Fy| ~0.1 of
# max |Fx| here) 3.1e-3 / 3.6e-2 of its own scale -- the 16-bit rounding of
# the stored offsets, not an error of the arithmetic
# Stochastic rounding moves a value by up to one 16-bit step instead of half
# of one: twice the round-to-nearest tolerances.
STORAGE = [(lbm.LBM_F16_OFS, 2e-3, 2e-4, 1e-2), (lbm.LBM_BF16_OFS, 2e-2, 2e-3, 1e-1),
           (lbm.LBM_F64, 1e-12, 1e-12, 1e-12), (lbm.LBM_F16_SR, 4e-3, 4e-4, 2e-2),
           (lbm.LBM_BF16_SR, 4e-2, 4e-3, 2e-1)]


@pytest.mark.parametrize("storage,tol,tol_F,tol_Fy", STORAGE, ids=["f16", "bf16", "f64", "f16sr", "bf16sr"])
@pytest.mark.parametrize("kname,kw", KERNELS, ids=[k[0] for k in KERNELS])
def test_storage_forms_match_oracle(storage, tol, tol_F, tol_Fy, kname, kw):
    wl = W.random_case(300, 41, seed=33, bc=W.BC_FREESLIP, D=8)
    pops, F, fields, _ = gpu_run(wl, 60, storage=storage, **kw)
    compare(wl, 60, pops, F, fields, tol_f=tol * wl.U, tol_F=tol_F, storage=storage, tol_Fy=tol_Fy)


def test_full_size_lattice_sampled_windows():
    """The 16000 x 8000 throughput lattice in the benchmark's launch shape,
    checked on sampled windows.  After s steps a node depends only on the
    initial state within s nodes, so the oracle run on a crop that adds
    s + 2 nodes around a window (real boundaries kept where the window
    touches them) reproduces the full lattice inside the window exactly.
    The cylinder window holds every link, so the force history is compared
    too."""
    wl = W.THROUGHPUT_D400
    s, m = 3, 5
    nx, ny = wl.nx, wl.ny
    rho, u, v = wl.initial_fields()
    mask = wl.mask()
    lat = lbm.lattice_for(wl)
    lat.init_fields(rho, u, v)
    lat.step(s)
    lat.sync()
    F = lat.forces_raw(0, s + 1)
    r = wl.D // 2
    windows = [
        ("inlet-bottom", 0, 0, 48, 24), ("inlet-top", 0, ny - 24, 48, 24),
        ("outlet-bottom", nx - 48, 0, 48, 24), ("outlet-top", nx - 48, ny - 24, 48, 24),
        ("bottom-row", 8000, 0, 64, 16), ("top-row", 8000, ny - 16, 64, 16),
        ("tile-seam", 7 * 1024 - 40, 6000, 80, 16), ("interior", 12345, 2345, 64, 32),
        ("cylinder", wl.xc - r - 4, wl.yc - r - 4, 2 * r + 9, 2 * r + 9),
    ]
    for name, x0, y0, w, h in windows:
        win = lat.get_window(x0, y0, w, h)
        cx0, cy0 = max(0, x0 - m), max(0, y0 - m)
        cx1, cy1 = min(nx, x0 + w + m), min(ny, y0 + h + m)
        o = O.Oracle(cx1 - cx0, cy1 - cy0, wl.tau, wl.U, bc_y=wl.bc, mask=mask[cy0:cy1, cx0:cx1])
        o.init_equilibrium(rho[cy0:cy1, cx0:cx1], u[cy0:cy1, cx0:cx1], v[cy0:cy1, cx0:cx1])
        Fo = o.run(s)
        o.collide()
        Fo = np.vstack([Fo, o.force()[None, :]])
        ref = o.get_fs()[:, y0 - cy0:y0 - cy0 + h, x0 - cx0:x0 - cx0 + w]
        f = offsets_to_f(win, wl.U)
        fluid = mask[y0:y0 + h, x0:x0 + w] == 0
        df = np.max(np.abs(f - ref)[:, fluid])
        assert df <= 1e-6 * wl.U, (name, df)
        if name == "cylinder":
            assert np.max(np.abs(F - Fo)) <= 1e-6 * np.max(np.abs(Fo)), (F, Fo)
    lat.close()


@pytest.mark.parametrize("storage", [lbm.LBM_F32, lbm.LBM_F16_OFS, lbm.LBM_BF16_OFS, lbm.LBM_F16_SR])
def test_bulk_store_kernel_matches_direct(storage):
    """TMA loads + TMA bulk stores: the same per-node arithmetic, identical bits."""
    shapes = lbm.lbm_kernel_shapes(lbm.LBM_KERNEL_TMA_BULK)
    assert len(shapes) >= 3
    for wl in (W.random_case(613, 57, seed=21, bc=W.BC_FREESLIP, D=10),
               W.random_case(769, 33, seed=8, bc=W.BC_ZOUHE, D=8),   # outlet alone at a 768-node tile start
               W.random_case(1025, 29, seed=9, bc=W.BC_PERIODIC, D=8)):
        ref, Fr, _, _ = gpu_run(wl, 25, kernel=lbm.LBM_KERNEL_DIRECT, storage=storage)
        for shape in shapes:
            for ctas in (1, 2):
                for coll in (lbm.LBM_COLLIDE_BGK,):
                    pops, F, _, info = gpu_run(wl, 25, kernel=lbm.LBM_KERNEL_TMA_BULK, shape=shape,
                                               ctas_per_sm=ctas, storage=storage, collision=coll)
                    assert info["kernel"] == lbm.LBM_KERNEL_TMA_BULK
                    assert np.array_equal(pops.view(np.uint8), ref.view(np.uint8)), (wl.name, shape, ctas)
                    assert np.array_equal(F, Fr), (wl.name, shape, ctas)


def test_bulk_store_kernel_mrt_matches_oracle():
    wl = W.random_case(300, 41, seed=501, bc=W.BC_ZOUHE, D=8, tau=0.56)
    pops, F, fields, _ = gpu_run(wl, 60, kernel=lbm.LBM_KERNEL_TMA_BULK, **MRT)
    compare(wl, 60, pops, F, fields, tol_f=1e-5 * wl.U, tol_F=1e-4, mrt=True)
