"""Failure detection and checkpointing, in forms that cannot fault the GPU.

* Checkpoints carry a header and a checksum: a round trip is bitwise (the
  populations, the step count and the force history), and a truncated,
  corrupted or foreign image is refused with LBM_ERR_ARG.
* A NaN written into the populations from the host is caught by the step's
  stability check (LBM_ERR_UNSTABLE).
* A bounded device wait that runs out (a row tile whose copies the producer
  announces but never issues, with a short wait limit) ends the step with
  LBM_ERR_TIMEOUT; the context stays usable afterwards.
* The float collision's -1/rho (reciprocal estimate plus one Newton-Raphson
  step) stays within one ulp of the exact quotient for every float in
  [0.5, 1.5], and the packed pair lane gives the same bits.
"""
import numpy as np
import pytest

from paper_2605_02185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_02185_gb300 import lbm  # noqa: E402


def fresh(wl, **kw):
    lat = lbm.lattice_for(wl, **kw)
    lat.init_fields(*wl.initial_fields())
    return lat


@pytest.mark.parametrize("storage", [lbm.LBM_F32, lbm.LBM_F16_OFS], ids=["f32", "f16"])
def test_checkpoint_round_trip_is_bitwise(storage):
    wl = W.random_case(301, 61, seed=9, bc=W.BC_ZOUHE, D=10)
    ref = fresh(wl, storage=storage)
    ref.step(40)
    ref.sync()
    want_pops, want_F = ref.get_populations(), ref.forces_raw(0, 41)
    ref.close()
    a = fresh(wl, storage=storage)
    a.step(17)
    image = a.checkpoint()
    a.close()
    b = lbm.lattice_for(wl, storage=storage)
    b.restore(image)
    assert b.force_count() == 18
    b.step(23)
    b.sync()
    assert np.array_equal(b.get_populations().view(np.uint8), want_pops.view(np.uint8))
    # the whole history: restored entries 0..17 and stepped entries 18..40
    assert np.array_equal(b.forces_raw(0, 41), want_F)
    b.close()


def test_damaged_or_foreign_checkpoint_is_refused():
    wl = W.random_case(157, 43, seed=4, bc=W.BC_FREESLIP, D=8)
    a = fresh(wl)
    a.step(9)
    image = a.checkpoint()
    before = a.get_populations()
    cases = {
        "truncated": image[:-5],
        "header only": image[:88],
        "padded": image + b"\0" * 8,
        "one flipped bit in the populations": image[:1000] + bytes([image[1000] ^ 4]) + image[1001:],
        "one flipped bit in the history": image[:-3] + bytes([image[-3] ^ 1]) + image[-2:],
        "bad magic": b"X" + image[1:],
        "empty": b"",
    }
    for name, bad in cases.items():
        with pytest.raises(lbm.LBMError) as e:
            a.restore(bad)
        assert e.value.code == lbm.LBM_ERR_ARG, name
    # the refused loads left the context as it was
    assert np.array_equal(a.get_populations(), before)
    a.close()
    # an intact image of another lattice (other tau) is refused too
    import dataclasses
    other = lbm.lattice_for(dataclasses.replace(wl, tau=0.61))
    with pytest.raises(lbm.LBMError) as e:
        other.restore(image)
    assert e.value.code == lbm.LBM_ERR_ARG
    other.close()


def test_nan_written_from_the_host_is_reported_unstable():
    wl = W.random_case(157, 43, seed=4, bc=W.BC_FREESLIP, D=8)
    lat = fresh(wl)
    lat.step(3)
    pops = lat.get_populations()
    n = lat.force_count()
    pops[5, 20, 30] = np.nan  # one population of one fluid node
    assert wl.mask()[20, 30] == 0
    lat.set_populations(pops, n)
    lat.step(1)
    with pytest.raises(lbm.LBMError) as e:
        lat.sync()
    assert e.value.code == lbm.LBM_ERR_UNSTABLE
    lat.close()


@pytest.mark.parametrize("kernel", [lbm.LBM_KERNEL_TMA, lbm.LBM_KERNEL_TMA_BULK], ids=["tma", "tma_bulk"])
def test_bounded_wait_that_runs_out_reports_timeout(kernel):
    wl = W.random_case(613, 57, seed=21, bc=W.BC_FREESLIP, D=10)
    ref = fresh(wl, kernel=kernel)
    ref.step(5)
    ref.sync()
    want = ref.get_populations()
    ref.close()
    lat = lbm.lattice_for(wl, kernel=kernel)
    try:
        lat.init_fields(*wl.initial_fields())
        lbm.lbm_set_fault_injection(lat.h, 7, 0.05)  # tile 7: announced, never copied; 50 ms waits
        lat.step(1)
        with pytest.raises(lbm.LBMError) as e:
            lat.sync()
        assert e.value.code == lbm.LBM_ERR_TIMEOUT
        # back to normal operation: the same context steps correctly again
        lbm.lbm_set_fault_injection(lat.h, -1, 0.0)
        lat.init_fields(*wl.initial_fields())
        lat.step(5)
        lat.sync()
        assert np.array_equal(lat.get_populations(), want)
    finally:
        lat.close()
    direct = lbm.lattice_for(wl, kernel=lbm.LBM_KERNEL_DIRECT)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_set_fault_injection(direct.h, 0, 0.05)
    assert e.value.code == lbm.LBM_ERR_ARG
    direct.close()


def test_negative_reciprocal_within_one_ulp_for_every_density():
    lo = np.array(0.5, np.float32).view(np.uint32)
    hi = np.array(1.5, np.float32).view(np.uint32)
    x = np.arange(lo, hi + 1, dtype=np.uint32).view(np.float32)
    xd = torch.from_numpy(x).cuda()
    y1 = torch.empty_like(xd)
    y2 = torch.empty_like(xd)
    lbm.lbm_probe_neg_recip(xd.data_ptr(), y1.data_ptr(), y2.data_ptr(), x.size)
    torch.cuda.synchronize()
    y1, y2 = y1.cpu().numpy(), y2.cpu().numpy()
    assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))  # the pair lane reproduces one lane
    exact = -1.0 / x.astype(np.float64)
    rounded = exact.astype(np.float32)
    ulp = np.spacing(np.abs(rounded)).astype(np.float64)
    err = np.abs(y1.astype(np.float64) - exact) / ulp
    exact_share = float(np.mean(y1 == rounded))
    print(f"-1/x on {x.size} floats in [0.5, 1.5]: max error {err.max():.4f} ulp, "
          f"correctly rounded {100 * exact_share:.3f} %")
    assert err.max() < 1.0, err.max()
    # and nearly always the correctly rounded quotient
    assert exact_share > 0.99


@pytest.mark.parametrize("storage", [lbm.LBM_F16_SR, lbm.LBM_BF16_SR], ids=["f16sr", "bf16sr"])
def test_stochastic_rounding_is_unbiased_and_brackets_the_value(storage):
    """Each stored value is one of the two 16-bit neighbours of the float
    being stored (toward zero, or one step further out), and over many
    salts it averages to that float."""
    rng = np.random.default_rng(3)
    vals = np.array([1.234567e-3, -7.654321e-5, 0.0123456, -0.0021, 3.0e-6, 0.25], np.float32)
    n = 200_000
    x = np.repeat(vals, n)
    salt = rng.integers(0, 2 ** 32, x.size, dtype=np.uint64).astype(np.uint32)
    xd, sd = torch.from_numpy(x).cuda(), torch.from_numpy(salt.view(np.int32)).cuda()
    out = torch.empty(x.size, dtype=torch.int16, device="cuda")
    lbm.lbm_probe_stochastic_round(storage, xd.data_ptr(), sd.data_ptr(), out.data_ptr(), x.size)
    torch.cuda.synchronize()
    bits = out.cpu().numpy().view(np.uint16)
    if storage == lbm.LBM_F16_SR:  # binary16 of 4096 x the offset
        scaled = (x * np.float32(4096)).astype(np.float32)
        t = scaled.astype(np.float16)
        out_of = np.abs(t.astype(np.float32)) > np.abs(scaled)
        t[out_of] = np.nextafter(t[out_of], np.float16(0))
        u = np.nextafter(t, np.where(scaled < 0, np.float16(-np.inf), np.float16(np.inf)).astype(np.float16))
        got = bits.view(np.float16).astype(np.float64) / 4096.0
        lo, hi = t.astype(np.float64) / 4096.0, u.astype(np.float64) / 4096.0
    else:  # bfloat16: truncation toward zero, or one step further out
        tb = x.view(np.uint32) & np.uint32(0xFFFF0000)
        got = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        lo = tb.view(np.float32).astype(np.float64)
        hi = (tb + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    assert np.all((got == lo) | (got == hi))
    for j, v in enumerate(vals):
        g = got[j * n:(j + 1) * n]
        gap = abs(hi[j * n] - lo[j * n])
        # the mean lands on v within 5 standard errors of a two-point draw
        assert abs(g.mean() - float(v)) <= 5 * 0.5 * gap / np.sqrt(n), (v, g.mean(), gap)
