"""Batched step: many lattices of different size, Re and boundary mode in one
launch per step, checked against single-lattice runs and the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_02185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_02185_gb300 import lbm  # noqa: E402


def mixed_cases():
    return [
        W.random_case(37, 23, seed=1, bc=W.BC_FREESLIP, D=6),
        W.random_case(613, 57, seed=2, bc=W.BC_ZOUHE, D=10, U=0.05, tau=0.7),
        W.random_case(257, 31, seed=3, bc=W.BC_PERIODIC, D=8),
        W.random_case(1025, 41, seed=4, bc=W.BC_FREESLIP, D=12, U=0.06, tau=0.56),
        W.random_case(300, 77, seed=5, bc=W.BC_ZOUHE, D=14),
    ]


def single(wl, steps, **kw):
    lat = lbm.lattice_for(wl, **kw)
    lat.init_fields(*wl.initial_fields())
    lat.step(steps)
    lat.sync()
    out = lat.get_populations(), lat.forces_raw(0, steps + 1)
    lat.close()
    return out


@pytest.mark.parametrize("kernel,shape,graph", [
    (lbm.LBM_KERNEL_TMA, None, 0), (lbm.LBM_KERNEL_TMA, (8, 1, 8), -1), (lbm.LBM_KERNEL_TMA, (16, 2, 3), 4),
    (lbm.LBM_KERNEL_DIRECT, None, 0)])
def test_batch_equals_single_lattices(kernel, shape, graph):
    cases = mixed_cases()
    steps = 25
    b = lbm.Batch(cases, kernel=kernel, shape=shape, graph_steps=graph)
    try:
        b.init_all()
        b.step(steps)
        b.sync()
        got = [(b.get_populations(c), b.forces_raw(c)) for c in range(len(cases))]
        info = b.kernel_info()
    finally:
        b.close()
    for c, wl in enumerate(cases):
        kw = dict(kernel=kernel)
        if kernel == lbm.LBM_KERNEL_TMA:
            kw.update(shape=(info["consumer_warps"], info["cells_per_thread"], info["stages"]),
                      ctas_per_sm=info["ctas_per_sm"])
        ref = single(wl, steps, **kw)
        assert np.array_equal(got[c][0], ref[0]), c
        assert np.array_equal(got[c][1], ref[1]), c


def test_batch_matches_oracle():
    cases = mixed_cases()[:3]
    steps = 40
    b = lbm.Batch(cases)
    b.init_all()
    b.step(steps)
    b.sync()
    for c, wl in enumerate(cases):
        o = O.Oracle(wl.nx, wl.ny, wl.tau, wl.U, bc_y=wl.bc, mask=wl.mask())
        o.init_equilibrium(*wl.initial_fields())
        Fo = o.run(steps)
        _, uo, vo = o.fields()
        _, u, v = b.fields(c)
        fluid = wl.mask() == 0
        du = max(np.max(np.abs(u - uo)[fluid]), np.max(np.abs(v - vo)[fluid]))
        assert du <= 1e-5 * wl.U, (c, du)
        F = b.forces_raw(c, 0, steps)
        assert np.max(np.abs(F - Fo)) <= 1e-4 * np.max(np.abs(Fo)), c
    b.close()


def test_batch_of_paper_boxes_and_autotune(tmp_path, monkeypatch):
    from paper_2605_02185_gb300 import autotune
    monkeypatch.setenv("GBLBM_TUNE_CACHE", str(tmp_path / "tune.json"))
    cases = W.batched_cases(6, seed=4)
    b = lbm.Batch(cases, collision=lbm.LBM_COLLIDE_MRT)  # MRT keeps the low-tau cases stable
    b.init_all()
    nodes, bytes_step = b.nodes()
    assert nodes == sum(w.nx * w.ny for w in cases)
    assert bytes_step == 72.0 * nodes
    best = autotune.tune(b, [(w.nx, w.ny) for w in cases], lbm.LBM_F32, b.stream, steps=4, warmup=2)
    assert best["ms_per_step"] > 0
    again = autotune.tune(b, [(w.nx, w.ny) for w in cases], lbm.LBM_F32, b.stream)
    assert again["shape"] == best["shape"] and again["kind"] == best["kind"]  # served from the cache
    before = [lbm.lbm_force_count(b.case(c)) for c in range(len(cases))]
    b.step(10)
    b.sync()
    for c in range(len(cases)):
        assert lbm.lbm_force_count(b.case(c)) == before[c] + 10
        cd, cl = b.forces(c)
        assert np.all(np.isfinite(cd))
    b.close()


def test_batch_reinit_at_odd_parity():
    cases = mixed_cases()[:2]
    b = lbm.Batch(cases, graph_steps=-1)
    b.init_all()
    b.step(3)  # odd parity now
    b.init_fields(0, *cases[0].initial_fields())
    b.init_fields(1, *cases[1].initial_fields())
    b.step(5)
    b.sync()
    got = [b.get_populations(c) for c in range(2)]
    b.close()
    info_ref = [single(w, 5, kernel=lbm.LBM_KERNEL_TMA) for w in cases]
    for c in range(2):
        np.testing.assert_allclose(got[c], info_ref[c][0], rtol=0, atol=1e-7)
