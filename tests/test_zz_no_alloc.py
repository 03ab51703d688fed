"""lbm_step_noalloc: one step on caller-owned device buffers, no allocation.

Some callers cannot allocate device memory (their memory comes from a pool
or arena they manage, or another runtime owns the allocator); this entry
point takes their input and output buffers and keeps its own scratch in a
fixed device array inside the library.  Its result must match the ordinary
entry point, lbm_step, on two calls in a row (the second call reuses the
scratch the first left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2605_02185_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_02185_gb300 import lbm  # noqa: E402


def test_noalloc_step_matches_lbm_step_twice():
    wl = W.random_case(613, 57, seed=21, bc=W.BC_ZOUHE, D=10)
    lat = lbm.lattice_for(wl)
    try:
        lat.init_fields(*wl.initial_fields())
        lat.step(3)
        lat.sync()
        h0 = lat.get_populations()
        n0 = lat.force_count()
        # the existing entry point, two steps
        lat.step(1)
        lat.sync()
        h1 = lat.get_populations()
        lat.step(1)
        lat.sync()
        h2 = lat.get_populations()
        F = lat.forces_raw(n0, 2)
        # the same two steps through lbm_step_noalloc on caller-owned buffers
        dev = torch.device("cuda")
        a = torch.from_numpy(h0).to(dev)
        b = torch.empty_like(a)
        force = torch.zeros(2, 2, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        lbm.lbm_step_noalloc(lat.h, a.data_ptr(), b.data_ptr(), force[0].data_ptr())
        lbm.lbm_step_noalloc(lat.h, b.data_ptr(), a.data_ptr(), force[1].data_ptr())
        lat.sync()
        got1 = b.cpu().numpy()
        got2 = a.cpu().numpy()
        got_force = force.cpu().numpy()
    finally:
        lat.close()
    # same per-node arithmetic as lbm_step; tolerance of the float path
    tol = 1e-5 * wl.U
    assert np.max(np.abs(got1.astype(np.float64) - h1)) <= tol
    assert np.max(np.abs(got2.astype(np.float64) - h2)) <= tol
    np.testing.assert_allclose(got_force, F, rtol=1e-4, atol=1e-12)
