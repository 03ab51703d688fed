"""Learned warm start end to end on a reduced problem (D = 20, 800 x 400,
Re in [60, 85], where the cold start reaches a clean limit cycle): snapshots
from the batched solver, training with the library's tensor-core kernels,
warm vs cold start to periodic shedding on held-out Re."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2605_02185_gb300 import warmstart as WS  # noqa: E402


def test_warm_start_gains_over_cold_start():
    cfg = WS.Config(D=20, re_hi=85.0, train_cases=12, snapshots=9000, replay=512, iters=3000, batch=4,
                    stride=37, spinup_max=300_000, eval_max=200_000, chunk=500)
    dev = torch.device("cuda")
    net, info = WS.train(cfg, dev, log=lambda m: None)
    first, last = info["losses"][0][1], info["losses"][-1][1]
    assert last < 0.1 * first, info["losses"]
    rows, summary = WS.evaluate(net, cfg, n_eval=2, device=dev, log=lambda m: None)
    for r in rows:
        assert r["cold"]["steps"] is not None  # the judge itself reached periodic shedding
        assert r["warm"]["steps"] is not None
        # the acceptance rule: mean drag, lift amplitude and Strouhal number
        # of the converged cycle each within 1 % of the cold start's
        print(f"warm start Re {r['Re']:.1f}: drift {r['drift']}, steps {r['cold']['steps']} -> "
              f"{r['warm']['steps']}")
        assert all(r["drift"][k] <= 0.01 for k in ("cd_mean", "cl_amp", "st")), r
        assert r["accepted"]
    # the gain: fewer steps to periodic shedding from the prediction
    assert np.median([r["step_speedup"] for r in rows]) > 1.0, rows
