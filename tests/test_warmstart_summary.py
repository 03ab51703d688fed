"""Host logic of the warm-start evaluation: the gain of a case counts the
fallback to a cold start when the prediction is rejected or never becomes
periodic, and only cases whose cold start became periodic are judged."""
import math

import pytest

ws = pytest.importorskip("paper_2605_02185_gb300.warmstart")


def case(cold_s, warm_s, accepted, cold_periodic=True, limit_s=None, step_speedup=None):
    r = {"cold": {"wall_s": cold_s}, "warm": {"wall_s": warm_s}, "accepted": accepted,
         "cold_periodic": cold_periodic}
    if limit_s is not None:
        r["warm"]["limit_s"] = limit_s
    if accepted:
        r["step_speedup"] = step_speedup
        r["time_speedup"] = cold_s / warm_s
    return r


def test_gain_counts_the_fallback():
    rows = [case(4.0, 1.0, True, step_speedup=5.0),         # accepted: cold / warm
            case(3.0, 1.0, False),                          # rejected: cold / (warm + cold)
            case(2.0, None, False, limit_s=10.0),           # warm never periodic: cold / (limit + cold)
            case(None, None, False, cold_periodic=False)]   # cold never periodic: not judged
    s = ws.summarize(rows)
    assert (s["cases"], s["cold_periodic"], s["accepted"]) == (4, 3, 1)
    assert [r["gain"] for r in rows[:3]] == [4.0, 0.75, 2.0 / 12.0]
    assert "gain" not in rows[3]
    assert s["median_gain_all_judged"] == 0.75
    assert math.isclose(s["total_time_speedup"], 9.0 / 17.0)
    assert s["median_step_speedup_accepted"] == 5.0
    assert s["median_time_speedup_accepted"] == 4.0


def test_nothing_judged():
    s = ws.summarize([case(None, None, False, cold_periodic=False)])
    assert s["cold_periodic"] == 0 and s["median_gain_all_judged"] is None and s["total_time_speedup"] is None
