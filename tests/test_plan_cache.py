"""The autotuner's plan cache (host logic, no GPU): a shape class is
measured once, then read back; the key holds every input the plan depends
on; an unreadable cache counts as empty."""
import json

from paper_2407_11290_gb300 import ttcross


class FakeCross:
    """Stands in for a TTCross: records the tuner's calls."""

    def __init__(self, n, plan=(32, 6, 1.5)):
        self.n = n
        self.plan = plan
        self.tuned = 0
        self.set = []

    def autotune(self, eps, max_rank, grid, stream):
        self.tuned += 1
        return self.plan

    def set_plan(self, te, qs):
        self.set.append((te, qs))


def test_measured_once_then_cached(tmp_path, monkeypatch):
    path = tmp_path / "plans.json"
    monkeypatch.setenv("TTCROSS_PLAN_CACHE", str(path))
    tc = FakeCross([64] * 6)
    assert ttcross.tuned_plan(tc, 1e-8, 64, [2] * 6, "fp64", "stored") == (32, 6, "measured")
    assert tc.tuned == 1 and path.exists()
    assert ttcross.tuned_plan(tc, 1e-8, 64, [2] * 6, "fp64", "stored") == (32, 6, "cache")
    assert tc.tuned == 1 and tc.set == [(32, 6)]
    # another eps, precision, grid or form is another class
    for args in [(1e-9, 64, [2] * 6, "fp64", "stored"), (1e-8, 64, [2] * 6, "split", "stored"),
                 (1e-8, 64, None, "fp64", "stored"), (1e-8, 64, [2] * 6, "fp64", "recompute"),
                 (1e-8, 32, [2] * 6, "fp64", "stored")]:
        assert ttcross.tuned_plan(tc, *args)[2] == "measured"
    assert tc.tuned == 6
    assert len(json.loads(path.read_text())) == 6


def test_unreadable_cache_is_empty(tmp_path, monkeypatch):
    path = tmp_path / "plans.json"
    path.write_text("{not json")
    monkeypatch.setenv("TTCROSS_PLAN_CACHE", str(path))
    tc = FakeCross([32] * 4, plan=(64, 4, 2.0))
    assert ttcross.tuned_plan(tc, 1e-6, 64, None, "split", "stored") == (64, 4, "measured")
    assert json.loads(path.read_text())  # rewritten as valid JSON
