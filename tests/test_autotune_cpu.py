"""Autotuner logic without a GPU: the fastest candidate is chosen and remembered."""
import json

import pytest

torch = pytest.importorskip("torch")


class _FakeSolver:
    nprob, ncell, device = 10, 1000, "cpu"

    def __init__(self):
        self.tuning = None

    def set_tuning(self, cand):
        self.tuning = cand


def test_pick_and_cache(tmp_path, monkeypatch):
    from paper_2003_09145_gb300 import autotune
    monkeypatch.setenv("TENO_AUTOTUNE_CACHE", str(tmp_path / "t.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    times = {(64, 4): 3.0, (128, 4): 1.5, (256, 2): 1.5, (128, 8): 2.0}
    calls = []

    def timer(solver, U, cand, steps):
        calls.append(cand)
        return times[cand]

    s = _FakeSolver()
    best = autotune.tune_batched(s, None, candidates=list(times), timer=timer)
    assert best == (128, 4) and s.tuning == (128, 4)        # first of the tied minimum
    data = json.load(open(tmp_path / "t.json"))
    assert data["FakeGPU"]["batch:nprob=10:ncell=1000"]["best"] == [128, 4]
    n = len(calls)
    assert autotune.tune_batched(_FakeSolver(), None, candidates=list(times), timer=timer) == (128, 4)
    assert len(calls) == n                                  # served from the cache
