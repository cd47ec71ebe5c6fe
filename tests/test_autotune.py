"""Host logic of the launch-shape autotuner: selection and the JSON cache (no GPU)."""
import json

import pytest

from paper_2109_07719_gb300 import autotune as at


class FakeSim:
    def __init__(self, B=4096):
        self.B = B
        self.signature = (B, 7, 7, 7 * B, "fp32", "abc")
        self.calls = []

    def set_launch(self, threads=0, persistent=False):
        self.calls.append((threads, persistent))
        self.launch = (threads, persistent)


def test_choose_picks_fastest_and_breaks_ties_by_order():
    times = {(32, False): 2.0, (64, False): 1.0, (128, True): 1.0}
    assert at.choose(times) == (64, False)
    with pytest.raises(ValueError):
        at.choose({})


def test_autotune_times_candidates_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    sim = FakeSim()
    cost = {(32, False): 3.0, (64, False): 2.0, (128, False): 2.5, (32, True): 1.5,
            (64, True): 4.0, (128, True): 5.0}
    seen = []

    def timer(s, cand):
        seen.append(cand)
        return cost[cand]

    best = at.autotune(sim, None, None, timer=timer, device_name="GB300")
    assert best == (32, True)
    assert sim.launch == (32, True)
    assert sorted(seen) == sorted(cost)
    table = json.load(open(tmp_path / "tune.json"))
    assert len(table) == 1
    # second call: served from the cache, no timing
    sim2 = FakeSim()
    best2 = at.autotune(sim2, None, None, timer=lambda s, c: pytest.fail("timed again"),
                        device_name="GB300")
    assert best2 == (32, True) and sim2.calls == [(32, True)]
    # another GPU name is another key
    sim3 = FakeSim()
    at.autotune(sim3, None, None, timer=timer, device_name="other")
    assert len(json.load(open(tmp_path / "tune.json"))) == 2


def test_small_batches_skip_oversized_blocks(tmp_path, monkeypatch):
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    sim = FakeSim(B=20)
    seen = []
    at.autotune(sim, None, None, timer=lambda s, c: seen.append(c) or 1.0, device_name="x",
                use_cache=False)
    assert all(c[0] == 32 for c in seen)
