"""Host logic of the launch-shape autotuner: selection and the JSON cache (no GPU)."""
import json

import pytest

from paper_2109_07719_gb300 import autotune as at


class FakeSim:
    """Records the launch controls; ``pipelines`` / ``aligns`` say whether the
    model's shape lets the pipelined or the world-aligned kernels run (the
    library refuses the tape space otherwise, as the binding reports)."""

    def __init__(self, B=4096, pipelines=True, aligns=True):
        self.B = B
        self.signature = (B, 7, 7, 7 * B, "fp32", "abc")
        self.calls = []
        self.pipelines = pipelines
        self.aligns = aligns
        self.space = "auto"

    def set_launch(self, threads=0, persistent=False):
        self.calls.append((threads, persistent, self.space))
        self.launch = (threads, persistent)

    def set_tape_space(self, space="auto"):
        from paper_2109_07719_gb300 import SimError
        self.space = space
        if (space == "pipelined" and not self.pipelines) or (space.startswith("aligned") and not self.aligns):
            raise SimError(f"{space}: this model cannot run on these kernels")

    def last_storage(self):
        mode = {"pipelined": "pipelined", "aligned": "aligned_shared",
                "aligned_pipelined": "aligned_pipelined_shared"}.get(self.space, "shared")
        return mode, mode


def test_choose_picks_fastest_and_breaks_ties_by_order():
    times = {(32, False, 1): 2.0, (64, False, 1): 1.0, (128, True, 1): 1.0, (32, True, 2): 1.0}
    assert at.choose(times) == (64, False, 1)
    with pytest.raises(ValueError):
        at.choose({})


def test_autotune_times_candidates_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    sim = FakeSim()
    cost = {(32, False, 1): 3.0, (64, False, 1): 2.0, (128, False, 1): 2.5, (32, True, 1): 1.5,
            (64, True, 1): 4.0, (128, True, 1): 5.0, (32, False, 2): 1.6, (32, True, 2): 1.7,
            (32, False, 3): 1.8, (64, False, 3): 1.9, (32, True, 3): 2.1, (64, True, 3): 2.2,
            (32, False, 4): 1.55, (64, False, 4): 1.65, (32, True, 4): 1.75, (64, True, 4): 1.85,
            (32, False, 5): 1.52, (32, True, 5): 1.51}
    seen = []

    def timer(s, cand):
        seen.append(cand)
        return cost[cand]

    best = at.autotune(sim, None, None, timer=timer, device_name="GB300")
    assert best == (32, True, 1)
    assert sim.launch == (32, True) and sim.space == "one_warp"
    assert sorted(seen) == sorted(cost)
    table = json.load(open(tmp_path / "tune.json"))
    assert len(table) == 1
    # second call: served from the cache, no timing
    sim2 = FakeSim()
    best2 = at.autotune(sim2, None, None, timer=lambda s, c: pytest.fail("timed again"),
                        device_name="GB300")
    assert best2 == (32, True, 1) and sim2.calls == [(32, True, "one_warp")]
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


def test_two_lanes_win_where_the_model_pipelines(tmp_path, monkeypatch):
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    cost = lambda s, c: 1.0 if c[2] == 2 else 2.0          # noqa: E731
    sim = FakeSim()
    assert at.autotune(sim, None, None, timer=cost, device_name="x") == (32, False, 2)
    assert sim.space == "pipelined"
    assert json.load(open(tmp_path / "tune.json")).popitem()[1]["kernels"] == 2
    # the cache entry restores the tape mode too
    sim2 = FakeSim()
    at.autotune(sim2, None, None, timer=lambda s, c: pytest.fail("timed again"), device_name="x")
    assert sim2.space == "pipelined" and sim2.launch == (32, False)


def test_world_aligned_kernels_are_a_candidate(tmp_path, monkeypatch):
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    sim = FakeSim()
    best = at.autotune(sim, None, None, timer=lambda s, c: 1.0 if c == (64, True, 3) else 2.0, device_name="x")
    assert best == (64, True, 3) and sim.space == "aligned" and sim.launch == (64, True)


def test_candidates_the_model_cannot_run_are_dropped(tmp_path, monkeypatch):
    """A model neither the pipelined nor the world-aligned kernels can run (the
    library refuses those tape spaces): only the one-warp kernels are kept."""
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    sim = FakeSim(pipelines=False, aligns=False)
    seen = []
    best = at.autotune(sim, None, None, timer=lambda s, c: seen.append(c) or (1.0 if c[2] != 1 else 2.0),
                       device_name="x")
    assert best[2] == 1 and sim.space == "one_warp"
    # the automatic choice is timed too, and dropped: it ran the one-warp kernels
    assert all(c[2] in (1, 5) for c in seen)
    kept = json.load(open(tmp_path / "tune.json")).popitem()[1]["seconds"]
    assert kept and all(key.endswith("/one_warp") for key in kept)


def test_old_cache_entries(tmp_path, monkeypatch):
    """Entries written before the kernel family was recorded: no key means the
    one-warp kernels, a 'lanes' key of 2 the pipelined ones."""
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    sim = FakeSim()
    at.save_cache({at.cache_key(sim.signature, "x"): {"threads": 64, "persistent": False}})
    assert at.autotune(sim, None, None, timer=None, device_name="x") == (64, False, 1)
    assert sim.space == "one_warp"
    at.save_cache({at.cache_key(sim.signature, "y"): {"threads": 32, "persistent": True, "lanes": 2}})
    assert at.autotune(sim, None, None, timer=None, device_name="y") == (32, True, 2)
    assert sim.space == "pipelined"
