"""bench.py's CPU baseline legs (no GPU): the oracle timed in one process on one
thread, and on every host core as spawned single-threaded processes that start
together at a barrier."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _args():
    return types.SimpleNamespace(config=2, precision="fp32", contacts=False, limits=False)


def test_one_core_baseline():
    import bench
    import torch
    before = torch.get_num_threads()
    r = bench.cpu_baseline(_args(), budget_s=1.0, threads=1)
    assert r["cores"] == 1 and r["kind"] == "oracle" and r["value"] > 0
    assert torch.get_num_threads() == before          # the thread count is restored


def test_all_core_baseline_runs_one_process_per_core():
    import bench
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    r = bench.cpu_baseline(_args(), budget_s=1.0)
    if "process pool unavailable" in r["sample"]:
        pytest.skip(r["sample"])
    assert r["cores"] == n and r["value"] > 0
    assert f"in each of {n} single-threaded processes" in r["sample"]
