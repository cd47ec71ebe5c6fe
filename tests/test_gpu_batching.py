"""Batching machinery on the GPU: slot packing of uneven trees, persistent
scheduling, CUDA-graph capture and the autotuner leave every result unchanged."""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


def _setup(cfg=4, B=300, T=30, precision="fp32"):
    from paper_2109_07719_gb300 import Simulator
    kw = dict(B=B, T=T, precision=precision)
    if cfg == 4:
        kw["dof_hi"] = 40
    work = wl.config(cfg, **kw)
    sim = Simulator(work.model, precision=precision)
    dt, dev = sim.dtype, sim.device
    q0 = torch.tensor(work.q0, dtype=dt, device=dev)
    qd0 = torch.tensor(work.qd0, dtype=dt, device=dev)
    tau = work.tau(device="cpu").to(dt).to(dev)
    return work, sim, q0, qd0, tau


def _run(sim, q0, qd0, tau, k=1):
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=k)
    g = sim.backward(ck, tau, torch.ones_like(qT), torch.ones_like(qdT), k=k)
    torch.cuda.synchronize()
    return (qT, qdT) + tuple(g)


def test_slot_order_sorts_by_link_count():
    work, sim, *_ = _setup()
    order = sim.slot_order()
    nl = np.diff(work.model.sys_link_offset)
    assert sorted(order.tolist()) == list(range(sim.B))
    assert np.all(np.diff(nl[order]) <= 0)


@pytest.mark.parametrize("threads", [32, 64, 128])
def test_persistent_schedule_matches_grid(threads):
    work, sim, q0, qd0, tau = _setup()
    ref = _run(sim, q0, qd0, tau)
    sim.set_launch(threads, persistent=True)
    out = _run(sim, q0, qd0, tau)
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    out2 = _run(sim, q0, qd0, tau, k=1)     # the ticket is reset between launches
    for a, b in zip(ref, out2):
        assert torch.equal(a, b)


def test_cuda_graph_capture_replays_the_same_step():
    work, sim, q0, qd0, tau = _setup(cfg=2, B=200)
    ref = _run(sim, q0, qd0, tau)
    outs = {}
    static_q0 = q0.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        _run(sim, static_q0, qd0, tau)       # warm up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        qT, qdT, ck, _ = sim.rollout(static_q0, qd0, tau)
        gr = sim.backward(ck, tau, torch.ones_like(qT), torch.ones_like(qdT))
        outs["v"] = (qT, qdT) + tuple(gr)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, outs["v"]):
        assert torch.equal(a, b)
    # new inputs copied into the static buffer flow through the replay
    static_q0.add_(0.01)
    g.replay()
    torch.cuda.synchronize()
    ref2 = _run(sim, static_q0, qd0, tau)
    for a, b in zip(ref2, outs["v"]):
        assert torch.equal(a, b)


def test_autotune_keeps_results(tmp_path, monkeypatch):
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    work, sim, q0, qd0, tau = _setup()
    from paper_2109_07719_gb300 import autotune as at
    best = sim.autotune(q0, qd0, T_probe=4, reps=1)
    assert best[2] in (1, 3, 4, 5) and best in at.CANDIDATES   # trees: not the link-frame pipelined kernels
    out = _run(sim, q0, qd0, tau)
    sim.set_launch(32, False)                               # the same kernels at the default shape
    ref = _run(sim, q0, qd0, tau)
    for a, b in zip(ref, out):
        assert torch.equal(a, b)


def test_autotune_lanes_on_chains(tmp_path, monkeypatch):
    """Serial chains: the one-warp, pipelined and world-aligned kernels are all
    timed; the pick runs with the matching kernels and gives the results of the
    one-lane path (to FP32 round-off)."""
    from paper_2109_07719_gb300 import autotune as at
    monkeypatch.setenv("ABASIM_TUNE_CACHE", str(tmp_path / "tune.json"))
    work, sim, q0, qd0, tau = _setup(cfg=2, B=256, T=20)
    sim.set_tape_space("one_warp")
    ref = _run(sim, q0, qd0, tau)
    assert "pipelined" not in sim.last_storage()
    best = sim.autotune(q0, qd0, T_probe=4, reps=1)
    out = _run(sim, q0, qd0, tau)
    assert (sim.last_storage()[0] == "pipelined") == (best[2] in (2, 5))
    assert sim.last_storage()[0].startswith("aligned") == (best[2] in (3, 4))
    assert sim.last_storage()[1].startswith("aligned_pipelined") == (best[2] in (4, 5))
    entry = next(iter(at.load_cache().values()))
    assert any(key.endswith("/pipelined") for key in entry["seconds"])
    assert any(key.endswith("/aligned") for key in entry["seconds"])
    for a, b in zip(ref, out):
        err = float((a - b).abs().max() / (b.abs().max() + 1e-30))
        assert err < 1e-5


@pytest.mark.parametrize("cfg", [2, 3, 4])
def test_shared_memory_tape_matches_global(cfg):
    """The per-step tape in shared memory or in global scratch gives the same
    results (the two are separately compiled kernels, so to FP32 round-off)."""
    work, sim, q0, qd0, tau = _setup(cfg=cfg, B=96, T=40)
    sim.set_tape_space("global")
    ref = _run(sim, q0, qd0, tau)
    sim.set_tape_space("one_warp")
    out = _run(sim, q0, qd0, tau)
    for a, b in zip(ref, out):
        err = float((a - b).abs().max() / (b.abs().max() + 1e-30))
        assert err < 1e-5
