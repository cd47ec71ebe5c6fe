"""Host logic of bench.py's extra measurements, with a stand-in for the
simulator that checks arguments the way the binding does (device, dtype,
contiguity, shape) and returns deterministic outputs: the per-output error
against the FP64 path indexes the sampled systems consistently, and the
checkpoint-interval sweep passes its own buffers (no GPU)."""
import types

import numpy as np
import pytest
import torch

import bench
import workloads as wl


class FakeSim:
    def __init__(self, model, precision="fp32", integrator="semi"):
        self.model = model
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.device = torch.device("cpu")
        self.B = model.n_systems
        self.nq_max, self.nv_max = model.nq_max, model.nv_max
        self.n_links = model.n_links_total

    @property
    def nx(self):
        return self.nq_max + self.nv_max

    def _arg(self, t, shape, name):
        assert t.device == self.device and t.dtype == self.dtype and t.is_contiguous(), name
        assert tuple(t.shape) == tuple(shape), (name, tuple(t.shape), shape)

    def empty(self, *shape):
        return torch.empty(shape, dtype=self.dtype)

    def ckpt_bytes(self, T, k):
        return (T + k - 1) // k * self.nx * self.B * self.dtype.itemsize

    def work_bytes(self, k):
        return 0 if k == 1 else k * self.nx * self.B * self.dtype.itemsize

    def rollout(self, q0, qd0, tau, k=1, traj=False, out=None):
        T = tau.shape[0]
        self._arg(q0, (self.nq_max, self.B), "q0")
        self._arg(qd0, (self.nv_max, self.B), "qd0")
        self._arg(tau, (T, self.nv_max, self.B), "tau")
        ck = torch.cat([torch.cat([q0, qd0])[None] + t for t in range(0, T, k)]) if T else self.empty(0, self.nx, self.B)
        return q0 + T, qd0 + T, ck, None

    def status(self):
        return np.zeros(self.B, np.int32)

    def backward(self, ck, tau, gqT, gqdT, k=1, **kw):
        T = tau.shape[0]
        self._arg(gqT, (self.nq_max, self.B), "gqT")
        self._arg(gqdT, (self.nv_max, self.B), "gqdT")
        assert ck.shape[0] == (T + k - 1) // k
        return gqT * 2, gqdT * 3, tau * 4, torch.ones(self.n_links, dtype=self.dtype)


def test_precision_error_compares_the_sampled_systems(monkeypatch):
    import paper_2109_07719_gb300 as pkg
    monkeypatch.setattr(pkg, "Simulator", FakeSim)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    work = wl.config(4, B=40, T=600, precision="fp32")
    sim = FakeSim(work.model)
    q0 = torch.tensor(work.q0, dtype=torch.float32)
    qd0 = torch.tensor(work.qd0, dtype=torch.float32)
    tau = work.tau(dtype=torch.float32)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
    ones = torch.ones_like(qT)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, ones, torch.zeros_like(qdT))
    args = types.SimpleNamespace(k=1, precision="fp32")
    r = bench.precision_error(sim, work, args, (qT, qdT, gq0, gqd0, gtau, gm), ck, tau)
    nv = work.model.nv_per_system()
    assert nv.min() in r["dof"] and nv.max() in r["dof"]
    # the stand-in returns the same functions of the same inputs on both sides
    for name, err in r["per_output"].items():
        assert err < 1e-6, (name, err)
    assert set(r["by_horizon"]) == {"250", "500"}
    assert r["within_tolerance"] and r["largest_horizon_within_tolerance"] == 600


def test_checkpoint_sweep_uses_its_own_buffers():
    work = wl.config(2, B=8, T=20, precision="fp32")
    sim = FakeSim(work.model)
    seen = []

    def step(evs=None, kk=1, ckb=None, wbuf=None):
        seen.append((kk, tuple(ckb.shape)))
        if evs:
            for e in evs:
                e.record()

    class Ev:
        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self, stream=None):
            import time
            self.t = time.perf_counter()

        def elapsed_time(self, other):
            return 1e3 * (other.t - self.t) + 1e-3

    import bench as b
    orig = torch.cuda.Event
    try:
        torch.cuda.Event = Ev
        sync = torch.cuda.synchronize
        torch.cuda.synchronize = lambda: None
        out = b.checkpoint_sweep(sim, step, 20, 8, torch.zeros(4), [10, 7])
    finally:
        torch.cuda.Event = orig
        torch.cuda.synchronize = sync
    assert set(out) == {"10", "7"}
    assert seen == [(10, (2, sim.nx, 8)), (10, (2, sim.nx, 8)), (7, (3, sim.nx, 8)), (7, (3, sim.nx, 8))]
    assert out["7"]["ckpt_bytes"] == 3 * sim.nx * 8 * 4
