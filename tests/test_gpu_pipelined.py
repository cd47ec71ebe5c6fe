"""The pipelined two-warp adjoint (one warp recomputes step t while the other
differentiates step t + 1) against the single-warp adjoint and the FP64 oracle,
through the C ABI: ragged batches, horizons of 1 and 2 steps, persistent
scheduling, per-step objective terms and the FP32 + FP64 D-solve mode."""
import numpy as np
import pytest
import torch

import workloads as wl
from tests._parity import oracle_backward, check

pytestmark = pytest.mark.gpu


def _run(sim, space, q0, qd0, tau, gqT, gqdT, g_traj=None, persistent=False):
    sim.set_tape_space(space)
    sim.set_launch(32, persistent)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=1)
    out = sim.backward(ck, tau, gqT, gqdT, k=1, g_traj=g_traj)
    torch.cuda.synchronize()
    return out


def _setup(B, T, precision="fp32", seed=3):
    from paper_2109_07719_gb300 import Simulator
    work = wl.config(2, B=B, T=T, precision=precision, seed=wl.SEED_BASE + seed)
    sim = Simulator(work.model, precision=precision)
    dt, dev = sim.dtype, sim.device
    q0 = torch.tensor(work.q0, dtype=dt, device=dev)
    g = torch.Generator().manual_seed(seed)
    qd0 = (0.5 * torch.randn(work.qd0.shape, generator=g, dtype=torch.float64)).to(dt).to(dev)
    tau = work.tau(device=dev, dtype=dt)
    gqT = torch.randn(q0.shape, generator=g, dtype=torch.float64).to(dt).to(dev)
    gqdT = torch.randn(qd0.shape, generator=g, dtype=torch.float64).to(dt).to(dev)
    return work, sim, q0, qd0, tau, gqT, gqdT


@pytest.mark.parametrize("B,T", [(100, 37), (32, 1), (33, 2), (4096, 20)])
@pytest.mark.parametrize("precision", ["fp32", "fp32_d64"])
def test_pipelined_matches_single_warp(B, T, precision):
    work, sim, q0, qd0, tau, gqT, gqdT = _setup(B, T, precision)
    a = _run(sim, "shared", q0, qd0, tau, gqT, gqdT)
    b = _run(sim, "pipelined", q0, qd0, tau, gqT, gqdT)
    for name, x, y in zip(("gq0", "gqd0", "gtau", "gmass"), a, b):
        check(name, y.cpu().numpy(), x.cpu().numpy(), 1e-5)
    assert sim.status().sum() == 0


def test_pipelined_persistent_equals_grid():
    work, sim, q0, qd0, tau, gqT, gqdT = _setup(300, 25)
    a = _run(sim, "pipelined", q0, qd0, tau, gqT, gqdT, persistent=False)
    b = _run(sim, "pipelined", q0, qd0, tau, gqT, gqdT, persistent=True)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_pipelined_per_step_objective():
    work, sim, q0, qd0, tau, gqT, gqdT = _setup(70, 15)
    g = torch.Generator().manual_seed(9)
    gtraj = torch.randn((16, sim.nx, sim.B), generator=g, dtype=torch.float64).to(sim.dtype).to(sim.device)
    a = _run(sim, "shared", q0, qd0, tau, gqT, gqdT, g_traj=gtraj)
    b = _run(sim, "pipelined", q0, qd0, tau, gqT, gqdT, g_traj=gtraj)
    for name, x, y in zip(("gq0", "gqd0", "gtau", "gmass"), a, b):
        check(name, y.cpu().numpy(), x.cpu().numpy(), 1e-5)


def test_pipelined_against_oracle():
    """FP32 pipelined gradients against the FP64 oracle within the FP32 bound (1e-2)."""
    work, sim, q0, qd0, tau, gqT, gqdT = _setup(64, 60, seed=5)
    gq0, gqd0, gtau, gm = _run(sim, "pipelined", q0, qd0, tau, gqT, gqdT)
    sel = [0, 31, 63]
    h = [x.double().cpu().numpy() for x in (q0, qd0, tau, gqT, gqdT)]
    o = oracle_backward(work.model, sel, h[0], h[1], h[2], h[3], h[4])
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], 1e-2)
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], 1e-2)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-2)


def test_pipelined_refuses_what_it_cannot_run():
    from paper_2109_07719_gb300 import SimError
    work, sim, q0, qd0, tau, gqT, gqdT = _setup(40, 12)
    sim.set_tape_space("pipelined")
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=3)
    with pytest.raises(SimError, match="pipelined"):
        sim.backward(ck, tau, gqT, gqdT, k=3)


# ---------------------------------------------------------------- pipelined rollout

@pytest.mark.parametrize("B,T", [(100, 37), (32, 1), (33, 2)])
@pytest.mark.parametrize("precision", ["fp32", "fp32_d64"])
def test_pipelined_rollout_matches_single_warp(B, T, precision):
    """Forward rollout split over an inertia warp and a bias warp against the
    one-warp rollout: final state, checkpoints and trajectory."""
    work, sim, q0, qd0, tau, gqT, gqdT = _setup(B, T, precision)
    outs = {}
    for space in ("shared", "pipelined"):
        sim.set_tape_space(space)
        outs[space] = sim.rollout(q0, qd0, tau, k=1, traj=True)
        torch.cuda.synchronize()
        assert sim.last_storage()[0] == space
    for name, x, y in zip(("qT", "qdT", "ckpt", "traj"), outs["shared"], outs["pipelined"]):
        check(name, y.cpu().numpy(), x.cpu().numpy(), 1e-5)


def test_pipelined_rollout_persistent_and_interval():
    work, sim, q0, qd0, tau, gqT, gqdT = _setup(300, 23)
    sim.set_tape_space("pipelined")
    sim.set_launch(32, False)
    a = sim.rollout(q0, qd0, tau, k=5)
    sim.set_launch(32, True)
    b = sim.rollout(q0, qd0, tau, k=5)
    torch.cuda.synchronize()
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    sim.set_launch(32, False)
    c = sim.rollout(q0, qd0, tau, k=1)
    assert torch.equal(a[2], c[2][::5])


@pytest.mark.parametrize("n,expect", [(14, "pipelined"), (15, None)])
def test_pipelined_rollout_chain_length_limit(n, expect):
    from paper_2109_07719_gb300 import Simulator
    work = wl.serial_chains(B=40, T=12, n=n, precision="fp32")
    sim = Simulator(work.model, precision="fp32")
    dev = sim.device
    q0 = torch.tensor(work.q0, dtype=torch.float32, device=dev)
    qd0 = torch.tensor(work.qd0, dtype=torch.float32, device=dev)
    tau = work.tau(device=dev, dtype=torch.float32)
    a = sim.rollout(q0, qd0, tau)
    torch.cuda.synchronize()
    mode = sim.last_storage()[0]
    if expect:
        assert mode == expect
        sim.set_tape_space("global")          # a 14-link one-warp tape does not fit on chip
        b = sim.rollout(q0, qd0, tau)
        for x, y in zip(a[:2], b[:2]):
            check("state", x.cpu().numpy(), y.cpu().numpy(), 1e-5)
    else:
        assert mode != "pipelined"


def _mixed_chains(B3=37, B7=30, T=21):
    """A batch of 3-link and 7-link serial chains (tiles mixing both lengths after
    slot packing): the model descriptions concatenated system by system."""
    a = wl.serial_chains(B=B3, T=T, n=3, precision="fp32")
    c = wl.serial_chains(B=B7, T=T, n=7, precision="fp32", seed=wl.SEED_BASE + 11)
    ma, mc = a.model, c.model
    off = np.concatenate([ma.sys_link_offset, ma.sys_link_offset[-1] + mc.sys_link_offset[1:]]).astype(np.int32)
    cat = lambda f: np.concatenate([getattr(ma, f), getattr(mc, f)])  # noqa: E731
    m = wl.ModelDesc(off, cat("parent"), cat("joint_type"), cat("axis"), cat("X_tree"), cat("mass"), cat("com"),
                     cat("I_com"), ma.dt, ma.gravity, "mixed_chains")
    q0 = np.zeros((7, B3 + B7))
    q0[:3, :B3] = a.q0
    q0[:, B3:] = c.q0
    return m, q0, np.zeros((7, B3 + B7))


def test_pipelined_kernels_with_mixed_chain_lengths():
    from paper_2109_07719_gb300 import Simulator
    m, q0h, qd0h = _mixed_chains()
    sim = Simulator(m, precision="fp32")
    dev = sim.device
    g = torch.Generator().manual_seed(21)
    q0 = torch.tensor(q0h, dtype=torch.float32, device=dev)
    qd0 = torch.tensor(0.3 * np.random.default_rng(4).standard_normal(qd0h.shape), dtype=torch.float32, device=dev)
    nv = torch.tensor(m.nv_per_system())
    mask = (torch.arange(7)[:, None] < nv[None, :]).float().to(dev)
    qd0 = qd0 * mask
    tau = torch.randn((21, 7, sim.B), generator=g).float().to(dev) * mask
    gqT, gqdT = torch.ones_like(q0) * mask, torch.ones_like(qd0) * mask
    outs = {}
    for space in ("global", "pipelined"):
        sim.set_tape_space(space)
        qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
        gr = sim.backward(ck, tau, gqT, gqdT)
        torch.cuda.synchronize()
        outs[space] = (qT, qdT) + tuple(gr)
        assert sim.last_storage() == ((space, space) if space == "pipelined" else ("global", "global"))
    for name, x, y in zip(("qT", "qdT", "gq0", "gqd0", "gtau", "gmass"), outs["global"], outs["pipelined"]):
        check(name, y.cpu().numpy(), x.cpu().numpy(), 1e-5)
    assert sim.status().sum() == 0
