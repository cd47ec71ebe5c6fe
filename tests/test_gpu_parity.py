"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle,
element by element on seeded inputs.

Tolerances (relative, max-norm per output tensor): the FP64 path must match
states within 1e-8 and gradients within 1e-6; the FP32 path states within
1e-3 and gradients within 1e-2.  Batch sizes span several 32-system blocks
with a ragged tail.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from tests._parity import oracle_forward, oracle_backward, check, mass_grad_of

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-8, 1e-6), "fp32": (1e-3, 1e-2)}


def _sim(work, precision="fp64", integrator="semi"):
    from paper_2109_07719_gb300 import Simulator
    return Simulator(work.model, precision=precision, integrator=integrator)


def _inputs(work, sim, T):
    """Device inputs in the simulator's dtype, and the same values in FP64 for the oracle."""
    q0 = torch.tensor(work.q0).to(sim.dtype)
    qd0 = torch.tensor(work.qd0)
    # a non-zero initial velocity exercises the Coriolis terms from step 0
    g = torch.Generator().manual_seed(work.seed + 3)
    qd0 = (qd0 + 0.5 * torch.randn(qd0.shape, generator=g, dtype=torch.float64)).to(sim.dtype)
    nv = work.model.nv_per_system()
    qd0 = qd0 * (torch.arange(work.model.nv_max)[:, None] < torch.tensor(nv)[None, :]).to(sim.dtype)
    tau = work.tau(T=T).to(sim.dtype)
    host = [x.double().numpy() for x in (q0, qd0, tau)]
    dev = [x.to(sim.device).contiguous() for x in (q0, qd0, tau)]
    return dev, host


CASES = {  # cfg: (B, T) for the full-oracle comparisons
    1: (1, 1000),
    2: (70, 120),
    3: (37, 80),
    4: (40, 40),
    5: (35, 40),
}


def _work(cfg, B, T, precision="fp64"):
    if cfg == 1:
        return wl.config(1, B=B, T=T)
    if cfg == 4:
        return wl.config(4, B=B, T=T, dof_hi=24, precision=precision)
    return wl.config(cfg, B=B, T=T, precision=precision)


@pytest.mark.parametrize("cfg", [1, 2, 3, 4, 5])
def test_single_step_fp64(cfg):
    B = CASES[cfg][0]
    work = _work(cfg, B, 1)
    sim = _sim(work)
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, 1)
    q1, qd1 = sim.step(q0, qd0, tau[0])
    torch.cuda.synchronize()
    oq, oqd = oracle_forward(work.model, list(range(B)), hq, hqd, ht)
    check("q1", q1.cpu().numpy(), oq, 1e-12)
    check("qd1", qd1.cpu().numpy(), oqd, 1e-12)


@pytest.mark.parametrize("cfg", [1, 2, 3, 4, 5])
def test_rollout_and_adjoint_fp64(cfg):
    B, T = CASES[cfg]
    work = _work(cfg, B, T)
    sim = _sim(work)
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    qT, qdT, ck, traj = sim.rollout(q0, qd0, tau, k=1, traj=True)
    g = torch.Generator().manual_seed(17)
    gqT = torch.randn(qT.shape, generator=g, dtype=torch.float64)
    gqdT = torch.randn(qdT.shape, generator=g, dtype=torch.float64)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT.to(sim.device), gqdT.to(sim.device), k=1)
    torch.cuda.synchronize()
    systems = list(range(B))
    oq, oqd = oracle_forward(work.model, systems, hq, hqd, ht)
    ts, tg = TOL["fp64"]
    check("qT", qT.cpu().numpy(), oq, ts)
    check("qdT", qdT.cpu().numpy(), oqd, ts)
    assert torch.equal(traj[-1][:sim.nq_max], qT) and torch.equal(traj[0][:sim.nq_max], q0)
    assert torch.equal(ck[0], traj[0])
    gsys = systems if cfg != 2 else systems[::5] + [B - 1]
    o = oracle_backward(work.model, gsys, hq, hqd, ht, gqT.numpy(), gqdT.numpy())
    check("gq0", gq0.cpu().numpy()[:, gsys], o["gq0"], tg)
    check("gqd0", gqd0.cpu().numpy()[:, gsys], o["gqd0"], tg)
    check("gtau", gtau.cpu().numpy()[:, :, gsys], o["gtau"], tg)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), gsys)
    check("gmass", np.concatenate([gmd[s] for s in gsys]), np.concatenate([o["gm"][s] for s in gsys]), tg)
    assert sim.status().sum() == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_oblique_joint_axes(precision):
    """Revolute axes in arbitrary directions, among them -z, a hair off -z, -x and
    +z: the library re-expresses each link in a frame whose z axis is the joint
    axis, which must leave states and gradients unchanged (FP32 runs the
    pipelined chain kernels)."""
    B, T = 40, 60
    work = wl.config(2, B=B, T=T, precision=precision)
    rng = np.random.default_rng(77)
    ax = rng.standard_normal(work.model.axis.shape)
    ax[:4] = [(0, 0, -1), (0, 1e-7, -1), (-1, 0, 0), (0, 0, 1)]
    work.model.axis = ax / np.linalg.norm(ax, axis=1, keepdims=True)
    sim = _sim(work, precision)
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=1)
    g = torch.Generator().manual_seed(5)
    gqT = torch.randn(qT.shape, generator=g, dtype=torch.float64)
    gqdT = torch.randn(qdT.shape, generator=g, dtype=torch.float64)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT.to(sim.dtype).to(sim.device), gqdT.to(sim.dtype).to(sim.device))
    torch.cuda.synchronize()
    ts, tg = TOL[precision]
    oq, oqd = oracle_forward(work.model, list(range(B)), hq, hqd, ht)
    check("qT", qT.cpu().numpy(), oq, ts)
    check("qdT", qdT.cpu().numpy(), oqd, ts)
    sel = [0, 1, 17, B - 1]
    o = oracle_backward(work.model, sel, hq, hqd, ht, gqT.to(sim.dtype).double().numpy(),
                        gqdT.to(sim.dtype).double().numpy())
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], tg)
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], tg)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], tg)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), sel)
    check("gmass", np.concatenate([gmd[s] for s in sel]), np.concatenate([o["gm"][s] for s in sel]), tg)
    assert sim.status().sum() == 0


def test_headline_configuration_full_size_sampled():
    """The chain configuration at full size -- 4096 serial 7-DOF chains,
    T = 1000, FP32, k = 1, automatic kernel choice (the link-frame pipelined rollout and the
    world-aligned pipelined adjoint) --
    against the FP64 oracle on sampled systems: the final state of every 64th system
    and the last, and the gradients of the first, a middle and the last system (first
    tile, a middle tile, the ragged end of the slot order)."""
    from paper_2109_07719_gb300 import Simulator
    work = wl.config(2)
    B, T = work.model.n_systems, work.T
    assert (B, T) == (4096, 1000)
    sim = Simulator(work.model, precision="fp32")
    dev = sim.device
    q0 = torch.tensor(work.q0, dtype=torch.float32)
    qd0 = torch.tensor(work.qd0, dtype=torch.float32)
    tau = work.tau().float()
    g = torch.Generator().manual_seed(41)
    gqT = torch.randn(q0.shape, generator=g, dtype=torch.float64).float()
    gqdT = torch.randn(qd0.shape, generator=g, dtype=torch.float64).float()
    qT, qdT, ck, _ = sim.rollout(q0.to(dev), qd0.to(dev), tau.to(dev), k=1)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau.to(dev), gqT.to(dev), gqdT.to(dev), k=1)
    torch.cuda.synchronize()
    assert sim.last_storage() == ("pipelined", "aligned_pipelined_shared")
    assert sim.status().sum() == 0
    h = [x.double().numpy() for x in (q0, qd0, tau, gqT, gqdT)]
    ts, tg = TOL["fp32"]
    sel = list(range(0, B, 64)) + [B - 1]
    oq, oqd = oracle_forward(work.model, sel, h[0], h[1], h[2])
    check("qT", qT.cpu().numpy()[:, sel], oq, ts)
    check("qdT", qdT.cpu().numpy()[:, sel], oqd, ts)
    gsel = [0, B // 2 - 1, B - 1]
    o = oracle_backward(work.model, gsel, h[0], h[1], h[2], h[3], h[4])
    check("gq0", gq0.cpu().numpy()[:, gsel], o["gq0"], tg)
    check("gqd0", gqd0.cpu().numpy()[:, gsel], o["gqd0"], tg)
    check("gtau", gtau.cpu().numpy()[:, :, gsel], o["gtau"], tg)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), gsel)
    check("gmass", np.concatenate([gmd[s] for s in gsel]), np.concatenate([o["gm"][s] for s in gsel]), tg)


@pytest.mark.parametrize("cfg", [2, 3])
def test_explicit_euler_fp64(cfg):
    B, T = 33, 50
    work = _work(cfg, B, T)
    sim = _sim(work, integrator="explicit")
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
    gqT = torch.ones_like(qT)
    gqdT = torch.zeros_like(qdT)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT, gqdT)
    oq, oqd = oracle_forward(work.model, list(range(B)), hq, hqd, ht, "explicit")
    check("qT", qT.cpu().numpy(), oq, 1e-8)
    sel = [0, 13, 32]
    o = oracle_backward(work.model, sel, hq, hqd, ht, np.ones_like(hq), np.zeros_like(hqd), "explicit")
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], 1e-6)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-6)


@pytest.mark.parametrize("cfg,k", [(2, 7), (2, 10), (3, 10), (4, 4), (5, 16)])
def test_checkpoint_interval_gives_same_gradients(cfg, k):
    """Segment replay from every k-th state reproduces the k = 1 gradients to
    round-off (the replay runs the same formulas inside another kernel, where the
    compiler may contract multiply-adds differently), with T not a multiple of k."""
    B, T = 41, 53
    work = _work(cfg, B, T)
    sim = _sim(work)
    (q0, qd0, tau), _ = _inputs(work, sim, T)
    qT, qdT, ck1, _ = sim.rollout(q0, qd0, tau, k=1)
    qTk, qdTk, ckk, _ = sim.rollout(q0, qd0, tau, k=k)
    assert torch.equal(qT, qTk) and torch.equal(qdT, qdTk)
    assert ckk.shape[0] == (T + k - 1) // k
    assert torch.equal(ckk, ck1[::k])
    gqT, gqdT = torch.ones_like(qT), -torch.ones_like(qdT)
    a = sim.backward(ck1, tau, gqT, gqdT, k=1)
    b = sim.backward(ckk, tau, gqT, gqdT, k=k)
    for name, x, y in zip(("gq0", "gqd0", "gtau", "gmass"), a, b):
        check(name, y.cpu().numpy(), x.cpu().numpy(), 1e-10)


def test_per_step_objective_terms():
    """g_traj adds dPhi/dx^t at every t: equals the sum of separate seeds."""
    B, T = 35, 30
    work = _work(2, B, T)
    sim = _sim(work)
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    qT, qdT, ck, traj = sim.rollout(q0, qd0, tau, traj=True)
    gt = torch.zeros_like(traj)
    t_mid = 11
    gt[t_mid, :sim.nq_max] = 1.0
    z = torch.zeros_like(qT)
    zd = torch.zeros_like(qdT)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, z, zd, g_traj=gt)
    # the same objective as a rollout of t_mid steps with a terminal seed
    qm, qdm, ckm, _ = sim.rollout(q0, qd0, tau[:t_mid].contiguous())
    ref = sim.backward(ckm, tau[:t_mid].contiguous(), torch.ones_like(qm), zd)
    assert torch.allclose(gq0, ref[0], rtol=1e-12, atol=1e-12)
    assert torch.allclose(gtau[:t_mid], ref[2], rtol=1e-12, atol=1e-12)
    assert torch.count_nonzero(gtau[t_mid:]) == 0


def test_fp32_path_error_report():
    """FP32 path vs the FP64 oracle on 7-DOF chains over 200 steps."""
    B, T = 70, 200
    work = _work(2, B, T, "fp32")
    sim = _sim(work, "fp32")
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
    gqT = torch.ones_like(qT)
    gqdT = torch.zeros_like(qdT)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT, gqdT)
    ts, tg = TOL["fp32"]
    oq, oqd = oracle_forward(work.model, list(range(B)), hq, hqd, ht)
    rep = {}
    check("qT", qT.cpu().numpy(), oq, ts, rep)
    check("qdT", qdT.cpu().numpy(), oqd, ts, rep)
    sel = [0, 31, 69]
    o = oracle_backward(work.model, sel, hq, hqd, ht, np.ones_like(hq), np.zeros_like(hqd))
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], tg, rep)
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], tg, rep)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], tg, rep)
    print("fp32 relative errors:", rep)


def test_zero_steps_and_single_system():
    work = _work(2, 1, 5)
    sim = _sim(work)
    (q0, qd0, tau), _ = _inputs(work, sim, 5)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau[:0].contiguous(), ckpt=False)
    assert torch.equal(qT, q0) and torch.equal(qdT, qd0)
    a = torch.ones_like(q0)
    b = torch.full_like(qd0, 2.0)
    ck = torch.empty(0, sim.nx, 1, dtype=sim.dtype, device=sim.device)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau[:0].contiguous(), a, b)
    assert torch.equal(gq0, a) and torch.equal(gqd0, b) and torch.count_nonzero(gm) == 0


def test_nonfinite_input_is_isolated_and_flagged():
    B, T = 40, 20
    work = _work(2, B, T)
    sim = _sim(work)
    (q0, qd0, tau), _ = _inputs(work, sim, T)
    clean = sim.rollout(q0, qd0, tau)
    assert sim.status().sum() == 0
    bad = tau.clone()
    bad[5, 3, 17] = float("nan")
    dirty = sim.rollout(q0, qd0, bad)
    flags = sim.status()
    assert flags[17] == 1 and flags.sum() == 1
    keep = [b for b in range(B) if b != 17]
    assert torch.equal(clean[0][:, keep], dirty[0][:, keep])
    sim.clear_status()
    assert sim.status().sum() == 0


def test_set_masses_matches_model_masses():
    B, T = 33, 25
    work = _work(3, B, T)
    sim = _sim(work)
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    m2 = work.model.mass * (1.0 + 0.2 * np.sin(np.arange(work.model.n_links_total)))
    sim.set_masses(torch.tensor(m2, device=sim.device))
    qT, qdT, _, _ = sim.rollout(q0, qd0, tau)
    work.model.mass[:] = m2
    oq, oqd = oracle_forward(work.model, list(range(B)), hq, hqd, ht)
    check("qT", qT.cpu().numpy(), oq, 1e-8)


def test_autograd_double_pendulum_full_horizon():
    """The double-pendulum workload as specified: FP64, 1000 steps, loss sum q_T^2,
    gradients w.r.t. q0, qd0 and every torque, through torch.autograd."""
    from paper_2109_07719_gb300 import Rollout
    work = wl.config(1)
    sim = _sim(work)
    q0 = torch.tensor(work.q0, device=sim.device, requires_grad=True)
    qd0 = torch.tensor(work.qd0, device=sim.device, requires_grad=True)
    tau = work.tau().to(sim.device).requires_grad_(True)
    qT, qdT = Rollout.apply(sim, q0, qd0, tau)
    (qT ** 2).sum().backward()
    hq, hqd, ht = work.q0, work.qd0, work.tau().numpy()
    oq, _ = oracle_forward(work.model, [0], hq, hqd, ht)
    check("qT", qT.detach().cpu().numpy(), oq, 1e-8)
    o = oracle_backward(work.model, [0], hq, hqd, ht, 2 * oq, np.zeros_like(hqd))
    check("gq0", q0.grad.cpu().numpy(), o["gq0"], 1e-6)
    check("gqd0", qd0.grad.cpu().numpy(), o["gqd0"], 1e-6)
    check("gtau", tau.grad.cpu().numpy(), o["gtau"], 1e-6)


@pytest.mark.parametrize("cfg", [2, 3, 5])
def test_fp32_with_fp64_d_solves(cfg):
    """SIM_FP32_D64: FP32 storage and arithmetic with the articulated-inertia D
    solves in FP64; same tolerances as the FP32 path."""
    B, T = 40, 100
    work = _work(cfg, B, T, "fp32_d64")
    sim = _sim(work, "fp32_d64")
    assert sim.dtype == torch.float32
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
    gqT = torch.ones_like(qT)
    gqdT = torch.zeros_like(qdT)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT, gqdT)
    ts, tg = TOL["fp32"]
    oq, oqd = oracle_forward(work.model, list(range(B)), hq, hqd, ht)
    rep = {}
    check("qT", qT.cpu().numpy(), oq, ts, rep)
    check("qdT", qdT.cpu().numpy(), oqd, ts, rep)
    sel = [0, 21, 39]
    o = oracle_backward(work.model, sel, hq, hqd, ht, np.ones_like(hq), np.zeros_like(hqd))
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], tg, rep)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], tg, rep)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), sel)
    check("gmass", np.concatenate([gmd[s] for s in sel]), np.concatenate([o["gm"][s] for s in sel]), tg, rep)
    print(f"fp32_d64 cfg {cfg} relative errors:", rep)


@pytest.mark.parametrize("cfg,k", [(2, 7), (3, 10)])
def test_quadratic_replay_gives_same_gradients(cfg, k):
    """The supplement's recompute-from-checkpoint scheme and the one-pass segment
    replay give the same gradients (to round-off), T not a multiple of k."""
    B, T = 37, 53
    work = _work(cfg, B, T)
    sim = _sim(work)
    (q0, qd0, tau), _ = _inputs(work, sim, T)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=k)
    gqT, gqdT = torch.ones_like(qT), -torch.ones_like(qdT)
    a = sim.backward(ck, tau, gqT, gqdT, k=k)
    sim.set_replay("quadratic")
    b = sim.backward(ck, tau, gqT, gqdT, k=k)
    sim.set_replay("segment")
    for name, x, y in zip(("gq0", "gqd0", "gtau", "gmass"), a, b):
        check(name, y.cpu().numpy(), x.cpu().numpy(), 1e-10)


@pytest.mark.parametrize("cfg", [2, 4])
def test_joint_damping_fp64(cfg):
    """Viscous joint damping (joint force tau - b qd) forward and adjoint."""
    B, T = 37, 60
    work = _work(cfg, B, T)
    work.model = work.model.with_damping(seed=cfg + 20)
    sim = _sim(work)
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
    gqT = torch.ones_like(qT)
    gqdT = torch.ones_like(qdT)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT, gqdT)
    oq, oqd = oracle_forward(work.model, list(range(B)), hq, hqd, ht)
    check("qT", qT.cpu().numpy(), oq, 1e-8)
    check("qdT", qdT.cpu().numpy(), oqd, 1e-8)
    sel = [0, 17, 36]
    o = oracle_backward(work.model, sel, hq, hqd, ht, np.ones_like(hq), np.ones_like(hqd))
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], 1e-6)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-6)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), sel)
    check("gmass", np.concatenate([gmd[s] for s in sel]), np.concatenate([o["gm"][s] for s in sel]), 1e-6)


def test_trajectory_objective_through_autograd():
    """A per-step cost sum_t |q^t|^2 + |qd^t|^2 through RolloutTrajectory equals
    the oracle's gradient of the same objective (per-step seeds g_traj)."""
    from paper_2109_07719_gb300 import RolloutTrajectory
    B, T = 9, 40
    work = _work(2, B, T)
    sim = _sim(work)
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    q0.requires_grad_(True)
    tau.requires_grad_(True)
    mass = torch.tensor(work.model.mass, device=sim.device, requires_grad=True)
    traj = RolloutTrajectory.apply(sim, q0, qd0, tau, mass, 1)
    (traj ** 2).sum().backward()
    from oracle.dynamics import OracleModel
    from oracle.rollout import rollout, rollout_backward
    om = OracleModel(work.model, list(range(B)))
    oq = torch.tensor(hq[:om.nq].T)
    oqd = torch.tensor(hqd[:om.nv].T)
    ot = torch.tensor(ht).permute(0, 2, 1).contiguous()
    with torch.no_grad():
        _, _, otraj = rollout(om, oq, oqd, ot)
    g_traj = [(2 * x[0], 2 * x[1]) for x in otraj]
    g = rollout_backward(om, oq, oqd, ot, torch.zeros_like(oq), torch.zeros_like(oqd), g_traj=g_traj)
    check("gq0", q0.grad.cpu().numpy()[:om.nq].T, g[0].numpy(), 1e-6)
    check("gtau", tau.grad.cpu().numpy().transpose(0, 2, 1), g[2].numpy(), 1e-6)
    gm = mass.grad.cpu().numpy().reshape(B, om.N)
    check("gmass", gm, g[3].numpy(), 1e-6)


def test_maximum_link_count():
    """Systems at the 255-link limit (a serial chain), mixed with short ones."""
    import numpy as np
    work = wl.config(4, B=34, T=6, dof_lo=250, dof_hi=255, precision="fp64")
    sim = _sim(work)
    assert sim.n_links == int(np.diff(work.model.sys_link_offset).sum())
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, 6)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, torch.ones_like(qT), torch.zeros_like(qdT))
    sel = [0, 33]
    oq, oqd = oracle_forward(work.model, sel, hq, hqd, ht, fd="aba")
    check("qT", qT.cpu().numpy()[:, sel], oq, 1e-8)
    check("qdT", qdT.cpu().numpy()[:, sel], oqd, 1e-8)
    o = oracle_backward(work.model, sel[:1], hq, hqd, ht, np.ones_like(hq), np.zeros_like(hqd), fd="aba")
    check("gtau", gtau.cpu().numpy()[:, :, sel[:1]], o["gtau"], 1e-6)


def test_call_argument_errors_are_reported():
    from paper_2109_07719_gb300 import SimError, lib
    work = _work(2, 4, 3)
    sim = _sim(work)
    (q0, qd0, tau), _ = _inputs(work, sim, 3)
    with pytest.raises(SimError):
        sim.rollout(q0.float(), qd0, tau)                      # wrong dtype
    with pytest.raises(SimError):
        sim.step(q0, qd0, tau)                                  # wrong torque shape
    assert lib.sim_rollout(sim._h, None, None, None, 3, 1, None, None, None, None, None) == -1
    assert lib.sim_rollout(sim._h, q0.data_ptr(), qd0.data_ptr(), tau.data_ptr(), 3, 0, None,
                           q0.data_ptr(), qd0.data_ptr(), None, None) == -1      # k < 1
    assert b"k >= 1" in lib.sim_last_error(sim._h)
    with pytest.raises(SimError, match="workspace"):
        qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=2)
        sim.backward(ck, tau, qT, qdT, k=2, work=torch.empty(1, dtype=torch.uint8, device=sim.device))
