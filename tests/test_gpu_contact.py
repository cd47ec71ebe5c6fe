"""GPU parity of the constraint path (sphere contacts against the ground plane
and revolute joint limits, the MLCP of Sec. 3.1 Eq. 8 solved by projected
Gauss-Seidel) and of its adjoint, through the C ABI, against the CPU FP64 oracle.

Inputs: the floating-base quadruped (13 links, a 2 cm sphere on each foot) with
straight legs, its base lowered so that in some systems the lowest foot starts
4 mm inside the ground and in the others 2-9 mm above it, falling at 1 m/s, so
contacts are active from step 0 in some systems and appear during the rollout
in others.  Joint limits: 7-DOF chains with every other joint limited to
[-0.4, 0.4] and q0 ~ U(-1, 1), and the quadrupeds with knee and hip-pitch
limits that the straight legs violate.  The batches span two 32-system blocks
with a ragged tail.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.contact import contact_points
from oracle.dynamics import OracleModel
from tests._parity import oracle_forward, oracle_backward, check, mass_grad_of

pytestmark = pytest.mark.gpu


def _touching(B=37, T=25, seed=0):
    """Workload and FP64 host inputs (q0, qd0, tau) of the falling quadrupeds."""
    work = wl.config(3, B=B, T=T, contacts=True, precision="fp64")
    om = OracleModel(work.model, list(range(B)))
    q = torch.tensor(work.q0.T).clone()
    q[:, 7:] = 0.0
    _, phi = contact_points(om, q)
    g = torch.Generator().manual_seed(seed)
    clearance = torch.where(torch.arange(B) % 3 == 0, torch.full((B,), -0.004),
                            0.002 + 0.007 * torch.rand(B, generator=g, dtype=torch.float64))
    q[:, 2] -= phi.min(1).values - clearance
    qd = 0.2 * torch.randn(B, om.nv, generator=g, dtype=torch.float64)
    qd[:, 3:6] = 0.0
    qd[:, 5] = -1.0          # body-frame z: the bases start level, so this is downward
    q0 = np.ascontiguousarray(q.numpy().T)
    qd0 = np.ascontiguousarray(qd.numpy().T)
    tau = work.tau(T=T).numpy()
    return work, q0, qd0, tau


def _sim(work, precision="fp64"):
    from paper_2109_07719_gb300 import Simulator
    return Simulator(work.model, precision=precision)


def _dev(sim, *xs):
    return [torch.tensor(x).to(sim.dtype).to(sim.device).contiguous() for x in xs]


def test_contacts_are_exercised():
    """The input recipe gives contacts from step 0 and contacts that appear later."""
    work, q0, qd0, tau = _touching()
    om = OracleModel(work.model, list(range(work.model.n_systems)))
    _, phi0 = contact_points(om, torch.tensor(q0.T))
    qT, _ = oracle_forward(work.model, list(range(work.model.n_systems)), q0, qd0, tau)
    _, phiT = contact_points(om, torch.tensor(qT.T))
    touching0 = (phi0 < 0).any(1)
    assert 0 < int(touching0.sum()) < work.model.n_systems
    assert bool(((phiT < 0).any(1) & ~touching0).any())


def test_contact_rollout_and_adjoint_fp64():
    work, q0, qd0, tau = _touching()
    B = work.model.n_systems
    sim = _sim(work)
    dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
    qT, qdT, ck, _ = sim.rollout(dq0, dqd0, dtau, k=1)
    g = torch.Generator().manual_seed(11)
    gqT = torch.randn(qT.shape, generator=g, dtype=torch.float64)
    gqdT = torch.randn(qdT.shape, generator=g, dtype=torch.float64)
    gq0, gqd0, gtau, gm = sim.backward(ck, dtau, gqT.to(sim.device), gqdT.to(sim.device), k=1)
    torch.cuda.synchronize()
    systems = list(range(B))
    oq, oqd = oracle_forward(work.model, systems, q0, qd0, tau)
    check("qT", qT.cpu().numpy(), oq, 1e-8)
    check("qdT", qdT.cpu().numpy(), oqd, 1e-8)
    sel = [0, 1, 2, 3, 31, 32, 36]   # both kinds of system, both blocks, the ragged tail
    o = oracle_backward(work.model, sel, q0, qd0, tau, gqT.numpy(), gqdT.numpy())
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], 1e-6)
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], 1e-6)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-6)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), sel)
    check("gmass", np.concatenate([gmd[s] for s in sel]), np.concatenate([o["gm"][s] for s in sel]), 1e-6)
    assert sim.status().sum() == 0


def test_contact_single_step_fp64():
    work, q0, qd0, tau = _touching(B=40, T=1, seed=4)
    sim = _sim(work)
    dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
    q1, qd1 = sim.step(dq0, dqd0, dtau[0])
    torch.cuda.synchronize()
    oq, oqd = oracle_forward(work.model, list(range(40)), q0, qd0, tau)
    check("q1", q1.cpu().numpy(), oq, 1e-12)
    check("qd1", qd1.cpu().numpy(), oqd, 1e-10)


@pytest.mark.parametrize("replay,k", [("segment", 6), ("quadratic", 5)])
def test_contact_checkpoint_replay(replay, k):
    """Replaying contact steps from every k-th state reproduces the k = 1
    gradients to round-off."""
    work, q0, qd0, tau = _touching(B=35, T=23, seed=2)
    sim = _sim(work)
    dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
    qT, qdT, ck1, _ = sim.rollout(dq0, dqd0, dtau, k=1)
    _, _, ckk, _ = sim.rollout(dq0, dqd0, dtau, k=k)
    gqT, gqdT = torch.ones_like(qT), -torch.ones_like(qdT)
    a = sim.backward(ck1, dtau, gqT, gqdT, k=1)
    sim.set_replay(replay)
    b = sim.backward(ckk, dtau, gqT, gqdT, k=k)
    for name, x, y in zip(("gq0", "gqd0", "gtau", "gmass"), a, b):
        check(name, y.cpu().numpy(), x.cpu().numpy(), 1e-10)


@pytest.mark.parametrize("precision", ["fp32", "fp32_d64"])
def test_contact_fp32(precision):
    """FP32 storage (and FP32 with FP64 D-solves) through contact steps against
    the FP64 oracle: states within 1e-3, gradients within 1e-2 (relative, max-norm)."""
    work, q0, qd0, tau = _touching(B=37, T=25, seed=6)
    sim = _sim(work, precision)
    dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
    hq0, hqd0, htau = [x.double().cpu().numpy() for x in (dq0, dqd0, dtau)]
    qT, qdT, ck, _ = sim.rollout(dq0, dqd0, dtau)
    gqT = torch.ones_like(qT)
    gqdT = torch.ones_like(qdT)
    gq0, gqd0, gtau, gm = sim.backward(ck, dtau, gqT, gqdT)
    oq, oqd = oracle_forward(work.model, list(range(37)), hq0, hqd0, htau)
    check("qT", qT.cpu().numpy(), oq, 1e-3)
    check("qdT", qdT.cpu().numpy(), oqd, 1e-3)
    sel = [0, 4, 36]
    o = oracle_backward(work.model, sel, hq0, hqd0, htau, np.ones_like(hq0), np.ones_like(hqd0))
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], 1e-2)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-2)


def test_separated_spheres_change_nothing():
    """Spheres that never reach the ground leave states and gradients equal (to
    round-off) to those of the same model without spheres."""
    work = wl.config(3, B=33, T=30, contacts=True, precision="fp64")
    free = wl.config(3, B=33, T=30, precision="fp64")
    q0, qd0 = work.q0.copy(), work.qd0
    q0[2] += 10.0            # the base 10.5 m up: the feet stay far above the ground
    tau = work.tau().numpy()
    outs = []
    for w in (work, free):
        sim = _sim(w)
        dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
        qT, qdT, ck, _ = sim.rollout(dq0, dqd0, dtau)
        outs.append((qT, qdT) + tuple(sim.backward(ck, dtau, torch.ones_like(qT), torch.ones_like(qdT))))
    for name, x, y in zip(("qT", "qdT", "gq0", "gqd0", "gtau", "gmass"), *outs):
        check(name, x.cpu().numpy(), y.cpu().numpy(), 1e-12)


def test_jvp_of_contact_model_is_refused():
    from paper_2109_07719_gb300 import SimError
    work, q0, qd0, tau = _touching(B=4, T=1)
    sim = _sim(work)
    dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
    with pytest.raises(SimError, match="contact"):
        sim.jvp(dq0, dqd0, dtau[0], dq=torch.ones_like(dq0))


# ---------------------------------------------------------------- joint limits

def _limited_chains(B=37, T=40, seed=8):
    """7-DOF chains with every other joint limited to [-0.4, 0.4]: q0 ~ U(-1, 1)
    starts many joints outside their range, qd0 ~ N(0, 0.5^2)."""
    work = wl.config(2, B=B, T=T, precision="fp64")
    work.model = work.model.with_limits(-0.4, 0.4, every=2)
    g = np.random.default_rng(seed)
    qd0 = 0.5 * g.standard_normal(work.qd0.shape)
    return work, work.q0, qd0, work.tau().numpy()


def _with_leg_limits(work):
    """Knees limited to [-1, -0.02] (straight legs start above the range) and hip
    pitch to [-0.05, 0.05]."""
    md = work.model
    lim = np.tile(np.array([[-np.inf, np.inf]]), (md.n_links_total, 1))
    for b in range(md.n_systems):
        for leg in range(4):
            lim[md.sys_link_offset[b] + 3 + 3 * leg] = (-1.0, -0.02)
            lim[md.sys_link_offset[b] + 2 + 3 * leg] = (-0.05, 0.05)
    md.limits = lim
    return work


def _parity_fp64(work, q0, qd0, tau, sel, seed=13):
    sim = _sim(work)
    dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
    qT, qdT, ck, _ = sim.rollout(dq0, dqd0, dtau, k=1)
    g = torch.Generator().manual_seed(seed)
    gqT = torch.randn(qT.shape, generator=g, dtype=torch.float64)
    gqdT = torch.randn(qdT.shape, generator=g, dtype=torch.float64)
    gq0, gqd0, gtau, gm = sim.backward(ck, dtau, gqT.to(sim.device), gqdT.to(sim.device), k=1)
    torch.cuda.synchronize()
    oq, oqd = oracle_forward(work.model, list(range(work.model.n_systems)), q0, qd0, tau)
    check("qT", qT.cpu().numpy(), oq, 1e-8)
    check("qdT", qdT.cpu().numpy(), oqd, 1e-8)
    o = oracle_backward(work.model, sel, q0, qd0, tau, gqT.numpy(), gqdT.numpy())
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], 1e-6)
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], 1e-6)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-6)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), sel)
    check("gmass", np.concatenate([gmd[s] for s in sel]), np.concatenate([o["gm"][s] for s in sel]), 1e-6)
    assert sim.status().sum() == 0


def test_joint_limits_fp64():
    work, q0, qd0, tau = _limited_chains()
    _parity_fp64(work, q0, qd0, tau, [0, 5, 31, 32, 36])


def test_contacts_and_joint_limits_fp64():
    work, q0, qd0, tau = _touching(B=37, T=25, seed=9)
    work = _with_leg_limits(work)
    _parity_fp64(work, q0, qd0, tau, [0, 1, 3, 33, 36])


def test_joint_limits_checkpoint_replay():
    work, q0, qd0, tau = _limited_chains(B=35, T=29, seed=10)
    sim = _sim(work)
    dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
    qT, qdT, ck1, _ = sim.rollout(dq0, dqd0, dtau, k=1)
    _, _, ckk, _ = sim.rollout(dq0, dqd0, dtau, k=6)
    gqT, gqdT = torch.ones_like(qT), -torch.ones_like(qdT)
    a = sim.backward(ck1, dtau, gqT, gqdT, k=1)
    b = sim.backward(ckk, dtau, gqT, gqdT, k=6)
    for name, x, y in zip(("gq0", "gqd0", "gtau", "gmass"), a, b):
        check(name, y.cpu().numpy(), x.cpu().numpy(), 1e-10)


def test_joint_limits_fp32():
    work, q0, qd0, tau = _limited_chains(B=37, T=40, seed=12)
    sim = _sim(work, "fp32")
    dq0, dqd0, dtau = _dev(sim, q0, qd0, tau)
    hq0, hqd0, htau = [x.double().cpu().numpy() for x in (dq0, dqd0, dtau)]
    qT, qdT, ck, _ = sim.rollout(dq0, dqd0, dtau)
    gq0, gqd0, gtau, gm = sim.backward(ck, dtau, torch.ones_like(qT), torch.ones_like(qdT))
    oq, oqd = oracle_forward(work.model, list(range(37)), hq0, hqd0, htau)
    check("qT", qT.cpu().numpy(), oq, 1e-3)
    check("qdT", qdT.cpu().numpy(), oqd, 1e-3)
    sel = [0, 9, 36]
    o = oracle_backward(work.model, sel, hq0, hqd0, htau, np.ones_like(hq0), np.ones_like(hqd0))
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], 1e-2)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-2)
