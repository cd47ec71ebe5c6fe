"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test ties the oracle to something other than its own code: an independent
algorithm (CRBA+RNEA vs ABA), a textbook closed form (compound and double
pendulum), a conservation law (power balance, momentum), a small-angle period,
finite differences, forward-mode AD of the rollout (the dot-product test of the
adjoint recurrence), and the paper's printed adjoint rule of its worked example
(Sec. 3.1, Eq. 5-6).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from oracle.dynamics import OracleModel
from oracle.rollout import step, rollout, rollout_backward

torch.set_num_threads(1)


@pytest.fixture(autouse=True)
def _fp64_default_dtype():
    """FP64 as torch's default dtype for this module's tests only (restored after
    each test, so GPU tests collected later see the usual float32 default)."""
    prev = torch.get_default_dtype()
    torch.set_default_dtype(torch.float64)
    yield
    torch.set_default_dtype(prev)
G = 9.81


def _single_link(mass=1.0, l=1.0, g=(0.0, -G, 0.0), dt=1e-3):
    """One thin rod of length l on a revolute z joint, hanging along -y."""
    return wl.ModelDesc(np.array([0, 1], np.int32), np.array([-1], np.int32),
                        np.array([wl.REVOLUTE], np.int32), np.array([[0.0, 0, 1]]),
                        np.array([[1.0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]]), np.array([mass]),
                        np.array([[0.0, -l / 2, 0]]),
                        np.array([[mass * l * l / 12, 0, mass * l * l / 12, 0, 0, 0]]),
                        dt, np.array(g), "single_link")


def _om(work, systems=None):
    m = work.model
    systems = range(m.n_systems) if systems is None else systems
    return OracleModel(m, systems)


def _state(work, om, systems=None, seed=0):
    systems = list(range(work.model.n_systems)) if systems is None else list(systems)
    q = torch.tensor(work.q0[:om.nq, systems].T)
    g = torch.Generator().manual_seed(seed)
    qd = torch.randn(len(systems), om.nv, generator=g)
    tau = torch.randn(len(systems), om.nv, generator=g)
    return q, qd, tau


# ----------------------------------------------------------------- dynamics

@pytest.mark.parametrize("cfg", [1, 2, 3, 4, 5])
def test_aba_equals_crba_rnea(cfg):
    """Two independent algorithms for qdd agree to round-off."""
    work = wl.config(cfg, B=4) if cfg != 4 else wl.config(4, B=6, dof_hi=20)
    for s in range(work.model.n_systems):
        om = _om(work, [s])
        q, qd, tau = _state(work, om, [s], seed=s)
        a = oracle.fd_crba(om, q, qd, tau)
        b = oracle.aba(om, q, qd, tau)
        assert torch.allclose(a, b, rtol=1e-10, atol=1e-10 * a.abs().max())


def test_compound_pendulum_closed_form():
    """qdd = (tau - m g l_c sin q) / I_pivot, I_pivot = m l^2/3, l_c = l/2."""
    om = OracleModel(_single_link(mass=1.7, l=0.8), [0])
    q = torch.linspace(-3, 3, 13)[:, None]
    for qi in q:
        tau = torch.tensor([[0.37]])
        qdd = oracle.fd_crba(om, qi[None], torch.tensor([[2.0]]), tau)
        ip = 1.7 * 0.8 ** 2 / 3
        expect = (0.37 - 1.7 * G * 0.4 * math.sin(qi.item())) / ip
        assert abs(qdd.item() - expect) < 1e-12
        assert abs(oracle.aba(om, qi[None], torch.tensor([[2.0]]), tau).item() - expect) < 1e-12


def test_double_pendulum_textbook():
    """Planar double pendulum with rods: hand-written M(q), Coriolis and gravity."""
    work = wl.config(1, B=1)
    om = _om(work)
    m, l, lc, Ic = 1.0, 1.0, 0.5, 1.0 / 12
    rng = np.random.default_rng(5)
    for _ in range(10):
        t1, t2, d1, d2, u1, u2 = rng.uniform(-2, 2, 6)
        M = np.array([[2 * Ic + m * lc ** 2 + m * (l ** 2 + lc ** 2 + 2 * l * lc * math.cos(t2)),
                       Ic + m * (lc ** 2 + l * lc * math.cos(t2))],
                      [Ic + m * (lc ** 2 + l * lc * math.cos(t2)), Ic + m * lc ** 2]])
        h = -m * l * lc * math.sin(t2)
        C = np.array([h * (2 * d1 * d2 + d2 ** 2), -h * d1 ** 2])
        Gv = np.array([m * G * lc * math.sin(t1) + m * G * (l * math.sin(t1) + lc * math.sin(t1 + t2)),
                       m * G * lc * math.sin(t1 + t2)])
        expect = np.linalg.solve(M, np.array([u1, u2]) - C - Gv)
        q = torch.tensor([[t1, t2]])
        qd = torch.tensor([[d1, d2]])
        tau = torch.tensor([[u1, u2]])
        assert np.allclose(oracle.crba(om, q)[0].numpy(), M, atol=1e-13)
        assert np.allclose(oracle.fd_crba(om, q, qd, tau)[0].numpy(), expect, atol=1e-11)
        assert np.allclose(oracle.aba(om, q, qd, tau)[0].numpy(), expect, atol=1e-11)


def test_small_angle_period():
    """Period of the compound pendulum -> 2 pi sqrt(2 l / (3 g)) as amplitude -> 0."""
    om = OracleModel(_single_link(), [0])
    q = torch.tensor([[1e-3]])
    qd = torch.zeros(1, 1)
    tau = torch.zeros(1, 1)
    crossings = []
    prev = q.item()
    t = 0
    while len(crossings) < 21:
        q, qd = step(om, q, qd, tau)
        t += 1
        cur = q.item()
        if prev > 0 >= cur or prev < 0 <= cur:
            crossings.append((t - 1) + prev / (prev - cur))
        prev = cur
    period = 2 * (crossings[-1] - crossings[0]) / (len(crossings) - 1) * om.dt
    expect = 2 * math.pi * math.sqrt(2 * 1.0 / (3 * G))
    assert abs(period - expect) / expect < 1e-3


def _power_balance(om, q, qd, tau, s=1e-5):
    """(E(step(+s)) - E(step(-s))) / 2s, the rate of change of energy along the flow."""
    dt0 = om.dt
    om.dt = s
    qp, qdp = step(om, q, qd, tau)
    om.dt = -s
    qm, qdm = step(om, q, qd, tau)
    om.dt = dt0
    return (oracle.energy(om, qp, qdp) - oracle.energy(om, qm, qdm)) / (2 * s)


@pytest.mark.parametrize("cfg", [1, 2, 3, 5])
def test_power_balance(cfg):
    """dE/dt = qd . tau: joint torques are the only source of work."""
    work = wl.config(cfg, B=3) if cfg != 1 else wl.config(1, B=1)
    om = _om(work)
    q, qd, tau = _state(work, om, seed=cfg)
    if cfg in (3, 5):
        tau[:, :6] = 0.0  # the base is unactuated
        q[:, 3:7] = q[:, 3:7] + 0.1 * torch.randn(q.shape[0], 4)
        q[:, 3:7] = q[:, 3:7] / q[:, 3:7].norm(dim=1, keepdim=True)
    rate = _power_balance(om, q, qd, tau)
    power = (qd * tau).sum(1)
    scale = 1 + power.abs().max()
    assert torch.allclose(rate, power, atol=1e-6 * scale), (rate, power)


@pytest.mark.parametrize("cfg", [2, 3])
def test_damped_power_balance(cfg):
    """With viscous joint damping b: dE/dt = qd . tau - sum b qd^2."""
    work = wl.config(cfg, B=3)
    work.model = work.model.with_damping(seed=cfg)
    om = _om(work)
    q, qd, tau = _state(work, om, seed=cfg + 10)
    if cfg == 3:
        tau[:, :6] = 0.0
    rate = _power_balance(om, q, qd, tau)
    power = (qd * tau).sum(1) - (om.damping * qd * qd).sum(1)
    assert (om.damping > 0).any()
    assert torch.allclose(rate, power, atol=1e-6 * (1 + power.abs().max())), (rate, power)


@pytest.mark.parametrize("cfg", [3, 5])
def test_momentum_conservation_rate(cfg):
    """With g = 0 and an unactuated base, joint torques are internal: dh/dt = 0."""
    work = wl.config(cfg, B=2)
    work.model.gravity[:] = 0.0
    om = _om(work)
    q, qd, tau = _state(work, om, seed=11)
    tau[:, :6] = 0.0
    s = 1e-5
    om.dt = s
    qp, qdp = step(om, q, qd, tau)
    om.dt = -s
    qm, qdm = step(om, q, qd, tau)
    rate = (oracle.spatial_momentum(om, qp, qdp) - oracle.spatial_momentum(om, qm, qdm)) / (2 * s)
    h = oracle.spatial_momentum(om, q, qd)
    assert rate.abs().max() < 1e-6 * (1 + h.abs().max())
    # and a torque on the base does change it
    tau[:, 3] = 1.0
    om.dt = s
    qp, qdp = step(om, q, qd, tau)
    om.dt = -s
    qm, qdm = step(om, q, qd, tau)
    rate = (oracle.spatial_momentum(om, qp, qdp) - oracle.spatial_momentum(om, qm, qdm)) / (2 * s)
    assert rate.abs().max() > 0.5


def _energy_deviation(work, om, steps, every=10, integrator="semi"):
    q = torch.tensor(work.q0.T)
    qd = torch.zeros(q.shape[0], om.nv)
    tau = torch.zeros(q.shape[0], om.nv)
    E0 = oracle.energy(om, q, qd)
    scale = float(om.mass.sum(1).max()) * G * 1.0   # m g l with l = 1 m
    dev = []
    for t in range(steps):
        q, qd = step(om, q, qd, tau, integrator)
        if t % every == 0:
            dev.append((oracle.energy(om, q, qd) - E0).abs().max().item() / scale)
    return np.array(dev)


def test_bounded_energy_drift():
    """Semi-implicit Euler on the frictionless, unforced double pendulum keeps the
    energy error under 0.5% of m g l over 1e4 steps at dt = 1e-3, while plain
    explicit Euler gains energy several times faster.  (In velocity form with a
    configuration-dependent M the scheme is not symplectic, so the bound is first
    order in dt rather than drift-free; see the dt-scaling test.)"""
    work = wl.config(1, B=1)
    om = _om(work)
    dev = _energy_deviation(work, om, 10000, every=50)
    assert dev.max() < 5e-3
    dev_x = _energy_deviation(work, om, 2000, every=50, integrator="explicit")
    assert dev_x.max() > 3 * dev[:40].max()


@pytest.mark.parametrize("cfg,steps", [(1, 1500), (2, 400)])
def test_energy_error_first_order_in_dt(cfg, steps):
    """Halving dt halves the energy error over the same interval (first-order method)."""
    work = wl.config(cfg, B=1)
    om = _om(work)
    d1 = _energy_deviation(work, om, steps, every=5).max()
    om.dt = om.dt / 2
    d2 = _energy_deviation(work, om, 2 * steps, every=10).max()
    assert 1.6 < d1 / d2 < 2.4, (d1, d2)


# ---------------------------------------------------------------- gradients

def _loss_and_grads(om, q0, qd0, tau, wq, wqd, integrator="semi"):
    def phi(q0_, qd0_, tau_, m_):
        qT, qdT, _ = rollout(om, q0_, qd0_, tau_, integrator, mass=m_, keep=False)
        return (qT ** 2).sum() + (wq * qT).sum() + (wqd * qdT).sum()
    with torch.no_grad():
        qT, qdT, _ = rollout(om, q0, qd0, tau, integrator, keep=False)
    g = rollout_backward(om, q0, qd0, tau, 2 * qT + wq, wqd, integrator=integrator)
    return phi, g


@pytest.mark.parametrize("cfg,T,integrator,damped", [(1, 40, "semi", False), (2, 15, "semi", False),
                                                     (3, 10, "semi", False), (5, 6, "semi", False),
                                                     (2, 10, "explicit", False), (2, 12, "semi", True)])
def test_adjoint_matches_central_fd(cfg, T, integrator, damped):
    """Gradients w.r.t. q0, qd0, tau and link masses vs central differences along
    random directions (FP64, h = 1e-6: truncation O(h^2))."""
    work = wl.config(cfg, B=2) if cfg != 1 else wl.config(1, B=1)
    if damped:
        work.model = work.model.with_damping(seed=4)
    om = _om(work)
    q0, qd0, _ = _state(work, om, seed=3)
    gen = torch.Generator().manual_seed(9)
    tau = torch.randn(T, om.B, om.nv, generator=gen)
    wq = torch.randn(om.B, om.nq, generator=gen)
    wqd = torch.randn(om.B, om.nv, generator=gen)
    phi, (gq0, gqd0, gtau, gm) = _loss_and_grads(om, q0, qd0, tau, wq, wqd, integrator)
    m0 = om.mass.clone()
    h = 1e-6
    for k in range(3):
        dq = torch.randn(q0.shape, generator=gen)
        dqd = torch.randn(qd0.shape, generator=gen)
        dtau = torch.randn(tau.shape, generator=gen)
        dm = torch.randn(m0.shape, generator=gen) * 0.1
        if cfg in (3, 5):
            dq[:, 3:7] = 0.0  # keep the quaternion on the unit sphere
        fd = (phi(q0 + h * dq, qd0 + h * dqd, tau + h * dtau, m0 + h * dm)
              - phi(q0 - h * dq, qd0 - h * dqd, tau - h * dtau, m0 - h * dm)) / (2 * h)
        an = (gq0 * dq).sum() + (gqd0 * dqd).sum() + (gtau * dtau).sum() + (gm * dm).sum()
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k, fd.item(), an.item())


def test_adjoint_closed_form_free_rod():
    """One rod on a revolute joint, no gravity: qdd = tau / I_pivot, so with
    semi-implicit Euler q_T = q0 + T dt qd0 + dt^2/I sum_t (T - t) tau_t."""
    mass, l, T = 1.3, 0.9, 25
    om = OracleModel(_single_link(mass=mass, l=l, g=(0.0, 0.0, 0.0)), [0])
    gen = torch.Generator().manual_seed(1)
    tau = torch.randn(T, 1, 1, generator=gen)
    q0 = torch.tensor([[0.2]])
    qd0 = torch.tensor([[0.5]])
    gq0, gqd0, gtau, gm = rollout_backward(om, q0, qd0, tau, torch.ones(1, 1), torch.zeros(1, 1))
    dt = om.dt
    ip = mass * l * l / 3
    t = torch.arange(T, dtype=torch.float64)
    assert abs(gq0.item() - 1.0) < 1e-14
    assert abs(gqd0.item() - T * dt) < 1e-14
    assert torch.allclose(gtau[:, 0, 0], dt * dt * (T - t) / ip, rtol=1e-12)
    # mass enters with the COM and the rotational inertia about it held fixed,
    # so dI_pivot/dm = l_c^2 = l^2/4
    s = (dt * dt * (T - t) * tau[:, 0, 0]).sum()
    expect = -s / ip ** 2 * (l / 2) ** 2
    assert abs(gm.item() - expect) < 1e-12 * abs(expect)


def test_crossf_adjoint_matches_worked_example():
    """Sec. 3.1 worked example: p = f + v x* h with motion v = (w1, v1) and force
    h = (w2, v2); the pull-back of (wbar, vbar) printed in Eq. 6."""
    gen = torch.Generator().manual_seed(2)
    v = torch.randn(6, generator=gen, requires_grad=True)
    hf = torch.randn(6, generator=gen, requires_grad=True)
    f = torch.randn(6, generator=gen, requires_grad=True)
    pbar = torch.randn(6, generator=gen)
    p = f + oracle.crossf(v) @ hf
    gv, gh, gf = torch.autograd.grad(p, (v, hf, f), pbar)
    w1, v1, w2, v2 = v[:3].detach(), v[3:].detach(), hf[:3].detach(), hf[3:].detach()
    wb, vb = pbar[:3], pbar[3:]
    cr = torch.linalg.cross
    assert torch.allclose(gv[:3], -cr(wb, w2) - cr(vb, v2))
    assert torch.allclose(gv[3:], -cr(wb, v2))
    assert torch.allclose(gh[:3], cr(wb, w1))
    assert torch.allclose(gh[3:], cr(wb, v1) + cr(vb, w1))
    assert torch.allclose(gf, pbar)


def test_plucker_transform_matches_st_apply():
    """The oracle's 6x6 motion transform equals the supplement's st_apply formula
    [E a1; E (a2 - r x a1)] and its transpose equals st_apply_trans."""
    gen = torch.Generator().manual_seed(4)
    E = torch.linalg.qr(torch.randn(3, 3, generator=gen))[0]
    r = torch.randn(3, generator=gen)
    a = torch.randn(6, generator=gen)
    X = oracle.xform(E, r)
    b = X @ a
    assert torch.allclose(b[:3], E @ a[:3])
    assert torch.allclose(b[3:], E @ (a[3:] - torch.linalg.cross(r, a[:3])))
    bt = X.T @ a
    assert torch.allclose(bt[:3], E.T @ a[:3] + torch.linalg.cross(r, E.T @ a[3:]))
    assert torch.allclose(bt[3:], E.T @ a[3:])


def test_quaternion_mul_vec_matches_supplement():
    """quat (x) (v, 0) written out component-wise as the supplement's mul_vec."""
    gen = torch.Generator().manual_seed(6)
    q = torch.randn(4, generator=gen)
    v = torch.randn(3, generator=gen)
    r = oracle.quat_mul(q, torch.cat([v, torch.zeros(1)]))
    x, y, z, w = q
    expect = torch.stack([w * v[0] + y * v[2] - z * v[1], w * v[1] + z * v[0] - x * v[2],
                          w * v[2] + x * v[1] - y * v[0], -x * v[0] - y * v[1] - z * v[2]])
    assert torch.allclose(r, expect)


@pytest.mark.parametrize("cfg,T,integrator", [(1, 30, "semi"), (2, 10, "semi"), (2, 8, "explicit"),
                                              (3, 6, "semi"), (5, 4, "semi")])
def test_adjoint_dot_product_with_forward_mode(cfg, T, integrator):
    """The oracle's adjoint recurrence against forward-mode AD of its own rollout
    (torch.func.jvp, a differentiation mode the recurrence does not use):
    <ybar, J xdot> = <J^T ybar, xdot> for random tangents of q0, qd0, every tau and
    the link masses, to round-off -- no finite-difference truncation."""
    work = wl.config(cfg, B=2) if cfg != 1 else wl.config(1, B=1)
    om = _om(work)
    q0, qd0, _ = _state(work, om, seed=5)
    gen = torch.Generator().manual_seed(11)
    tau = torch.randn(T, om.B, om.nv, generator=gen)
    wq = torch.randn(om.B, om.nq, generator=gen)
    wqd = torch.randn(om.B, om.nv, generator=gen)
    m0 = om.mass.clone()
    dq = torch.randn(q0.shape, generator=gen)
    dqd = torch.randn(qd0.shape, generator=gen)
    dtau = torch.randn(tau.shape, generator=gen)
    dm = 0.1 * torch.randn(m0.shape, generator=gen)

    def final_state(q, qd, ta, m):
        qT, qdT, _ = rollout(om, q, qd, ta, integrator, mass=m, keep=False)
        return qT, qdT

    _, (tq, tqd) = torch.func.jvp(final_state, (q0, qd0, tau, m0), (dq, dqd, dtau, dm))
    lhs = (wq * tq).sum() + (wqd * tqd).sum()
    gq0, gqd0, gtau, gm = rollout_backward(om, q0, qd0, tau, wq, wqd, integrator=integrator)
    rhs = (gq0 * dq).sum() + (gqd0 * dqd).sum() + (gtau * dtau).sum() + (gm * dm).sum()
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(rhs)), (lhs.item(), rhs.item())


def test_double_pendulum_gradient_by_brute_force():
    """The small-case configuration (one double pendulum, Phi = sum q_T^2, T = 1000):
    the oracle's gradient with respect to every one of its 2 + 2 + 2000 inputs
    (q0, qd0, every torque) against central differences, all 4008 perturbed rollouts
    run as the systems of one batched oracle rollout."""
    T, h = 1000, 1e-5
    base = wl.config(1, B=1, T=T)
    q0 = torch.tensor(base.q0[:, 0])
    qd0 = torch.tensor(base.qd0[:, 0])
    tau = base.tau(T=T)[:, :, 0]
    n_in = 4 + 2 * T
    B = 2 * n_in
    work = wl.config(1, B=B, T=T)
    assert np.array_equal(work.model.mass, np.tile(base.model.mass, B))   # one model, B copies
    om = OracleModel(work.model, range(B))
    x = torch.cat([q0, qd0, tau.reshape(-1)]).repeat(B, 1)
    i = torch.arange(n_in)
    x[2 * i, i] += h
    x[2 * i + 1, i] -= h
    qT, _, _ = rollout(om, x[:, :2], x[:, 2:4], x[:, 4:].reshape(B, T, 2).permute(1, 0, 2).contiguous(),
                       keep=False)
    phi = (qT ** 2).sum(1)
    fd = (phi[0::2] - phi[1::2]) / (2 * h)
    om1 = OracleModel(base.model, [0])
    qT1, qdT1, _ = rollout(om1, q0[None], qd0[None], tau[:, None, :], keep=False)
    gq0, gqd0, gtau, _ = rollout_backward(om1, q0[None], qd0[None], tau[:, None, :], 2 * qT1,
                                          torch.zeros_like(qdT1))
    an = torch.cat([gq0[0], gqd0[0], gtau[:, 0, :].reshape(-1)])
    assert float((fd - an).abs().max() / an.abs().max()) < 1e-7
