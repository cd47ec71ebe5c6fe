"""Pins of the oracle's contact resolution (Sec. 3.1 MLCP solved by projected
Gauss-Seidel) against closed forms and the complementarity conditions."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.contact import contact_points, contact_velocity_change, contact_jacobian
from oracle.dynamics import OracleModel, crba
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


def _ball(mass=2.0, radius=0.1, mu=0.5, erp=0.0, g=(0.0, 0.0, -9.81), dt=1e-3):
    """One free body with its COM at the body origin and a contact sphere there."""
    I = [0.02, 0.03, 0.04, 0.0, 0.0, 0.0]
    m = wl.ModelDesc(np.array([0, 1], np.int32), np.array([-1], np.int32),
                     np.array([wl.FREE], np.int32), np.zeros((1, 3)),
                     np.array([[1.0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]]), np.array([mass]),
                     np.zeros((1, 3)), np.array([I]), dt, np.array(g), "ball")
    m.contact = np.array([[0.0, 0.0, 0.0, radius]])
    m.friction, m.erp, m.pgs_iterations = mu, erp, 20
    return m


def _quat(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


@pytest.mark.parametrize("vt,expect_stick", [((0.05, -0.02), True), ((3.0, 1.0), False)])
def test_ball_impact_closed_form(vt, expect_stick):
    """A point-mass ball hitting the ground: A = 1/m, so the impulse is
    lambda_n = -m (v*_z + erp/dt phi) and the friction impulse is -m v*_t boxed
    by mu lambda_n, component by component."""
    mass, radius, mu, erp, dt = 2.0, 0.1, 0.5, 0.2, 1e-3
    om = OracleModel(_ball(mass, radius, mu, erp, dt=dt), [0])
    rng = np.random.default_rng(1)
    quat = _quat(rng)
    z = radius - 0.003                                   # 3 mm penetration
    q = torch.tensor([[0.1, -0.2, z, *quat]])
    R = torch.tensor(__import__("oracle").spatial.quat_to_R(torch.tensor(quat)).numpy())
    v_world = torch.tensor([vt[0], vt[1], -1.5])
    w_body = torch.zeros(3)       # no spin: no gyroscopic or body-frame coupling terms
    qd = torch.cat([w_body, R.T @ v_world])[None]
    tau = torch.zeros(1, 6)
    q1, qd1 = step(om, q, qd, tau)
    v_star = v_world + dt * torch.tensor([0.0, 0.0, -9.81])
    phi = z - radius
    ln = -mass * (v_star[2] + erp / dt * phi)
    lt = torch.clamp(-mass * v_star[:2], -mu * ln, mu * ln)
    v_expect = v_star + torch.cat([lt, ln[None]]) / mass
    v_got = R @ qd1[0, 3:]          # quaternion changes only by dt w: compare in the old frame
    assert torch.allclose(qd1[0, :3], w_body, atol=1e-12)
    assert torch.allclose(v_got, v_expect, atol=1e-12)
    if expect_stick:
        assert torch.allclose(v_got[:2], torch.zeros(2), atol=1e-12)
    else:
        assert abs(abs(float(lt[0])) - mu * float(ln)) < 1e-12


def test_no_contact_when_separated():
    """Contact spheres above the ground leave the step identical to the contact-free one."""
    work = wl.config(3, B=2, contacts=True)
    om = OracleModel(work.model, [0, 1])
    free = wl.config(3, B=2)
    om0 = OracleModel(free.model, [0, 1])
    q = torch.tensor(work.q0.T)
    qd = 0.1 * torch.randn(2, om.nv, generator=torch.Generator().manual_seed(0))
    tau = torch.randn(2, om.nv, generator=torch.Generator().manual_seed(1))
    tau[:, :6] = 0
    _, phi = contact_points(om, q)
    assert bool((phi > 0).all())
    a = step(om, q, qd, tau)
    b = step(om0, q, qd, tau)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def _touching_quadruped(B=3, seed=0, mu=0.8):
    work = wl.config(3, B=B, contacts=True)
    work.model.friction = mu
    om = OracleModel(work.model, list(range(B)))
    q = torch.tensor(work.q0.T)
    q[:, 7:] = 0.0                                    # legs straight down
    _, phi = contact_points(om, q)
    q[:, 2] -= phi.min(1).values + 0.004              # lowest foot 4 mm into the ground
    g = torch.Generator().manual_seed(seed)
    qd = 0.2 * torch.randn(B, om.nv, generator=g)
    qd[:, 5] = -1.0                                   # falling
    return work, om, q, qd


def test_pgs_solves_the_normal_lcp():
    """Frictionless, enough sweeps: lambda >= 0, a = A lambda + b >= 0 on active
    normals, lambda_n a_n = 0 (the LCP the MLCP reduces to)."""
    work, om, q, qd = _touching_quadruped(mu=0.0)
    om.pgs_iterations = 400
    dv, lam = contact_velocity_change(om, q, qd)
    _, phi = contact_points(om, q)
    active = phi < 0
    assert int(active.sum()) >= 4
    J = contact_jacobian(om, q)
    M = crba(om, q)
    A = J @ torch.linalg.solve(M, J.transpose(-1, -2))
    b = (J @ qd[..., None])[..., 0]
    b[:, 2::3] += om.erp / om.dt * torch.clamp(phi, max=0.0)
    a = (A @ lam[..., None])[..., 0] + b
    ln, an = lam[:, 2::3], a[:, 2::3]
    assert bool((ln >= 0).all())
    assert bool((an[active] > -1e-8).all())
    assert float((ln * an)[active].abs().max()) < 1e-8
    assert float(lam[:, 0::3].abs().max()) == 0.0 and float(lam[:, 1::3].abs().max()) == 0.0
    # the impulse removes kinetic energy (erp = 0: a purely inelastic, frictionless impact)
    om.erp = 0.0
    dv, lam = contact_velocity_change(om, q, qd)
    v1 = qd + dv
    e0 = 0.5 * (qd[:, None] @ M @ qd[..., None]).squeeze()
    e1 = 0.5 * (v1[:, None] @ M @ v1[..., None]).squeeze()
    assert bool((e1 <= e0 + 1e-12).all())


def test_friction_box_is_respected():
    work, om, q, qd = _touching_quadruped(mu=0.3, seed=3)
    qd[:, 3:5] = 2.0                                   # sliding sideways
    dv, lam = contact_velocity_change(om, q, qd)
    ln = lam[:, 2::3]
    for k in (0, 1):
        assert bool((lam[:, k::3].abs() <= 0.3 * ln + 1e-12).all())
    assert float(ln.max()) > 0


def test_contact_gradient_matches_central_fd():
    """Gradient of a rollout through contact steps vs central differences (small h
    keeps the active set fixed)."""
    work, om, q0, qd0 = _touching_quadruped(B=2, seed=5)
    T = 6
    gen = torch.Generator().manual_seed(2)
    tau = torch.randn(T, 2, om.nv, generator=gen)
    tau[:, :, :6] = 0
    wq = torch.randn(2, om.nq, generator=gen)
    wqd = torch.randn(2, om.nv, generator=gen)

    def phi_fn(q0_, qd0_, tau_, m_):
        qT, qdT, _ = rollout(om, q0_, qd0_, tau_, mass=m_, keep=False)
        return (wq * qT).sum() + (wqd * qdT).sum()

    g = rollout_backward(om, q0, qd0, tau, wq, wqd)
    m0 = om.mass.clone()
    h = 1e-7
    for k in range(2):
        dq = torch.randn(q0.shape, generator=gen)
        dq[:, 3:7] = 0
        dqd = torch.randn(qd0.shape, generator=gen)
        dtau = torch.randn(tau.shape, generator=gen)
        dtau[:, :, :6] = 0
        dm = 0.1 * torch.randn(m0.shape, generator=gen)
        fd = (phi_fn(q0 + h * dq, qd0 + h * dqd, tau + h * dtau, m0 + h * dm)
              - phi_fn(q0 - h * dq, qd0 - h * dqd, tau - h * dtau, m0 - h * dm)) / (2 * h)
        an = (g[0] * dq).sum() + (g[1] * dqd).sum() + (g[2] * dtau).sum() + (g[3] * dm).sum()
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (fd.item(), an.item())
