"""Pins of the oracle's joint-limit rows (unilateral rows of the Sec. 3.1 MLCP,
solved by projected Gauss-Seidel together with the contact rows) against closed
forms, the complementarity conditions and finite differences."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.contact import contact_velocity_change, limit_gaps, limit_jacobian
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


def _pendulum(lo, hi, m=1.5, l=0.8, erp=0.2, dt=1e-3):
    """One rod on a revolute joint about z, COM l/2 below the pivot at q = 0,
    gravity along -y: I_pivot = m l^2 / 12 + m (l/2)^2 = m l^2 / 3."""
    md = wl.ModelDesc(np.array([0, 1], np.int32), np.array([-1], np.int32),
                      np.array([wl.REVOLUTE], np.int32), np.array([[0.0, 0.0, 1.0]]),
                      np.array([[1.0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]]), np.array([m]),
                      np.array([[0.0, -l / 2, 0.0]]), np.array([[m * l * l / 12, 1e-9, m * l * l / 12, 0, 0, 0]]),
                      dt, np.array([0.0, -9.81, 0.0]), "rod")
    md.limits = np.array([[lo, hi]])
    md.erp = erp
    return md


@pytest.mark.parametrize("side", ["lower", "upper"])
def test_pendulum_pushed_back_into_range(side):
    """1 DOF: A = 1/I_pivot, so an active limit row gives lambda = -I_pivot b and
    the new velocity qd' = -s (erp/dt) phi, whatever the unconstrained motion."""
    m, l, erp, dt = 1.5, 0.8, 0.2, 1e-3
    lo, hi = -0.5, 0.7
    md = _pendulum(lo, hi, m, l, erp, dt)
    om = OracleModel(md, [0])
    if side == "lower":
        q, qd, s, phi = lo - 0.01, -0.5, 1.0, -0.01
    else:
        q, qd, s, phi = hi + 0.02, 0.3, -1.0, -0.02
    qq, qqd = torch.tensor([[q]]), torch.tensor([[qd]])
    tau = torch.tensor([[0.3]])
    I_piv = m * l * l / 3
    qdd_free = (0.3 - m * 9.81 * (l / 2) * np.sin(q)) / I_piv          # closed form, no limit
    v_star = qd + dt * qdd_free
    b = s * v_star + erp / dt * phi
    lam = -I_piv * b
    assert lam > 0
    q1, qd1 = step(om, qq, qqd, tau)
    assert abs(float(qd1[0, 0]) - (-s * erp / dt * phi)) < 1e-12
    assert abs(float(qd1[0, 0]) - (v_star + s * lam / I_piv)) < 1e-12
    assert abs(float(q1[0, 0]) - (q + dt * float(qd1[0, 0]))) < 1e-15


def test_separating_joint_is_left_alone():
    """A joint outside its range but moving back fast enough needs no impulse:
    the step equals the limit-free one."""
    md = _pendulum(-0.5, 0.7)
    free = _pendulum(-np.inf, np.inf)
    q, qd, tau = torch.tensor([[-0.51]]), torch.tensor([[5.0]]), torch.tensor([[0.0]])
    a = step(OracleModel(md, [0]), q, qd, tau)
    b = step(OracleModel(free, [0]), q, qd, tau)
    assert torch.allclose(a[0], b[0], atol=1e-15) and torch.allclose(a[1], b[1], atol=1e-15)


def test_limits_in_range_change_nothing():
    work = wl.config(2, B=3, T=1)
    lim = work.model.with_limits(-10.0, 10.0)
    q = torch.tensor(work.q0.T)
    qd = 0.3 * torch.randn(3, 7, generator=torch.Generator().manual_seed(0))
    tau = torch.randn(3, 7, generator=torch.Generator().manual_seed(1))
    a = step(OracleModel(lim.subset([0, 1, 2]), [0, 1, 2]), q, qd, tau)
    b = step(OracleModel(work.model, [0, 1, 2]), q, qd, tau)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_limit_rows_solve_the_lcp():
    """Chains with every joint limited to [-0.3, 0.3] and q0 ~ U(-1, 1): many rows
    active at once; 400 sweeps satisfy lambda >= 0, a = A lambda + b >= 0 on the
    active rows and lambda a = 0."""
    work = wl.config(2, B=4, T=1)
    md = work.model.with_limits(-0.3, 0.3)
    om = OracleModel(md, [0, 1, 2, 3])
    om.pgs_iterations = 400
    q = torch.tensor(work.q0.T)
    qd = 0.5 * torch.randn(4, 7, generator=torch.Generator().manual_seed(3))
    s, phi = limit_gaps(om, q)
    active = phi < 0
    assert int(active.sum()) >= 8
    dv, lam = contact_velocity_change(om, q, qd)
    J = limit_jacobian(om, q)
    M = crba(om, q)
    A = J @ torch.linalg.solve(M, J.transpose(-1, -2))
    b = (J @ qd[..., None])[..., 0] + om.erp / om.dt * torch.clamp(phi, max=0.0)
    a = (A @ lam[..., None])[..., 0] + b
    assert bool((lam >= 0).all())
    assert float(lam[~active].abs().max()) == 0.0
    assert bool((a[active] > -1e-8).all())
    assert float((lam * a)[active].abs().max()) < 1e-8
    # the impulse only ever pushes a violated joint back towards its range
    dq = torch.stack([dv[:, om.vs[l].start] for l in om.limit_links], 1)
    assert bool((dq * s >= -1e-12)[active].all())


def _fd_check(om, q0, qd0, tau, free_dofs, gen, h=1e-7, tol=1e-5):
    B = q0.shape[0]
    wq = torch.randn(B, om.nq, generator=gen)
    wqd = torch.randn(B, om.nv, generator=gen)

    def phi_fn(q0_, qd0_, tau_, m_):
        qT, qdT, _ = rollout(om, q0_, qd0_, tau_, mass=m_, keep=False)
        return (wq * qT).sum() + (wqd * qdT).sum()

    g = rollout_backward(om, q0, qd0, tau, wq, wqd)
    m0 = om.mass.clone()
    for _ in range(2):
        dq = torch.randn(q0.shape, generator=gen) * free_dofs["q"]
        dqd = torch.randn(qd0.shape, generator=gen)
        dtau = torch.randn(tau.shape, generator=gen) * free_dofs["tau"]
        dm = 0.1 * torch.randn(m0.shape, generator=gen)
        fd = (phi_fn(q0 + h * dq, qd0 + h * dqd, tau + h * dtau, m0 + h * dm)
              - phi_fn(q0 - h * dq, qd0 - h * dqd, tau - h * dtau, m0 - h * dm)) / (2 * h)
        an = (g[0] * dq).sum() + (g[1] * dqd).sum() + (g[2] * dtau).sum() + (g[3] * dm).sum()
        assert abs(fd - an) <= tol * max(1.0, abs(an)), (fd.item(), an.item())


def test_limit_gradient_matches_central_fd():
    work = wl.config(2, B=2, T=6)
    md = work.model.with_limits(-0.4, 0.4, every=2)
    om = OracleModel(md, [0, 1])
    gen = torch.Generator().manual_seed(4)
    q0 = torch.tensor(work.q0.T)
    qd0 = 0.5 * torch.randn(2, 7, generator=gen)
    s, phi = limit_gaps(om, q0)
    assert bool((phi < -0.05).any())
    tau = torch.randn(6, 2, 7, generator=gen)
    _fd_check(om, q0, qd0, tau, {"q": torch.ones(1), "tau": torch.ones(1)}, gen)


def test_contacts_and_limits_together_fd():
    """Feet on the ground and every knee past its upper limit in the same MLCP."""
    work = wl.config(3, B=2, T=5, contacts=True)
    md = work.model
    lim = np.tile(np.array([[-np.inf, np.inf]]), (md.n_links_total, 1))
    for b in range(2):
        for leg in range(4):
            lim[md.sys_link_offset[b] + 3 + 3 * leg] = (-1.0, -0.02)     # knees straight: above the range
    md.limits = lim
    om = OracleModel(md, [0, 1])
    from oracle.contact import contact_points
    q = torch.tensor(work.q0.T)
    q[:, 7:] = 0.0
    _, phi = contact_points(om, q)
    q[:, 2] -= phi.min(1).values + 0.004
    gen = torch.Generator().manual_seed(5)
    qd = 0.2 * torch.randn(2, om.nv, generator=gen)
    qd[:, 5] = -1.0
    tau = torch.randn(5, 2, om.nv, generator=gen)
    tau[:, :, :6] = 0
    qmask = torch.ones(om.nq)
    qmask[3:7] = 0
    tmask = torch.ones(om.nv)
    tmask[:6] = 0
    _fd_check(om, q, qd, tau, {"q": qmask, "tau": tmask}, gen)
