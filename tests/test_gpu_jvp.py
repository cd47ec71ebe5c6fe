"""Forward-mode derivative of one step (sim_step_jvp) on the GPU: against central
differences of the FP64 oracle, against the reverse-mode adjoint through the
dot-product test <J dx, ybar> = <dx, J^T ybar>, and FP32 against FP64."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.dynamics import OracleModel
from oracle.rollout import step

pytestmark = pytest.mark.gpu


def _case(cfg, B, precision):
    from paper_2109_07719_gb300 import Simulator
    work = wl.config(cfg, B=B, T=1, precision=precision) if cfg != 4 else \
        wl.config(4, B=B, T=1, dof_hi=20, precision=precision)
    sim = Simulator(work.model, precision=precision)
    m = work.model
    rng = np.random.default_rng(cfg)
    nq, nv = m.nq_max, m.nv_max
    q = work.q0.copy()
    qd = 0.5 * rng.standard_normal((nv, B))
    tau = rng.standard_normal((nv, B))
    dq = rng.standard_normal((nq, B))
    dqd = rng.standard_normal((nv, B))
    dtau = rng.standard_normal((nv, B))
    for b, (a, c) in enumerate(zip(m.nq_per_system(), m.nv_per_system())):
        qd[c:, b] = tau[c:, b] = dqd[c:, b] = dtau[c:, b] = 0
        dq[a:, b] = 0
    if m.joint_type[0] == wl.FREE:
        dq[3:7] = 0          # keep the quaternion on the unit sphere
    dev = lambda x: torch.tensor(x, dtype=sim.dtype, device=sim.device)  # noqa: E731
    return work, sim, (q, qd, tau, dq, dqd, dtau), [dev(x) for x in (q, qd, tau, dq, dqd, dtau)]


@pytest.mark.parametrize("cfg", [2, 3, 4, 5])
def test_jvp_matches_oracle_central_differences(cfg):
    B = 40
    work, sim, host, d = _case(cfg, B, "fp64")
    q1, qd1, dq1, dqd1 = sim.jvp(*d)
    r1, rd1 = sim.step(*d[:3])
    assert torch.allclose(q1, r1, rtol=1e-13, atol=1e-13) and torch.allclose(qd1, rd1, rtol=1e-13, atol=1e-13)
    q, qd, tau, dq, dqd, dtau = host
    m = work.model
    h = 1e-6
    worst = 0.0
    for b in range(0, B, 7):
        om = OracleModel(m, [b])
        a, c = om.nq, om.nv

        def f(s):
            x = step(om, torch.tensor(q[:a, b] + s * dq[:a, b])[None],
                     torch.tensor(qd[:c, b] + s * dqd[:c, b])[None],
                     torch.tensor(tau[:c, b] + s * dtau[:c, b])[None])
            return torch.cat([x[0][0], x[1][0]]).numpy()

        fd = (f(h) - f(-h)) / (2 * h)
        got = np.concatenate([dq1[:a, b].cpu().numpy(), dqd1[:c, b].cpu().numpy()])
        worst = max(worst, np.abs(fd - got).max() / np.abs(fd).max())
    assert worst < 1e-7, worst


@pytest.mark.parametrize("cfg", [2, 3, 5])
def test_jvp_vjp_dot_product(cfg):
    """<J dx, ybar> = <dx, J^T ybar>: forward mode against the hand-derived adjoint."""
    B = 33
    work, sim, host, (q, qd, tau, dq, dqd, dtau) = _case(cfg, B, "fp64")
    _, _, dq1, dqd1 = sim.jvp(q, qd, tau, dq, dqd, dtau)
    g = torch.Generator().manual_seed(3)
    yq = torch.randn(dq1.shape, generator=g, dtype=torch.float64).to(sim.device)
    yqd = torch.randn(dqd1.shape, generator=g, dtype=torch.float64).to(sim.device)
    tau1 = tau[None].contiguous()
    qT, qdT, ck, _ = sim.rollout(q, qd, tau1)
    gq, gqd, gtau, _ = sim.backward(ck, tau1, yq, yqd, mass_grad=False)
    lhs = (dq1 * yq).sum(0) + (dqd1 * yqd).sum(0)
    rhs = (dq * gq).sum(0) + (dqd * gqd).sum(0) + (dtau * gtau[0]).sum(0)
    assert torch.allclose(lhs, rhs, rtol=1e-10, atol=1e-10 * float(lhs.abs().max()))


def test_jvp_fp32_against_fp64():
    B = 64
    _, s64, _, d64 = _case(2, B, "fp64")
    _, s32, _, d32 = _case(2, B, "fp32")
    a = s64.jvp(*d64)
    b = s32.jvp(*d32)
    for x, y in zip(a, b):
        err = float((x - y.double()).abs().max() / x.abs().max())
        assert err < 1e-4
