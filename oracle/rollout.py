"""Time integration, rollouts and the adjoint recurrence (FP64, CPU).

States are batch-first here: q [B, nq], qd [B, nv], tau [T, B, nv].

Integrator (Sec. 3.1 names explicit Euler with df^k/dx^k = I and prints no
formula).  Reading: semi-implicit (symplectic) Euler by default,
qd' = qd + dt qdd(q, qd, tau); q' = q + dt qd'; plain explicit Euler
(q' = q + dt qd) is the alternative.  Free joints integrate the body-frame
velocity the same way, then p' = p + dt R(quat) v' and
quat' = normalize(quat + dt/2 quat (x) (w', 0)) (the supplement's quaternion
``mul_vec`` is quat (x) (w, 0)).  The torque u^k acts over step k -> k+1
(Sec. 2: f^{k+1}(u^k, x^k, x^{k+1}) = 0).

Gradients (Sec. 3.1 Eq. 3-4, Sec. 3.2 Eq. 7): only the state at the start of
each step is kept; during backprop each step is recomputed from its stored
state and the adjoint R^{k+1} = xbar^{k+1} is pulled back through it.
"""
from __future__ import annotations

import torch

from .dynamics import OracleModel, FREE, fd_crba, aba, crba, jcalc, link_world_poses
from .spatial import quat_to_R, quat_mul, crossm


def qdd_of(model, q, qd, tau, fd="crba", mass=None):
    if fd == "crba":
        return fd_crba(model, q, qd, tau, mass)
    if fd == "aba":
        return aba(model, q, qd, tau, mass)
    raise ValueError(fd)


def step(model: OracleModel, q, qd, tau, integrator="semi", fd="crba", mass=None):
    """One time step x^k -> x^{k+1}; joint forces are tau - b qd (viscous damping);
    contact and joint-limit impulses (if the model has contact spheres or limits)
    change the velocity by M^-1 J^T lambda, applied as an extra acceleration over
    the step."""
    qdd = qdd_of(model, q, qd, tau - model.damping * qd, fd, mass)
    dt = model.dt
    if model.contact_links or model.limit_links:
        from .contact import contact_velocity_change
        dv, _ = contact_velocity_change(model, q, qd + dt * qdd, mass)
        qdd = qdd + dv / dt
    qd_new = qd + dt * qdd
    qv = qd_new if integrator == "semi" else qd
    parts = []
    for i in range(model.N):
        qi = q[:, model.qs[i]]
        vi = qv[:, model.vs[i]]
        if model.jtype[i] == FREE:
            p, quat = qi[:, 0:3], qi[:, 3:7]
            w, v = vi[:, 0:3], vi[:, 3:6]
            p_new = p + dt * (quat_to_R(quat) @ v[..., None])[..., 0]
            wq = torch.cat([w, torch.zeros_like(w[:, :1])], -1)
            raw = quat + 0.5 * dt * quat_mul(quat, wq)
            quat_new = raw / torch.linalg.norm(raw, dim=-1, keepdim=True)
            parts.append(torch.cat([p_new, quat_new], -1))
        else:
            parts.append(qi + dt * vi)
    return torch.cat(parts, -1), qd_new


def rollout(model, q0, qd0, tau, integrator="semi", fd="crba", mass=None, keep=True):
    """Run T = len(tau) steps; returns (qT, qdT, [(q^t, qd^t) for t = 0..T])."""
    q, qd = q0, qd0
    traj = [(q, qd)] if keep else None
    for t in range(tau.shape[0]):
        q, qd = step(model, q, qd, tau[t], integrator, fd, mass)
        if keep:
            traj.append((q, qd))
    return q, qd, traj


def rollout_backward(model, q0, qd0, tau, gqT, gqdT, g_traj=None, integrator="semi",
                     fd="crba", mass=None):
    """Adjoint of a rollout.

    Objective seeds: dPhi/dq^T = gqT, dPhi/dqd^T = gqdT, plus optional per-step
    terms g_traj = [(gq^t, gqd^t) for t = 0..T].  Returns the gradients with
    respect to q^0, qd^0, every tau^t and every link mass: (gq0, gqd0, gtau, gmass).
    """
    m0 = model.mass if mass is None else mass
    with torch.no_grad():
        _, _, traj = rollout(model, q0, qd0, tau, integrator, fd, m0)
    T = tau.shape[0]
    gq, gqd = gqT.clone(), gqdT.clone()
    if g_traj is not None:
        gq = gq + g_traj[T][0]
        gqd = gqd + g_traj[T][1]
    gtau = torch.zeros_like(tau)
    gmass = torch.zeros_like(m0)
    for t in reversed(range(T)):
        q = traj[t][0].detach().requires_grad_(True)
        qd = traj[t][1].detach().requires_grad_(True)
        ut = tau[t].detach().requires_grad_(True)
        m = m0.detach().requires_grad_(True)
        with torch.enable_grad():
            qn, qdn = step(model, q, qd, ut, integrator, fd, m)
            dq, dqd, du, dm = torch.autograd.grad((qn, qdn), (q, qd, ut, m), (gq, gqd),
                                                  allow_unused=True)
        gq, gqd = dq, dqd
        if g_traj is not None:
            gq = gq + g_traj[t][0]
            gqd = gqd + g_traj[t][1]
        gtau[t] = du
        gmass = gmass + dm
    return gq, gqd, gtau, gmass


def energy(model, q, qd, mass=None):
    """Total mechanical energy 1/2 qd^T M qd + V, V = -sum_i m_i g . c_i(world)."""
    M = crba(model, q, mass)
    T = 0.5 * (qd[:, None, :] @ M @ qd[..., None])[:, 0, 0]
    E, r, _ = link_world_poses(model, q)
    com_w = r + (E.transpose(-1, -2) @ model.com[..., None])[..., 0]
    m = model.mass if mass is None else mass
    V = -(m[..., None] * com_w * model.gravity).sum((-1, -2))
    return T + V


def spatial_momentum(model, q, qd, mass=None):
    """Total spatial momentum in world coordinates, sum_i X_i0^T (I_i v_i)."""
    Xs, Ss = jcalc(model, q)
    I = model.inertias(mass)
    _, _, X0 = link_world_poses(model, q)
    v = [None] * model.N
    h = 0
    for i in range(model.N):
        vJ = (Ss[i] @ qd[:, model.vs[i]][..., None])[..., 0]
        p = model.parents[i]
        v[i] = vJ if p < 0 else (Xs[i] @ v[p][..., None])[..., 0] + vJ
        hi = (I[:, i] @ v[i][..., None])
        h = h + (X0[i].transpose(-1, -2) @ hi)[..., 0]
    return h


__all__ = ["step", "rollout", "rollout_backward", "energy", "spatial_momentum", "crossm"]
