"""Forward dynamics of one batch of identically shaped kinematic trees (FP64, CPU).

Two independent routes to qdd:
* ``fd_crba``: the plain definition qdd = M(q)^-1 (tau - C(q, qd)), with M from
  the composite-rigid-body algorithm, C = RNEA(q, qd, 0) (gravity included) and a
  Cholesky solve;
* ``aba``: Featherstone's Articulated Body Algorithm, the method the paper
  builds on (Sec. 2 "Articulated body dynamics"): outward kinematics/velocity
  pass, inward articulated-inertia pass, outward acceleration pass (Sec. 3.1,
  Fig. 1).

Joint models (a reading of the paper, which names no joint convention):
* revolute about unit axis a (link frame): E_J = R(a, q)^T, r_J = 0, S = [a; 0];
* free (floating base): q = (p, quaternion x y z w), the base pose in the world;
  E_J = R(quat)^T, r_J = p; qd = body-frame spatial velocity (w, v); S = 1_6.
Link i's transform from its parent is X_i = X_J(q_i) X_tree,i.  Gravity enters
as the fictitious base acceleration a_0 = [0; -g].  Viscous joint damping b (a
joint force -b qd on revolute joints) is applied by the integrator step.
"""
from __future__ import annotations

import torch

from .spatial import xform, spatial_inertia, rot_axis_angle, quat_to_E, crossm, crossf

REVOLUTE = 0
FREE = 1


class OracleModel:
    """Per-link parameters of ``len(systems)`` systems that share one topology,
    as FP64 tensors with the system index leading."""

    def __init__(self, desc, systems):
        systems = [int(s) for s in systems]
        off = desc.sys_link_offset
        n = off[systems[0] + 1] - off[systems[0]]
        rows = []
        for s in systems:
            idx = list(range(off[s], off[s + 1]))
            if len(idx) != n:
                raise ValueError("systems do not share a topology")
            rows.append(idx)
        rows = torch.as_tensor(rows)
        first = rows[0].tolist()
        self.parents = [int(desc.parent[i]) for i in first]
        self.jtype = [int(desc.joint_type[i]) for i in first]
        for r in rows.tolist():
            if [int(desc.parent[i]) for i in r] != self.parents or \
               [int(desc.joint_type[i]) for i in r] != self.jtype:
                raise ValueError("systems do not share a topology")
        f64 = torch.float64
        t = lambda a: torch.as_tensor(a, dtype=f64)[rows]  # noqa: E731
        self.B = len(systems)
        self.N = n
        self.axis = t(desc.axis)
        Xt = t(desc.X_tree)
        self.E_tree = Xt[..., :9].reshape(self.B, n, 3, 3)
        self.r_tree = Xt[..., 9:]
        self.mass = t(desc.mass)
        self.com = t(desc.com)
        I6 = t(desc.I_com)
        xx, yy, zz, xy, xz, yz = [I6[..., k] for k in range(6)]
        self.Ic = torch.stack([torch.stack([xx, xy, xz], -1),
                               torch.stack([xy, yy, yz], -1),
                               torch.stack([xz, yz, zz], -1)], -2)
        self.gravity = torch.as_tensor(desc.gravity, dtype=f64)
        self.dt = float(desc.dt)
        damp = getattr(desc, "damping", None)
        self.link_damping = t(damp) if damp is not None else torch.zeros(self.B, n, dtype=f64)
        self.qs, self.vs = [], []
        qo = vo = 0
        for j in self.jtype:
            nq, nv = (7, 6) if j == FREE else (1, 1)
            self.qs.append(slice(qo, qo + nq))
            self.vs.append(slice(vo, vo + nv))
            qo += nq
            vo += nv
        self.nq, self.nv = qo, vo
        # contact spheres (links whose radius is >= 0) and solver parameters
        ct = getattr(desc, "contact", None)
        cts = t(ct) if ct is not None else None
        self.contact_links = [] if cts is None else [i for i in range(n) if float(cts[0, i, 3]) >= 0]
        for r in range(self.B):
            if cts is not None and [i for i in range(n) if float(cts[r, i, 3]) >= 0] != self.contact_links:
                raise ValueError("systems do not share a topology")
        if self.contact_links:
            self.contact_p = cts[:, self.contact_links, :3]
            self.contact_r = cts[:, self.contact_links, 3]
        # revolute joints with position limits (lo, hi; +-inf: none on that side)
        lim = getattr(desc, "limits", None)
        lims = t(lim) if lim is not None else None
        fin = lambda r: [i for i in range(n) if self.jtype[i] == REVOLUTE  # noqa: E731
                         and bool(torch.isfinite(lims[r, i]).any())]
        self.limit_links = [] if lims is None else fin(0)
        for r in range(self.B):
            if lims is not None and fin(r) != self.limit_links:
                raise ValueError("systems do not share a topology")
        if self.limit_links:
            self.limit_lo = lims[:, self.limit_links, 0]
            self.limit_hi = lims[:, self.limit_links, 1]
        self.friction = float(getattr(desc, "friction", 0.8))
        self.pgs_iterations = int(getattr(desc, "pgs_iterations", 20))
        self.erp = float(getattr(desc, "erp", 0.2))
        # viscous damping per velocity coordinate (revolute joints only)
        self.damping = torch.zeros(self.B, vo, dtype=f64)
        for i, j in enumerate(self.jtype):
            if j != FREE:
                self.damping[:, self.vs[i]] = self.link_damping[:, i:i + 1]

    def inertias(self, mass=None):
        """Spatial inertia of every link [B, N, 6, 6]; ``mass`` [B, N] overrides."""
        m = self.mass if mass is None else mass
        return spatial_inertia(m, self.com, self.Ic)

    def a0(self):
        """Fictitious base acceleration [0; -g], expanded to [B, 6]."""
        a = torch.zeros(self.B, 6, dtype=torch.float64)
        a[:, 3:] = -self.gravity
        return a


def jcalc(model: OracleModel, q):
    """Link transforms X_i = X_J(q_i) X_tree,i [B,6,6] and motion subspaces S_i [B,6,nd]."""
    Xs, Ss = [], []
    for i in range(model.N):
        qi = q[:, model.qs[i]]
        Xtree = xform(model.E_tree[:, i], model.r_tree[:, i])
        if model.jtype[i] == REVOLUTE:
            a = model.axis[:, i]
            EJ = rot_axis_angle(a, qi[:, 0]).transpose(-1, -2)
            XJ = xform(EJ, torch.zeros_like(a))
            S = torch.cat([a, torch.zeros_like(a)], -1)[..., None]
        else:
            XJ = xform(quat_to_E(qi[:, 3:7]), qi[:, 0:3])
            S = torch.eye(6, dtype=q.dtype).expand(q.shape[0], 6, 6)
        Xs.append(XJ @ Xtree)
        Ss.append(S)
    return Xs, Ss


def _mv(M, v):
    return (M @ v[..., None])[..., 0]


def rnea(model: OracleModel, q, qd, qdd, mass=None):
    """Inverse dynamics tau = M qdd + C(q, qd) with gravity (Newton-Euler)."""
    Xs, Ss = jcalc(model, q)
    I = model.inertias(mass)
    N = model.N
    v, a, f = [None] * N, [None] * N, [None] * N
    for i in range(N):
        vJ = _mv(Ss[i], qd[:, model.vs[i]])
        aJ = _mv(Ss[i], qdd[:, model.vs[i]])
        p = model.parents[i]
        vp = torch.zeros_like(vJ) if p < 0 else v[p]
        ap = model.a0() if p < 0 else a[p]
        v[i] = _mv(Xs[i], vp) + vJ
        a[i] = _mv(Xs[i], ap) + aJ + _mv(crossm(v[i]), vJ)
        f[i] = _mv(I[:, i], a[i]) + _mv(crossf(v[i]), _mv(I[:, i], v[i]))
    tau = [None] * N
    for i in reversed(range(N)):
        tau[i] = _mv(Ss[i].transpose(-1, -2), f[i])
        p = model.parents[i]
        if p >= 0:
            f[p] = f[p] + _mv(Xs[i].transpose(-1, -2), f[i])
    return torch.cat(tau, -1)


def crba(model: OracleModel, q, mass=None):
    """Joint-space inertia matrix M(q) [B, nv, nv] (composite rigid bodies)."""
    Xs, Ss = jcalc(model, q)
    I = model.inertias(mass)
    N = model.N
    Ic = [I[:, i] for i in range(N)]
    for i in reversed(range(N)):
        p = model.parents[i]
        if p >= 0:
            Ic[p] = Ic[p] + Xs[i].transpose(-1, -2) @ Ic[i] @ Xs[i]
    rows = [[None] * N for _ in range(N)]
    for i in range(N):
        F = Ic[i] @ Ss[i]
        rows[i][i] = Ss[i].transpose(-1, -2) @ F
        j = i
        while model.parents[j] >= 0:
            F = Xs[j].transpose(-1, -2) @ F
            j = model.parents[j]
            rows[i][j] = F.transpose(-1, -2) @ Ss[j]
            rows[j][i] = rows[i][j].transpose(-1, -2)
    B = q.shape[0]
    for i in range(N):
        for j in range(N):
            if rows[i][j] is None:
                ni = Ss[i].shape[-1]
                nj = Ss[j].shape[-1]
                rows[i][j] = torch.zeros(B, ni, nj, dtype=q.dtype)
    return torch.cat([torch.cat(r, -1) for r in rows], -2)


def fd_crba(model: OracleModel, q, qd, tau, mass=None):
    """qdd = M^-1 (tau - C): the plain definition of forward dynamics."""
    M = crba(model, q, mass)
    C = rnea(model, q, qd, torch.zeros_like(qd), mass)
    L = torch.linalg.cholesky(M)
    return torch.cholesky_solve((tau - C)[..., None], L)[..., 0]


def aba(model: OracleModel, q, qd, tau, mass=None):
    """Articulated Body Algorithm: three passes over the tree (Sec. 3.1)."""
    Xs, Ss = jcalc(model, q)
    I = model.inertias(mass)
    N = model.N
    v, c, IA, pA = [None] * N, [None] * N, [None] * N, [None] * N
    # pass 1, root to leaves: velocities, velocity-product accelerations, bias forces
    for i in range(N):
        vJ = _mv(Ss[i], qd[:, model.vs[i]])
        p = model.parents[i]
        v[i] = vJ if p < 0 else _mv(Xs[i], v[p]) + vJ
        c[i] = _mv(crossm(v[i]), vJ)
        IA[i] = I[:, i]
        pA[i] = _mv(crossf(v[i]), _mv(I[:, i], v[i]))
    # pass 2, leaves to root: articulated inertias and bias forces
    U, Dinv, u = [None] * N, [None] * N, [None] * N
    for i in reversed(range(N)):
        S = Ss[i]
        U[i] = IA[i] @ S
        D = S.transpose(-1, -2) @ U[i]
        Dinv[i] = torch.linalg.inv(D)
        u[i] = tau[:, model.vs[i]] - _mv(S.transpose(-1, -2), pA[i])
        p = model.parents[i]
        if p >= 0:
            Ia = IA[i] - U[i] @ Dinv[i] @ U[i].transpose(-1, -2)
            pa = pA[i] + _mv(Ia, c[i]) + _mv(U[i] @ Dinv[i], u[i])
            XT = Xs[i].transpose(-1, -2)
            IA[p] = IA[p] + XT @ Ia @ Xs[i]
            pA[p] = pA[p] + _mv(XT, pa)
    # pass 3, root to leaves: accelerations
    a = [None] * N
    qdd = [None] * N
    for i in range(N):
        p = model.parents[i]
        ap = _mv(Xs[i], model.a0() if p < 0 else a[p]) + c[i]
        qdd[i] = _mv(Dinv[i], u[i] - _mv(U[i].transpose(-1, -2), ap))
        a[i] = ap + _mv(Ss[i], qdd[i])
    return torch.cat(qdd, -1)


def link_world_poses(model: OracleModel, q):
    """World->link transforms of every link, as (E [B,N,3,3], origin r [B,N,3])."""
    Xs, _ = jcalc(model, q)
    X0 = [None] * model.N
    for i in range(model.N):
        p = model.parents[i]
        X0[i] = Xs[i] if p < 0 else Xs[i] @ X0[p]
    Es, rs = [], []
    for X in X0:
        E = X[:, :3, :3]
        rx = -E.transpose(-1, -2) @ X[:, 3:, :3]      # X21 = -E rx
        rs.append(torch.stack([rx[:, 2, 1], rx[:, 0, 2], rx[:, 1, 0]], -1))
        Es.append(E)
    return torch.stack(Es, 1), torch.stack(rs, 1), X0
