"""Seeded synthetic workloads: model trees, initial states and joint torques.

This module only draws random numbers and lays them out; it holds none of the
dynamics (no spatial algebra, no inertia assembly, no integration).  Both the
CPU oracle and the CUDA path read their inputs from here, so a mistake in
either side cannot leak into the other through shared arithmetic.

Model description (one batch of ``n_systems`` independent articulated bodies,
links stored CSR by system, each system's links in topological order):

  sys_link_offset  int32 [B+1]   first link of each system
  parent           int32 [L]     parent link index *within the system*, -1 = world
  joint_type       int32 [L]     REVOLUTE (1 position, 1 velocity coordinate) or
                                 FREE (7 positions p, quaternion x y z w; 6 velocities
                                 omega, v in body coordinates)
  axis             f64  [L,3]    unit joint axis (revolute), in the link frame
  X_tree           f64  [L,12]   parent frame -> joint frame: E row-major (9), r (3)
  mass             f64  [L]
  com              f64  [L,3]    centre of mass in the link frame
  I_com            f64  [L,6]    rotational inertia about the COM: xx yy zz xy xz yz
  damping          f64  [L]      viscous joint damping b (joint force -b qd), or None
  contact          f64  [L,4]    contact sphere of a link against the ground z = 0:
                                 centre in the link frame (3), radius (< 0: none); or None
  limits           f64  [L,2]    revolute joint position limits lo < hi (+-inf: none); or None
  friction, pgs_iterations, erp  contact solver parameters (Coulomb coefficient,
                                 Gauss-Seidel sweeps, penetration correction rate)

State layout (structure of arrays, system index fastest, zero padded to the
batch maximum): q [nq_max, B], qd [nv_max, B], tau [T, nv_max, B].

The five workloads follow the paper's experiment families (double pendulum,
serial chains, a floating-base quadruped of the Laikago's 19/18 coordinate
size, uneven random trees, a floating-base humanoid); sizes are fixed here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

REVOLUTE = 0
FREE = 1

SEED_BASE = 2109077190

JOINT_NQ = {REVOLUTE: 1, FREE: 7}
JOINT_NV = {REVOLUTE: 1, FREE: 6}


@dataclass
class ModelDesc:
    sys_link_offset: np.ndarray
    parent: np.ndarray
    joint_type: np.ndarray
    axis: np.ndarray
    X_tree: np.ndarray
    mass: np.ndarray
    com: np.ndarray
    I_com: np.ndarray
    dt: float
    gravity: np.ndarray
    name: str = ""
    damping: np.ndarray = None
    contact: np.ndarray = None
    friction: float = 0.8
    pgs_iterations: int = 20
    erp: float = 0.2
    limits: np.ndarray = None

    @property
    def n_systems(self) -> int:
        return int(len(self.sys_link_offset) - 1)

    @property
    def n_links_total(self) -> int:
        return int(self.sys_link_offset[-1])

    def links(self, b: int) -> range:
        return range(int(self.sys_link_offset[b]), int(self.sys_link_offset[b + 1]))

    def nq_per_system(self) -> np.ndarray:
        per_link = np.where(self.joint_type == FREE, 7, 1)
        return np.add.reduceat(per_link, self.sys_link_offset[:-1]).astype(np.int64)

    def nv_per_system(self) -> np.ndarray:
        per_link = np.where(self.joint_type == FREE, 6, 1)
        return np.add.reduceat(per_link, self.sys_link_offset[:-1]).astype(np.int64)

    @property
    def nq_max(self) -> int:
        return int(self.nq_per_system().max())

    @property
    def nv_max(self) -> int:
        return int(self.nv_per_system().max())

    def subset(self, systems) -> "ModelDesc":
        """The model restricted to the listed systems (in that order)."""
        systems = [int(s) for s in systems]
        idx = np.concatenate([np.arange(self.sys_link_offset[s], self.sys_link_offset[s + 1])
                              for s in systems])
        counts = [self.sys_link_offset[s + 1] - self.sys_link_offset[s] for s in systems]
        off = np.zeros(len(systems) + 1, np.int32)
        off[1:] = np.cumsum(counts)
        return ModelDesc(off, self.parent[idx].copy(), self.joint_type[idx].copy(),
                         self.axis[idx].copy(), self.X_tree[idx].copy(), self.mass[idx].copy(),
                         self.com[idx].copy(), self.I_com[idx].copy(), self.dt,
                         self.gravity.copy(), self.name + "[subset]",
                         None if self.damping is None else self.damping[idx].copy(),
                         None if self.contact is None else self.contact[idx].copy(),
                         self.friction, self.pgs_iterations, self.erp,
                         None if self.limits is None else self.limits[idx].copy())

    def with_limits(self, lo: float, hi: float, every: int = 1) -> "ModelDesc":
        """A copy with position limits [lo, hi] on every ``every``-th revolute joint
        of each system (counting from its first link)."""
        m = ModelDesc(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        lim = np.tile(np.array([[-np.inf, np.inf]]), (self.n_links_total, 1))
        for b in range(self.n_systems):
            for j, i in enumerate(self.links(b)):
                if self.joint_type[i] == REVOLUTE and j % every == 0:
                    lim[i] = (lo, hi)
        m.limits = lim
        m.name = self.name + "_limits"
        return m

    def with_damping(self, seed: int, lo: float = 0.05, hi: float = 0.5) -> "ModelDesc":
        """A copy with viscous damping ~ U(lo, hi) on every revolute joint."""
        rng = np.random.default_rng(seed)
        d = rng.uniform(lo, hi, self.n_links_total) * (self.joint_type == REVOLUTE)
        m = ModelDesc(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        m.damping = d
        return m


@dataclass
class Workload:
    model: ModelDesc
    q0: np.ndarray           # [nq_max, B] float64
    qd0: np.ndarray          # [nv_max, B] float64
    T: int
    tau_sigma: float
    seed: int
    precision: str           # "fp64" | "fp32" | "fp32_d64"
    tau_mask: np.ndarray = field(default=None)  # [nv_max, B] 1 where a torque is drawn

    def in_slot_order(self) -> "Workload":
        """The same systems laid out by link count, longest first (stable), the
        order in which the library packs systems into warps: a caller that keeps
        its per-system arrays in this order gives every warp 32 consecutive
        systems, so state, torque, checkpoint and gradient accesses are whole
        cache lines.  Torques are drawn afresh for the new order (same
        distribution); initial states move with their systems."""
        nl = np.diff(self.model.sys_link_offset)
        order = np.argsort(-nl, kind="stable")
        m = self.model.subset(order)
        m.name = self.model.name
        return Workload(m, np.ascontiguousarray(self.q0[:, order]), np.ascontiguousarray(self.qd0[:, order]),
                        self.T, self.tau_sigma, self.seed, self.precision,
                        None if self.tau_mask is None else np.ascontiguousarray(self.tau_mask[:, order]))

    def tau(self, T: int | None = None, device="cpu", dtype=None):
        """Joint torques [T, nv_max, B] drawn N(0, tau_sigma^2) from a seeded torch
        generator on ``device``; entries outside ``tau_mask`` are zero."""
        import torch
        T = self.T if T is None else T
        dtype = dtype or torch.float64
        g = torch.Generator(device=device)
        g.manual_seed(self.seed + 7)
        B = self.model.n_systems
        nv = self.model.nv_max
        t = torch.randn((T, nv, B), generator=g, device=device, dtype=torch.float64)
        t.mul_(self.tau_sigma)
        t.mul_(torch.as_tensor(self.tau_mask, device=device, dtype=torch.float64))
        return t.to(dtype)


# ---------------------------------------------------------------- helpers

def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n orthogonal 3x3 matrices from the QR of Gaussians, sign fixed, det +1."""
    a = rng.standard_normal((n, 3, 3))
    qm, rm = np.linalg.qr(a)
    qm = qm * np.sign(np.diagonal(rm, axis1=1, axis2=2))[:, None, :]
    neg = np.linalg.det(qm) < 0
    qm[neg, :, 0] *= -1
    return qm


def _random_inertias(rng, n, lo, hi) -> np.ndarray:
    """n SPD 3x3 matrices with eigenvalues ~ U(lo, hi), as [n, 6] (xx yy zz xy xz yz)."""
    Q = _random_rotations(rng, n)
    lam = rng.uniform(lo, hi, (n, 3))
    M = np.einsum('nij,nj,nkj->nik', Q, lam, Q)
    return np.stack([M[:, 0, 0], M[:, 1, 1], M[:, 2, 2], M[:, 0, 1], M[:, 0, 2], M[:, 1, 2]], 1)


def _units(rng, n) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _assemble(counts, parent, jtype, axis, r, mass, com, Ic, dt, gravity, name) -> ModelDesc:
    n = len(parent)
    Xt = np.zeros((n, 12))
    Xt[:, [0, 4, 8]] = 1.0
    Xt[:, 9:] = r
    off = np.zeros(len(counts) + 1, np.int32)
    off[1:] = np.cumsum(counts)
    return ModelDesc(off, np.asarray(parent, np.int32), np.asarray(jtype, np.int32),
                     np.asarray(axis, float).reshape(n, 3), Xt, np.asarray(mass, float),
                     np.asarray(com, float).reshape(n, 3), np.asarray(Ic, float).reshape(n, 6),
                     float(dt), np.asarray(gravity, float), name)


def _state_arrays(model: ModelDesc):
    B = model.n_systems
    return np.zeros((model.nq_max, B)), np.zeros((model.nv_max, B)), np.zeros((model.nv_max, B))


def _random_tree_params(rng, parents_local, first, off_lo=0.1, off_hi=0.4, m_lo=0.5, m_hi=2.0,
                        ilo=0.01, ihi=0.1):
    """Per-link random parameters for revolute trees given local parent indices
    (concatenated over systems) and a flag marking each system's first link:
    axis ~ U{x,y,z}; joint offset = random unit direction x U(off_lo, off_hi)
    (zero for the root); COM at half the first child's offset (own draw for leaves);
    mass ~ U(m_lo, m_hi); I_com SPD with eigenvalues ~ U(ilo, ihi)."""
    n = len(parents_local)
    axis = np.eye(3)[rng.integers(3, size=n)]
    offs = _units(rng, n) * rng.uniform(off_lo, off_hi, (n, 1))
    own = _units(rng, n) * rng.uniform(off_lo, off_hi, (n, 1))
    mass = rng.uniform(m_lo, m_hi, n)
    Ic = _random_inertias(rng, n, ilo, ihi)
    sys_start = np.maximum.accumulate(np.where(first, np.arange(n), 0))
    com = own / 2
    first_child = np.full(n, -1)
    for i in range(n - 1, -1, -1):          # lowest-index child wins
        p = parents_local[i]
        if p >= 0:
            first_child[sys_start[i] + p] = i
    has = first_child >= 0
    com[has] = offs[first_child[has]] / 2
    r = np.where(first[:, None], 0.0, offs)
    return axis, r, mass, com, Ic


# ---------------------------------------------------------------- workloads

def double_pendulum(B: int = 1, T: int = 1000, seed: int = SEED_BASE + 1) -> Workload:
    """Planar double pendulum: two revolute z joints, unit masses, 1 m thin rods
    (COM at mid length, I_xx = I_zz = m l^2/12, I_yy = 0), q = 0 hangs down along -y,
    gravity -9.81 along y; q0 ~ U(-1, 1), qd0 = 0, torques ~ N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    l, m = 1.0, 1.0
    Ic = [m * l * l / 12, 0.0, m * l * l / 12, 0.0, 0.0, 0.0]
    model = _assemble([2] * B, [-1, 0] * B, [REVOLUTE] * (2 * B), [(0, 0, 1)] * (2 * B),
                      [(0, 0, 0), (0, -l, 0)] * B, [m] * (2 * B), [(0, -l / 2, 0)] * (2 * B),
                      [Ic] * (2 * B), 1e-3, (0.0, -9.81, 0.0), "double_pendulum")
    q0, qd0, mask = _state_arrays(model)
    q0[:] = rng.uniform(-1, 1, q0.shape)
    mask[:] = 1.0
    return Workload(model, q0, qd0, T, 0.1, seed, "fp64", mask)


def serial_chains(B: int = 4096, T: int = 1000, n: int = 7, seed: int = SEED_BASE + 2,
                  precision: str = "fp32") -> Workload:
    """B serial n-DOF revolute chains with per-system random parameters
    (axes from {x, y, z}, masses U(0.5, 2), inertia eigenvalues U(0.01, 0.1),
    offsets U(0.1, 0.4) m); gravity -9.81 z; q0 ~ U(-1, 1), qd0 = 0, torques N(0, 1)."""
    rng = np.random.default_rng(seed)
    parents = np.tile(np.arange(-1, n - 1), B)
    first = np.tile(np.arange(n) == 0, B)
    axis, r, mass, com, Ic = _random_tree_params(rng, parents, first)
    model = _assemble([n] * B, parents, np.zeros(n * B), axis, r, mass, com, Ic, 1e-3,
                      (0.0, 0.0, -9.81), f"serial_chains_{n}dof")
    q0, qd0, mask = _state_arrays(model)
    q0[:] = rng.uniform(-1, 1, q0.shape)
    mask[:] = 1.0
    return Workload(model, q0, qd0, T, 1.0, seed, precision, mask)


def quadruped(B: int = 8192, T: int = 2000, seed: int = SEED_BASE + 3,
              precision: str = "fp32_d64", contacts: bool = False) -> Workload:
    """Floating-base quadruped: 10 kg 0.5 x 0.3 x 0.15 m box base on a free joint,
    hips at (+-0.25, +-0.15, 0); each leg hip roll (x), hip pitch (y), knee pitch (y)
    with 0.2 m thigh and calf, leg link masses U(0.5, 1.5), inertia eigenvalues
    U(0.001, 0.01); 19 position and 18 velocity coordinates.  Base starts 0.5 m up,
    identity orientation, legs U(-0.3, 0.3), at rest; leg torques N(0, 1).
    Contact-free."""
    rng = np.random.default_rng(seed)
    a, b, c, mb = 0.5, 0.3, 0.15, 10.0
    Ib = [mb / 12 * (b * b + c * c), mb / 12 * (a * a + c * c), mb / 12 * (a * a + b * b), 0, 0, 0]
    par1 = [-1]
    ax1 = [(0, 0, 0)]
    r1 = [(0, 0, 0)]
    com1 = [(0, 0, 0)]
    for sx in (1, -1):
        for sy in (1, -1):
            base = len(par1)
            par1 += [0, base, base + 1]
            ax1 += [(1, 0, 0), (0, 1, 0), (0, 1, 0)]
            r1 += [(sx * a / 2, sy * b / 2, 0), (0, 0, 0), (0, 0, -0.2)]
            com1 += [(0, 0, 0), (0, 0, -0.1), (0, 0, -0.1)]
    nl = len(par1)
    mass = rng.uniform(0.5, 1.5, (B, nl))
    mass[:, 0] = mb
    Ic = _random_inertias(rng, B * nl, 0.001, 0.01).reshape(B, nl, 6)
    Ic[:, 0] = Ib
    jt = [FREE] + [REVOLUTE] * (nl - 1)
    model = _assemble([nl] * B, par1 * B, jt * B, ax1 * B, r1 * B, mass.reshape(-1),
                      com1 * B, Ic.reshape(-1, 6), 5e-4, (0.0, 0.0, -9.81), "quadruped")
    if contacts:
        # 2 cm foot spheres at the ends of the calves (the last link of each leg)
        ct = np.full((nl, 4), -1.0)
        for leg in range(4):
            ct[3 + 3 * leg] = (0.0, 0.0, -0.2, 0.02)
        model.contact = np.tile(ct, (B, 1))
        model.name = "quadruped_contact"
    q0, qd0, mask = _state_arrays(model)
    q0[2, :] = 0.5
    q0[6, :] = 1.0
    q0[7:, :] = rng.uniform(-0.3, 0.3, q0[7:].shape)
    mask[6:, :] = 1.0
    return Workload(model, q0, qd0, T, 1.0, seed, precision, mask)


def uneven_trees(B: int = 16384, T: int = 5000, seed: int = SEED_BASE + 4,
                 dof_lo: int = 2, dof_hi: int = 64, precision: str = "fp32") -> Workload:
    """B revolute trees, DOF ~ U{dof_lo..dof_hi}, per-system branch factor ~ U{1..3}:
    each new link attaches to a uniformly chosen earlier link that has fewer children
    than the branch factor (factor 1 gives a serial chain); link parameters as for
    the serial chains."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(dof_lo, dof_hi + 1, B)
    bfs = rng.integers(1, 4, B)
    parents = []
    for n, bf in zip(ns.tolist(), bfs.tolist()):
        kids = [0] * n
        parents.append(-1)
        open_ = [0]
        draws = rng.random(n)
        for i in range(1, n):
            j = min(int(draws[i] * len(open_)), len(open_) - 1) if bf > 1 else len(open_) - 1
            p = open_[j]
            kids[p] += 1
            if kids[p] >= bf:
                open_.pop(j)
            open_.append(i)
            parents.append(p)
    parents = np.asarray(parents)
    first = parents < 0
    axis, r, mass, com, Ic = _random_tree_params(rng, parents, first)
    model = _assemble(ns, parents, np.zeros(len(parents)), axis, r, mass, com, Ic, 1e-3,
                      (0.0, 0.0, -9.81), "uneven_trees")
    q0, qd0, mask = _state_arrays(model)
    nq = model.nq_per_system()
    q0[:] = rng.uniform(-1, 1, q0.shape) * (np.arange(model.nq_max)[:, None] < nq[None, :])
    mask[:] = (np.arange(model.nv_max)[:, None] < model.nv_per_system()[None, :])
    return Workload(model, q0, qd0, T, 1.0, seed, precision, mask)


def humanoid(B: int = 1024, T: int = 50000, seed: int = SEED_BASE + 5,
             precision: str = "fp32") -> Workload:
    """Floating-base humanoid: pelvis on a free joint, a 2-joint waist (z, y) to a
    chest, two 4-joint arms (x, y, z, elbow y) on the chest, two 6-joint legs
    (hip x, y, z, knee y, ankle y, x) on the pelvis: 22 revolute joints, 29 position
    and 28 velocity coordinates; link masses U(1, 8) kg, inertia eigenvalues
    U(0.01, 0.1).  Pelvis starts 1 m up, upright, joints U(-0.1, 0.1), at rest;
    joint torques N(0, 1)."""
    rng = np.random.default_rng(seed)
    par, ax, r, com = [-1], [(0, 0, 0)], [(0, 0, 0)], [(0, 0, 0)]

    def add(parent, axis, rr, cc):
        par.append(parent)
        ax.append(axis)
        r.append(rr)
        com.append(cc)
        return len(par) - 1

    w1 = add(0, (0, 0, 1), (0, 0, 0.1), (0, 0, 0))
    chest = add(w1, (0, 1, 0), (0, 0, 0), (0, 0, 0.2))
    for sy in (1, -1):
        s1 = add(chest, (1, 0, 0), (0, sy * 0.2, 0.35), (0, 0, 0))
        s2 = add(s1, (0, 1, 0), (0, 0, 0), (0, 0, 0))
        s3 = add(s2, (0, 0, 1), (0, 0, 0), (0, 0, -0.15))
        add(s3, (0, 1, 0), (0, 0, -0.3), (0, 0, -0.15))
    for sy in (1, -1):
        h1 = add(0, (1, 0, 0), (0, sy * 0.1, -0.1), (0, 0, 0))
        h2 = add(h1, (0, 1, 0), (0, 0, 0), (0, 0, 0))
        h3 = add(h2, (0, 0, 1), (0, 0, 0), (0, 0, -0.2))
        kn = add(h3, (0, 1, 0), (0, 0, -0.4), (0, 0, -0.2))
        a1 = add(kn, (0, 1, 0), (0, 0, -0.4), (0, 0, 0))
        add(a1, (1, 0, 0), (0, 0, 0), (0.05, 0, -0.05))
    nl = len(par)
    mass = rng.uniform(1, 8, B * nl)
    Ic = _random_inertias(rng, B * nl, 0.01, 0.1)
    jt = [FREE] + [REVOLUTE] * (nl - 1)
    model = _assemble([nl] * B, par * B, jt * B, ax * B, r * B, mass, com * B, Ic, 1e-3,
                      (0.0, 0.0, -9.81), "humanoid")
    q0, qd0, mask = _state_arrays(model)
    q0[2, :] = 1.0
    q0[6, :] = 1.0
    q0[7:, :] = rng.uniform(-0.1, 0.1, q0[7:].shape)
    mask[6:, :] = 1.0
    return Workload(model, q0, qd0, T, 1.0, seed, precision, mask)


CONFIGS = {
    1: double_pendulum,
    2: serial_chains,
    3: quadruped,
    4: uneven_trees,
    5: humanoid,
}


def config(i: int, **kw) -> Workload:
    """Workload ``i`` (1..5) at its full size, or scaled by keyword (B=, T=)."""
    return CONFIGS[i](**kw)
