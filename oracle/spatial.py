"""Plain dense spatial algebra (Featherstone 6D vectors), batched over a leading dim.

Conventions (Sec. 3.1, Eq. 5, and the supplementary spatial-algebra operators):
* a spatial motion or force vector is [angular (3); linear (3)];
* a coordinate transform is the pair (E, r): rotation E from the parent frame
  to the child frame and child origin r in parent coordinates; it acts on motion
  vectors as [E a1; E(a2 - r x a1)] (the supplement's ``st_apply``), i.e. the
  6x6 matrix X = [E 0; -E rx E]; forces transform with X^-T;
* the spatial inertia of a body with mass m, centre of mass c and rotational
  inertia I_c about c is [I_c + m cx cx^T, m cx; m cx^T, m 1];
* motion cross product v x m = [w x m_w; w x m_v + v x m_w] (``sm_crossm``),
  force cross product v x* f = [w x f_n + v x f_f; w x f_f] (``sm_crossf``, Eq. 5).
Everything is written as full matrices so it can be checked by eye.
"""
import torch


def skew(v):
    """[..., 3] -> [..., 3, 3] with skew(a) @ b == a x b."""
    z = torch.zeros_like(v[..., 0])
    x, y, w = v[..., 0], v[..., 1], v[..., 2]
    return torch.stack([
        torch.stack([z, -w, y], -1),
        torch.stack([w, z, -x], -1),
        torch.stack([-y, x, z], -1)], -2)


def crossm(v):
    """6x6 matrix of the motion cross product v x (.)."""
    w, u = v[..., :3], v[..., 3:]
    W, U = skew(w), skew(u)
    Z = torch.zeros_like(W)
    return torch.cat([torch.cat([W, Z], -1), torch.cat([U, W], -1)], -2)


def crossf(v):
    """6x6 matrix of the force cross product v x* (.) = -crossm(v)^T."""
    return -crossm(v).transpose(-1, -2)


def xform(E, r):
    """Motion transform X = [E 0; -E rx E] for rotation E [...,3,3], offset r [...,3]."""
    Z = torch.zeros_like(E)
    return torch.cat([torch.cat([E, Z], -1), torch.cat([-E @ skew(r), E], -1)], -2)


def spatial_inertia(m, c, Ic):
    """[..] mass, [..,3] COM, [..,3,3] inertia about COM -> [..,6,6]."""
    C = skew(c)
    m3 = m[..., None, None]
    eye = torch.eye(3, dtype=c.dtype).expand(C.shape)
    top = torch.cat([Ic + m3 * (C @ C.transpose(-1, -2)), m3 * C], -1)
    bot = torch.cat([m3 * C.transpose(-1, -2), m3 * eye], -1)
    return torch.cat([top, bot], -2)


def rot_axis_angle(axis, theta):
    """Active rotation about unit ``axis`` by ``theta`` (Rodrigues)."""
    K = skew(axis)
    eye = torch.eye(3, dtype=axis.dtype).expand(K.shape)
    s = torch.sin(theta)[..., None, None]
    c = torch.cos(theta)[..., None, None]
    return eye + s * K + (1 - c) * (K @ K)


def quat_to_R(q):
    """Unit quaternion (x, y, z, w) -> rotation matrix taking body to world."""
    x, y, z, w = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        torch.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        torch.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], -2)


def quat_to_E(q):
    """World -> body coordinate rotation E = R(q)^T."""
    return quat_to_R(q).transpose(-1, -2)


def quat_mul(a, b):
    """Hamilton product of quaternions stored (x, y, z, w)."""
    av, aw = a[..., :3], a[..., 3:]
    bv, bw = b[..., :3], b[..., 3:]
    v = aw * bv + bw * av + torch.linalg.cross(av, bv, dim=-1)
    w = aw * bw - (av * bv).sum(-1, keepdim=True)
    return torch.cat([v, w], -1)
