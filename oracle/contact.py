"""Contact and joint-limit resolution by a mixed linear complementarity problem
solved with projected Gauss-Seidel (Sec. 3.1 "Collision resolution", Eq. 8;
supplement Sec. D, Alg. 1), plain CPU FP64.  Test infrastructure only: imported
by the tests, the smoke check and the benchmark's CPU baseline.

Reading (the paper names the MLCP a = A x + b, 0 <= a _|_ x >= 0, c- <= x <= c+,
with A the inertial matrix and b the relative velocities, and gives no contact
model parameters):
* contact candidates are spheres (centre p_c in a link's frame, radius r) against
  the ground plane z = 0; the gap is phi = y_z - r with y the sphere centre in the
  world; a candidate is active when phi < 0;
* joint limits (the paper lists them among the constraints the LCP handles) are
  rows on revolute joints with limits lo < hi: the gap is phi = q - lo below the
  range (row J = +e_j) or phi = hi - q above it (row J = -e_j), active when
  phi < 0; the row's impulse is >= 0, like a normal row;
* the unknowns x are impulses lambda: 3 per contact (world x, y tangent, z
  normal), then one per limit row; A = J M^-1 J^T with J stacking the world-frame
  velocity Jacobian of the sphere centres and the limit rows;
  b = J v* + (erp/dt) min(phi, 0) on the normal and limit rows, where
  v* = qd + dt qdd is the velocity after the unconstrained step;
* the normal impulse is >= 0 and complementary to the normal velocity; the
  friction impulses are boxed by c-+ = -+mu lambda_n (the box uses the current
  normal impulse, as PGS does);
* PGS runs a fixed number of sweeps: over the active contacts (normal row
  first, then x and y), then over the active limit rows; the post-constraint
  velocity is v* + M^-1 J^T lambda.
The impulse folds into the step as an extra acceleration M^-1 J^T lambda / dt.
"""
from __future__ import annotations

import torch

from .dynamics import crba, jcalc, link_world_poses


def contact_points(model, q):
    """World sphere centres y [B, C, 3] and gaps phi [B, C] of the contact candidates."""
    E, o, _ = link_world_poses(model, q)
    ys = []
    for c, l in enumerate(model.contact_links):
        p = model.contact_p[:, c]
        ys.append(o[:, l] + (E[:, l].transpose(-1, -2) @ p[..., None])[..., 0])
    y = torch.stack(ys, 1)
    return y, y[..., 2] - model.contact_r


def limit_gaps(model, q):
    """Per limited joint: the row sign s [B, K] (+1 below the range, -1 above it)
    and the gap phi [B, K] = s (q - the violated limit), negative when violated."""
    qj = torch.stack([q[:, model.qs[l].start] for l in model.limit_links], 1)
    below = qj - model.limit_lo
    above = model.limit_hi - qj
    s = torch.where(below < 0, torch.ones_like(qj), torch.where(above < 0, -torch.ones_like(qj),
                                                                torch.ones_like(qj)))
    phi = torch.where(below < 0, below, torch.where(above < 0, above, torch.minimum(below, above)))
    return s, phi


def point_velocities(model, q, v):
    """World velocity of every sphere centre for generalized velocity v: [B, C, 3]."""
    Xs, Ss = jcalc(model, q)
    E, _, _ = link_world_poses(model, q)
    vel = [None] * model.N
    for i in range(model.N):
        vJ = (Ss[i] @ v[:, model.vs[i]][..., None])[..., 0]
        p = model.parents[i]
        vel[i] = vJ if p < 0 else (Xs[i] @ vel[p][..., None])[..., 0] + vJ
    out = []
    for c, l in enumerate(model.contact_links):
        w, lin = vel[l][:, :3], vel[l][:, 3:]
        pv = lin + torch.linalg.cross(w, model.contact_p[:, c], dim=-1)
        out.append((E[:, l].transpose(-1, -2) @ pv[..., None])[..., 0])
    return torch.stack(out, 1)


def contact_jacobian(model, q):
    """J [B, 3C, nv]: rows (contact c, world axis x/y/z) of the sphere-centre velocity."""
    B, nv = q.shape[0], model.nv
    cols = []
    for j in range(nv):
        e = torch.zeros(B, nv, dtype=q.dtype)
        e[:, j] = 1.0
        cols.append(point_velocities(model, q, e).reshape(B, -1))
    return torch.stack(cols, -1)


def limit_jacobian(model, q):
    """J [B, K, nv]: row k is s_k e_j for limited joint k (coordinate j)."""
    s, _ = limit_gaps(model, q)
    J = torch.zeros(q.shape[0], len(model.limit_links), model.nv, dtype=q.dtype)
    for k, l in enumerate(model.limit_links):
        J[:, k, model.vs[l].start] = s[:, k]
    return J


def pgs(A, b, active, mu, iterations, n_contacts):
    """Projected Gauss-Seidel on the boxed MLCP; A [B, n, n], b [B, n], active
    [B, C + K].  Rows 3c (x), 3c+1 (y) tangent and 3c+2 (z) normal of contact c,
    then one row per limit (rows 3C..3C+K-1)."""
    Bn, n = b.shape
    C = n_contacts
    lam = torch.zeros_like(b)
    act = active.to(b.dtype)

    def update(lam, r, lo, hi, on):
        s = lam[:, r] - ((A[:, r] * lam).sum(-1) + b[:, r]) / A[:, r, r]
        if hi is None:
            new = torch.clamp(s, min=0.0) * on
        else:
            new = torch.maximum(torch.minimum(s, hi), lo) * on
        return torch.cat([lam[:, :r], new[:, None], lam[:, r + 1:]], 1)

    for _ in range(iterations):
        for c in range(C):
            rn = 3 * c + 2
            lam = update(lam, rn, None, None, act[:, c])
            for rt in (3 * c, 3 * c + 1):
                hi = mu * lam[:, rn]
                lam = update(lam, rt, -hi, hi, act[:, c])
        for k in range(n - 3 * C):
            lam = update(lam, 3 * C + k, None, None, act[:, C + k])
    return lam


def contact_velocity_change(model, q, v_star, mass=None):
    """M^-1 J^T lambda: the velocity change the contact and limit impulses cause,
    and lambda."""
    C = len(model.contact_links)
    phis = []
    if C:
        phis.append(contact_points(model, q)[1])
    if model.limit_links:
        phis.append(limit_gaps(model, q)[1])
    phi = torch.cat(phis, 1)
    active = phi < 0
    n = 3 * C + len(model.limit_links)
    if not bool(active.any()):       # no active row anywhere: lambda = 0 and M^-1 J^T lambda = 0
        return torch.zeros_like(v_star), torch.zeros(q.shape[0], n, dtype=q.dtype)
    Js, bs = [], []
    k = model.erp / model.dt
    if C:
        Jc = contact_jacobian(model, q)
        bc = (Jc @ v_star[..., None])[..., 0].clone()
        bc[:, 2::3] = bc[:, 2::3] + k * torch.clamp(phi[:, :C], max=0.0)
        Js.append(Jc)
        bs.append(bc)
    if model.limit_links:
        Jl = limit_jacobian(model, q)
        Js.append(Jl)
        bs.append((Jl @ v_star[..., None])[..., 0] + k * torch.clamp(phi[:, C:], max=0.0))
    J = torch.cat(Js, 1)
    b = torch.cat(bs, 1)
    M = crba(model, q, mass)
    L = torch.linalg.cholesky(M)
    W = torch.cholesky_solve(J.transpose(-1, -2), L)           # M^-1 J^T
    A = J @ W
    lam = pgs(A, b, active, model.friction, model.pgs_iterations, C)
    return (W @ lam[..., None])[..., 0], lam
