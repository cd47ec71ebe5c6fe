"""Contact resolution by a mixed linear complementarity problem solved with
projected Gauss-Seidel (Sec. 3.1 "Collision resolution", Eq. 8; supplement
Sec. D, Alg. 1), plain CPU FP64.

Reading (the paper names the MLCP a = A x + b, 0 <= a _|_ x >= 0, c- <= x <= c+,
with A the inertial matrix and b the relative velocities, and gives no contact
model parameters):
* contact candidates are spheres (centre p_c in a link's frame, radius r) against
  the ground plane z = 0; the gap is phi = y_z - r with y the sphere centre in the
  world; a candidate is active when phi < 0;
* the unknowns x are contact impulses lambda (3 per contact: world x, y tangent,
  z normal); A = J M^-1 J^T with J the world-frame velocity Jacobian of the
  sphere centres; b = J v* + (erp/dt) min(phi, 0) e_z, where v* = qd + dt qdd is
  the velocity after the unconstrained step;
* the normal impulse is >= 0 and complementary to the normal velocity; the
  friction impulses are boxed by c-+ = -+mu lambda_n (the box uses the current
  normal impulse, as PGS does);
* PGS runs a fixed number of sweeps over the active contacts, normal row first,
  then x and y; the post-contact velocity is v* + M^-1 J^T lambda.
The contact impulse folds into the step as an extra acceleration M^-1 J^T lambda / dt.
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


def pgs(A, b, active, mu, iterations):
    """Projected Gauss-Seidel on the boxed MLCP; A [B, 3C, 3C], b [B, 3C],
    active [B, C].  Rows of contact c: 3c (x), 3c+1 (y) tangent, 3c+2 (z) normal."""
    B, n = b.shape
    C = n // 3
    lam = torch.zeros_like(b)
    act = active.to(b.dtype)
    for _ in range(iterations):
        for c in range(C):
            rn = 3 * c + 2
            s = lam[:, rn] - ((A[:, rn] * lam).sum(-1) + b[:, rn]) / A[:, rn, rn]
            ln = torch.clamp(s, min=0.0) * act[:, c]
            lam = torch.cat([lam[:, :rn], ln[:, None], lam[:, rn + 1:]], 1)
            for rt in (3 * c, 3 * c + 1):
                s = lam[:, rt] - ((A[:, rt] * lam).sum(-1) + b[:, rt]) / A[:, rt, rt]
                hi = mu * lam[:, rn]
                lt = torch.maximum(torch.minimum(s, hi), -hi) * act[:, c]
                lam = torch.cat([lam[:, :rt], lt[:, None], lam[:, rt + 1:]], 1)
    return lam


def contact_velocity_change(model, q, v_star, mass=None):
    """M^-1 J^T lambda: the velocity change the contact impulses cause."""
    y, phi = contact_points(model, q)
    active = phi < 0
    J = contact_jacobian(model, q)
    M = crba(model, q, mass)
    L = torch.linalg.cholesky(M)
    W = torch.cholesky_solve(J.transpose(-1, -2), L)           # M^-1 J^T
    A = J @ W
    b = (J @ v_star[..., None])[..., 0]
    b = b.clone()
    b[:, 2::3] = b[:, 2::3] + (model.erp / model.dt) * torch.clamp(phi, max=0.0)
    lam = pgs(A, b, active, model.friction, model.pgs_iterations)
    return (W @ lam[..., None])[..., 0], lam
