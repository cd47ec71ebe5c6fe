"""Helpers shared by the GPU parity tests: run the CPU FP64 oracle on chosen
systems of a workload (grouped by topology), and compare per output tensor."""
from __future__ import annotations

from collections import defaultdict

import numpy as np
import torch

from oracle.dynamics import OracleModel
from oracle.rollout import rollout, rollout_backward

torch.set_num_threads(1)


def groups(model, systems):
    g = defaultdict(list)
    for s in systems:
        r = model.links(s)
        ct = () if model.contact is None else tuple(model.contact[r.start:r.stop, 3] >= 0)
        lm = () if getattr(model, "limits", None) is None else \
            tuple(np.isfinite(model.limits[r.start:r.stop]).any(1))
        key = (tuple(model.parent[r.start:r.stop]), tuple(model.joint_type[r.start:r.stop]), ct, lm)
        g[key].append(int(s))
    return list(g.values())


def oracle_forward(model, systems, q0, qd0, tau, integrator="semi", fd="crba"):
    """Final states of the listed systems, padded SoA [nq_max, S], [nv_max, S]."""
    nqm, nvm = q0.shape[0], qd0.shape[0]
    S = len(systems)
    qT = np.zeros((nqm, S))
    qdT = np.zeros((nvm, S))
    col = {s: i for i, s in enumerate(systems)}
    for grp in groups(model, systems):
        om = OracleModel(model, grp)
        oq = torch.tensor(q0[:om.nq, grp].T)
        oqd = torch.tensor(qd0[:om.nv, grp].T)
        ot = torch.tensor(tau[:, :om.nv, grp]).permute(0, 2, 1).contiguous()
        with torch.no_grad():
            a, b, _ = rollout(om, oq, oqd, ot, integrator, fd, keep=False)
        for j, s in enumerate(grp):
            qT[:om.nq, col[s]] = a[j].numpy()
            qdT[:om.nv, col[s]] = b[j].numpy()
    return qT, qdT


def oracle_backward(model, systems, q0, qd0, tau, gqT, gqdT, integrator="semi", fd="crba"):
    """Gradients of <gqT, q^T> + <gqdT, qd^T> for the listed systems."""
    nqm, nvm = q0.shape[0], qd0.shape[0]
    T = tau.shape[0]
    S = len(systems)
    out = dict(gq0=np.zeros((nqm, S)), gqd0=np.zeros((nvm, S)), gtau=np.zeros((T, nvm, S)), gm={})
    col = {s: i for i, s in enumerate(systems)}
    for grp in groups(model, systems):
        om = OracleModel(model, grp)
        oq = torch.tensor(q0[:om.nq, grp].T)
        oqd = torch.tensor(qd0[:om.nv, grp].T)
        ot = torch.tensor(tau[:, :om.nv, grp]).permute(0, 2, 1).contiguous()
        g = rollout_backward(om, oq, oqd, ot, torch.tensor(gqT[:om.nq, grp].T),
                             torch.tensor(gqdT[:om.nv, grp].T), integrator=integrator, fd=fd)
        for j, s in enumerate(grp):
            c = col[s]
            out["gq0"][:om.nq, c] = g[0][j].numpy()
            out["gqd0"][:om.nv, c] = g[1][j].numpy()
            out["gtau"][:, :om.nv, c] = g[2][:, j].numpy()
            out["gm"][s] = g[3][j].numpy()
    return out


def rel_err(gpu, ref, floor=1e-12):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if gpu.shape != ref.shape:
        raise AssertionError(f"shape {gpu.shape} vs {ref.shape}")
    if not np.all(np.isfinite(gpu)):
        return float("inf")
    return float(np.abs(gpu - ref).max() / max(np.abs(ref).max(), floor))


def check(name, gpu, ref, tol, report=None):
    e = rel_err(gpu, ref)
    if report is not None:
        report[name] = e
    assert e <= tol, f"{name}: relative error {e:.3e} > {tol:.1e}"
    return e


def mass_grad_of(model, gmass, systems):
    """Per-system slices of a CSR per-link array."""
    return {s: np.asarray(gmass[model.sys_link_offset[s]:model.sys_link_offset[s + 1]]) for s in systems}
