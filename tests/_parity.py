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


# ------------------------------------------------------------------ parallel oracle
# Large parity cases run the oracle on many systems; each topology group is
# independent, so groups are spread over a pool of spawned worker processes
# (spawn, never fork: the parent already holds a CUDA context).

def _fwd_job(args):
    model, grp, q0, qd0, tau, integrator, fd = args
    torch.set_num_threads(1)
    return grp, oracle_forward(model, grp, q0, qd0, tau, integrator, fd)


def _bwd_job(args):
    model, grp, q0, qd0, tau, gqT, gqdT, integrator, fd = args
    torch.set_num_threads(1)
    return grp, oracle_backward(model, grp, q0, qd0, tau, gqT, gqdT, integrator, fd)


def _pool_map(fn, jobs, workers):
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    workers = max(1, min(workers or (os.cpu_count() or 1), len(jobs)))
    if workers == 1:
        return [fn(j) for j in jobs]
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, jobs))


def oracle_forward_parallel(model, systems, q0, qd0, tau, integrator="semi", fd="aba", workers=None):
    """oracle_forward over a spawned process pool (one job per topology group,
    largest first); same result layout."""
    nqm, nvm = q0.shape[0], qd0.shape[0]
    col = {s: i for i, s in enumerate(systems)}
    grps = sorted(groups(model, systems), key=lambda g: -len(model.links(g[0])) * len(g))
    sub = lambda x, g: np.ascontiguousarray(x[..., g])  # noqa: E731
    jobs = [(model, list(range(len(g))), sub(q0, g), sub(qd0, g), sub(tau, g), integrator, fd) for g in grps]
    jobs = [(model.subset(g),) + j[1:] for g, j in zip(grps, jobs)]
    qT = np.zeros((nqm, len(systems)))
    qdT = np.zeros((nvm, len(systems)))
    for g, (_, (a, b)) in zip(grps, _pool_map(_fwd_job, jobs, workers)):
        for j, s in enumerate(g):
            qT[:a.shape[0], col[s]] = a[:, j]
            qdT[:b.shape[0], col[s]] = b[:, j]
    return qT, qdT


def oracle_backward_parallel(model, systems, q0, qd0, tau, gqT, gqdT, integrator="semi", fd="crba",
                             workers=None):
    """oracle_backward over a spawned process pool, one job per system."""
    nqm, nvm = q0.shape[0], qd0.shape[0]
    T = tau.shape[0]
    S = len(systems)
    out = dict(gq0=np.zeros((nqm, S)), gqd0=np.zeros((nvm, S)), gtau=np.zeros((T, nvm, S)), gm={})
    sub = lambda x, s: np.ascontiguousarray(x[..., [s]])  # noqa: E731
    jobs = [(model.subset([s]), [0], sub(q0, s), sub(qd0, s), sub(tau, s), sub(gqT, s), sub(gqdT, s),
             integrator, fd) for s in systems]
    for i, (s, (_, o)) in enumerate(zip(systems, _pool_map(_bwd_job, jobs, workers))):
        out["gq0"][:, i] = o["gq0"][:, 0]
        out["gqd0"][:, i] = o["gqd0"][:, 0]
        out["gtau"][:, :, i] = o["gtau"][:, :, 0]
        out["gm"][s] = o["gm"][0]
    return out
