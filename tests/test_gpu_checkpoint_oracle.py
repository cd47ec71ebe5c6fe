"""GPU parity against the CPU FP64 oracle for the cases the k = 1 tests do not
reach directly.

1. Checkpoint interval k > 1 (Sec. 3.2 Eq. 7; the supplement's Sec. B): the
   segment replay and the supplement's quadratic recompute are compared with
   the oracle's gradient itself (which does not depend on k), not only with the
   GPU's own k = 1 run; chains, uneven trees and quadrupeds with foot contacts,
   T not a multiple of k, FP64 at the FP64 bounds (states 1e-8, gradients 1e-6).
2. The uneven-tree workload in FP32 (the precision it is specified in) over
   the full DOF range 2..64, several hundred systems: the final state of every
   system and the gradients of three systems, among them a 64-DOF tree, within
   the FP32 bounds (states 1e-3, gradients 1e-2).  The oracle runs over a pool
   of spawned processes.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from tests._parity import (check, mass_grad_of, oracle_backward, oracle_backward_parallel,
                           oracle_forward, oracle_forward_parallel)

pytestmark = pytest.mark.gpu


def _inputs(work, sim, T, q0=None, qd0=None, tau=None):
    q0 = torch.tensor(work.q0 if q0 is None else q0).to(sim.dtype)
    if qd0 is None:
        g = torch.Generator().manual_seed(work.seed + 9)
        nv = work.model.nv_per_system()
        mask = (torch.arange(work.model.nv_max)[:, None] < torch.tensor(nv)[None, :]).double()
        qd0 = (0.5 * torch.randn(work.qd0.shape, generator=g, dtype=torch.float64) * mask).to(sim.dtype)
    else:
        qd0 = torch.tensor(qd0).to(sim.dtype)
    tau = (work.tau(T=T) if tau is None else torch.tensor(tau)).to(sim.dtype)
    host = [x.double().numpy() for x in (q0, qd0, tau)]
    dev = [x.to(sim.device).contiguous() for x in (q0, qd0, tau)]
    return dev, host


def _contact_work(B, T):
    from oracle.contact import contact_points
    from oracle.dynamics import OracleModel
    work = wl.config(3, B=B, T=T, contacts=True, precision="fp64")
    om = OracleModel(work.model, list(range(B)))
    q = torch.tensor(work.q0.T).clone()
    q[:, 7:] = 0.0
    _, phi = contact_points(om, q)
    g = torch.Generator().manual_seed(3)
    clearance = torch.where(torch.arange(B) % 3 == 0, torch.full((B,), -0.004),
                            0.002 + 0.007 * torch.rand(B, generator=g, dtype=torch.float64))
    q[:, 2] -= phi.min(1).values - clearance
    qd = 0.2 * torch.randn(B, om.nv, generator=g, dtype=torch.float64)
    qd[:, 3:6] = 0.0
    qd[:, 5] = -1.0
    return work, np.ascontiguousarray(q.numpy().T), np.ascontiguousarray(qd.numpy().T)


def _work(kind, B, T):
    if kind == "chains":
        return wl.config(2, B=B, T=T, precision="fp64"), None, None
    if kind == "trees":
        return wl.config(4, B=B, T=T, dof_hi=24, precision="fp64"), None, None
    return _contact_work(B, T)


@pytest.mark.parametrize("kind,k,replay", [("chains", 7, "segment"), ("chains", 10, "segment"),
                                           ("chains", 100, "segment"), ("trees", 10, "segment"),
                                           ("contact", 10, "segment"), ("chains", 7, "quadratic"),
                                           ("trees", 10, "quadratic"), ("contact", 7, "quadratic")])
def test_checkpoint_interval_against_oracle(kind, k, replay):
    from paper_2109_07719_gb300 import Simulator
    B, T = 37, (123 if k == 100 else 53)          # T not a multiple of k; a ragged second tile
    work, q0h, qd0h = _work(kind, B, T)
    sim = Simulator(work.model, precision="fp64")
    sim.set_replay(replay)
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T, q0h, qd0h)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=k)
    assert ck.shape[0] == (T + k - 1) // k
    g = torch.Generator().manual_seed(23)
    gqT = torch.randn(qT.shape, generator=g, dtype=torch.float64)
    gqdT = torch.randn(qdT.shape, generator=g, dtype=torch.float64)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT.to(sim.device), gqdT.to(sim.device), k=k)
    torch.cuda.synchronize()
    assert sim.status().sum() == 0
    oq, oqd = oracle_forward(work.model, list(range(B)), hq, hqd, ht)
    check("qT", qT.cpu().numpy(), oq, 1e-8)
    check("qdT", qdT.cpu().numpy(), oqd, 1e-8)
    sel = [0, 1, 18, B - 1]
    o = oracle_backward(work.model, sel, hq, hqd, ht, gqT.numpy(), gqdT.numpy())
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], 1e-6)
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], 1e-6)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-6)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), sel)
    check("gmass", np.concatenate([gmd[s] for s in sel]), np.concatenate([o["gm"][s] for s in sel]), 1e-6)


def test_uneven_trees_fp32_full_dof_range():
    """320 trees with DOF ~ U{2..64} (branch factors 1..3) in FP32, T = 12: the
    launch the full-size run takes for trees this large (slot packing by link
    count, the batch's longest tree 64 links), against the FP64 oracle."""
    from paper_2109_07719_gb300 import Simulator
    B, T = 320, 12
    work = wl.config(4, B=B, T=T, precision="fp32")
    assert work.model.nv_max == 64
    sim = Simulator(work.model, precision="fp32")
    (q0, qd0, tau), (hq, hqd, ht) = _inputs(work, sim, T)
    qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=1)
    g = torch.Generator().manual_seed(29)
    gqT = torch.randn(qT.shape, generator=g, dtype=torch.float64).float()
    gqdT = torch.randn(qdT.shape, generator=g, dtype=torch.float64).float()
    nv = work.model.nv_per_system()
    mask_q = (np.arange(work.model.nq_max)[:, None] < work.model.nq_per_system()[None, :])
    mask_v = (np.arange(work.model.nv_max)[:, None] < nv[None, :])
    gqT *= torch.tensor(mask_q, dtype=torch.float32)
    gqdT *= torch.tensor(mask_v, dtype=torch.float32)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, gqT.to(sim.device), gqdT.to(sim.device), k=1)
    torch.cuda.synchronize()
    assert sim.status().sum() == 0
    rep = {}
    oq, oqd = oracle_forward_parallel(work.model, list(range(B)), hq, hqd, ht)
    check("qT", qT.cpu().numpy(), oq, 1e-3, rep)
    check("qdT", qdT.cpu().numpy(), oqd, 1e-3, rep)
    big = int(np.flatnonzero(nv == 64)[0])
    sel = [int(np.argmin(nv)), int(np.flatnonzero(nv == 33)[0]) if (nv == 33).any() else B // 2, big]
    o = oracle_backward_parallel(work.model, sel, hq, hqd, ht, gqT.double().numpy(), gqdT.double().numpy())
    check("gq0", gq0.cpu().numpy()[:, sel], o["gq0"], 1e-2, rep)
    check("gqd0", gqd0.cpu().numpy()[:, sel], o["gqd0"], 1e-2, rep)
    check("gtau", gtau.cpu().numpy()[:, :, sel], o["gtau"], 1e-2, rep)
    gmd = mass_grad_of(work.model, gm.cpu().numpy(), sel)
    check("gmass", np.concatenate([gmd[s] for s in sel]), np.concatenate([o["gm"][s] for s in sel]), 1e-2, rep)
    print("uneven trees fp32 relative errors:", rep)
