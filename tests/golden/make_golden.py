"""Writes the golden fixtures of this directory from the CPU FP64 oracle alone
(no CUDA code is imported): final states and gradients of three small rollouts,
each tied to the paper passage it exercises.  Run from the repository root:

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as wl                                     # noqa: E402
from oracle.contact import contact_points                  # noqa: E402
from oracle.dynamics import OracleModel                    # noqa: E402
from oracle.rollout import rollout, rollout_backward       # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def golden_model(name):
    """The one-system model description of fixture `name` (seeded generators)."""
    if name.startswith("double_pendulum"):
        return wl.config(1).model.subset([0])
    if name.startswith("quadruped_contact"):
        return wl.config(3, B=1, T=12, contacts=True, precision="fp64").model.subset([0])
    w = wl.config(2, B=1, T=20, precision="fp64")
    return w.model.with_limits(-0.4, 0.4).subset([0])


def case(name, cite, work, q0, qd0, tau, gq_of_qT, gqd_of_qdT):
    """Rollout of system 0 and the gradients of <gqT, q^T> + <gqdT, qd^T>."""
    m = work.model.subset([0])
    om = OracleModel(m, [0])
    q = torch.tensor(q0[:om.nq, :1].T)
    qd = torch.tensor(qd0[:om.nv, :1].T)
    t = torch.tensor(tau[:, :om.nv, :1]).permute(0, 2, 1).contiguous()
    with torch.no_grad():
        qT, qdT, _ = rollout(om, q, qd, t, keep=False)
    gqT, gqdT = gq_of_qT(qT), gqd_of_qdT(qdT)
    g = rollout_backward(om, q, qd, t, gqT, gqdT)
    return {"name": name, "cite": cite, "dt": m.dt, "T": int(t.shape[0]),
            "q0": q[0].tolist(), "qd0": qd[0].tolist(), "tau": t[:, 0].tolist(),
            "gqT": gqT[0].tolist(), "gqdT": gqdT[0].tolist(),
            "qT": qT[0].tolist(), "qdT": qdT[0].tolist(),
            "gq0": g[0][0].tolist(), "gqd0": g[1][0].tolist(), "gtau": g[2][:, 0].tolist(),
            "gmass": g[3][0].tolist()}


def main():
    torch.set_default_dtype(torch.float64)   # the oracle's precision; only when run as a script
    out = []
    # 1. the double pendulum: Phi = sum q_T^2, gradients w.r.t. q0, qd0, every torque (Sec. 2 Eq. 1-2,
    #    Sec. 3.1 Eq. 3-4, Sec. 3.2 Eq. 7)
    w = wl.config(1)
    tau = w.tau().numpy()
    out.append(case("double_pendulum_1000_steps", "Sec. 2 Eq. 1-2; Sec. 3.1 Eq. 3-6; Sec. 3.2 Eq. 7",
                    w, w.q0, w.qd0, tau, lambda qT: 2 * qT, lambda qdT: torch.zeros_like(qdT)))
    # 2. a quadruped landing on its feet: contacts resolved as the Sec. 3.1 MLCP (Eq. 8) by PGS
    w = wl.config(3, B=1, T=12, contacts=True, precision="fp64")
    om = OracleModel(w.model, [0])
    q = torch.tensor(w.q0.T).clone()
    q[:, 7:] = 0.0
    _, phi = contact_points(om, q)
    q[:, 2] -= phi.min(1).values + 0.003
    qd = torch.zeros(1, om.nv)
    qd[:, 5] = -0.5
    out.append(case("quadruped_contact_12_steps", "Sec. 3.1 Eq. 8 (MLCP), supplement Alg. 1 (PGS)",
                    w, q.numpy().T, qd.numpy().T, w.tau().numpy(), lambda qT: torch.ones_like(qT),
                    lambda qdT: torch.ones_like(qdT)))
    # 3. a 7-DOF chain with joint limits as unilateral MLCP rows
    w = wl.config(2, B=1, T=20, precision="fp64")
    w.model = w.model.with_limits(-0.4, 0.4)
    qd0 = np.full(w.qd0.shape, 0.3)
    out.append(case("limited_chain_20_steps", "Sec. 3.1 Eq. 8 (joint limits as LCP rows)",
                    w, w.q0, qd0, w.tau().numpy(), lambda qT: torch.ones_like(qT),
                    lambda qdT: torch.ones_like(qdT)))
    for c in out:
        with open(os.path.join(HERE, c["name"] + ".json"), "w") as f:
            json.dump(c, f, indent=0)
        print("wrote", c["name"])


if __name__ == "__main__":
    main()
