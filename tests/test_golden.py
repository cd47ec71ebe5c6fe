"""The golden fixtures (tests/golden/, written by make_golden.py from the CPU
oracle): the oracle reproduces them (a regression pin of the oracle), and on a
GPU the CUDA path in FP64 matches them within the FP64 bounds (states 1e-8,
gradients 1e-6)."""
import json
import os
import sys

import numpy as np
import pytest
import torch

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
from make_golden import golden_model  # noqa: E402

from oracle.dynamics import OracleModel  # noqa: E402
from oracle.rollout import rollout, rollout_backward  # noqa: E402

NAMES = ["double_pendulum_1000_steps", "quadruped_contact_12_steps", "limited_chain_20_steps"]


def _load(name):
    with open(os.path.join(HERE, name + ".json")) as f:
        return json.load(f)


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-12))


@pytest.mark.parametrize("name", NAMES)
def test_oracle_reproduces_golden(name):
    g = _load(name)
    m = golden_model(name)
    om = OracleModel(m, [0])
    q = torch.tensor([g["q0"]], dtype=torch.float64)
    qd = torch.tensor([g["qd0"]], dtype=torch.float64)
    t = torch.tensor(g["tau"], dtype=torch.float64)[:, None, :]
    with torch.no_grad():
        qT, qdT, _ = rollout(om, q, qd, t, keep=False)
    r = rollout_backward(om, q, qd, t, torch.tensor([g["gqT"]], dtype=torch.float64),
                         torch.tensor([g["gqdT"]], dtype=torch.float64))
    for key, val in (("qT", qT[0]), ("qdT", qdT[0]), ("gq0", r[0][0]), ("gqd0", r[1][0]),
                     ("gtau", r[2][:, 0]), ("gmass", r[3][0])):
        assert _rel(val.numpy(), g[key]) < 1e-12, key


@pytest.mark.gpu
@pytest.mark.parametrize("name", NAMES)
def test_cuda_path_matches_golden(name):
    from paper_2109_07719_gb300 import Simulator
    g = _load(name)
    sim = Simulator(golden_model(name), precision="fp64")
    dev = sim.device
    col = lambda v: torch.tensor(v, dtype=torch.float64, device=dev)[:, None].contiguous()  # noqa: E731
    tau = torch.tensor(g["tau"], dtype=torch.float64, device=dev)[:, :, None].contiguous()
    qT, qdT, ck, _ = sim.rollout(col(g["q0"]), col(g["qd0"]), tau)
    gq0, gqd0, gtau, gm = sim.backward(ck, tau, col(g["gqT"]), col(g["gqdT"]))
    torch.cuda.synchronize()
    for key, val, tol in (("qT", qT[:, 0], 1e-8), ("qdT", qdT[:, 0], 1e-8), ("gq0", gq0[:, 0], 1e-6),
                          ("gqd0", gqd0[:, 0], 1e-6), ("gtau", gtau[:, :, 0], 1e-6), ("gmass", gm, 1e-6)):
        err = _rel(val.cpu().numpy(), g[key])
        assert err < tol, (key, err)
