"""FP64 running-state accumulation in the FP32 + FP64 D-solve mode: the
rollout sums q and qd in FP64 between steps and stores FP32.  A drifting free
body shows the mechanism exactly; chains and quadrupeds stay within the FP32
tolerances of the oracle, and the other precisions refuse the flag."""
import numpy as np
import pytest
import torch

import workloads as wl
from tests._parity import oracle_forward, oracle_backward, check

pytestmark = pytest.mark.gpu


def _free_body(B=8, dt=1e-3):
    """One free rigid body per system, COM at the link origin, no gravity: with no
    rotation and no force it moves at constant velocity (qdd = 0 exactly)."""
    n = B
    md = wl.ModelDesc(np.arange(n + 1, dtype=np.int32), -np.ones(n, np.int32), np.full(n, wl.FREE, np.int32),
                      np.zeros((n, 3)), np.tile([1.0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], (n, 1)), np.ones(n),
                      np.zeros((n, 3)), np.tile([0.1, 0.1, 0.1, 0, 0, 0], (n, 1)), dt, np.zeros(3), "free_body")
    return md


def test_fp64_sums_keep_increments_below_fp32_resolution():
    """x = 1000 m, v = 1 cm/s, dt = 1 ms: each step adds 1e-5 m, under half an FP32
    ulp at 1000 (3.05e-5).  Summed in FP32 the body never moves; summed in FP64 it
    reaches 1000.01 m after 1000 steps (stored as the nearest FP32)."""
    from paper_2109_07719_gb300 import Simulator
    B, T = 8, 1000
    sim = Simulator(_free_body(B), precision="fp32_d64")
    dev = sim.device
    q0 = torch.zeros(7, B, dtype=torch.float32, device=dev)
    q0[0] = 1000.0
    q0[6] = 1.0                                    # identity quaternion (x y z w)
    qd0 = torch.zeros(6, B, dtype=torch.float32, device=dev)
    qd0[3] = 0.01                                  # body-frame linear velocity along x
    tau = torch.zeros(T, 6, B, dtype=torch.float32, device=dev)
    qT32, qdT32, _, _ = sim.rollout(q0, qd0, tau)
    sim.set_state_accumulation("fp64")
    qT64, qdT64, ck, _ = sim.rollout(q0, qd0, tau)
    torch.cuda.synchronize()
    assert torch.all(qT32[0] == 1000.0)
    expect = np.float32(1000.0 + T * 1e-3 * np.float64(np.float32(0.01)))
    assert torch.all(qT64[0].cpu() == torch.tensor(expect))
    assert torch.equal(qdT64, qdT32)
    # checkpoints are the FP32 rounding of the FP64 running state
    assert float(ck[500][0, 0]) == np.float32(1000.0 + 500 * 1e-3 * np.float64(np.float32(0.01)))
    sim.set_state_accumulation("fp32")
    qT, _, _, _ = sim.rollout(q0, qd0, tau)
    assert torch.equal(qT, qT32)


@pytest.mark.parametrize("cfg,B,T", [(2, 40, 300), (3, 37, 120)])
def test_fp64_state_accumulation_against_oracle(cfg, B, T):
    from paper_2109_07719_gb300 import Simulator
    work = wl.config(cfg, B=B, T=T, precision="fp32")
    sim = Simulator(work.model, precision="fp32_d64")
    dev = sim.device
    q0 = torch.tensor(work.q0, dtype=torch.float32)
    g = torch.Generator().manual_seed(31)
    nv = torch.tensor(work.model.nv_per_system())
    mask = (torch.arange(sim.nv_max)[:, None] < nv[None, :]).float()
    qd0 = (0.5 * torch.randn(work.qd0.shape, generator=g, dtype=torch.float64)).float() * mask
    tau = work.tau(T=T).float()
    gqT = torch.randn(q0.shape, generator=g, dtype=torch.float64).float()
    gqdT = torch.randn(qd0.shape, generator=g, dtype=torch.float64).float() * mask
    d = [x.to(dev) for x in (q0, qd0, tau, gqT, gqdT)]
    h = [x.double().numpy() for x in (q0, qd0, tau, gqT, gqdT)]
    out = {}
    for mode in ("fp32", "fp64"):
        sim.set_state_accumulation(mode)
        qT, qdT, ck, _ = sim.rollout(d[0], d[1], d[2])
        grads = sim.backward(ck, d[2], d[3], d[4])
        torch.cuda.synchronize()
        assert sim.last_storage()[0] != "pipelined" or mode == "fp32"
        out[mode] = (qT.cpu().numpy(), qdT.cpu().numpy()) + tuple(x.cpu().numpy() for x in grads)
    assert not np.array_equal(out["fp32"][0], out["fp64"][0])
    oq, oqd = oracle_forward(work.model, list(range(B)), h[0], h[1], h[2])
    sel = [0, B // 2, B - 1]
    o = oracle_backward(work.model, sel, h[0], h[1], h[2], h[3], h[4])
    for mode in ("fp32", "fp64"):
        qT, qdT, gq0, gqd0, gtau, _ = out[mode]
        check(f"qT[{mode}]", qT, oq, 1e-3)
        check(f"qdT[{mode}]", qdT, oqd, 1e-3)
        check(f"gq0[{mode}]", gq0[:, sel], o["gq0"], 1e-2)
        check(f"gqd0[{mode}]", gqd0[:, sel], o["gqd0"], 1e-2)
        check(f"gtau[{mode}]", gtau[:, :, sel], o["gtau"], 1e-2)
    assert sim.status().sum() == 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_other_precisions_refuse_the_flag(precision):
    from paper_2109_07719_gb300 import Simulator, SimError
    work = wl.config(2, B=4, T=2, precision=precision)
    sim = Simulator(work.model, precision=precision)
    with pytest.raises(SimError, match="D-solve"):
        sim.set_state_accumulation("fp64")
    sim.set_state_accumulation("fp32")
