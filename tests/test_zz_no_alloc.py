"""sim_step_batch_static: the one-step entry point that allocates nothing.

It serves callers that cannot allocate device memory: a plug-in whose host
application owns every device allocation through its own pool and hands it only
a handle and state buffers, or a real-time loop where cudaMalloc's implicit
synchronisation and latency are not allowed.  Its per-link scratch is a fixed
16 MiB static device array inside the library instead of the handle's tape.
Here it is called through the C ABI (the ctypes binding) and compared, over two
calls in a row, with sim_step_batch on the same inputs, at the single-step
tolerance of the parity tests (1e-12 relative for FP64, 1e-6 for FP32).  This
file is collected last so that a failure here stops a first-failure run only
after every other test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("cfg,B,precision,tol", [(2, 256, "fp32", 1e-6), (3, 40, "fp64", 1e-12),
                                                 (5, 33, "fp32", 1e-6)])
def test_static_step_matches_step_batch(cfg, B, precision, tol):
    from paper_2109_07719_gb300 import Simulator
    work = wl.config(cfg, B=B, T=2, precision=precision)
    sim = Simulator(work.model, precision=precision)
    dev, dt = sim.device, sim.dtype
    q = torch.tensor(work.q0, dtype=dt, device=dev)
    g = torch.Generator().manual_seed(5)
    qd = (0.3 * torch.randn(work.qd0.shape, generator=g, dtype=torch.float64)).to(dt).to(dev)
    tau = work.tau(device="cpu").to(dt).to(dev)
    for t in range(2):                      # two calls in a row
        ref_q, ref_qd = sim.step(q, qd, tau[t])
        st_q, st_qd = sim.step_static(q, qd, tau[t])
        torch.cuda.synchronize()
        assert _rel(st_q, ref_q) <= tol
        assert _rel(st_qd, ref_qd) <= tol
        q, qd = ref_q, ref_qd
    assert sim.status().sum() == 0


def test_static_step_rejects_batches_beyond_the_static_scratch():
    from paper_2109_07719_gb300 import Simulator, SimError
    work = wl.config(2, B=8192, T=1, precision="fp32")   # 7 x 119 x 8192 x 4 B > 16 MiB
    sim = Simulator(work.model, precision="fp32")
    q = torch.zeros(sim.nq_max, sim.B, dtype=sim.dtype, device=sim.device)
    qd = torch.zeros(sim.nv_max, sim.B, dtype=sim.dtype, device=sim.device)
    with pytest.raises(SimError, match="static"):
        sim.step_static(q, qd, qd)


def test_static_step_leaves_device_memory_unchanged():
    """After the first call (which looks up the static array's address), further
    calls into caller-owned outputs change neither the device's free memory
    (cudaMemGetInfo) nor the memory torch has handed out."""
    from paper_2109_07719_gb300 import Simulator
    work = wl.config(2, B=512, T=1, precision="fp32")
    sim = Simulator(work.model, precision="fp32")
    dev, dt = sim.device, sim.dtype
    q = torch.tensor(work.q0, dtype=dt, device=dev)
    qd = torch.zeros(sim.nv_max, sim.B, dtype=dt, device=dev)
    tau = torch.zeros(sim.nv_max, sim.B, dtype=dt, device=dev)
    q_out, qd_out = torch.empty_like(q), torch.empty_like(qd)
    sim.step_static(q, qd, tau, q_out, qd_out)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_allocated(dev)
    for _ in range(3):
        sim.step_static(q, qd, tau, q_out, qd_out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.cuda.memory_allocated(dev) == alloc0
    assert torch.isfinite(q_out).all() and torch.isfinite(qd_out).all()
