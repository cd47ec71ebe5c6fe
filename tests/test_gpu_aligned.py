"""The world-aligned kernels (link frames with the world's orientation and their
origin at the joint; the inward recursion translates instead of rotating)
against the link-frame kernels and between their own launch variants, through
the C ABI.  Their parity with the oracle is covered wherever the automatic
choice runs them (every revolute model without contacts or limits:
test_gpu_parity.py, test_gpu_checkpoint_oracle.py, test_golden.py)."""
import numpy as np
import pytest
import torch

import workloads as wl
from tests._parity import check

pytestmark = pytest.mark.gpu


def _setup(work, precision, integrator="semi", seed=7):
    from paper_2109_07719_gb300 import Simulator
    sim = Simulator(work.model, precision=precision, integrator=integrator)
    dt, dev = sim.dtype, sim.device
    g = torch.Generator().manual_seed(seed)
    nv = torch.tensor(work.model.nv_per_system())
    mask_v = (torch.arange(work.model.nv_max)[:, None] < nv[None, :]).double()
    nq = torch.tensor(work.model.nq_per_system())
    mask_q = (torch.arange(work.model.nq_max)[:, None] < nq[None, :]).double()
    q0 = torch.tensor(work.q0).to(dt).to(dev)
    qd0 = (0.5 * torch.randn(work.qd0.shape, generator=g, dtype=torch.float64) * mask_v).to(dt).to(dev)
    tau = work.tau(device="cpu").to(dt).to(dev)
    gqT = (torch.randn(work.q0.shape, generator=g, dtype=torch.float64) * mask_q).to(dt).to(dev)
    gqdT = (torch.randn(work.qd0.shape, generator=g, dtype=torch.float64) * mask_v).to(dt).to(dev)
    return sim, q0, qd0, tau, gqT, gqdT


def _run(sim, space, q0, qd0, tau, gqT, gqdT, k=1, threads=32, persistent=False):
    sim.set_tape_space(space)
    sim.set_launch(threads, persistent)
    qT, qdT, ck, traj = sim.rollout(q0, qd0, tau, k=k, traj=True)
    g = sim.backward(ck, tau, gqT, gqdT, k=k)
    torch.cuda.synchronize()
    return (qT, qdT, traj) + tuple(g)


NAMES = ("qT", "qdT", "traj", "gq0", "gqd0", "gtau", "gmass")


@pytest.mark.parametrize("case", ["pendulum", "chains", "trees", "damped_trees", "explicit_chains"])
def test_aligned_matches_link_frame_fp64(case):
    """Two formulations of the same step: FP64 states within 1e-10 and gradients
    within 1e-9 (relative, max norm) over 40 steps."""
    integ = "explicit" if case == "explicit_chains" else "semi"
    if case == "pendulum":
        work = wl.config(1, B=3, T=40)
    elif case in ("chains", "explicit_chains"):
        work = wl.config(2, B=45, T=40, precision="fp64")
    else:
        work = wl.config(4, B=45, T=40, dof_hi=20, precision="fp64")
        if case == "damped_trees":
            work.model = work.model.with_damping(seed=31)
    sim, *x = _setup(work, "fp64", integ)
    a = _run(sim, "one_warp", *x)
    b = _run(sim, "aligned", *x)
    assert sim.last_storage()[1].startswith("aligned")
    for name, u, v in zip(NAMES, a, b):
        check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-10 if name in ("qT", "qdT", "traj") else 1e-9)
    assert sim.status().sum() == 0


def test_aligned_fp32_matches_link_frame():
    work = wl.config(4, B=70, T=30, dof_hi=30, precision="fp32")
    sim, *x = _setup(work, "fp32")
    a = _run(sim, "one_warp", *x)
    b = _run(sim, "aligned", *x)
    for name, u, v in zip(NAMES, a, b):
        check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-4)


def test_tape_on_chip_and_in_global_memory_agree():
    """7-link chains: one 32-system tile per block keeps the tape on chip; two
    tiles per block do not fit, so the same kernels keep it in global memory."""
    work = wl.config(2, B=100, T=25, precision="fp32")
    sim, *x = _setup(work, "fp32")
    a = _run(sim, "aligned", *x, threads=32)
    assert sim.last_storage() == ("aligned_shared", "aligned_shared")
    b = _run(sim, "aligned", *x, threads=128)
    assert sim.last_storage()[1] == "aligned_global"
    for name, u, v in zip(NAMES, a, b):
        check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-5)


@pytest.mark.parametrize("threads", [32, 64])
def test_persistent_schedule_matches_grid(threads):
    work = wl.config(4, B=200, T=20, dof_hi=40, precision="fp32")
    sim, *x = _setup(work, "fp32")
    a = _run(sim, "aligned", *x, threads=threads)
    b = _run(sim, "aligned", *x, threads=threads, persistent=True)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


@pytest.mark.parametrize("k", [5, 16])
def test_segment_and_quadratic_replay_match_every_step_checkpoints(k):
    work = wl.config(4, B=40, T=37, dof_hi=24, precision="fp64")
    sim, *x = _setup(work, "fp64")
    a = _run(sim, "aligned", *x, k=1)
    b = _run(sim, "aligned", *x, k=k)
    sim.set_replay("quadratic")
    c = _run(sim, "aligned", *x, k=k)
    sim.set_replay("segment")
    for name, u, v, w in zip(NAMES, a, b, c):
        check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-12)
        check(name, w.cpu().numpy(), u.cpu().numpy(), 1e-12)


def test_per_step_objective_terms():
    work = wl.config(2, B=33, T=20, precision="fp64")
    sim, q0, qd0, tau, gqT, gqdT = _setup(work, "fp64")
    g = torch.Generator().manual_seed(3)
    gtraj = torch.randn((21, sim.nx, sim.B), generator=g, dtype=torch.float64).to(sim.device)
    outs = []
    for space in ("one_warp", "aligned"):
        sim.set_tape_space(space)
        qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
        outs.append(sim.backward(ck, tau, gqT, gqdT, g_traj=gtraj))
    for name, u, v in zip(NAMES[3:], *outs):
        check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-9)


def test_aligned_refuses_other_models():
    from paper_2109_07719_gb300 import SimError
    for work in (wl.config(3, B=4, T=3, precision="fp64"),
                 wl.config(2, B=4, T=3, precision="fp64")):
        if work.model.name.startswith("serial"):
            work.model = work.model.with_limits(-0.5, 0.5)
        sim, q0, qd0, tau, gqT, gqdT = _setup(work, "fp64")
        sim.set_tape_space("aligned")
        with pytest.raises(SimError, match="world-aligned"):
            sim.rollout(q0, qd0, tau)
        sim.set_tape_space("auto")
        qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
        sim.backward(ck, tau, gqT, gqdT)
        torch.cuda.synchronize()
        assert not any(m.startswith("aligned") for m in sim.last_storage())


@pytest.mark.parametrize("space", ["aligned", "one_warp"])
def test_keeping_the_system_order_gives_the_same_results(space):
    """SIM_KEEP_SYSTEM_ORDER packs 32 consecutive systems per warp (lanes walking
    different numbers of links) instead of sorting by link count."""
    from paper_2109_07719_gb300 import Simulator
    work = wl.config(4, B=150, T=25, dof_hi=30, precision="fp32")
    a_sim, *x = _setup(work, "fp32")
    a = _run(a_sim, space, *x)
    b_sim = Simulator(work.model, precision="fp32", keep_order=True)
    assert list(b_sim.slot_order()) == list(range(150))
    b = _run(b_sim, space, *x)
    for name, u, v in zip(NAMES, a, b):
        check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-6)
    assert b_sim.status().sum() == 0


# ---------------------------------------------------------------- pipelined adjoint

@pytest.mark.parametrize("cfg,B,T,precision", [(2, 100, 37, "fp32"), (2, 33, 1, "fp32"), (2, 40, 2, "fp64"),
                                               (4, 150, 23, "fp32"), (4, 70, 9, "fp32_d64"), (1, 3, 30, "fp64")])
def test_pipelined_adjoint_matches_one_warp(cfg, B, T, precision):
    """Two warps per tile (recompute of step t beside the adjoint of step t + 1,
    tapes on chip for the 7-link chains, in global memory for the trees) against
    the one-warp world-aligned adjoint: the same formulas, so equal to round-off."""
    kw = dict(B=B, T=T) if cfg == 1 else dict(B=B, T=T, precision=precision)
    if cfg == 4:
        kw["dof_hi"] = 40
    work = wl.config(cfg, **kw)
    sim, *x = _setup(work, precision)
    a = _run(sim, "aligned", *x)
    assert sim.last_storage()[1].startswith("aligned_") and "pipelined" not in sim.last_storage()[1]
    b = _run(sim, "aligned_pipelined", *x)
    assert sim.last_storage()[1].startswith("aligned_pipelined")
    tol = 1e-12 if precision == "fp64" else 1e-6
    for name, u, v in zip(NAMES, a, b):
        check(name, v.cpu().numpy(), u.cpu().numpy(), tol)
    assert sim.status().sum() == 0


def test_pipelined_adjoint_persistent_and_per_step_terms():
    work = wl.config(4, B=200, T=15, dof_hi=30, precision="fp32")
    sim, q0, qd0, tau, gqT, gqdT = _setup(work, "fp32")
    g = torch.Generator().manual_seed(13)
    gtraj = torch.randn((16, sim.nx, sim.B), generator=g, dtype=torch.float64).float().to(sim.device)
    outs = []
    for space, persistent in (("aligned", False), ("aligned_pipelined", False), ("aligned_pipelined", True)):
        sim.set_tape_space(space)
        sim.set_launch(32, persistent)
        qT, qdT, ck, _ = sim.rollout(q0, qd0, tau)
        outs.append(sim.backward(ck, tau, gqT, gqdT, g_traj=gtraj))
        torch.cuda.synchronize()
    for u, v in zip(outs[1], outs[2]):
        assert torch.equal(u, v)
    for name, u, v in zip(NAMES[3:], outs[0], outs[1]):
        check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-6)


def _nested_trees(big=True, reps=8, precision="fp64", seed=11):
    """Trees whose stack of parent values runs deep, repeated with fresh link
    parameters: a caterpillar (each spine link's first child continues the spine,
    its leaf comes later, so every spine link keeps a stack entry: depth 19, or 3
    for the small one), a star, a forest of three roots, a chain and a random tree
    with up to three children per link."""
    if big:
        cat = [-1] + list(range(0, 19)) + list(range(0, 20))
        rng0 = np.random.default_rng(seed)
        rnd, kids, open_ = [-1], [0] * 30, [0]
        for i in range(1, 30):
            j = int(rng0.integers(len(open_)))
            p = open_[j]
            rnd.append(p)
            kids[p] += 1
            if kids[p] >= 3:
                open_.pop(j)
            open_.append(i)
        shapes = [cat, [-1] + [0] * 8, [-1, 0, 0, -1, 3, 3, 5, -1, 7], [-1] + list(range(0, 14)), rnd]
    else:
        shapes = [[-1, 0, 1, 2, 0, 1, 2, 3], [-1, 0, 0, 0, 0], [-1, 0, 0, -1, 3, 3, 5, -1, 7]]
    shapes = shapes * reps
    counts = [len(s) for s in shapes]
    parents = np.concatenate([np.asarray(s) for s in shapes])
    starts = np.zeros(len(parents), bool)
    starts[np.cumsum([0] + counts[:-1])] = True
    rng = np.random.default_rng(seed + 1)
    axis, r, mass, com, Ic = wl._random_tree_params(rng, parents, starts)
    r[parents < 0] = 0.0
    model = wl._assemble(counts, parents, np.zeros(len(parents)), axis, r, mass, com, Ic, 1e-3,
                         (0.0, 0.0, -9.81), "nested_trees")
    q0, qd0, mask = wl._state_arrays(model)
    q0[:] = rng.uniform(-1, 1, q0.shape) * (np.arange(model.nq_max)[:, None] < model.nq_per_system()[None, :])
    mask[:] = (np.arange(model.nv_max)[:, None] < model.nv_per_system()[None, :])
    return wl.Workload(model, q0, qd0, 30, 1.0, seed, precision, mask)


@pytest.mark.parametrize("big", [True, False])
def test_deeply_nested_trees_fp64(big):
    """The stack of parent values at depth 19 (and in shared memory for the small
    trees), stars, forests: the world-aligned kernels, one-warp and pipelined,
    against the link-frame kernels (which keep one accumulator per branching
    link) within 1e-10 (states) and 1e-9 (gradients)."""
    work = _nested_trees(big)
    sim, *x = _setup(work, "fp64")
    a = _run(sim, "one_warp", *x)
    for space in ("aligned", "aligned_pipelined"):
        b = _run(sim, space, *x)
        assert sim.last_storage()[1].startswith(space)
        for name, u, v in zip(NAMES, a, b):
            check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-10 if name in ("qT", "qdT", "traj") else 1e-9)
    assert sim.status().sum() == 0


def test_deeply_nested_trees_fp32_interleaved_adjoint():
    """FP32 with the tapes in global memory, where the adjoint interleaves two
    links' independent work: against the FP32 link-frame kernels."""
    work = _nested_trees(True, precision="fp32")
    sim, *x = _setup(work, "fp32")
    a = _run(sim, "one_warp", *x)
    b = _run(sim, "aligned_pipelined", *x)
    assert sim.last_storage()[1] == "aligned_pipelined_global"
    for name, u, v in zip(NAMES, a, b):
        check(name, v.cpu().numpy(), u.cpu().numpy(), 1e-4)
