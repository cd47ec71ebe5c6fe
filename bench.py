"""Throughput of batched forward + adjoint rollouts on one GPU.

One step = one forward rollout of T steps with a checkpoint every k steps, plus
the adjoint rollout (recompute + hand-derived adjoint) that returns gradients
with respect to the initial state, every joint torque and every link mass, for
a batch of B independent articulated systems.  Default workload: the largest
single-GPU configuration, 16384 uneven revolute trees with DOF ~ U{2..64}
(branch factors 1..3), dt 1e-3, T = 5000, FP32, k = 1.

Prints one JSON line.  `--impl reference` times the CPU FP64 oracle on a bounded
sample of the same workload instead.  `--gpus N` without a launcher starts N
ranks itself (one process per GPU, each on its own batch).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s fwd+adjoint"

# Algorithmic FLOPs per system-step of the kernels' formulation, from the
# counting build of the step functions (paper_2109_07719_gb300/flopcount.cpp):
# per revolute link with a parent / revolute root / free root, for the forward
# step (kinematics + three passes + integration) and for the adjoint step.
FLOPS = None  # filled by _flop_table()


def _flop_table():
    path = os.path.join(ROOT, "paper_2109_07719_gb300", "flops.json")
    with open(path) as f:
        return json.load(f)


def flops_per_system_step(model, kind):
    """kind: 'fwd' / 'adj' (link-frame step: forward, adjoint without its recompute)
    or 'wfwd' / 'wrec' / 'wadj' (world-aligned step: the rollout's step, the
    adjoint's recompute, the adjoint step; revolute joints only)."""
    import numpy as np
    tab = _flop_table()[kind]
    jt = np.asarray(model.joint_type)
    par = np.asarray(model.parent)
    n_free = int((jt == 1).sum())
    n_rev_root = int(((jt == 0) & (par < 0)).sum())
    n_rev = int(((jt == 0) & (par >= 0)).sum())
    if n_free and "free_root" not in tab:
        raise ValueError(f"{kind}: no FLOP count for free joints")
    return (tab["rev"] * n_rev + tab["rev_root"] * n_rev_root + tab.get("free_root", 0) * n_free) / model.n_systems


def kernel_flops(model, storage):
    """(rollout kernel, its FLOPs per system-step, adjoint kernel, its FLOPs per
    system-step) for the storage modes the last launches reported."""
    fwd_aligned = storage[0].startswith("aligned")
    bwd_aligned = storage[1].startswith("aligned")
    kf = "k_wrollout" if fwd_aligned else ("k_rollout_pipe" if storage[0] == "pipelined" else "k_rollout")
    kb = ("k_wbackward_pipe" if storage[1].startswith("aligned_pipelined") else "k_wbackward") if bwd_aligned else \
        ("k_backward_pipe" if storage[1] == "pipelined" else "k_backward")
    ff = flops_per_system_step(model, "wfwd" if fwd_aligned else "fwd")
    fb = (flops_per_system_step(model, "wrec") + flops_per_system_step(model, "wadj")) if bwd_aligned else \
        (flops_per_system_step(model, "fwd") + flops_per_system_step(model, "adj"))
    return kf, ff, kb, fb


def source_digest() -> str:
    """Digest of the CUDA sources, to tell whether stored ncu counters still apply."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2109_07719_gb300", "csrc", "*"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload_name: str, B: int, T: int, precision: str, k: int):
    """DRAM bytes per launch of `kernel` from a committed ncu capture taken on this
    workload with the current sources (profiles/traffic_*.json), else None.  A
    record either holds per-launch bytes at one horizon or, for captures taken at
    a short horizon, bytes per step, scaled here to T steps (the kernels stream the
    same per-step traffic at every step)."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "traffic_*.json"))):
        with open(path) as f:
            rec = json.load(f)
        match = rec.get("match", {})
        if not (match.get("workload") == workload_name and match.get("n_systems") == B and
                match.get("precision") == precision and match.get("k") == k and
                match.get("horizon") in (None, T)):
            continue
        if rec.get("source_sha256_16") != source_digest():
            return None
        kr = rec["kernels"].get(kernel, {})
        if "traffic_bytes_per_step" in kr:
            return kr["traffic_bytes_per_step"] * T
        return kr.get("traffic_bytes_per_launch")
    return None


def _clock_sampler(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]]
    while not stop.is_set():
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=5)
            if r.returncode == 0 and r.stdout.strip():
                out.append([x.strip() for x in r.stdout.strip().split(",")])
        except Exception:
            pass
        stop.wait(0.2)


def _clocks_summary(samples):
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    import statistics
    sm = [float(s[0]) for s in samples if s[0].replace(".", "").isdigit()]
    mx = [float(s[1]) for s in samples if s[1].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for s in samples for i in range(4) if len(s) > 4 + i and s[4 + i] == "Active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def workload(cfg: int, precision: str, B=None, T=None, rank: int = 0, contacts: bool = False,
             limits: bool = False, slot_order: bool = False):
    """The workload of this rank: ranks simulate disjoint batches (their own seed).
    ``limits``: every revolute joint limited to [-0.5, 0.5] rad (chains and the
    quadruped, at most 12 limited joints per system).  ``slot_order``: the batch
    laid out by link count, as the library packs it (mixed-size batches)."""
    import workloads as wl
    kw = {"seed": wl.SEED_BASE + cfg + 1000 * rank}
    if contacts:
        if cfg != 3:
            raise SystemExit("--contacts applies to the quadruped workload (--config 3)")
        kw["contacts"] = True
    if B:
        kw["B"] = B
    if T:
        kw["T"] = T
    if cfg != 1:
        kw["precision"] = precision
    work = wl.config(cfg, **kw)
    if slot_order:
        work = work.in_slot_order()
    if limits:
        if cfg not in (2, 3):
            raise SystemExit("--limits applies to the chain and quadruped workloads (--config 2 or 3)")
        work.model = work.model.with_limits(-0.5, 0.5)
    return work


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2109_07719_gb300 import Simulator

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
        ws = dist.get_world_size()                 # the ranks that joined the process group
    peak = fp_peak(args.precision) if rank == 0 else None   # before any timing: the probe fills the GPU
    work = workload(args.config, args.precision, args.batch, args.horizon, rank, args.contacts, args.limits,
                    args.slot_layout)
    m = work.model
    T, k = work.T, args.k
    free0 = torch.cuda.mem_get_info()[0]
    sim = Simulator(m, precision=args.precision, keep_order=args.keep_order)
    handle_bytes = free0 - torch.cuda.mem_get_info()[0]
    sim.set_tape_space(args.tape)
    sim.set_replay(args.replay)
    if args.prefetch is not None:
        sim.set_prefetch(args.prefetch)
    if args.state_accumulation != "fp32":
        sim.set_state_accumulation(args.state_accumulation)
    tuned = None
    if args.autotune:
        from paper_2109_07719_gb300 import autotune as _at
        best = sim.autotune(torch.tensor(work.q0, dtype=sim.dtype, device=sim.device),
                            torch.tensor(work.qd0, dtype=sim.dtype, device=sim.device))
        tuned = {"threads": best[0], "schedule": "persistent" if best[1] else "grid",
                 "kernels": _at.TAPE_SPACE[best[2]]}
    elif args.block or args.persistent:
        sim.set_launch(args.block, args.persistent)
    dev, dt = sim.device, sim.dtype
    B = sim.B
    q0 = torch.tensor(work.q0, dtype=dt, device=dev)
    qd0 = torch.tensor(work.qd0, dtype=dt, device=dev)
    tau = work.tau(device=dev, dtype=dt)
    # output and scratch buffers, allocated once (the calls allocate nothing)
    qT, qdT = sim.empty(sim.nq_max, B), sim.empty(sim.nv_max, B)
    ck = sim.empty((T + k - 1) // k, sim.nx, B)
    gq0, gqd0 = sim.empty(sim.nq_max, B), sim.empty(sim.nv_max, B)
    gtau = sim.empty(T, sim.nv_max, B)
    gm = sim.empty(sim.n_links)
    wb = sim.work_bytes(k)
    work_buf = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    gqT = torch.ones_like(qT)
    gqdT = torch.zeros_like(qdT)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(evs=None, kk=k, ckb=ck, wbuf=work_buf):
        if evs:
            evs[0].record(stream)
        sim.rollout(q0, qd0, tau, k=kk, out=(qT, qdT, ckb, None))
        if evs:
            evs[1].record(stream)
        sim.backward(ckb, tau, gqT, gqdT, k=kk, work=wbuf, out=(gq0, gqd0, gtau, gm))
        if evs:
            evs[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    graph = None
    if args.graph:
        # the whole step (forward rollout, adjoint rollout, mass-gradient gather) as one
        # CUDA graph: the calls allocate nothing, so they capture as plain kernel nodes
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()
    stop = threading.Event()
    samples = []
    th = threading.Thread(target=_clock_sampler, args=(stop, samples), daemon=True)
    th.start()
    time.sleep(0.3)
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.reset_peak_memory_stats()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))            # evict L2 between timed steps (not timed)
        step(events[i])
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    stop.set()
    th.join()
    peak_torch = torch.cuda.max_memory_allocated()
    fwd_ms = [e[0].elapsed_time(e[1]) for e in events]
    adj_ms = [e[1].elapsed_time(e[2]) for e in events]
    graph_ms = None
    if graph is not None:   # the same step replayed as one CUDA graph
        n_rep = min(args.steps, 2)
        gev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n_rep)]
        for i in range(n_rep):
            flush.fill_(float(i))
            gev[i][0].record(stream)
            graph.replay()
            gev[i][1].record(stream)
        torch.cuda.synchronize()
        graph_ms = float(np.mean([a.elapsed_time(b) for a, b in gev]))
        del graph
    step_ms = float(np.sum(fwd_ms) + np.sum(adj_ms)) / args.steps
    step_ms, units = aggregate(step_ms, B * T, dev)
    flags = sim.status()
    value = units / (step_ms / 1e3)
    storage = sim.last_storage()
    k_sweep = None
    if args.k_sweep and rank == 0:
        k_sweep = checkpoint_sweep(sim, step, T, B, flush, [int(x) for x in args.k_sweep.split(",")])
    grad_err = None
    if args.grad_check and rank == 0:
        grad_err = precision_error(sim, work, args, (qT, qdT, gq0, gqd0, gtau, gm), ck, tau)
    del ck, work_buf, gtau
    e2e = None
    if args.e2e:
        torch.cuda.empty_cache()
        e2e = run_e2e(sim, work, k, args.steps, tau.cpu().pin_memory(), q0.cpu().pin_memory(),
                      qd0.cpu().pin_memory())
    if rank != 0:
        return None
    kf, f_fwd, kb, f_bwd = kernel_flops(m, storage)
    adj_flops = B * T * f_bwd
    adj_s = float(np.mean(adj_ms)) / 1e3
    clocks = _clocks_summary(samples)
    achieved = adj_flops / adj_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp32_d64": "f32+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": m.name, "n_systems": B, "horizon": T, "dt": m.dt, "checkpoint_interval": k,
                   "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "block": sim.launch[0], "schedule": "persistent" if sim.launch[1] else "grid",
                   "slot_order": "system" if args.keep_order else "link count",
                   "batch_layout": "by link count (the packing order)" if args.slot_layout else "as generated",
                   "tape": args.tape, "autotuned": tuned, "replay": args.replay, "prefetch": args.prefetch, "state_accumulation": args.state_accumulation,
                   "storage": {"rollout": storage[0], "adjoint": storage[1]},
                   "cuda_graph": bool(args.graph), "contacts": bool(args.contacts),
                   "joint_limits": bool(args.limits)},
        "fwd_env_steps_per_s": B * T / (float(np.mean(fwd_ms)) / 1e3),
        "ms_fwd": float(np.mean(fwd_ms)), "ms_adj": float(np.mean(adj_ms)),
        "ms_per_step_cuda_graph": graph_ms,
        "roofline": {"bound": "alu", "kernel": kb, "achieved": achieved, "peak": peak["tflops"],
                     "unit": "TFLOP/s", "frac": achieved / peak["tflops"],
                     "traffic": measured_traffic(kb, m.name, B, T, args.precision, k),
                     "flops_per_system_step": {kf: f_fwd, kb: f_bwd},
                     "peak_note": peak["note"] + ("; the FLOP count covers the ABA step only, not the constraint "
                                                  "solve" if args.contacts or args.limits else ""),
                     "peaks_measured": {x: (peak.get("probe") or {}).get(x) for x in ("fp32_tflops", "fp64_tflops")},
                     "rollout": {"kernel": kf, "achieved": B * T * f_fwd / (float(np.mean(fwd_ms)) / 1e3) / 1e12,
                                 "frac": B * T * f_fwd / (float(np.mean(fwd_ms)) / 1e3) / 1e12 / peak["tflops"]}},
        "peak_mem_bytes": {"device_total": int(peak_torch + handle_bytes), "torch_allocator": int(peak_torch),
                           "handle": int(handle_bytes),
                           "note": "peak of the timed steps: inputs, checkpoints, outputs, the 256 MB L2-flush "
                                   "buffer (torch's allocator) and the handle's own buffers (model constants, "
                                   "tape scratch)"},
        "grad_rel_err": grad_err,
        "k_sweep": k_sweep,
        "e2e": e2e,
        "gpu_launches": args.steps * 3,
        "clocks": clocks,
        "nonfinite_systems": int((flags != 0).sum()),
        "nonfinite_ids": [int(i) for i in np.flatnonzero(np.asarray(flags) != 0)[:16]],
    }
    if args.plain:
        pl = plain_per_system(work, args, k, n_sys=args.plain_systems, tau_dev=tau)
        line["plain_per_system"] = pl
        line["vs_plain_per_system"] = value / pl["value"]
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
        one = cpu_baseline(args, budget_s=8.0, threads=1)
        line["cpu_baseline"]["one_core"] = {"value": one["value"], "unit": one["unit"], "cores": 1}
    return line


def checkpoint_sweep(sim, step, T, B, flush, ks):
    """Time per bench step with a checkpoint every k steps (Sec. 3.2 Eq. 7 and the
    supplement's Sec. B): one warm-up and one timed step per k, own checkpoint and
    workspace buffers; the checkpoint memory is ceil(T/k) states."""
    import torch
    out = {}
    for kk in ks:
        ckb = sim.empty((T + kk - 1) // kk, sim.nx, B)
        wbuf = torch.empty(max(sim.work_bytes(kk), 1), dtype=torch.uint8, device=sim.device)
        step(kk=kk, ckb=ckb, wbuf=wbuf)
        torch.cuda.synchronize()
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        step(ev, kk=kk, ckb=ckb, wbuf=wbuf)
        torch.cuda.synchronize()
        out[str(kk)] = {"ms_fwd": ev[0].elapsed_time(ev[1]), "ms_adj": ev[1].elapsed_time(ev[2]),
                        "env_steps_per_s": B * T / (ev[0].elapsed_time(ev[2]) / 1e3),
                        "ckpt_bytes": int(sim.ckpt_bytes(T, kk)), "work_bytes": int(sim.work_bytes(kk))}
        del ckb, wbuf
    return out


def _rel(a, b, floor=1e-12):
    """max |a - b| / max(max |b|, floor): the per-output relative error."""
    import numpy as np
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if not np.all(np.isfinite(a)):
        return float("inf")
    return float(np.abs(a - b).max() / max(np.abs(b).max(), floor))


def precision_error(sim, work, args, outs, ck, tau_dev, n_sample=8, horizons=(250, 500, 1000, 2000)):
    """Per-output relative error of the FP32 (or FP64) path against the library's
    FP64 path (whose parity with the CPU FP64 oracle, states 1e-8 and gradients
    1e-6, the GPU tests check), after the timed region, on sampled systems -- the
    smallest, the largest and others spread over the link counts.  Reported at the
    full horizon (the timed run's own outputs against an FP64 handle of those
    systems from the same inputs and seeds) and, because a long chaotic horizon
    can amplify any rounding beyond the bounds, at shorter horizons too: there both
    sides rerun the sampled systems (same kernels, one handle per precision), and
    the FP64 run's own sensitivity (the same run with q0 perturbed by 1e-12
    relative) says how much the dynamics amplify a perturbation by then.  The
    largest horizon whose errors meet the bounds is reported (the survey's reading
    for chaotic workloads)."""
    import numpy as np
    import torch
    from paper_2109_07719_gb300 import Simulator
    m = work.model
    T, k = work.T, args.k
    nv = m.nv_per_system()
    order = np.argsort(nv, kind="stable")
    pick = np.unique(np.round(np.linspace(0, len(order) - 1, n_sample)).astype(int))
    sel = sorted({int(order[i]) for i in pick})
    sub = m.subset(sel)
    ref = Simulator(sub, precision="fp64")
    low = Simulator(sub, precision=args.precision)
    dev = ref.device
    nqs, nvs = ref.nq_max, ref.nv_max
    # the timed run's inputs for these systems (rounded to its precision), in FP64 and its own dtype
    q0 = torch.tensor(np.ascontiguousarray(work.q0[:nqs, sel]), dtype=sim.dtype, device=dev).contiguous()
    qd0 = torch.tensor(np.ascontiguousarray(work.qd0[:nvs, sel]), dtype=sim.dtype, device=dev).contiguous()
    tau_s = tau_dev[:, :nvs][:, :, torch.tensor(sel, device=tau_dev.device)].to(dev).contiguous()
    q64, qd64, tau64 = q0.double().contiguous(), qd0.double().contiguous(), tau_s.double().contiguous()
    tol = (1e-8, 1e-6) if args.precision == "fp64" else (1e-3, 1e-2)
    lo = m.sys_link_offset

    def grads_err(a, b, gma, gmb):
        return {"qT": _rel(a[0].cpu(), b[0].cpu()), "qdT": _rel(a[1].cpu(), b[1].cpu()),
                "gq0": _rel(a[2].cpu(), b[2].cpu()), "gqd0": _rel(a[3].cpu(), b[3].cpu()),
                "gtau": _rel(a[4].cpu(), b[4].cpu()), "gmass": _rel(gma, gmb)}

    def within(e):
        return bool(max(e["qT"], e["qdT"]) <= tol[0] and max(e["gq0"], e["gqd0"], e["gtau"], e["gmass"]) <= tol[1])

    def run(h_sim, q, qd, tt):
        qT, qdT, ckh, _ = h_sim.rollout(q, qd, tt, k=1)
        g = h_sim.backward(ckh, tt, torch.ones_like(qT), torch.zeros_like(qdT), k=1)
        return (qT, qdT) + tuple(g[:3]), g[3], ckh

    # full horizon: the timed run's own outputs
    r64, gm64, ck64 = run(ref, q64, qd64, tau64)
    qTp, _, ckp, _ = ref.rollout(q64 * (1 + 1e-12), qd64, tau64, k=1)
    torch.cuda.synchronize()
    qT32, qdT32, gq0, gqd0, gtau, gm = outs
    cols = torch.tensor(sel, device=qT32.device)
    mine = (qT32[:nqs, cols], qdT32[:nvs, cols], gq0[:nqs, cols], gqd0[:nvs, cols], gtau[:, :nvs][:, :, cols])
    gmm = np.concatenate([gm.cpu().numpy()[lo[s]:lo[s + 1]] for s in sel])
    full = grads_err(mine, r64, gmm, gm64.cpu().numpy())
    out = {"reference": "the library's FP64 path (oracle parity checked in the GPU tests)", "systems": sel,
           "dof": [int(nv[s]) for s in sel], "tolerance": {"states": tol[0], "gradients": tol[1]},
           "per_output": full, "horizon": T, "within_tolerance": within(full),
           "fp64_self_sensitivity": _rel(ckp[-1].cpu(), ck64[-1].cpu()) if T > 0 else 0.0,
           "nonfinite_in_fp64": int((ref.status() != 0).sum()), "by_horizon": {}}
    best = None
    for h in sorted(x for x in horizons if x < T):
        a, gma, _ = run(low, q0, qd0, tau_s[:h].contiguous())
        b, gmb, _ = run(ref, q64, qd64, tau64[:h].contiguous())
        torch.cuda.synchronize()
        e = grads_err(a, b, gma.cpu().numpy(), gmb.cpu().numpy())
        e["fp64_self_sensitivity"] = _rel(ckp[h].cpu(), ck64[h].cpu())
        e["within_tolerance"] = within(e)
        out["by_horizon"][str(h)] = e
        if e["within_tolerance"]:
            best = h
    if out["within_tolerance"]:
        best = T
    out["largest_horizon_within_tolerance"] = best
    del ref, low
    return out


def plain_per_system(work, args, k, n_sys=64, tau_dev=None):
    """The same kernels with one system per launch (a 1-system handle each), systems
    run one after another: the per-system GPU version the batched path is compared
    with.  n_sys systems are timed and the rate is per env-step (extrapolation to the
    whole batch is linear: the launches are serial)."""
    import numpy as np
    import torch
    from paper_2109_07719_gb300 import Simulator
    m = work.model
    T = work.T
    sims, bufs, taus = [], [], []
    if tau_dev is None:
        tau_dev = work.tau(device="cuda", dtype=torch.float64 if args.precision == "fp64" else torch.float32)
    for b in range(min(n_sys, m.n_systems)):
        sim = Simulator(m.subset([b]), precision=args.precision)
        if args.state_accumulation != "fp32":
            sim.set_state_accumulation(args.state_accumulation)
        dev, dt = sim.device, sim.dtype
        q0 = torch.tensor(np.ascontiguousarray(work.q0[:sim.nq_max, b:b + 1]), dtype=dt, device=dev).contiguous()
        qd0 = torch.tensor(np.ascontiguousarray(work.qd0[:sim.nv_max, b:b + 1]), dtype=dt, device=dev).contiguous()
        sims.append(sim)
        bufs.append((q0, qd0))
        taus.append(tau_dev[:, :sim.nv_max, b:b + 1].to(dt).contiguous())

    def run_all():
        for sim, (q0, qd0), tau in zip(sims, bufs, taus):
            qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=k)
            sim.backward(ck, tau, torch.ones_like(qT), torch.zeros_like(qdT), k=k)

    run_all()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run_all()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": len(sims) * T / (ms / 1e3), "unit": "env-steps/s", "systems_timed": len(sims),
            "ms": ms, "note": "one system per launch (rollout + adjoint), systems serial; "
                              "rate per env-step from the timed systems"}


def aggregate(step_ms: float, units: int, device="cpu"):
    """Whole-job timing over ranks: the slowest rank's time per step and the env-steps
    all ranks processed (each rank runs its own batch, no data exchange)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return step_ms, units
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


_PEAKS = {}


def measure_fma_peaks():
    """FP32 and FP64 FMA throughput of this GPU from the library's probe
    (paper_2109_07719_gb300/_lib/fma_peak, built with the library), with the SM
    clock sampled while it runs; None if the probe is missing or fails."""
    if "probe" in _PEAKS:
        return _PEAKS["probe"]
    from paper_2109_07719_gb300 import build as b
    res = None
    if os.path.exists(b.FMA_PEAK):
        stop, samples = threading.Event(), []
        th = threading.Thread(target=_clock_sampler, args=(stop, samples), daemon=True)
        th.start()
        try:
            r = subprocess.run([b.FMA_PEAK], capture_output=True, text=True, timeout=120)
            if r.returncode == 0:
                res = json.loads(r.stdout.strip().splitlines()[-1])
        except (subprocess.TimeoutExpired, ValueError, IndexError):
            res = None
        stop.set()
        th.join()
        if res is not None:
            res["clocks"] = _clocks_summary(samples)
    _PEAKS["probe"] = res
    return res


def fp_peak(precision):
    """The roofline denominator: the FMA throughput measured on this GPU by the
    probe (FP32 for the FP32 storage modes, FP64 for the FP64 one); if the probe
    is unavailable, the nominal unit counts x the maximum clock (152 SMs x 128
    FP32 lanes x 2 FLOP x 2.07 GHz; FP64 the nominal 1.25 TFLOP/s), said so."""
    p = measure_fma_peaks()
    key = "fp64_tflops" if precision == "fp64" else "fp32_tflops"
    if p is not None and p.get(key):
        clk = p.get("clocks", {})
        return {"tflops": p[key], "note": f"measured: FMA-chain probe on this GPU ({key}; median SM clock "
                                          f"{clk.get('sm_mhz')} MHz during the probe)", "probe": p}
    if precision == "fp64":
        return {"tflops": 1.25, "note": "nominal FP64 vector rate of GB300 (1.25 TFLOP/s): probe unavailable"}
    return {"tflops": 152 * 128 * 2 * 2.07e9 / 1e12,
            "note": "nominal: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz (probe unavailable)"}


def run_e2e(sim, work, k, steps, tau_h, q0_h, qd0_h):
    """Same metric through the public API with host inputs: every step copies its
    (q0, qd0, tau) from pinned host memory to the device, runs Rollout forward and
    backward, and reads the gradients back to pinned host memory, all inside the
    timed region.  The copies run on a second stream, overlapped with the
    neighbouring steps' compute (double-buffered device inputs and host outputs),
    as a training loop that streams batches would."""
    import torch
    from paper_2109_07719_gb300 import Rollout
    dev = sim.device
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    ins = [tuple(torch.empty(x.shape, dtype=x.dtype, device=dev) for x in (q0_h, qd0_h, tau_h)) for _ in range(2)]
    outs = [(torch.empty(q0_h.shape, dtype=q0_h.dtype).pin_memory(),
             torch.empty(tau_h.shape, dtype=tau_h.dtype).pin_memory()) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def upload(i):
        b = i % 2
        with torch.cuda.stream(copy):
            if i >= 2:
                copy.wait_event(ev_free[b])            # step i - 2 is done with these buffers
            for dst, src in zip(ins[b], (q0_h, qd0_h, tau_h)):
                dst.copy_(src, non_blocking=True)
            ev_in[b].record(copy)

    def run(n):
        """n pipelined steps; seconds from before the first upload to the last download."""
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upload(0)
        for i in range(n):
            b = i % 2
            if i + 1 < n:
                upload(i + 1)
            comp.wait_event(ev_in[b])
            q0 = ins[b][0].detach().requires_grad_(True)
            qd0 = ins[b][1].detach().requires_grad_(True)
            tau = ins[b][2].detach().requires_grad_(True)
            qT, qdT = Rollout.apply(sim, q0, qd0, tau, None, k)
            qT.sum().backward()
            gq, gtau = q0.grad, tau.grad
            ev_free[b].record(comp)
            with torch.cuda.stream(copy):
                copy.wait_event(ev_free[b])
                if i >= 2:
                    ev_out[b].synchronize()            # the host buffers of step i - 2 are read
                outs[b][0].copy_(gq, non_blocking=True)
                outs[b][1].copy_(gtau, non_blocking=True)
                gq.record_stream(copy)
                gtau.record_stream(copy)
                ev_out[b].record(copy)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    run(1)                                             # warm-up, untimed
    elapsed = run(steps)
    s = elapsed / steps
    es = tau_h.element_size()
    return {"value": sim.B * work.T / s, "unit": "env-steps/s",
            "h2d_bytes_per_step": (q0_h.numel() + qd0_h.numel() + tau_h.numel()) * es,
            "d2h_bytes_per_step": (q0_h.numel() + tau_h.numel()) * es,
            "copies": "per step, on a second stream overlapped with the neighbouring steps' compute"}


ORACLE_SAMPLE = {4: (4, 5)}   # systems, steps of one oracle rollout of the CPU baseline (default 16, 20)


def _oracle_sample_size(config):
    return ORACLE_SAMPLE.get(config, (16, 20))


def _oracle_sample(config, precision, contacts, limits):
    """The CPU baseline's unit of work: forward + adjoint of a few systems of the
    workload over a few steps through the FP64 oracle (CRBA + RNEA forward,
    per-step recompute + reverse-mode step adjoint), one oracle batch per
    topology.  For the uneven trees the systems are spread over the link counts
    (the oracle's cost grows with them)."""
    import numpy as np
    import torch
    from oracle.dynamics import OracleModel
    from oracle.rollout import rollout_backward
    nsys, T = _oracle_sample_size(config)
    work = workload(config, precision, None if config == 4 else nsys, T, contacts=contacts, limits=limits)
    m = work.model
    if config == 4:
        order = np.argsort(m.nv_per_system(), kind="stable")
        sys_ = sorted(int(order[i]) for i in np.round(np.linspace(0, len(order) - 1, nsys)).astype(int))
    else:
        sys_ = list(range(min(nsys, m.n_systems)))
    tau = work.tau(T=T)
    groups = {}
    off = m.sys_link_offset
    for s in sys_:
        key = (tuple(m.parent[off[s]:off[s + 1]]), tuple(m.joint_type[off[s]:off[s + 1]]))
        groups.setdefault(key, []).append(s)

    def once():
        for grp in groups.values():
            om = OracleModel(m, grp)
            q0 = torch.tensor(work.q0[:om.nq, grp].T)
            qd0 = torch.tensor(work.qd0[:om.nv, grp].T)
            ot = tau[:, :om.nv, grp].permute(0, 2, 1).contiguous()
            rollout_backward(om, q0, qd0, ot, torch.ones_like(q0), torch.zeros_like(qd0))
        return len(sys_) * T

    return once


def _oracle_worker(config, precision, contacts, limits, budget_s, barrier, results):
    """One single-threaded process of the all-core baseline: waits for the others,
    then counts the env-steps it completes in budget_s."""
    import torch
    torch.set_num_threads(1)
    once = _oracle_sample(config, precision, contacts, limits)
    barrier.wait(timeout=600)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        done += once()
    results.put((done, time.perf_counter() - t0))


def cpu_baseline(args, budget_s: float = 15.0, threads: int | None = None):
    """The FP64 oracle on a bounded sample of the workload, scaled to env-steps/s:
    one process on one thread (threads=1), or one single-threaded process per host
    core, parallel over copies of the sample (the oracle batches its systems in
    small tensors, which intra-op threads barely speed up).  The process pool is
    started with spawn (this process may already hold a CUDA context)."""
    contacts, limits = getattr(args, "contacts", False), getattr(args, "limits", False)
    nsys, T = _oracle_sample_size(args.config)
    what = (f"{nsys} systems x {T} steps of the same workload, repeated for {budget_s:.0f} s "
            f"(FP64 CRBA+RNEA forward, per-step recompute + reverse-mode step adjoint)")
    if threads == 1:
        import torch
        prev = torch.get_num_threads()
        torch.set_num_threads(1)
        try:
            once = _oracle_sample(args.config, args.precision, contacts, limits)
            done, t0 = 0, time.perf_counter()
            while time.perf_counter() - t0 < budget_s:
                done += once()
            el = time.perf_counter() - t0
        finally:
            torch.set_num_threads(prev)
        return {"value": done / el, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
                "sample": what + ", one process"}
    import multiprocessing as mp
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(n + 1), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, daemon=True,
                         args=(args.config, args.precision, contacts, limits, budget_s, barrier, results))
             for _ in range(n)]
    try:
        for p in procs:
            p.start()
        barrier.wait(timeout=600)
        got = [results.get(timeout=budget_s + 300) for _ in range(n)]
    except Exception as e:  # a worker that failed to start or finish: report one process instead
        for p in procs:
            if p.is_alive():
                p.terminate()
        one = cpu_baseline(args, budget_s, threads=1)
        one["sample"] += f" (process pool unavailable: {type(e).__name__})"
        return one
    for p in procs:
        p.join(timeout=30)
    return {"value": sum(d / el for d, el in got), "unit": "env-steps/s", "cores": n, "kind": "oracle",
            "sample": what + f", in each of {n} single-threaded processes at once"}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return None
    cb = cpu_baseline(args, budget_s=max(5.0, 10.0 * args.steps / max(args.steps, 1)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "env-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.config, args.precision, 4, 1,
                                            contacts=getattr(args, "contacts", False),
                                            limits=getattr(args, "limits", False)).model.name,
                       "note": "CPU FP64 oracle, bounded sample"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def memory_sweep(args):
    """Peak device memory of one forward + adjoint rollout versus horizon (Table 1's
    'Ours' column shape): torch's allocator peak (inputs, outputs, checkpoints,
    workspace) plus the handle's own buffers (model constants, per-step tape)."""
    import torch
    from paper_2109_07719_gb300 import Simulator
    torch.cuda.set_device(0)
    horizons = [int(x) for x in args.horizons.split(",")]
    lines = []
    for T in horizons:
        work = workload(args.config, args.precision, args.batch, T)
        m = work.model
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        free0 = torch.cuda.mem_get_info()[0]
        sim = Simulator(m, precision=args.precision)
        handle_bytes = free0 - torch.cuda.mem_get_info()[0]
        dt, dev = sim.dtype, sim.device
        q0 = torch.tensor(work.q0, dtype=dt, device=dev)
        qd0 = torch.tensor(work.qd0, dtype=dt, device=dev)
        tau = work.tau(device=dev, dtype=dt)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()   # drop the input generator's temporaries
        t0 = time.perf_counter()
        qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=args.k)
        g = sim.backward(ck, tau, torch.ones_like(qT), torch.zeros_like(qdT), k=args.k)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        peak = torch.cuda.max_memory_allocated() - base
        line = {"metric": "peak device memory vs horizon", "workload": m.name, "n_systems": sim.B,
                "horizon": T, "checkpoint_interval": args.k, "precision": args.precision,
                "peak_torch_bytes": int(peak), "handle_bytes": int(handle_bytes),
                "ckpt_bytes": int(sim.ckpt_bytes(T, args.k)), "tau_bytes": int(tau.numel() * tau.element_size()),
                "seconds_fwd_adj": el}
        lines.append(line)
        print(json.dumps(line))
        del sim, q0, qd0, tau, qT, qdT, ck, g
    if len(lines) > 1:
        a, b = lines[0], lines[-1]
        slope = (b["peak_torch_bytes"] - a["peak_torch_bytes"]) / (b["horizon"] - a["horizon"])
        print(json.dumps({"metric": "peak memory growth per step", "bytes_per_step": slope,
                          "bytes_per_step_per_system": slope / a["n_systems"]}))


def launch_ranks(n: int, fn, fn_args=(), backend_env=None, port=None):
    """Run fn(*fn_args) in n spawned processes, one per rank, with the
    torch.distributed environment a launcher would give them (RANK, LOCAL_RANK,
    WORLD_SIZE, MASTER_ADDR = 127.0.0.1, MASTER_PORT).  Returns the exit codes.
    Spawn, never fork: a parent that touched CUDA cannot fork children that use it."""
    import multiprocessing as mp
    import socket
    if port is None:
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = []
    for r in range(n):
        env = {"RANK": str(r), "LOCAL_RANK": str(r), "WORLD_SIZE": str(n), "LOCAL_WORLD_SIZE": str(n),
               "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), **(backend_env or {})}
        p = ctx.Process(target=_rank_entry, args=(env, fn, fn_args))
        p.start()
        procs.append(p)
    for p in procs:
        p.join()
    return [p.exitcode for p in procs]


def _rank_entry(env, fn, fn_args):
    os.environ.update(env)
    fn(*fn_args)


def _rank_bench(args):
    line = run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4,
                    help="workload 1..5 (default 4: 16384 uneven trees, T = 5000, the largest single-GPU one)")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp32_d64"])
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--horizon", type=int, default=None)
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--k-sweep", default=None,
                    help="also time one step at each of these checkpoint intervals (default 10,100 for --config 4)")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--persistent", action="store_true")
    ap.add_argument("--keep-order", action="store_true",
                    help="pack systems in their own order (coalesced streams) instead of by link count")
    ap.add_argument("--slot-layout", action=argparse.BooleanOptionalAction, default=None,
                    help="lay the batch out by link count, the library's packing order, so each warp's "
                         "streams are whole cache lines (default: on for the uneven trees, --config 4)")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=None,
                    help="time the kernel families and launch shapes on a short probe and keep the fastest "
                         "(default: on for the uneven-tree batch, whose configuration names autotuned grouping)")
    ap.add_argument("--tape", default="auto",
                    choices=["auto", "global", "shared", "pipelined", "one_warp", "aligned", "aligned_pipelined"])
    ap.add_argument("--prefetch", type=int, default=None,
                    help="links ahead the world-aligned global-tape passes prefetch (library default 2; 0: off)")
    ap.add_argument("--state-accumulation", default="fp32", choices=["fp32", "fp64"],
                    help="running-state sums of the fp32_d64 precision (fp64: summed in FP64, stored FP32)")
    ap.add_argument("--replay", default="segment", choices=["segment", "quadratic"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-plain", dest="plain", action="store_false")
    ap.add_argument("--plain-systems", type=int, default=8,
                    help="systems timed one per launch for the per-system comparison")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-grad-check", dest="grad_check", action="store_false",
                    help="skip the per-output error against the FP64 path on sampled systems")
    ap.add_argument("--graph", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the step captured as one CUDA graph (two replays after the timed steps)")
    ap.add_argument("--contacts", action=argparse.BooleanOptionalAction, default=None,
                    help="quadruped with foot contact spheres, the contact solve running every step "
                         "(default: on for --config 3, whose specification includes foot contacts)")
    ap.add_argument("--limits", action="store_true", help="revolute joints limited to [-0.5, 0.5] rad")
    ap.add_argument("--memory-sweep", action="store_true")
    ap.add_argument("--horizons", default="1000,5000,10000,50000")
    args = ap.parse_args()
    if args.contacts is None:
        args.contacts = args.config == 3
    if args.slot_layout is None:
        args.slot_layout = args.config == 4
    if args.autotune is None:  # a forced kernel family or launch shape is kept as given
        args.autotune = args.config == 4 and args.tape == "auto" and not (args.block or args.persistent)
    if args.k_sweep is None:
        args.k_sweep = "10,100" if args.config == 4 and args.k == 1 else ""
    args.warmup = max(args.warmup, 3)
    if args.memory_sweep:
        memory_sweep(args)
        return
    if args.impl == "ours" and args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        import torch
        if torch.cuda.device_count() < args.gpus:
            raise SystemExit(f"--gpus {args.gpus}: only {torch.cuda.device_count()} CUDA device(s) visible")
        codes = launch_ranks(args.gpus, _rank_bench, (args,))
        if any(codes):
            raise SystemExit(f"a rank failed: exit codes {codes}")
        return
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
