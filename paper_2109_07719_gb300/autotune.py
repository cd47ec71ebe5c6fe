"""Launch-shape autotuner for the batched rollout kernels.

Times a short forward + adjoint rollout for each candidate -- the kernel family
(the link-frame one-warp kernels, one lane per system; the link-frame pipelined
kernels, two warps per 32-system tile, for short serial chains; the
world-aligned kernels for revolute models without contacts or limits, one lane
per system or with the two-warp pipelined adjoint; the library's automatic
choice per direction), threads per block (systems per block) and grid or
persistent schedule -- and keeps the fastest.  A candidate whose kernels the
model cannot run (the library refuses the launch, or the pipelined space ran
nothing pipelined) is dropped.  Results are cached in a JSON file keyed by the
batch signature (systems, padded sizes, links, precision, link-count histogram)
and the GPU name, so a model is tuned once per device type.
"""
from __future__ import annotations

import json
import os

# (threads per block, persistent schedule, kernel family): 1 the link-frame
# one-warp kernels, 2 the link-frame pipelined kernels (two lanes per system),
# 3 the world-aligned kernels, 4 the world-aligned kernels with the pipelined
# adjoint (two lanes per system in the adjoint), 5 the library's automatic choice
# in each direction (which may mix families, e.g. the link-frame pipelined rollout
# with the world-aligned pipelined adjoint)
CANDIDATES = [(32, False, 1), (64, False, 1), (128, False, 1), (32, True, 1), (64, True, 1), (128, True, 1),
              (32, False, 2), (32, True, 2), (32, False, 3), (64, False, 3), (32, True, 3), (64, True, 3),
              (32, False, 4), (64, False, 4), (32, True, 4), (64, True, 4), (32, False, 5), (32, True, 5)]
TAPE_SPACE = {1: "one_warp", 2: "pipelined", 3: "aligned", 4: "aligned_pipelined", 5: "auto"}


def cache_path() -> str:
    return os.environ.get("ABASIM_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "abasim", "tune.json"))


def cache_key(signature, device_name: str) -> str:
    return json.dumps([list(signature), device_name])


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(table: dict, path=None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(times: dict):
    """The fastest candidate; ties go to the earlier (simpler) entry."""
    best = None
    for cand in CANDIDATES:
        t = times.get(cand)
        if t is not None and (best is None or t < times[best]):
            best = cand
    if best is None:
        raise ValueError("no candidate was timed")
    return best


def apply(sim, cand):
    threads, persistent, lanes = cand
    sim.set_tape_space(TAPE_SPACE[lanes])
    sim.set_launch(threads, persistent)


def autotune(sim, q0, qd0, T_probe: int = 16, reps: int = 3, k: int = 1, use_cache: bool = True,
             timer=None, device_name: str | None = None):
    """Select and apply the fastest candidate for ``sim``; returns (threads, persistent, lanes).

    ``timer(sim, cand)`` may replace the GPU measurement; it returns seconds."""
    import torch
    name = device_name or torch.cuda.get_device_name(sim.device)
    key = cache_key(sim.signature, name)
    table = load_cache() if use_cache else {}
    if key in table:
        e = table[key]
        best = (e["threads"], e["persistent"], e.get("kernels", e.get("lanes", 1)))
        apply(sim, best)
        return best
    if timer is None:
        timer = _gpu_timer(q0, qd0, T_probe, reps, k)
    from . import SimError
    times = {}
    for cand in CANDIDATES:
        if cand[2] != 2 and cand[0] > 32 and cand[0] // 2 >= sim.B:
            continue
        try:
            apply(sim, cand)
            t = timer(sim, cand)
        except SimError:
            continue                                   # the model cannot run on these kernels
        if cand[2] == 2 and "pipelined" not in sim.last_storage():
            continue                                   # ran one-lane in a direction: not this candidate
        if cand[2] == 5 and not any(s.startswith(("pipelined", "aligned")) for s in sim.last_storage()):
            continue                                   # the automatic choice was the one-warp family
        times[cand] = t
    best = choose(times)
    apply(sim, best)
    if use_cache:
        table[key] = {"threads": best[0], "persistent": best[1], "kernels": best[2],
                      "seconds": {f"{c[0]}/{'persistent' if c[1] else 'grid'}/{TAPE_SPACE[c[2]]}": t
                                  for c, t in times.items()}}
        save_cache(table)
    return best


def _gpu_timer(q0, qd0, T_probe, reps, k):
    import torch

    def timer(sim, cand):
        tau = torch.zeros(T_probe, sim.nv_max, sim.B, dtype=sim.dtype, device=sim.device)
        ones = torch.zeros(sim.nq_max, sim.B, dtype=sim.dtype, device=sim.device)
        zd = torch.zeros(sim.nv_max, sim.B, dtype=sim.dtype, device=sim.device)

        def once():
            qT, qdT, ck, _ = sim.rollout(q0, qd0, tau, k=k)
            sim.backward(ck, tau, ones, zd, k=k, mass_grad=False)

        once()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            once()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3)
        return best

    return timer
