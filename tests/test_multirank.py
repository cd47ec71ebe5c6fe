"""The N-GPU bench path on CPU ranks (gloo, world size 2): each rank runs its own
disjoint batch and the job's time is the slowest rank's, its env-steps the sum."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    work = bench.workload(2, "fp32", B=8, T=3, rank=rank)
    step_ms, units = bench.aggregate(10.0 * (rank + 1), 8 * 3)
    masses = torch.tensor(work.model.mass)
    gathered = [torch.zeros_like(masses) for _ in range(world)]
    dist.all_gather(gathered, masses)
    out[rank] = (step_ms, units, bool(torch.equal(gathered[0], gathered[1])))
    dist.destroy_process_group()


def test_two_rank_aggregation_and_disjoint_batches():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        step_ms, units, same = res[r]
        assert step_ms == 20.0          # the slowest rank
        assert units == 2 * 8 * 3       # both ranks' env-steps
        assert not same                 # different systems on each rank



def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate(3.5, 42) == (3.5, 42)


def test_bench_launches_its_own_ranks(tmp_path):
    """bench.py --gpus N without an external launcher starts N spawned ranks with
    the launcher's environment (here two gloo ranks on the CPU): every rank joins
    the process group, sees its own RANK / LOCAL_RANK and the loopback master."""
    import json
    import bench
    from tests._rank_probe import gloo_rank
    codes = bench.launch_ranks(2, gloo_rank, (str(tmp_path),))
    assert codes == [0, 0]
    seen = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(seen):
        assert d == {"rank": r, "world": 2, "sum": 3.0, "env_rank": str(r), "local_rank": str(r),
                     "master": "127.0.0.1"}
