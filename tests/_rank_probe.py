"""A rank body for the CPU test of bench.launch_ranks: joins the gloo process
group from the environment the launcher set, sums the ranks, and records what it
saw in a file per rank."""
import json
import os


def gloo_rank(outdir):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo")
    r, n = dist.get_rank(), dist.get_world_size()
    t = torch.tensor([float(r + 1)])
    dist.all_reduce(t)
    with open(os.path.join(outdir, f"rank{r}.json"), "w") as f:
        json.dump({"rank": r, "world": n, "sum": float(t.item()), "env_rank": os.environ["RANK"],
                   "local_rank": os.environ["LOCAL_RANK"], "master": os.environ["MASTER_ADDR"]}, f)
    dist.destroy_process_group()
