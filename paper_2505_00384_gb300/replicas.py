"""Replica runs on several GPUs (one process per GPU, launched by torchrun).

The pressure solve of one mesh does not shard here (one GPU per problem), so N
GPUs run N independent replicas of the workload; the only cross-rank step is
the timing: a barrier before and after the timed region and the maximum of the
per-rank times.  No collective touches the data path.
"""
import os


def env():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend="nccl"):
    """Join the default process group when launched with more than one rank;
    returns torch.distributed or None."""
    ws, _, _ = env()
    if ws <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend)
    return dist


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value, device="cpu"):
    """Maximum of a per-rank float over all ranks (the value itself without a group)."""
    if pg is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())
