"""Host-side logic of running the solver as independent replicas, one per
rank (weak scaling).  A single large instance does not shard without halo
exchanges and distributed transposes, so N GPUs run N independent solves;
the only collective is the reduction of the timing (max over ranks), which
is not on the data path.  Works with any torch.distributed backend (NCCL on
GPUs, gloo on CPU for the tests)."""

import os


def dist_env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, dist=None, device="cpu"):
    """Maximum of a float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist=None, device="cpu"):
    """Sum of a float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_this_rank, elapsed_ms_this_rank, dist=None, device="cpu"):
    """Whole-job throughput: units processed by all ranks / the slowest rank's
    time (the job ends when the last replica ends)."""
    units = sum_over_ranks(units_this_rank, dist, device)
    ms = max_over_ranks(elapsed_ms_this_rank, dist, device)
    return units / (ms / 1000.0), ms
