"""Bookkeeping for runs on several GPUs: one process per GPU, each running independent work.

The unfolded system of one instance is not split across GPUs (each RK4 stage would need an
all-gather of the whole state); what runs on several GPUs are independent replicas or disjoint
shares of independent instances (batched parameter sets, finite-difference perturbations,
parameter scans).  The only collectives are the ones that time the run: a barrier around the
timed region, the maximum of the elapsed times and the sum of the work done.
"""


def shard(n_items, rank, world):
    """Contiguous share [begin, end) of n_items independent items for `rank` of `world`; the first
    n_items % world ranks take one item more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} out of range for world size {world}")
    base, extra = divmod(n_items, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def reduce_timing(elapsed_ms, units, dist=None, device="cpu"):
    """(slowest rank's elapsed milliseconds, total units over ranks) of a timed region.

    `dist` is torch.distributed after init_process_group (None for one process); `device` is
    where the reduction tensors live (the rank's GPU under NCCL, "cpu" under gloo)."""
    if dist is None:
        return float(elapsed_ms), float(units)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def throughput(elapsed_ms, units, dist=None, device="cpu"):
    """Whole-job throughput: units done by all ranks per second of the slowest rank."""
    ms, total = reduce_timing(elapsed_ms, units, dist, device)
    return total / (ms * 1e-3)
