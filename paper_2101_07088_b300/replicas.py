"""Replicas across ranks (one process per GPU).

A solve does not shard: each rank solves its own independent system, with
its own seed, and no collective touches the data path. After timing, the job
reports the slowest rank's step time and counts every rank's charges (weak
scaling): value = sum_r n_r / max_r t_r.
"""


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s system: rank 0 keeps the workload's own seed."""
    return base_seed + 1000 * rank


def job_rate(local_ms: float, local_charges: int, dist=None, device=None):
    """(max step ms over ranks, total charges per second of the job).

    dist is torch.distributed (initialised) or None for one process; the two
    reductions (MAX of the time, SUM of the charges) run once per measurement.
    """
    if dist is None:
        return local_ms, local_charges / (local_ms * 1e-3)
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    c = torch.tensor([float(local_charges)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(c.item()) / (ms * 1e-3)
