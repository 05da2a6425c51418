"""One process per GPU: the batch of parameter samples is split by sample across ranks.
Samples are independent, so the data path needs no collective; the ranks only meet in a
barrier around the timed region and a max over their times."""
import numpy as np


def shard(theta, sys_id, rank, world):
    """Rank `rank`'s contiguous share of a global batch of world * B samples."""
    n = theta.shape[0]
    if n % world:
        raise ValueError(f"batch of {n} does not split over {world} ranks")
    B = n // world
    return np.ascontiguousarray(theta[rank * B:(rank + 1) * B]), \
        np.ascontiguousarray(sys_id[rank * B:(rank + 1) * B])


def max_over_ranks(value, dist, device="cpu"):
    """The largest of the ranks' values (a timing); the value itself with one rank."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])
