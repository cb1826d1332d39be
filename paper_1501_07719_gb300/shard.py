"""Time sharding of one observation over several processes (one GPU each).

The chi^2 of eq. 7 is a sum over timesteps, and every input of the RIME
except the sky model is indexed by time first (Table 2), so contiguous time
chunks are independent: each rank evaluates its chunk and one scalar sum
completes the chi^2 (the time subdivision of Sec. 4.4). The source gradient
sums the same way; the gains gradient stays with the rank that owns its
timesteps.
"""
from __future__ import annotations

import numpy as np

# arrays whose first axis is time
_TIME_FIRST = ("uvw", "pointing", "gains", "data", "weight", "noise")


def time_chunk(ntime: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous chunk [t0, t1) of rank `rank` out of `world`; chunk sizes
    differ by at most one and the chunks cover 0 .. ntime-1 in rank order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} out of range for world size {world}")
    base, extra = divmod(ntime, world)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def slice_observation(obs: dict, t0: int, t1: int) -> dict:
    """The inputs of timesteps t0 .. t1-1: every time-first array sliced, a
    time-varying brightness sliced along its time axis, the rest shared."""
    out = dict(obs)
    out["ntime"] = t1 - t0
    for key in _TIME_FIRST:
        if obs.get(key) is not None:
            out[key] = np.ascontiguousarray(obs[key][t0:t1])
    src = obs.get("sources")
    if src is not None and np.ndim(src["stokes"]) == 3:
        out["sources"] = dict(src, stokes=np.ascontiguousarray(src["stokes"][t0:t1]))
    return out


def reduce_sum(value: float, group=None) -> float:
    """Sum of one float64 scalar over the ranks of `group` (every rank gets
    the total). Uses a CPU tensor for gloo and a device tensor for nccl."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def reduce_max(value: float, group=None) -> float:
    """Maximum of one scalar over the ranks (for timing: the slowest rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_chi2(obs: dict, precision: int, group=None) -> float:
    """chi^2 of the whole observation evaluated as this rank's time chunk on
    its GPU (librime) plus a sum over ranks. obs holds the observation, data,
    weights, gains and sources as for Rime."""
    import torch.distributed as dist
    from .context import Rime
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    t0, t1 = time_chunk(int(obs["ntime"]), rank, world)
    part = 0.0
    if t1 > t0:
        sl = slice_observation(obs, t0, t1)
        r = Rime(sl, precision, data=sl["data"], weight=sl.get("weight"))
        if sl.get("gains") is not None:
            r.set_gains(sl["gains"])
        r.set_sources(sl["sources"])
        part = r.chi2()
        r.close()
    return reduce_sum(part, group)
