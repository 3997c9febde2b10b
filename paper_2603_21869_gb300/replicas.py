"""Several GPUs of one node: each rank steps its own cases (case-level
partitioning, no data-path collective).  Helpers for the rank setup, the
reductions of timings and counts over ranks, and a device-byte-balanced
partition of a fixed list of cases.  Backend nccl on GPUs; gloo (CPU
tensors) where no GPU is present."""
import os

import torch
import torch.distributed as dist


def setup(backend=None):
    """(rank, world, local_rank, initialised) from the torchrun environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return 0, 1, 0, False
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group("gloo")
    return rank, world, local, True


def _device():
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def max_over_ranks(x: float) -> float:
    """The slowest rank's time (the job is done when the last rank is)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def partition(weights, world):
    """Assign items (by weight, e.g. device bytes or cells) to `world` ranks:
    heaviest first, each to the least loaded rank (ties to the lower rank).
    Returns one list of item indices per rank, each in increasing order."""
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(weights)), key=lambda q: (-weights[q], q)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += weights[i]
    return [sorted(p) for p in parts]
