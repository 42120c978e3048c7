"""Host-side sharding of tracking work over the ranks of a torch.distributed job.

Under a fixed reference every frame is tracked on its own (Sec. III: the frames are
independent once the reference is fixed), so ranks split the work and exchange no frame
data: a frame stream is cut into contiguous blocks, or a camera set is dealt out to the
ranks, and the 24-byte records are gathered on the host afterwards. The tracking itself
runs in each rank's own CUDA context (libccst); this module only decides who tracks what
and puts the records back in the original order.
"""
from __future__ import annotations

import numpy as np


def frame_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of the frames rank `rank` tracks: contiguous blocks whose sizes differ by at
    most one, in rank order (rank 0 gets the first frames)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need n >= 0 and 0 <= rank < world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def camera_ranks(ncams: int, world: int) -> list[int]:
    """The rank that serves each camera: round robin over the ranks (camera c on rank
    c mod world), so each camera's frames stay on one device with its reference spectrum."""
    if world < 1 or ncams < 0:
        raise ValueError("need world >= 1 and ncams >= 0")
    return [c % world for c in range(ncams)]


def gather_records(local, world: int, rank: int):
    """Concatenate every rank's records in rank order on every rank.

    local: this rank's records (any numpy array; rows in the rank's own order). With
    world == 1 it is returned as is. Uses torch.distributed.all_gather_object, so it works
    over gloo (CPU) and NCCL."""
    if world == 1:
        return local
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, np.ascontiguousarray(local))
    return np.concatenate(parts)


def gather_camera_records(local: dict, world: int):
    """Merge per-camera records {camera: records} from every rank into one dict. Each
    camera lives on exactly one rank (camera_ranks), so keys never collide."""
    if world == 1:
        return dict(local)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, {k: np.ascontiguousarray(v) for k, v in local.items()})
    out = {}
    for p in parts:
        for k, v in p.items():
            if k in out:
                raise ValueError(f"camera {k} tracked on two ranks")
            out[k] = v
    return out
