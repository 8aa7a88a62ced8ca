"""Source sharding across ranks (one process per GPU).

Sources are independent until the final sum over sources (Section 1.1's
"running score"), so a multi-GPU run gives each rank whole batches of
sources and needs one reduction of the n FP64 partial BC vectors at the end.
Batches are dealt round-robin (batch i goes to rank i mod world) so that ranks
get the same number of batches to within one.
"""
from __future__ import annotations

import numpy as np


def shard_sources(sources, rank: int, world: int, batch: int) -> np.ndarray:
    """The sources rank `rank` of `world` runs: batches i with i % world == rank."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    src = np.asarray(sources, dtype=np.int32)
    nb = -(-src.size // batch)
    mine = [src[i * batch:(i + 1) * batch] for i in range(rank, nb, world)]
    return np.concatenate(mine) if mine else np.zeros(0, np.int32)


def reduce_partials(partial: np.ndarray, group=None) -> np.ndarray:
    """Sum every rank's partial BC vector in rank order (bit-reproducible for a
    fixed world size): gather to all ranks, then add rank 0, 1, ... in turn.
    Works on a gloo group (host tensors) and on an NCCL group (the vector goes
    through the current CUDA device)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return np.array(partial, dtype=np.float64, copy=True)
    t = torch.from_numpy(np.ascontiguousarray(partial, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        return reduce_partials_device(t.cuda(), group).cpu().numpy()
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out.numpy()


def reduce_partials_device(partial, group=None):
    """The rank-ordered sum of a tensor held by every rank (on the device for
    an NCCL group): one all-gather of the n-vectors, then rank 0, 1, ... added
    in turn, so every rank gets the same bits."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return partial.clone()
    parts = [torch.empty_like(partial) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, partial.contiguous(), group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out


def run_sharded_gpu(g, sources=None, batch: int = 256, flags: int = 0, group=None):
    """Multi-GPU betweenness: this rank's shard on its own GPU, then the
    rank-ordered sum. Returns the full BC vector on every rank."""
    import torch.distributed as dist
    from . import native
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    src = np.arange(g.n, dtype=np.int32) if sources is None else np.asarray(sources, np.int32)
    mine = shard_sources(src, rank, world, batch)
    with native.Graph.from_csr(g) as h:
        h.run(mine, batch=batch, flags=flags)
        part, _, _ = h.result()
    return reduce_partials(part, group)
