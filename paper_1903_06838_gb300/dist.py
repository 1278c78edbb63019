"""Several GPUs, one process each: frames are independent (the paper
processes every frame on its own), so each rank runs the chain on its own
contiguous block of frames with replicated pedestal and gain, and nothing
crosses ranks on the data path.  The one exchange is the merge of the
summaries: integer sums of the photon-count maps and of both histograms
(order-independent, so bit-exact), and the concatenation of the hit lists
with frame indices made global.  Uses torch.distributed (NCCL on GPUs, gloo
on CPU); argument marshalling only.
"""
from __future__ import annotations

import numpy as np


def shard(n_frames: int, world_size: int, rank: int) -> tuple[int, int]:
    """[first, last) frames of `rank` when n_frames are split into
    world_size contiguous blocks whose sizes differ by at most one."""
    if world_size < 1 or not 0 <= rank < world_size or n_frames < 0:
        raise ValueError("invalid shard request")
    base, extra = divmod(n_frames, world_size)
    first = rank * base + min(rank, extra)
    return first, first + base + (1 if rank < extra else 0)


def merge_summaries(count_map: np.ndarray, hist_pix: np.ndarray, hist_hit: np.ndarray,
                    group=None, device="cpu"):
    """All-reduce (sum) of one rank's summaries; returns the merged
    (count_map u64, hist_pix u64, hist_hit u64) on every rank."""
    import torch
    import torch.distributed as dist
    out = []
    for a in (count_map, hist_pix, hist_hit):
        t = torch.from_numpy(np.ascontiguousarray(a, np.int64)).to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out.append(t.cpu().numpy().astype(np.uint64))
    return tuple(out)


def gather_hits(hits: np.ndarray, dtype: np.dtype, group=None, device="cpu"):
    """Concatenation of every rank's hit records (rank order) on every rank.
    Records travel as raw bytes; sizes are exchanged first."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    raw = np.ascontiguousarray(hits).view(np.uint8).reshape(-1)
    n = torch.tensor([raw.size], dtype=torch.int64, device=device)
    sizes = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(ws)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(max(sizes), 1)
    buf = torch.zeros(cap, dtype=torch.uint8, device=device)
    buf[:raw.size] = torch.from_numpy(raw).to(device)
    parts = [torch.zeros(cap, dtype=torch.uint8, device=device) for _ in range(ws)]
    dist.all_gather(parts, buf, group=group)
    cat = np.concatenate([p.cpu().numpy()[:s] for p, s in zip(parts, sizes)])
    return cat.view(dtype)
