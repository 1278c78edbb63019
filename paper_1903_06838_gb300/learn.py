"""Host-side orchestration of the learned count / subpixel refinement.

Everything numeric runs in libpd's kernels (pd_process, pd_net_gather,
pd_net_train_step, pd_net_forward, pd_net_refine); this module only assembles
batches and labels.  Labels come from the generator's ground truth: the
photons whose landing pixel lies in the 3x3 window of a hit's seed give its
true count (clipped to 4) and, for single-photon hits, its true offset from
the seed pixel centre.
"""
from __future__ import annotations

import numpy as np

from . import pd, synth


def label_hits(det: synth.Detector, hits: np.ndarray, photons: np.ndarray):
    """(counts u8, targets float32 [n, 2], mask u8) for each hit."""
    C, R, M = det.cols, det.rows, det.n_modules
    mpx = R * C
    # photons keyed by (frame, module, landing row, landing col), sorted
    px = np.floor(photons["x"]).astype(np.int64)
    py = np.floor(photons["y"]).astype(np.int64)
    pkey = ((photons["frame"].astype(np.int64) * M + photons["module"].astype(np.int64)) * R
            + py) * C + px
    order = np.argsort(pkey, kind="stable")
    skey = pkey[order]
    n = len(hits)
    m, within = np.divmod(hits["pixel"].astype(np.int64), mpx)
    r0, c0 = np.divmod(within, C)
    base = hits["frame"].astype(np.int64) * M + m
    total = np.zeros(n, np.int64)
    first = np.full(n, -1, np.int64)  # a photon of the window (for single ones)
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            r, c = r0 + dr, c0 + dc
            ok = (r >= 0) & (r < R) & (c >= 0) & (c < C)
            k = (base * R + r) * C + c
            lo = np.searchsorted(skey, k, "left")
            hi = np.searchsorted(skey, k, "right")
            cnt = np.where(ok, hi - lo, 0)
            take = (cnt > 0) & (first < 0)
            first[take] = order[lo[take]]
            total += cnt
    counts = np.minimum(total, 4).astype(np.uint8)
    single = total == 1
    tgt = np.zeros((n, 2), np.float32)
    ph = photons[first[single]]
    tgt[single, 0] = ph["x"] - (c0[single] + 0.5)
    tgt[single, 1] = ph["y"] - (r0[single] + 0.5)
    mask = single.astype(np.uint8)
    return counts, tgt, mask


def hits_and_patches(ctx, det, frames_dev, frame_base=0):
    """Run the chain on device frames; returns (hits numpy, patches tensor
    [n, 25] on the device, hits tensor on the device)."""
    import torch
    n_frames = frames_dev.numel() // det.pixels_per_frame
    out = pd.process(ctx, frames_dev, frame_base=frame_base, cm=True)
    torch.cuda.synchronize()
    hits, n = out.hits_host()
    assert len(hits) == n
    patches = torch.empty((max(n, 1), 25), dtype=torch.float32, device=frames_dev.device)
    pd.pd_net_gather(ctx, frames_dev.data_ptr(), frame_base, out.cm.data_ptr(),
                     out.hits.data_ptr(), n, patches.data_ptr())
    torch.cuda.synchronize()
    return hits, patches[:n], out.hits[:n]


def make_set(det: synth.Detector, n_frames: int, first_frame: int = 0):
    """Generated frames -> (hits, patches on device, host labels, device labels)."""
    import torch
    ped, gain = synth.maps(det)
    raw, photons = synth.frames(det, ped, gain, first_frame, n_frames)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    dev = pd.frames_to_device(raw)
    hits, patches, _ = hits_and_patches(ctx, det, dev, first_frame)
    del dev
    counts, tgt, mask = label_hits(det, hits, photons)
    dev_labels = (torch.from_numpy(counts).cuda(), torch.from_numpy(tgt).cuda(),
                  torch.from_numpy(mask).cuda())
    return hits, patches, (counts, tgt, mask), dev_labels


def train(net, patches, dev_labels, steps: int, batch: int = 2048, lr: float = 2e-3,
          lam: float = 10.0, seed: int = 0, host_mask=None):
    """Adam steps over random mini-batches; returns the loss per step.  Every
    step's batch indices are drawn up front and uploaded once; each step's
    rows are gathered on the device (pd_net_take) and the losses stay on the
    device until the end, so the steps run back to back with no host work
    between them."""
    import torch
    counts, tgt, mask = dev_labels
    n = patches.shape[0]
    dev = patches.device
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, (steps, batch), dtype=np.int64).astype(np.uint32)
    m_host = host_mask if host_mask is not None else mask.cpu().numpy()
    n_reg = m_host[idx].astype(np.int64).sum(axis=1)
    idx_dev = torch.from_numpy(idx.view(np.int32)).to(dev)
    x = torch.empty((batch, 25), dtype=torch.float32, device=dev)
    c = torch.empty(batch, dtype=torch.uint8, device=dev)
    t = torch.empty((batch, 2), dtype=torch.float32, device=dev)
    m = torch.empty(batch, dtype=torch.uint8, device=dev)
    losses = torch.zeros(max(steps, 1), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for s in range(steps):
        pd.pd_net_take(patches.data_ptr(), counts.data_ptr(), tgt.data_ptr(), mask.data_ptr(),
                       idx_dev[s].data_ptr(), batch, x.data_ptr(), c.data_ptr(), t.data_ptr(),
                       m.data_ptr(), stream=stream)
        pd.pd_net_train_step(net, x.data_ptr(), c.data_ptr(), t.data_ptr(), m.data_ptr(),
                             batch, float(n_reg[s]), lam, lr, losses[s].data_ptr(),
                             stream=stream)
    return [float(v) for v in losses[:steps].cpu().numpy()]


def predict(net, patches):
    import torch
    n = patches.shape[0]
    out = torch.empty((max(n, 1), 7), dtype=torch.float32, device=patches.device)
    pd.pd_net_forward(net, patches.data_ptr(), n, out.data_ptr())
    torch.cuda.synchronize()
    return out[:n]
