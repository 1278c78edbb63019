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
    C = det.cols
    mpx = det.rows * det.cols
    # photons indexed by (frame, module, landing row, landing col)
    key = {}
    for i, ph in enumerate(photons):
        r, c = int(ph["y"]), int(ph["x"])
        key.setdefault((int(ph["frame"]), int(ph["module"]), r, c), []).append(i)
    n = len(hits)
    counts = np.zeros(n, np.uint8)
    tgt = np.zeros((n, 2), np.float32)
    mask = np.zeros(n, np.uint8)
    for j, h in enumerate(hits):
        m, within = divmod(int(h["pixel"]), mpx)
        r0, c0 = divmod(within, C)
        sel = []
        for dr in (-1, 0, 1):
            for dc in (-1, 0, 1):
                sel += key.get((int(h["frame"]), m, r0 + dr, c0 + dc), [])
        counts[j] = min(len(sel), 4)
        if len(sel) == 1:
            ph = photons[sel[0]]
            tgt[j] = (ph["x"] - (c0 + 0.5), ph["y"] - (r0 + 0.5))
            mask[j] = 1
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
    """Generated frames -> (hits, patches on device, labels)."""
    import torch
    ped, gain = synth.maps(det)
    raw, photons = synth.frames(det, ped, gain, first_frame, n_frames)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    dev = pd.frames_to_device(raw)
    hits, patches, _ = hits_and_patches(ctx, det, dev, first_frame)
    counts, tgt, mask = label_hits(det, hits, photons)
    dev_labels = (torch.from_numpy(counts).cuda(), torch.from_numpy(tgt).cuda(),
                  torch.from_numpy(mask).cuda())
    return hits, patches, (counts, tgt, mask), dev_labels


def train(net, patches, dev_labels, steps: int, batch: int = 2048, lr: float = 2e-3,
          lam: float = 10.0, seed: int = 0):
    """Adam steps over shuffled mini-batches; returns the loss per step."""
    import torch
    counts, tgt, mask = dev_labels
    n = patches.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=patches.device)
    losses = []
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).to(patches.device)
        x = patches[idx].contiguous()
        c = counts[idx].contiguous()
        t = tgt[idx].contiguous()
        m = mask[idx].contiguous()
        nreg = float(m.sum().item())
        loss.zero_()
        pd.pd_net_train_step(net, x.data_ptr(), c.data_ptr(), t.data_ptr(), m.data_ptr(),
                             batch, nreg, lam, lr, loss.data_ptr())
        losses.append(float(loss.item()))
    return losses


def predict(net, patches):
    import torch
    n = patches.shape[0]
    out = torch.empty((max(n, 1), 7), dtype=torch.float32, device=patches.device)
    pd.pd_net_forward(net, patches.data_ptr(), n, out.data_ptr())
    torch.cuda.synchronize()
    return out[:n]
