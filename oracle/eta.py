"""CPU oracle of the centroid linearisation — TEST INFRASTRUCTURE (only tests,
the smoke check and the benchmark's CPU baseline may import it; it shares no
code with the CUDA path).

The paper notes that the centre-of-mass offset of a photon's charge depends
nonlinearly on where the photon landed, and that the centroids must be
linearised to give positions (section "Photon Subpixel Resolution", Fig. f
and its caption); it gives no method.  Reading: with photons landing
uniformly inside the seed pixel, the true offset u in [-1/2, 1/2) and the
measured centroid d are related by a monotone map, so u = F(d) - 1/2 where F
is the cumulative distribution of d.  F is estimated per axis from the
single-photon hits (count == 1) of a calibration set: a histogram of d over
B bins spanning [-1, 1], interpolated linearly inside a bin.  B is odd: the
centroid has an atom at d = 0 (photons whose neighbours all stay below the
zero-suppression threshold), and with d = 0 in the middle of a bin that atom
maps to the middle of its probability mass rather than to its lower end.

Every step is float32 round-to-nearest in this order (numpy float32 scalars):
    t   = (d + 1) * (B * 0.5)
    k   = clamp(floor(t), 0, B - 1)                       bin
    phi = clamp(t - k, 0, 1)                              position in the bin
    F   = (C[k] + phi * h[k]) / N                         C: counts below bin k
    out = F - 1/2
Hits with count != 1, or a non-finite centroid, keep their centroid; the
others get flag bit LINEARISED (8) set.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32
LINEARISED = 8


def bin_of(d, bins: int):
    """(k, phi) of centroids d (float32 arrays), in the order above."""
    d = np.asarray(d, np.float32)
    t = (d + F32(1.0)) * (F32(bins) * F32(0.5))
    k = np.clip(np.floor(t), 0, bins - 1).astype(np.int64)
    phi = np.clip(t - k.astype(np.float32), F32(0.0), F32(1.0)).astype(np.float32)
    return k, phi


def accumulate(hist, hits, bins: int):
    """Add the single-photon hits' centroids to hist (uint32 [2][bins])."""
    sel = (hits["count"] == 1) & np.isfinite(hits["dx"]) & np.isfinite(hits["dy"])
    for axis, name in enumerate(("dx", "dy")):
        k, _ = bin_of(hits[name][sel], bins)
        np.add.at(hist[axis], k, 1)
    return hist


def linearise(hist, d, bins: int):
    """u for centroids d along one axis from that axis' histogram."""
    h = hist.astype(np.int64)
    n = int(h.sum())
    if n == 0:
        return np.asarray(d, np.float32).copy()
    below = np.concatenate([[0], np.cumsum(h)[:-1]])
    k, phi = bin_of(d, bins)
    num = below[k].astype(np.float32) + phi * h[k].astype(np.float32)
    return (num / F32(n) - F32(0.5)).astype(np.float32)


def apply(hist, hits, bins: int):
    """Copy of hits with dx, dy of single-photon hits linearised."""
    out = hits.copy()
    sel = (hits["count"] == 1) & np.isfinite(hits["dx"]) & np.isfinite(hits["dy"])
    out["dx"][sel] = linearise(hist[0], hits["dx"][sel], bins)
    out["dy"][sel] = linearise(hist[1], hits["dy"][sel], bins)
    out["flags"][sel] |= LINEARISED
    return out
