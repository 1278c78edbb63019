"""Matched-filter banks for the charge summing of section "Photon Charge
Summing" (Figs. d, e) and the centroids of Fig. f.

The paper shows its bank (F0, F1 of shape 4 x 5 x 1 x 6, F1Nmin, F1dx, F1dy)
only as a picture, so the bank is an input.  ``example_bank`` builds one with
six features, each a cloud shape anchored at one of its pixels:

    single pixel, horizontal pair, vertical pair, 2 x 2 square (3 or 4 of its
    pixels), 1 x 3 row, 2 x 3 block (5 or 6 of its pixels)

F1 is the shape's footprint (1 on its pixels), F0 the ring of pixels around
it that must be free of signal, F1Nmin the number of footprint pixels that
must carry signal, and F1dx, F1dy the column and row offsets of each
footprint pixel from the anchor, so that the centroid comes out relative to
the anchor pixel's centre.  The thresholds are chosen so that a cloud that
fits one of the shapes matches exactly one feature.

Tap (i, j) of a 4 x 5 filter applied at pixel (r, c) meets pixel
(r + i - 1, c + j - 2): the alignment of TF's conv2d with "SAME" padding.
"""
from __future__ import annotations

import numpy as np

ROW0, COL0 = 1, 2  # window position of the anchor pixel


def _feature(cells, nmin):
    """Filters of one feature from its footprint cells (dy, dx)."""
    f1 = np.zeros((4, 5), np.float32)
    for dy, dx in cells:
        f1[ROW0 + dy, COL0 + dx] = 1.0
    ring = np.zeros((4, 5), np.float32)
    for dy, dx in cells:
        for ry in (-1, 0, 1):
            for rx in (-1, 0, 1):
                i, j = ROW0 + dy + ry, COL0 + dx + rx
                if 0 <= i < 4 and 0 <= j < 5:
                    ring[i, j] = 1.0
    ring[f1 != 0] = 0.0
    rows = np.arange(4, dtype=np.float32)[:, None] - ROW0
    cols = np.arange(5, dtype=np.float32)[None, :] - COL0
    # (+ 0 turns the -0 of negative offsets times 0 into +0)
    return ring, f1, f1 * cols + np.float32(0), f1 * rows + np.float32(0), np.float32(nmin)


def example_bank() -> dict:
    """Six features (see the module text); arrays [6][4][5] and [6]."""
    shapes = [
        ([(0, 0)], 1),
        ([(0, 0), (0, 1)], 2),
        ([(0, 0), (1, 0)], 2),
        ([(0, 0), (0, 1), (1, 0), (1, 1)], 3),
        ([(0, -1), (0, 0), (0, 1)], 3),
        ([(dy, dx) for dy in (0, 1) for dx in (-1, 0, 1)], 5),
    ]
    feats = [_feature(c, n) for c, n in shapes]
    f0, f1, fdx, fdy, nmin = (np.stack(a) for a in zip(*feats))
    return dict(f0=f0, f1=f1, f1_dx=fdx, f1_dy=fdy, f1_nmin=nmin)
