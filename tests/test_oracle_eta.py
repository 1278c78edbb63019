"""Pins of the centroid linearisation oracle (oracle/eta.py) against what
the mathematics fixes: a uniform centroid maps to itself halved, a known
monotone distortion is undone, the map is monotone and spans [-1/2, 1/2],
the histogram counts exactly the single-photon hits."""
from __future__ import annotations

import numpy as np

from oracle import eta
from paper_1903_06838_gb300 import pd

B = 255


def _hits(dx, dy, count=None):
    h = np.zeros(len(dx), pd.HIT_DTYPE)
    h["dx"], h["dy"] = dx, dy
    h["count"] = 1 if count is None else count
    return h


def test_uniform_centroids_map_to_half():
    # centroids uniform on (-1, 1): F(d) = (d + 1) / 2, so u = d / 2
    m = 100_000
    d = (-1.0 + (np.arange(m) + 0.5) * (2.0 / m)).astype(np.float32)
    hist = eta.accumulate(np.zeros((2, B), np.uint32), _hits(d, d), B)
    u = eta.linearise(hist[0], d, B)
    assert np.max(np.abs(u - d / 2)) <= 1.0 / m + 2.0 ** -20


def test_known_distortion_is_undone():
    # true offsets u uniform in [-1/2, 1/2), measured d = sin(pi u), monotone
    rng = np.random.default_rng(0)
    u = rng.uniform(-0.5, 0.5, 400_000)
    d = np.sin(np.pi * u).astype(np.float32)
    hist = eta.accumulate(np.zeros((2, B), np.uint32), _hits(d, d), B)
    v = eta.linearise(hist[0], d, B)
    # linear interpolation inside bins of width 2/B plus sampling noise
    assert np.sqrt(np.mean((v - u) ** 2)) < 0.004
    assert np.max(np.abs(v - u)) < 0.02
    # without linearisation the error is far larger
    assert np.sqrt(np.mean((d / 2 - u) ** 2)) > 0.02


def test_map_is_monotone_and_spans_the_pixel():
    rng = np.random.default_rng(1)
    d = np.clip(rng.normal(0, 0.3, 50_000), -1, 1).astype(np.float32)
    hist = eta.accumulate(np.zeros((2, B), np.uint32), _hits(d, -d), B)
    grid = np.linspace(-1.2, 1.2, 10_001).astype(np.float32)
    v = eta.linearise(hist[0], grid, B)
    assert np.all(np.diff(v) >= 0)
    assert v[0] == np.float32(-0.5) and v[-1] == np.float32(0.5)
    # the ends of the range and beyond clip to the pixel edges
    assert eta.linearise(hist[0], np.float32([-1.0]), B)[0] == np.float32(-0.5)
    assert eta.linearise(hist[0], np.float32([1.0]), B)[0] == np.float32(0.5)


def test_only_single_photon_hits_count_and_change():
    d = np.float32([0.1, -0.3, 0.7, np.nan, 0.2])
    cnt = np.uint8([1, 2, 1, 1, 0])
    hits = _hits(d, d, cnt)
    hist = eta.accumulate(np.zeros((2, B), np.uint32), hits, B)
    assert hist[0].sum() == 2 and hist[1].sum() == 2
    k, _ = eta.bin_of(np.float32([0.1, 0.7]), B)
    assert hist[0][k[0]] == 1 and hist[0][k[1]] == 1
    out = eta.apply(hist, hits, B)
    assert out["dx"][1] == hits["dx"][1] and out["dx"][4] == hits["dx"][4]
    assert np.isnan(out["dx"][3])
    assert out["dx"][0] != hits["dx"][0]


def test_empty_histogram_is_the_identity():
    d = np.float32([0.25, -0.5])
    assert np.array_equal(eta.linearise(np.zeros(B, np.uint32), d, B), d)


def test_apply_flags_only_the_linearised_hits():
    d = np.float32([0.1, 0.2, np.inf])
    hits = _hits(d, d, np.uint8([1, 3, 1]))
    hits["flags"] = [1, 2, 0]
    hist = eta.accumulate(np.zeros((2, B), np.uint32), hits, B)
    out = eta.apply(hist, hits, B)
    assert list(out["flags"]) == [1 | eta.LINEARISED, 2, 0]
    assert pd.PD_HIT_LINEARISED == eta.LINEARISED


def test_atom_at_zero_maps_to_the_middle_of_its_mass():
    # 40 % of the centroids exactly 0 (all charge in the seed pixel), the rest
    # symmetric about 0: F jumps from 0.3 to 0.7 at d = 0, whose best
    # estimate is the middle of the jump, u = 0
    m = 30_000
    side = np.linspace(0.01, 0.99, m).astype(np.float32)
    d = np.concatenate([-side, side, np.zeros(40_000, np.float32)])
    hist = eta.accumulate(np.zeros((2, B), np.uint32), _hits(d, d), B)
    assert eta.linearise(hist[0], np.float32([0.0]), B)[0] == np.float32(0.0)
    # just off the atom the map leaves the jump's ends (within one bin's mass)
    lo, hi = eta.linearise(hist[0], np.float32([-0.01, 0.01]), B)
    assert -0.22 < lo < -0.19 and 0.19 < hi < 0.22


def test_one_bin_is_half_the_centroid():
    # a single bin spanning [-1, 1] interpolates the whole range linearly
    d = np.float32([-0.8, 0.0, 0.4, 1.0])
    hist = eta.accumulate(np.zeros((2, 1), np.uint32), _hits(d, d), 1)
    # (up to the float32 roundings of d + 1, the product by N and the quotient)
    assert np.max(np.abs(eta.linearise(hist[0], d, 1) - d / 2)) <= 2.0 ** -23
