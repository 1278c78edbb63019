"""Pins of the oracle's matched-filter charge summing (section "Photon
Charge Summing", Figs. d, e; centroids of Fig. f).

The filter model is checked against scipy's 2-D correlation (exact, on
integer signals), the TF "SAME" alignment of a 4 x 5 kernel against a delta
filter, the Valid logic (overflow ring, F1Nmin) and the feature sums on
hand-computed isolated cloud shapes with the example bank, so that a
misaligned or transposed window, a dropped term or a wrong comparison fails
at least one of them."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest
from scipy.signal import correlate2d

import oracle
from paper_1903_06838_gb300 import filters

F32 = np.float32
PH = 8.0


def _run(sig, bank, hist_bins=1296, n_frames=1):
    """Chain on integer-valued signal maps: pedestal 100, gain 1, no common
    mode, zero threshold 0.5, so s equals the given integers."""
    sig = np.asarray(sig)
    R, C = sig.shape[-2:]
    raw = (100 + sig).astype(np.uint16).reshape(n_frames, 1, R, C)
    g = oracle.geometry(1, R, C, R, C, oracle.CM_NONE)
    t = oracle.thresholds(1000.0, 0.5, 0.5, PH, hist_bins=hist_bins)
    ped = np.full((1, R, C), 100.0, np.float32)
    gain = np.ones((1, R, C), np.float32)
    return oracle.process(g, t, ped, gain, raw, filters=oracle.filters(**bank))


def _one_feature(f1, f0=None, fdx=None, fdy=None, nmin=-1e30):
    z = np.zeros((1, 4, 5), np.float32)
    return dict(f0=z if f0 is None else np.float32(f0)[None],
                f1=np.float32(f1)[None],
                f1_dx=z if fdx is None else np.float32(fdx)[None],
                f1_dy=z if fdy is None else np.float32(fdy)[None],
                f1_nmin=[nmin])


def test_delta_filter_fixes_the_same_padding_alignment():
    # tap (0, 0) meets pixel (r - 1, c - 2): a signal at (5, 7) lands at (6, 9)
    f1 = np.zeros((4, 5))
    f1[0, 0] = 1.0
    sig = np.zeros((12, 16), np.int64)
    sig[5, 7] = 40
    r = _run(sig, _one_feature(f1, nmin=1.0))
    assert r.n_hits == 1
    assert divmod(int(r.hits["pixel"][0]), 16) == (6, 9)
    assert r.hits["energy_kev"][0] == F32(40.0)


@pytest.mark.parametrize("seed", range(4))
def test_always_valid_feature_is_a_2d_correlation(seed):
    rng = np.random.default_rng(seed)
    R, C = 23, 37
    sig = np.where(rng.random((R, C)) < 0.15, rng.integers(1, 30, (R, C)), 0)
    f1 = rng.integers(-1, 4, (4, 5)).astype(np.float32)
    fdx = rng.integers(-3, 4, (4, 5)).astype(np.float32)
    fdy = rng.integers(-3, 4, (4, 5)).astype(np.float32)
    r = _run(sig, _one_feature(f1, fdx=fdx, fdy=fdy))
    pad = np.pad(sig.astype(np.float64), ((1, 2), (2, 2)))
    E = correlate2d(pad, f1, mode="valid")
    Mx = correlate2d(pad, fdx, mode="valid")
    My = correlate2d(pad, fdy, mode="valid")
    assert E.shape == (R, C)
    # seeds: every pixel whose sum is nonzero (the feature is always valid)
    assert r.n_seeds == int(np.count_nonzero(E))
    n = np.clip(np.rint(E / PH), 0, 255)
    exp = np.argwhere(n >= 1)
    got = sorted(divmod(int(p), C) for p in r.hits["pixel"])
    assert got == sorted(map(tuple, exp))
    for h in r.hits:
        rr, cc = divmod(int(h["pixel"]), C)
        assert h["energy_kev"] == F32(E[rr, cc])
        assert h["count"] == n[rr, cc]
        assert h["dx"] == F32(F32(Mx[rr, cc]) / F32(E[rr, cc]))
        assert h["dy"] == F32(F32(My[rr, cc]) / F32(E[rr, cc]))


SHAPES = {
    # name: cells (dy, dx) relative to the anchor, the matching feature
    "single": ([(0, 0)], 0),
    "h_pair": ([(0, 0), (0, 1)], 1),
    "v_pair": ([(0, 0), (1, 0)], 2),
    "l_shape": ([(0, 0), (0, 1), (1, 1)], 3),
    "square": ([(0, 0), (0, 1), (1, 0), (1, 1)], 3),
    "row3": ([(0, -1), (0, 0), (0, 1)], 4),
    "block2x3_5": ([(0, -1), (0, 0), (0, 1), (1, -1), (1, 0)], 5),
    "block2x3": ([(dy, dx) for dy in (0, 1) for dx in (-1, 0, 1)], 5),
}


@pytest.mark.parametrize("name", list(SHAPES))
def test_isolated_shape_matches_one_feature_at_its_anchor(name):
    cells, feat = SHAPES[name]
    rng = np.random.default_rng(len(name))
    sig = np.zeros((10, 12), np.int64)
    r0, c0 = 4, 5
    vals = rng.integers(3, 60, len(cells))
    for (dy, dx), v in zip(cells, vals):
        sig[r0 + dy, c0 + dx] = v
    r = _run(sig, filters.example_bank())
    assert r.n_seeds == 1 and r.n_hits == 1
    h = r.hits[0]
    assert divmod(int(h["pixel"]), 12) == (r0, c0)
    tot = int(vals.sum())
    assert h["energy_kev"] == F32(tot)
    mx = sum(int(v) * dx for (dy, dx), v in zip(cells, vals))
    my = sum(int(v) * dy for (dy, dx), v in zip(cells, vals))
    assert h["dx"] == F32(Fraction(mx, tot))
    assert h["dy"] == F32(Fraction(my, tot))
    assert h["npix"] == len(cells)
    assert h["count"] == int(np.rint(tot / PH)) or (tot / PH < 0.5 and r.n_hits == 0)


def test_touching_shapes_overflow_and_are_not_matched():
    # a single pixel next to a horizontal pair: each lies in the other's
    # ring, and together they fit no feature (a 1 x 3 row needs them in
    # one row with nothing around)
    sig = np.zeros((10, 12), np.int64)
    sig[4, 4] = 20
    sig[5, 5:7] = (15, 9)
    r = _run(sig, filters.example_bank())
    assert r.n_hits == 0 and r.n_seeds == 0


def test_nmin_and_overflow_comparisons():
    # one feature: F1 a 1 x 2 pair, F0 one pixel to its right
    f1 = np.zeros((4, 5))
    f1[1, 2:4] = 1.0
    f0 = np.zeros((4, 5))
    f0[1, 4] = 1.0
    sig = np.zeros((6, 10), np.int64)
    sig[2, 2:4] = (10, 10)
    # Size 2 >= 2 is valid (>=, not >), at the anchor (2, 2) only
    r = _run(sig, _one_feature(f1, f0=f0, nmin=2.0))
    assert [divmod(int(p), 10) for p in r.hits["pixel"]] == [(2, 2)]
    # a signal pixel in F0 at the anchor's right blocks it (== 0 required)
    sig[2, 4] = 1
    r = _run(sig, _one_feature(f1, f0=f0, nmin=2.0))
    assert (2, 2) not in [divmod(int(p), 10) for p in r.hits["pixel"]]
    # Size 2 < 2.5: not valid
    sig[2, 4] = 0
    assert _run(sig, _one_feature(f1, f0=f0, nmin=2.5)).n_seeds == 0


def test_features_add_up_in_order_and_zero_droplets_add_no_centroid():
    # two always-valid features at the same pixel: E adds, dx adds the two
    # centroids; a feature whose droplet is 0 adds 0 to dx
    sig = np.zeros((8, 8), np.int64)
    sig[3, 3] = 12
    sig[3, 4] = 4
    z = np.zeros((4, 5), np.float32)
    a = z.copy()
    a[1, 2] = 1.0
    a[1, 3] = 1.0
    adx = z.copy()
    adx[1, 3] = 1.0
    b = z.copy()
    b[1, 3] = 2.0
    bdx = z.copy()
    bdx[1, 3] = 3.0
    c = z.copy()
    c[3, 0] = 1.0      # never under signal at (3, 3): droplet 0
    cdx = z.copy()
    cdx[3, 0] = 5.0
    bank = dict(f0=np.stack([z, z, z]), f1=np.stack([a, b, c]),
                f1_dx=np.stack([adx, bdx, cdx]), f1_dy=np.stack([z, z, z]),
                f1_nmin=[1.0, 1.0, -1.0])
    r = _run(sig, bank)
    h = [x for x in r.hits if divmod(int(x["pixel"]), 8) == (3, 3)][0]
    assert h["energy_kev"] == F32(16 + 8)
    assert h["dx"] == F32(F32(4 / 16) + F32(12 / 8))
    assert h["npix"] == 2


def test_invalid_banks_are_rejected():
    bank = filters.example_bank()
    bad = dict(bank, f1=np.where(bank["f1"] > 0, np.inf, 0).astype(np.float32))
    with pytest.raises(ValueError):
        _run(np.zeros((4, 6), np.int64), bad)
    with pytest.raises(ValueError):
        _run(np.zeros((4, 6), np.int64), dict(bank, f1_nmin=[np.nan] * 6))
