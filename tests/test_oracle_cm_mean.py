"""Pins of the oracle's paper common mode (Fig. c: the mean of the background
pixels with the sqrt(group size) guard) and of its three stacked stages
(unit, module row, module column; section "Performance").

The estimator is checked against hand-computed worked examples, against an
exactly rounded sum in rational arithmetic, and the chain against noise-free
frames whose offsets are separable by construction, so that a stage applied
along the wrong axis, in the wrong order, without the guard or without the
cut fails."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import synth

F32 = np.float32


def _exact_mean(values, cut):
    """Independent statement of the estimator for values on a dyadic grid:
    the exact rational sum rounded once to binary32, then divided."""
    v = np.asarray(values, np.float32)
    sel = v[(v < F32(cut)) & (v > -np.inf)]
    total = sum((Fraction(float(x)) for x in sel), Fraction(0))
    s32 = F32(float(total))  # exact in binary64 here, so one rounding
    den = max(F32(len(sel)), np.sqrt(F32(len(v))))
    return F32(s32 / F32(den))


# --------------------------------------------------------------------------
# worked examples of the estimator
def test_guard_takes_sqrt_of_group_size():
    # 16 pixels, 3 of them below the cut: max(3, sqrt 16) = 4 -> 6 / 4
    v = [1.0, 2.0, 3.0] + [300.0] * 13
    assert oracle.paper_mean(v, 200.0) == F32(1.5)
    # all 4 pixels below: the plain mean (max(4, 2) = 4)
    assert oracle.paper_mean([1.0, 2.0, 3.0, 4.0], 200.0) == F32(2.5)
    # one of 9 below: divided by sqrt 9 = 3
    assert oracle.paper_mean([6.0] + [250.0] * 8, 200.0) == F32(2.0)
    # none below: 0
    assert oracle.paper_mean([250.0] * 5, 200.0) == F32(0.0)


def test_cut_is_strict_and_minus_infinity_is_left_out():
    assert oracle.paper_mean([200.0, 1.0, 3.0, 8.0], 200.0) == F32(4.0)
    assert oracle.paper_mean([-np.inf, 1.0, 2.0, 3.0], 200.0) == F32(2.0)
    assert oracle.paper_mean([np.nan, 1.0, 2.0, 3.0], 200.0) == F32(2.0)


def test_values_far_below_the_largest_fall_off_the_grid():
    # the grid of the sum is 2^(E - 38) with E = floor(log2 max|v|) = 10:
    # 2^-40 rounds to 0 there, so 1024 - 1024 + 2^-40 sums to 0
    v = [1024.0, -1024.0, 2.0 ** -40]
    assert oracle.paper_mean(v, 2048.0) == F32(0.0)
    # 2^-28 is the grid step itself and survives
    v = [1024.0, -1024.0, 2.0 ** -28]
    assert oracle.paper_mean(v, 2048.0) == F32(2.0 ** -28 / 3)


@pytest.mark.parametrize("seed", range(5))
def test_sum_is_the_exactly_rounded_sum(seed):
    # values on the 2^-8 grid, as d = raw - pedestal is for pedestals with
    # 8 fractional bits; the sum then is the exactly rounded sum
    rng = np.random.default_rng(seed)
    for n in (1, 7, 100, 4096, 35890):
        v = (rng.integers(-260_000, 60_000, n) / 256.0).astype(np.float32)
        got = oracle.paper_mean(v, 150.0)
        assert got == _exact_mean(v, 150.0), (n, got)
    # cancellation: the exact sum is tiny against the terms
    v = np.float32([1000.5, -1000.25, 0.00390625, 77.0, -77.0])
    assert oracle.paper_mean(v, 2000.0) == _exact_mean(v, 2000.0)


# --------------------------------------------------------------------------
# the chain in the two mean modes
def _thr(cut=200.0):
    return oracle.thresholds(cut, 0.8, 0.8, 8.0)


def _separable(R, C, ur, uc, rng):
    """Integer offsets a_unit + b_row + c_col with b summing to 0 over the
    module's rows and c summing to 0 over each unit's columns."""
    b = rng.integers(-6, 7, R).astype(np.int64)
    b[-1] -= b.sum()
    c = np.zeros(C, np.int64)
    for j in range(C // uc):
        cc = rng.integers(-6, 7, uc)
        cc[-1] -= cc.sum()
        c[j * uc:(j + 1) * uc] = cc
    a = rng.integers(-20, 21, (R // ur, C // uc)).astype(np.int64)
    off = np.repeat(np.repeat(a, ur, 0), uc, 1) + b[:, None] + c[None, :]
    return a, b, c, off


@pytest.mark.parametrize("shape", [(8, 12, 8, 6), (6, 10, 6, 10), (12, 8, 12, 4)])
def test_stacked_stages_recover_separable_offsets(shape):
    R, C, ur, uc = shape
    rng = np.random.default_rng(R * C)
    a, b, c, off = _separable(R, C, ur, uc, rng)
    ped = np.full((1, R, C), 1000.0, np.float32)
    gain = np.ones((1, R, C), np.float32)
    raw = (1000 + off).astype(np.uint16)[None, None]
    g = oracle.geometry(1, R, C, ur, uc, oracle.CM_MEAN_STACKED)
    r = oracle.process(g, _thr(), ped, gain, raw, want_corrected=True)
    upf = (R // ur) * (C // uc)
    assert r.cm.shape == (1, upf + R + C)
    np.testing.assert_array_equal(r.cm[0, :upf], a.reshape(-1).astype(np.float32))
    np.testing.assert_array_equal(r.cm[0, upf:upf + R], b.astype(np.float32))
    np.testing.assert_array_equal(r.cm[0, upf + R:], c.astype(np.float32))
    assert not np.any(r.corrected) and r.n_hits == 0
    # the single-stage mean removes only the unit terms
    g1 = oracle.geometry(1, R, C, ur, uc, oracle.CM_MEAN)
    r1 = oracle.process(g1, _thr(), ped, gain, raw, want_corrected=True)
    np.testing.assert_array_equal(r1.cm[0], a.reshape(-1).astype(np.float32))
    np.testing.assert_array_equal(r1.corrected.reshape(R, C),
                                  (b[:, None] + c[None, :]).astype(np.float32))


def test_stacked_guard_and_cut_per_stage():
    # 4 x 6 module, one unit.  Column 2 has photons (1000 ADU) in three of
    # its four rows: stage 3 sees one background pixel there and divides by
    # sqrt(4) = 2; rows 0..2 see one photon each, left out by the cut.
    R, C = 4, 6
    base = np.full((R, C), 10, np.int64)
    base[:, 4] += 4           # column term seen by stage 3
    base[0:3, 2] = 1000       # photons
    ped = np.zeros((1, R, C), np.float32)
    gain = np.ones((1, R, C), np.float32)
    raw = base.astype(np.uint16)[None, None]
    g = oracle.geometry(1, R, C, R, C, oracle.CM_MEAN_STACKED)
    r = oracle.process(g, _thr(200.0), ped, gain, raw)
    # stage 1: 21 background pixels (sum 21*10 + 4*4 = 226); guard sqrt(24)
    cm1 = F32(226.0) / F32(21.0)
    assert r.cm[0, 0] == cm1
    # stage 2, row 0: five background pixels d - cm1, guard sqrt(6)
    row0 = [F32(10) - cm1] * 4 + [F32(14) - cm1]
    row0 = [row0[0], row0[1], F32(1000) - cm1, row0[2], row0[3], row0[4]]
    assert r.cm[0, 1] == _exact_mean(np.float32(row0), 200.0)
    # stage 3, column 2: only row 3 is background -> (value) / 2
    cm2 = r.cm[0, 1:1 + R]
    v3 = (F32(10) - cm1) - cm2[3]
    assert r.cm[0, 1 + R + 2] == F32(float(v3) / 2.0)


@pytest.mark.parametrize("mode", [oracle.CM_MEAN, oracle.CM_MEAN_STACKED])
def test_mean_tracks_injected_offset(mode):
    """Synthetic banks with noise 4 ADU, injected offsets and photons at
    0.5 % occupancy: the paper's mean lands within a few standard errors of
    the offset plus the bias of the photon charge that stays below the cut
    (shared charge of about 200 ADU per photon, under 1.5 ADU per pixel),
    and that bias is upward."""
    det = synth.cspad_2p2m(n_modules=2).replace(seed=11)
    ped, gain = synth.maps(det)
    raw, _, cm_true = synth.frames(det, ped, gain, 0, 3, cm_truth=True)
    geo = dict(det.geometry(), cm_mode=mode)
    r = oracle.process(oracle.geometry(**geo), oracle.thresholds(**det.thresholds()),
                       ped, gain, raw)
    upf = det.units_per_frame
    n = det.unit_rows * det.unit_cols
    err = r.cm[:, :upf] - cm_true
    assert np.max(np.abs(err)) < 6 * det.noise_sigma / math.sqrt(n) + 1.5
    assert err.mean() > 0
    if mode == oracle.CM_MEAN_STACKED:
        # rows and columns carry no injected offset: residual terms of the
        # noise (4 / sqrt(185) ADU) and of sub-cut photon charge (one photon
        # per 185-pixel column on average, ~1 ADU each) only
        rest = np.abs(r.cm[:, upf:])
        assert rest.max() < 5.0 and np.median(rest) < 1.0


def test_mean_modes_reject_oversized_units():
    t = _thr()
    ped = np.zeros((1, 4, 4), np.float32)
    assert oracle.cm_values_per_frame(oracle.geometry(2, 4, 6, 2, 3, oracle.CM_MEAN_STACKED)) \
        == 2 * 4 + 2 * (4 + 6)
    with pytest.raises(ValueError):
        oracle.process(oracle.geometry(1, 4, 4, 4, 4, 4), t, ped, ped + 1,
                       np.zeros((1, 1, 4, 4), np.uint16))
