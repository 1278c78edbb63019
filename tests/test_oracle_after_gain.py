"""Pins of the oracle's processing in the paper's order (gain before common
mode, Fig. a; Fig. c takes the gain-corrected Frames1): with unit gains it
is the default order bit for bit in every common-mode mode; a hand-worked
unit fixes the selection on gain-corrected values, the exclusion of masked
pixels and their zero reading; and a gain spread leaves the residual the
default order removes."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import synth

F32 = np.float32


@pytest.mark.parametrize("mode", [oracle.CM_MEDIAN, oracle.CM_MEAN, oracle.CM_MEAN_STACKED])
def test_unit_gain_matches_the_default_order(mode):
    det = synth.cspad_2p2m(n_modules=2, gain_sigma=0.0, adu_per_kev=1.0, photon_kev=200.0,
                           seed=5)
    ped, gain = synth.maps(det)
    assert np.all(gain == 1.0)
    raw, _ = synth.frames(det, ped, gain, 0, 3)
    thr = det.thresholds()
    assert thr["cm_cut_kev"] == thr["cm_cut_adu"]
    res = []
    for ag in (0, 1):
        g = oracle.geometry(**dict(det.geometry(), cm_mode=mode, cm_after_gain=ag))
        res.append(oracle.process(g, oracle.thresholds(**thr), ped, gain, raw,
                                  want_corrected=True))
    a, b = res
    assert a.n_hits > 0 and a.hits.tobytes() == b.hits.tobytes()
    assert a.cm.tobytes() == b.cm.tobytes() and a.corrected.tobytes() == b.corrected.tobytes()
    np.testing.assert_array_equal(a.hist_pix, b.hist_pix)


def test_hand_worked_unit():
    # one row unit of 6 pixels: d = 10, 20, 30, 40, 50, 60 ADU; gains 10, 10,
    # 5, 10, 0 (masked), 2 ADU/keV -> e0 = 1, 2, 6, 4, -, 30 keV
    R, C = 1, 6
    ped = np.full((1, R, C), 100.0, np.float32)
    gain = np.float32([[[10, 10, 5, 10, 0, 2]]])
    raw = (100 + np.array([10, 20, 30, 40, 50, 60])).astype(np.uint16).reshape(1, 1, R, C)
    g = oracle.geometry(1, R, C, 1, C, oracle.CM_MEDIAN, 1)
    # cut 10 keV: the set is {1, 2, 6, 4} (30 is above, the masked pixel is
    # out); lower median of 4 values = the 2nd smallest = 2
    t = oracle.thresholds(1000.0, 0.5, 0.5, 8.0, cm_min_count=1, cm_cut_kev=10.0)
    r = oracle.process(g, t, ped, gain, raw, want_corrected=True)
    assert r.cm[0, 0] == F32(2.0)
    inv = [F32(1) / F32(v) if v else F32(0) for v in (10, 10, 5, 10, 0, 2)]
    e0 = [F32(d) * i for d, i in zip((10, 20, 30, 40, 50, 60), inv)]
    exp = [x - F32(2.0) for x in e0]
    exp[4] = F32(0.0)                     # the masked pixel reads 0
    np.testing.assert_array_equal(r.corrected.reshape(-1), np.array(exp, np.float32))
    # the same unit in the default order selects on d in ADU (cut 35 ADU):
    # {10, 20, 30} and the masked pixel's d = 50 is above it; median 20
    g0 = oracle.geometry(1, R, C, 1, C, oracle.CM_MEDIAN, 0)
    t0 = oracle.thresholds(35.0, 0.5, 0.5, 8.0, cm_min_count=1)
    assert oracle.process(g0, t0, ped, gain, raw).cm[0, 0] == F32(20.0)


def test_mean_skips_masked_pixels():
    # 4 pixels, one masked: the paper's mean over the 3 others, guard sqrt(4)
    ped = np.zeros((1, 1, 4), np.float32)
    gain = np.float32([[[1, 1, 0, 1]]])
    raw = np.array([3, 5, 1000, 7], np.uint16).reshape(1, 1, 1, 4)
    g = oracle.geometry(1, 1, 4, 1, 4, oracle.CM_MEAN, 1)
    t = oracle.thresholds(1e9, 0.5, 0.5, 8.0, cm_cut_kev=100.0)
    r = oracle.process(g, t, ped, gain, raw)
    assert r.cm[0, 0] == F32(15.0) / F32(3.0)


def test_gain_spread_leaves_the_offset_residual():
    # noise-free dark frames with an injected offset per row unit: the
    # default order removes it exactly; the paper's order leaves
    # offset * (inv_gain_p - median) on each pixel
    det = synth.asic_352x384(rows=16, occupancy=0.0, noise_sigma=0.0, seed=2)
    ped, gain = synth.maps(det)
    ped = np.rint(ped).astype(np.float32)
    raw, _, cm_true = synth.frames(det, ped, gain, 0, 2, cm_truth=True)
    t = oracle.thresholds(**det.thresholds())
    g0 = oracle.geometry(**det.geometry())
    g1 = oracle.geometry(**dict(det.geometry(), cm_after_gain=1))
    a = oracle.process(g0, t, ped, gain, raw, want_corrected=True)
    b = oracle.process(g1, t, ped, gain, raw, want_corrected=True)
    assert not np.any(a.corrected)
    off = np.abs(np.rint(cm_true)).max()
    resid = np.abs(b.corrected).max()
    assert 0 < resid < off * 0.2  # gain spread 3 %: residuals of a few % of the offset
