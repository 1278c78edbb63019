"""Pins of the oracle's auto-ranging multi-gain decoding (caption of Fig. b:
several darks and gains per pixel): one stage reduces to the single-gain
chain, hand-computed energies of every stage, the common mode taken from
stage-0 pixels only and subtracted from them only, corrupt stages read as
bad pixels, and bright spots read back at their deposited energy."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import synth

F32 = np.float32


def _geo(det, mode=oracle.CM_MEDIAN):
    return oracle.geometry(**dict(det.geometry(), cm_mode=mode))


@pytest.mark.parametrize("name", ["asic", "cspad"])
def test_one_stage_is_the_single_gain_chain(name):
    det = {"asic": synth.asic_352x384(rows=48), "cspad": synth.cspad_2p2m(n_modules=2)}[name]
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 3)
    assert raw.max() < 1 << 15
    t = oracle.thresholds(**det.thresholds())
    a = oracle.process(_geo(det), t, ped, gain, raw, want_corrected=True)
    b = oracle.process(_geo(det), t, ped[None], gain[None], raw, want_corrected=True,
                       n_gains=1, gain_shift=15)
    assert a.hits.tobytes() == b.hits.tobytes()
    assert a.corrected.tobytes() == b.corrected.tobytes() and a.cm.tobytes() == b.cm.tobytes()
    np.testing.assert_array_equal(a.hist_pix, b.hist_pix)


def test_stage_energies_and_common_mode_by_hand():
    # one row unit of 8 pixels: stage-0 pixels with d = 7, 5, 6, a stage-1
    # pixel, a stage-2 pixel and a corrupt stage 3; two more stage-0 pixels
    # above the cut
    det = synth.Detector(n_modules=1, rows=1, cols=8, unit_rows=1, unit_cols=8)
    ped = np.zeros((3, 1, 1, 8), np.float32)
    ped[0] = 100.0
    ped[1] = 50.0
    ped[2] = 20.0
    gain = np.zeros((3, 1, 1, 8), np.float32)
    gain[0] = 25.0
    gain[1] = 8.0
    gain[2] = 0.25
    sh = 14
    words = [107, 105, 106, (1 << sh) | 850, (2 << sh) | 520, (3 << sh) | 9000, 900, 950]
    raw = np.array(words, np.uint16).reshape(1, 1, 1, 8)
    t = oracle.thresholds(200.0, 0.5, 0.5, 8.0, cm_min_count=1)
    r = oracle.process(_geo(det), t, ped, gain, raw, want_corrected=True, n_gains=3,
                       gain_shift=sh)
    # common mode: lower median of the stage-0 values below the cut {7, 5, 6}
    assert r.cm[0, 0] == F32(6.0)
    inv = [F32(1) / F32(25), F32(1) / F32(8), F32(1) / F32(0.25)]
    exp = [(F32(7) - F32(6)) * inv[0], (F32(5) - F32(6)) * inv[0], (F32(6) - F32(6)) * inv[0],
           F32(800) * inv[1],                 # stage 1: no common mode
           F32(500) * inv[2],                 # stage 2
           F32(0),                            # corrupt stage: bad pixel
           (F32(800) - F32(6)) * inv[0], (F32(850) - F32(6)) * inv[0]]
    np.testing.assert_array_equal(r.corrected.reshape(-1), np.array(exp, np.float32))


def test_common_mode_ignores_other_stages():
    # 64-pixel rows: 40 stage-1 pixels with low readings would pull a median
    # over all pixels far down; the stage-0 median stays at the offset
    det = synth.Detector(n_modules=1, rows=2, cols=64, unit_rows=1, unit_cols=64)
    ped = np.zeros((2, 1, 2, 64), np.float32)
    ped[0] = 1000.0
    ped[1] = 0.0
    gain = np.ones((2, 1, 2, 64), np.float32)
    raw = np.full((1, 1, 2, 64), 1012, np.int64)
    raw[..., :40] = (1 << 14) | 3
    t = oracle.thresholds(200.0, 0.5, 0.5, 8.0)
    r = oracle.process(_geo(det), t, ped, gain, raw.astype(np.uint16), n_gains=2,
                       gain_shift=14, want_corrected=True)
    np.testing.assert_array_equal(r.cm, [[12.0, 12.0]])
    e = r.corrected.reshape(2, 64)
    assert np.all(e[:, 40:] == 0) and np.all(e[:, :40] == 3)


def test_bright_spots_read_back_at_their_energy():
    det = synth.asic_352x384(rows=96, occupancy=0.0, seed=4)
    ped, gain = synth.multigain_maps(det)
    raw, blob = synth.multigain_frames(det, ped, gain, 0, 2, bad_frac=0.0)
    stage = raw >> 14
    assert (stage == 1).sum() > 50 and (stage == 2).sum() > 20
    t = oracle.thresholds(**det.thresholds())
    r = oracle.process(_geo(det), t, ped, gain, raw, want_corrected=True, n_gains=3,
                       gain_shift=14)
    e = r.corrected.reshape(raw.shape)
    for g, tol in ((1, 3.0), (2, 60.0)):
        sel = stage == g
        # stage noise of 4 ADU at gain ratio 1/3 or 1/100 of 25 ADU/keV, plus
        # the stage-0 noise carried into the reading
        err = e[sel] - blob[sel]
        assert abs(err.mean()) < tol / 3 and np.abs(err).max() < 6 * tol


def test_mean_modes_and_bad_shifts_are_rejected():
    det = synth.asic_352x384(rows=8)
    ped, gain = synth.multigain_maps(det, 2)
    raw = np.zeros((1, 1, 8, 384), np.uint16)
    t = oracle.thresholds(**det.thresholds())
    with pytest.raises(ValueError):
        oracle.process(_geo(det, oracle.CM_MEAN), t, ped, gain, raw, n_gains=2, gain_shift=14)
    with pytest.raises(ValueError):
        oracle.process(_geo(det), t, ped, gain, raw, n_gains=2, gain_shift=16)
