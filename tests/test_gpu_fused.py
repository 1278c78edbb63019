"""The one-kernel chain (one CTA per frame and module; bank common mode, then a
band sweep through a ring of rows) against the oracle, bit for bit, and
against the two-kernel path on the same inputs.  The geometries cover a
partial and an exact last band, one and two banks per module, a 4-pixel chunk
that straddles the bank boundary, modules of 1 and 2 rows, common mode off,
the whole-bank select fallbacks and the seed-list overflow scan."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def D(**kw):
    base = dict(n_modules=2, unit_rows=None, occupancy=0.02)
    base.update(kw)
    if base["unit_rows"] is None:
        base["unit_rows"] = base["rows"]
    return synth.Detector(**base)


GEOMS = {
    "cspad_3_sensors": (synth.cspad_2p2m(n_modules=3, occupancy=0.01), 3),
    "banks_37x96_partial_band": (D(rows=37, cols=96, unit_cols=48), 3),
    "banks_36x100_straddle": (D(rows=36, cols=100, unit_cols=50), 3),
    "one_bank_20x64": (D(rows=20, cols=64, unit_cols=64, occupancy=0.05), 4),
    "two_rows_388": (D(rows=2, cols=388, unit_cols=194, occupancy=0.05), 5),
    "one_row_388": (D(rows=1, cols=388, unit_cols=194, occupancy=0.05), 5),
    "dense_scan_12x388": (D(rows=12, cols=388, unit_cols=194, occupancy=0.6,
                            cloud_sigma=0.2), 2),
    "big_bank_256x256": (D(n_modules=1, rows=256, cols=256, unit_cols=256,
                           occupancy=0.01), 2),
}


def _run(det, n, two_pass, geom_over=None, thr_over=None, ped_shift=0.0,
         integer_ped=False, flat=False):
    ped, gain = synth.maps(det)
    if integer_ped:
        ped = np.rint(ped).astype(np.float32)
    raw, _ = synth.frames(det, ped, gain, 0, n)
    if flat:
        raw[:] = np.rint(ped).astype(np.uint16)[None]
    ped_chain = (ped + np.float32(ped_shift)).astype(np.float32)
    geom = dict(det.geometry(), **(geom_over or {}))
    thr = dict(det.thresholds(), **(thr_over or {}))
    ctx = pd.pd_create(geom, ped_chain, gain, thr)
    pd.pd_set_tuning(ctx, two_pass=two_pass)
    if not two_pass:
        assert pd.pd_get_tuning(ctx)["two_pass"] == 0, "one-kernel path not available"
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped_chain, gain,
                         raw, want_corrected=True)
    hits, nh = out.hits_host()
    assert nh == ref.n_hits and len(hits) == nh
    assert sort_hits(hits).tobytes() == sort_hits(ref.hits).tobytes()
    assert out.cm.cpu().numpy().tobytes() == ref.cm.reshape(n, -1).tobytes()
    assert out.corrected.cpu().numpy().tobytes() == ref.corrected.reshape(n, -1).tobytes()
    cmap, hp, hh = pd.pd_get_summary(ctx)
    np.testing.assert_array_equal(cmap, ref.count_map)
    np.testing.assert_array_equal(hp, ref.hist_pix)
    np.testing.assert_array_equal(hh, ref.hist_hit)
    return ref


@pytest.mark.parametrize("two_pass", [0, 1])
@pytest.mark.parametrize("name", list(GEOMS))
def test_geometries_bit_exact(name, two_pass):
    det, n = GEOMS[name]
    ref = _run(det, n, two_pass)
    assert ref.n_hits > 0


def test_common_mode_off():
    det = synth.cspad_2p2m(n_modules=2)
    _run(det, 2, 0, geom_over=dict(cm_mode=pd.PD_CM_NONE))


def test_median_below_window_falls_back_to_whole_bank_select():
    # d is about -400 ADU, below the window [cut - 448, cut) = [-248, 200)
    det = synth.cspad_2p2m(n_modules=2)
    ref = _run(det, 2, 0, ped_shift=400.0)
    assert float(ref.cm.max()) < -248.0


def test_flat_frames_overflow_the_candidates():
    # every d of a bank equal: one bin holds the whole bank
    det = synth.cspad_2p2m(n_modules=2, noise_sigma=0.0)
    _run(det, 2, 0, integer_ped=True)


def test_small_flat_banks_rank_among_equal_values():
    # banks of 12 x 32 = 384 pixels, all equal: the candidate path ranks
    # hundreds of equal values
    det = D(rows=12, cols=64, unit_cols=32, noise_sigma=0.0, occupancy=0.0)
    _run(det, 2, 0, integer_ped=True, flat=True)


def test_min_count_not_reached():
    det = synth.cspad_2p2m(n_modules=1, occupancy=0.02)
    ref = _run(det, 2, 0, thr_over=dict(cm_min_count=40000))
    assert not ref.cm.any()


def test_ineligible_geometries_report_two_pass():
    det = synth.asic_352x384(rows=8)   # row units: not column banks
    ped, gain = synth.maps(det)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    assert pd.pd_get_tuning(ctx)["two_pass"] == 1
    det = synth.cspad_2p2m(n_modules=1)
    ped, gain = synth.maps(det)
    ctx = pd.pd_create(det.geometry(), ped, gain, dict(det.thresholds(), cm_cut_adu=200.3))
    assert pd.pd_get_tuning(ctx)["two_pass"] == 1
