"""CUDA path vs the CPU oracle, element by element, through the C ABI.

The plain chain is bit-exact: hit lists (after sorting by frame and pixel),
common mode, corrected frames, count map and both histograms must be equal
bit for bit.  Cases span several 16x64 tiles and ragged tails, row and bank
common-mode units, units too large to stage in shared memory, empty calls,
hit-capacity overflow, frame offsets and the host-buffer entry point.  The
full 2.2 Mpixel batch of 1024 frames runs in the benchmark's configuration
and is checked on sampled frames plus size-independent properties.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import pd, synth
from tests._cases import (expected_cm, expected_hits, load_cases, sort_hits,
                          sparse_to_dense)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = load_cases()


def _ctx(geom: dict, thr: dict, ped, gain):
    return pd.pd_create(geom, ped, gain, thr)


def _oracle(geom: dict, thr: dict, ped, gain, raw, **kw):
    return oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr),
                          ped, gain, raw, **kw)


def _compare(ctx, out, ref, n_frames, check_corrected=True):
    hits, n = out.hits_host()
    assert n == ref.n_hits
    assert len(hits) == n, "hit capacity too small for a full comparison"
    assert len(ref.hits) == n, "oracle hit capacity too small for a full comparison"
    assert sort_hits(hits).tobytes() == sort_hits(ref.hits).tobytes()
    got_cm = out.cm.cpu().numpy()
    assert got_cm.tobytes() == ref.cm.reshape(n_frames, -1).tobytes()
    if check_corrected and out.corrected is not None:
        got = out.corrected.cpu().numpy()
        assert got.tobytes() == ref.corrected.reshape(n_frames, -1).tobytes()
    cmap, hp, hh = pd.pd_get_summary(ctx)
    np.testing.assert_array_equal(cmap, ref.count_map)
    np.testing.assert_array_equal(hp, ref.hist_pix)
    np.testing.assert_array_equal(hh, ref.hist_hit)


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_golden_cases_on_gpu(case):
    geom, thr = case["geometry"], case["thresholds"]
    ctx = _ctx(geom, thr, case["ped_arr"], case["gain_arr"])
    dev = pd.frames_to_device(case["raw_arr"])
    out = pd.process(ctx, dev, hit_capacity=64, corrected=True, cm=True)
    torch.cuda.synchronize()
    hits, n = out.hits_host()
    exp = expected_hits(case)
    assert n == len(exp)
    assert sort_hits(hits).tobytes() == exp.tobytes()
    assert out.cm.cpu().numpy().tobytes() == expected_cm(case).tobytes()
    cmap, hp, hh = pd.pd_get_summary(ctx)
    bins = thr["hist_bins"]
    np.testing.assert_array_equal(hp, sparse_to_dense(case["expect"]["hist_pix"], bins))
    np.testing.assert_array_equal(hh, sparse_to_dense(case["expect"]["hist_hit"], bins))
    np.testing.assert_array_equal(
        cmap, sparse_to_dense(case["expect"]["count_map"], cmap.size, np.uint32))


WORKLOADS = {
    # the 16-frame single-ASIC workload in full
    "asic_352x384_x16": (synth.asic_352x384(), 16),
    "cspad_2modules_x4": (synth.cspad_2p2m(n_modules=2), 4),
    "epix_704x768_x2": (synth.epix_704x768(occupancy=0.02), 2),
    "asic16_x1": (synth.asic16_352x384(n_modules=3), 1),
    # ragged against 16x64 tiles; bank units of 37x15
    "ragged_37x45_banks": (synth.Detector(n_modules=3, rows=37, cols=45 + 3,
                                          unit_rows=37, unit_cols=16,
                                          occupancy=0.03), 5),
    "ragged_rows_odd": (synth.Detector(n_modules=1, rows=19, cols=104,
                                       unit_rows=1, unit_cols=52,
                                       occupancy=0.05, cloud_sigma=0.5), 7),
    # a 65536-pixel unit does not fit in shared memory (global-key path)
    "big_unit_256x256": (synth.Detector(n_modules=1, rows=256, cols=256,
                                        unit_rows=256, unit_cols=256,
                                        occupancy=0.01), 2),
    "high_occupancy_pileup": (synth.asic_352x384(rows=64, occupancy=0.1,
                                                 cloud_sigma_hi=0.5,
                                                 cloud_sigma=0.2), 3),
    # narrow units: a four-pixel chunk of the band stencil meets up to four
    # units of one column, two of two or three columns
    "column_units_48x64": (synth.Detector(n_modules=2, rows=48, cols=64,
                                          unit_rows=48, unit_cols=1,
                                          occupancy=0.02), 3),
    "two_column_units_40x96": (synth.Detector(n_modules=1, rows=40, cols=96,
                                              unit_rows=20, unit_cols=2,
                                              occupancy=0.02), 3),
    "three_column_units_33x72": (synth.Detector(n_modules=2, rows=33, cols=72,
                                                unit_rows=11, unit_cols=3,
                                                occupancy=0.02), 3),
}


@pytest.mark.parametrize("kernels", [1, 2], ids=["lean_pair", "earlier_pair"])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_generated_workloads_bit_exact(name, kernels):
    det, n = WORKLOADS[name]
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, n)
    geom, thr = det.geometry(), det.thresholds()
    ctx = _ctx(geom, thr, ped, gain)
    pd.pd_set_tuning(ctx, kernels=kernels)
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = _oracle(geom, thr, ped, gain, raw, want_corrected=True)
    assert ref.n_hits > 0 or name == "big_unit_256x256"
    _compare(ctx, out, ref, n)


# Special paths of the large-unit common-mode kernel and the band stencil.
def _run_case(det, n, ped_shift=0.0, thr_over=None, integer_ped=False):
    ped, gain = synth.maps(det)
    if integer_ped:
        ped = np.rint(ped).astype(np.float32)
    raw, _ = synth.frames(det, ped, gain, 0, n)
    ped_chain = (ped + np.float32(ped_shift)).astype(np.float32)
    geom, thr = det.geometry(), dict(det.thresholds(), **(thr_over or {}))
    ctx = _ctx(geom, thr, ped_chain, gain)
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = _oracle(geom, thr, ped_chain, gain, raw, want_corrected=True)
    _compare(ctx, out, ref, n)
    return ref


def test_bank_odd_columns_scalar_paths():
    # unit_cols odd (scalar common-mode loads), cols % 4 != 0 (scalar stencil)
    det = synth.Detector(n_modules=2, rows=64, cols=198, unit_rows=64,
                         unit_cols=99, occupancy=0.02)
    assert _run_case(det, 3).n_hits > 0


def test_bank_median_below_window_uses_whole_unit_select():
    # d is about -400 ADU, below the window [cut - 512, cut) = [-312, 200)
    det = synth.cspad_2p2m(n_modules=2)
    ref = _run_case(det, 2, ped_shift=400.0)
    assert ref.n_hits > 0 and float(ref.cm.max()) < -312.0


def test_bank_flat_frames_overflow_candidates():
    # no noise and integer pedestals: every d of a bank is the same value,
    # so one 1/8-ADU bin holds the whole bank (more than the candidate buffer)
    det = synth.cspad_2p2m(n_modules=2, noise_sigma=0.0)
    ref = _run_case(det, 2, integer_ped=True)
    assert ref.n_hits > 0


def test_bank_unanchored_cut_generic_path():
    det = synth.cspad_2p2m(n_modules=2)
    _run_case(det, 2, thr_over=dict(cm_cut_adu=200.3))


def test_bank_low_pedestals_keep_float_codes():
    # pedestals near 100 ADU: d = raw - ped is not exact in binary32 over the
    # whole window, so the bank median keeps its floating-point bin codes
    det = synth.cspad_2p2m(n_modules=2, ped_mean=120.0, ped_sigma=30.0)
    ref = _run_case(det, 2)
    assert ref.n_hits > 0 and ref.cm.any()


def test_bank_wide_pedestal_spread():
    # pedestals spread over thousands of ADU: the integer codes do not fit
    # 16-bit lanes and the context keeps the floating-point bank median
    det = synth.cspad_2p2m(n_modules=2)
    ped, gain = synth.maps(det)
    ped = (ped + np.linspace(0.0, 6000.0, ped.size).reshape(ped.shape)).astype(np.float32)
    raw, _ = synth.frames(det, ped, gain, 0, 2)
    geom, thr = det.geometry(), det.thresholds()
    ctx = _ctx(geom, thr, ped, gain)
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    _compare(ctx, out, _oracle(geom, thr, ped, gain, raw, want_corrected=True), 2)


def test_lean_stencil_candidate_list_overflow():
    # a bright flat region: every pixel of it passes the seed threshold, more
    # candidates than a tile's list holds, so the tile tests every own pixel
    det = synth.cspad_2p2m(n_modules=1)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 2)
    raw = raw.reshape(2, det.rows, det.cols)
    raw[0, 10:60, 20:300] = np.minimum(raw[0, 10:60, 20:300].astype(np.int64) + 60, 65535)
    geom, thr = det.geometry(), det.thresholds()
    ctx = _ctx(geom, thr, ped, gain)
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = _oracle(geom, thr, ped, gain, raw, want_corrected=True)
    _compare(ctx, out, ref, 2)


def test_bank_min_count_not_reached():
    det = synth.cspad_2p2m(n_modules=1, occupancy=0.02)
    ref = _run_case(det, 2, thr_over=dict(cm_min_count=40000))
    assert not ref.cm.any()


def test_rows_median_below_window_uses_radix_fallback():
    # row units: 1-ADU bins over [-128, 128), [128, cut = 200) open bin 255;
    # d is about -300 ADU
    det = synth.asic_352x384(rows=24)
    ref = _run_case(det, 2, ped_shift=300.0)
    assert ref.n_hits > 0 and float(ref.cm.max()) < -128.0


def test_rows_median_in_open_top_bin_uses_radix_fallback():
    # d is about +170 ADU: below the cut (200) but above the window's 1-ADU
    # bins [-128, 128), so the median lies in the open bin [127, 200)
    det = synth.asic_352x384(rows=24)
    ref = _run_case(det, 2, ped_shift=-170.0)
    assert ref.n_hits > 0 and float(ref.cm.max()) < 200.0
    assert np.mean(ref.cm > 128.0) > 0.9


@pytest.mark.parametrize("shift", [0.0, -97.5], ids=["median_near_zero", "median_at_the_cut"])
def test_rows_window_closed_at_a_low_cut(shift):
    # cut 100 ADU <= 128: the bins span [cut - 256, cut) and bin 255 is the
    # whole 1-ADU bin [99, 100); with d about 97.5 ADU half the values lie
    # above the cut and the median of the rest sits just below it
    det = synth.asic_352x384(rows=24)
    ref = _run_case(det, 2, ped_shift=shift, thr_over=dict(cm_cut_adu=100.0))
    assert float(ref.cm.max()) < 100.0


def test_rows_flat_frames_many_equal_values():
    # integer pedestals, no noise: every d of a row is equal (> 64 values in
    # one 1/64-ADU sub-bin)
    det = synth.epix_704x768(rows=16, noise_sigma=0.0)
    ref = _run_case(det, 2, integer_ped=True)
    assert ref.n_hits > 0


def test_rows_non_integer_cut_generic_kernel():
    det = synth.asic_352x384(rows=24)
    _run_case(det, 2, thr_over=dict(cm_cut_adu=200.25))


def test_cm_none_and_masked_pixels():
    det = synth.asic_352x384(rows=32)
    ped, gain = synth.maps(det)
    gain.reshape(-1)[::97] = 0.0
    gain.reshape(-1)[5] = -1.0
    raw, _ = synth.frames(det, ped, gain, 0, 3)
    geom = dict(det.geometry(), cm_mode=pd.PD_CM_NONE)
    thr = det.thresholds()
    ctx = _ctx(geom, thr, ped, gain)
    assert ctx.info.masked_pixels == len(range(0, gain.size, 97)) + 1
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = _oracle(dict(geom), thr, ped, gain, raw, want_corrected=True)
    _compare(ctx, out, ref, 3)


def test_empty_call_zeroes_count():
    det = synth.asic_352x384(rows=16)
    ped, gain = synth.maps(det)
    ctx = _ctx(det.geometry(), det.thresholds(), ped, gain)
    out = pd.Outputs(ctx, 0, 8)
    out.n_hits.fill_(1234)
    dummy = torch.zeros(8, dtype=torch.int16, device="cuda")
    pd.pd_process(ctx, dummy.data_ptr(), 0, 0, **out.ptrs())
    torch.cuda.synchronize()
    assert int(out.n_hits.item()) == 0
    cmap, hp, hh = pd.pd_get_summary(ctx)
    assert cmap.sum() == 0 and hp.sum() == 0 and hh.sum() == 0


def test_hit_capacity_overflow_keeps_true_count():
    det = synth.asic_352x384(rows=64, occupancy=0.03)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 2)
    ctx = _ctx(det.geometry(), det.thresholds(), ped, gain)
    ref = _oracle(det.geometry(), det.thresholds(), ped, gain, raw)
    cap = ref.n_hits // 3
    out = pd.process(ctx, pd.frames_to_device(raw), hit_capacity=cap)
    torch.cuda.synchronize()
    hits, n = out.hits_host()
    assert n == ref.n_hits and len(hits) == cap
    ref_set = {h.tobytes() for h in ref.hits}
    assert all(h.tobytes() in ref_set for h in hits)
    assert len({h.tobytes() for h in hits}) == cap


def test_frame_base_and_accumulation_over_calls():
    det = synth.cspad_2p2m(n_modules=1)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 5)
    geom, thr = det.geometry(), det.thresholds()
    ctx = _ctx(geom, thr, ped, gain)
    dev = pd.frames_to_device(raw)
    a = pd.process(ctx, dev[:2])
    b = pd.process(ctx, dev[2:], frame_base=2)
    torch.cuda.synchronize()
    ref = _oracle(geom, thr, ped, gain, raw)
    ha, _ = a.hits_host()
    hb, _ = b.hits_host()
    got = sort_hits(np.concatenate([ha, hb]))
    assert got.tobytes() == sort_hits(ref.hits).tobytes()
    cmap, hp, hh = pd.pd_get_summary(ctx)
    np.testing.assert_array_equal(cmap, ref.count_map)
    np.testing.assert_array_equal(hp, ref.hist_pix)
    np.testing.assert_array_equal(hh, ref.hist_hit)
    pd.pd_reset_summary(ctx)
    cmap, hp, hh = pd.pd_get_summary(ctx)
    assert cmap.sum() == 0 and hp.sum() == 0 and hh.sum() == 0


def test_host_buffer_entry_point():
    det = synth.epix_704x768()
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 150)  # > one 64 MB chunk
    geom, thr = det.geometry(), det.thresholds()
    ctx = _ctx(geom, thr, ped, gain)
    hits, n = pd.pd_process_host(ctx, raw, frame_base=10)
    sample = [0, 77, 149]
    ref = _oracle(geom, thr, ped, gain, raw[sample])
    got = hits[np.isin(hits["frame"], [10 + s for s in sample])]
    exp = ref.hits.copy()
    exp["frame"] = np.array([10 + sample[f] for f in ref.hits["frame"]], np.uint32)
    assert sort_hits(got).tobytes() == sort_hits(exp).tobytes()
    assert n == len(hits)
    # overflow through the host path reports the true count
    small, n2 = pd.pd_process_host(ctx, raw[:3], hit_capacity=10)
    assert len(small) == 10 and n2 > 10


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable_hits", "page_locked_hits"])
def test_host_path_hits_downloaded_during_uploads(pinned):
    """Five 64 MB chunks of 2.2 Mpx frames: the hits that come back chunk by
    chunk while later chunks upload are exactly the device path's, and a
    capacity that ends inside one chunk's download returns that many distinct
    records of the full list with the true count."""
    det = synth.cspad_2p2m(occupancy=0.01)
    ped, gain = synth.maps(det)
    n = 70  # 14 frames per chunk
    raw, _ = synth.frames(det, ped, gain, 0, n, truth=False)
    geom, thr = det.geometry(), det.thresholds()
    dev_ctx = _ctx(geom, thr, ped, gain)
    out = pd.process(dev_ctx, pd.frames_to_device(raw), hit_capacity=n * 65536)
    torch.cuda.synchronize()
    ref, n_ref = out.hits_host()
    assert n_ref == len(ref) > 0
    ctx = _ctx(geom, thr, ped, gain)
    cap = n * 65536
    buf = (torch.empty(cap * pd.HIT_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True).numpy()
           if pinned else np.empty(cap * pd.HIT_DTYPE.itemsize, np.uint8)).view(pd.HIT_DTYPE)
    hits, nh = pd.pd_process_host(ctx, raw, out=buf)
    assert nh == n_ref == len(hits)
    assert sort_hits(hits).tobytes() == sort_hits(ref).tobytes()
    part = n_ref // 3 + 7
    some, n2 = pd.pd_process_host(ctx, raw, hit_capacity=part)
    assert n2 == n_ref and len(some) == part
    keys = set(zip(ref["frame"].tolist(), ref["pixel"].tolist()))
    got = list(zip(some["frame"].tolist(), some["pixel"].tolist()))
    assert len(set(got)) == part and set(got) <= keys


def test_invalid_arguments_rejected():
    det = synth.asic_352x384(rows=16)
    ped, gain = synth.maps(det)
    bad = dict(det.geometry(), unit_cols=100)
    with pytest.raises(pd.PdError) as ei:
        pd.pd_create(bad, ped, gain, det.thresholds())
    assert ei.value.code == pd.PD_EINVAL
    bad_thr = dict(det.thresholds(), zero_thr_kev=2.0, seed_thr_kev=1.0)
    with pytest.raises(pd.PdError):
        pd.pd_create(det.geometry(), ped, gain, bad_thr)
    ctx = _ctx(det.geometry(), det.thresholds(), ped, gain)
    out = pd.Outputs(ctx, 1, 8)
    buf = torch.zeros(ctx.pixels_per_frame + 8, dtype=torch.int16, device="cuda")
    with pytest.raises(pd.PdError) as ei:
        pd.pd_process(ctx, buf.data_ptr() + 2, 1, 0, **out.ptrs())
    assert ei.value.code == pd.PD_EALIGN


def test_full_size_cspad_batch_sampled():
    """1024 frames of the 32x185x388 geometry in one call (the benchmark's
    launch): sampled frames equal the oracle bit for bit, and the summaries
    obey size-independent identities."""
    det = synth.cspad_2p2m()
    ped, gain = synth.maps(det)
    n = 1024
    raw, _ = synth.frames(det, ped, gain, 0, n, truth=False)
    geom, thr = det.geometry(), det.thresholds()
    ctx = _ctx(geom, thr, ped, gain)
    dev = pd.frames_to_device(raw)
    out = pd.process(ctx, dev, hit_capacity=n * 16384, cm=True)
    torch.cuda.synchronize()
    hits, nh = out.hits_host()
    assert nh == len(hits) > 0
    cm_all = out.cm.cpu().numpy()
    cmap, hp, hh = pd.pd_get_summary(ctx)
    assert hp.sum() == n * det.pixels_per_frame
    assert hh.sum() >= nh
    assert int(cmap.astype(np.int64).sum()) == int(hits["count"].astype(np.int64).sum())
    for f in (0, 1, 517, n - 1):
        ref = _oracle(geom, thr, ped, gain, raw[f:f + 1])
        mine = hits[hits["frame"] == f].copy()
        mine["frame"] = 0
        assert sort_hits(mine).tobytes() == sort_hits(ref.hits).tobytes()
        assert cm_all[f].tobytes() == ref.cm.reshape(-1).tobytes()


@pytest.mark.parametrize("tuning", [dict(chunk_frames=1, overlap=1, two_pass=0),
                                    dict(chunk_frames=1, overlap=1, two_pass=1),
                                    dict(chunk_frames=3, overlap=0, two_pass=1),
                                    dict(chunk_frames=2, band_rows=4, overlap=1, two_pass=1),
                                    dict(chunk_frames=5, band_rows=17, overlap=1, two_pass=1),
                                    # 82 loaded rows over 5 row lanes: more than 64 seed
                                    # candidates per thread, one CTA per SM
                                    dict(chunk_frames=4, band_rows=80, overlap=0, two_pass=1),
                                    # the lean stencil with 1- and 2-row bands (halo rows
                                    # by the last row lanes), and the earlier pair
                                    dict(chunk_frames=2, band_rows=1, overlap=1, two_pass=1),
                                    dict(chunk_frames=3, band_rows=2, overlap=0, two_pass=1),
                                    dict(chunk_frames=4, overlap=1, two_pass=1, kernels=2),
                                    dict(chunk_frames=1, band_rows=9, overlap=0, two_pass=1,
                                         kernels=2)])
def test_results_independent_of_tuning(tuning):
    """Chunking, band height, the two-stream overlap and the choice between
    the one-kernel chain and the kernel pair change only the launch schedule:
    hits (as a set), common mode and summaries are equal."""
    det = synth.cspad_2p2m(n_modules=3, occupancy=0.01)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 11)
    geom, thr = det.geometry(), det.thresholds()
    ctx = _ctx(geom, thr, ped, gain)
    pd.pd_set_tuning(ctx, **tuning)
    got = pd.pd_get_tuning(ctx)
    assert got["chunk_frames"] == tuning["chunk_frames"]
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = _oracle(geom, thr, ped, gain, raw, want_corrected=True)
    _compare(ctx, out, ref, 11)


@pytest.mark.parametrize("bins", [1, 4096])
def test_histogram_bin_count_extremes(bins):
    """One bin (every value clipped into it) and the maximum PD_MAX_HIST_BINS."""
    det = synth.cspad_2p2m(n_modules=2, occupancy=0.02)
    thr = dict(det.thresholds(), hist_bins=bins, hist_bin_kev=0.02 if bins > 1 else 1.0)
    assert bins <= pd.PD_MAX_HIST_BINS
    _run_case(det, 2, thr_over=thr)


def test_widest_module_band_stencil():
    """2048 columns per module (the widest the band stencil takes), row units
    of 512 pixels (the largest the row kernel takes)."""
    det = synth.Detector(n_modules=1, rows=12, cols=2048, unit_rows=1, unit_cols=512,
                         occupancy=0.02)
    ref = _run_case(det, 2)
    assert ref.n_hits > 0


@pytest.mark.parametrize("kernels", [1, 2], ids=["lean_pair", "earlier_pair"])
def test_histogram_bins_non_dyadic_width_on_gpu(kernels):
    """e values next to the edges of 0.05 keV bins from -4 keV (not dyadic):
    the pixel histogram holds them in the bins of the fused form
    floor(fma(e, 1/w, -lo/w)) worked out in exact rationals by the oracle's
    pin (the division form would put each in the neighbouring bin)."""
    vals = [(0.20000001788139343, 84), (-0.9000000953674316, 62), (0.44999998807907104, 89),
            (0.5499998927116394, 91), (-1.0000001192092896, 59), (-0.9500001072883606, 60),
            (0.0, 80), (0.0, 80)]
    C = len(vals)
    geom = dict(n_modules=1, rows=1, cols=C, unit_rows=1, unit_cols=C, cm_mode=pd.PD_CM_NONE)
    thr = dict(cm_cut_adu=100.0, zero_thr_kev=100.0, seed_thr_kev=100.0, photon_kev=1.0,
               hist_lo_kev=-4.0, hist_bin_kev=0.05, hist_bins=1296)
    ped = np.array([-v for v, _ in vals], np.float32).reshape(1, 1, C)
    gain = np.ones((1, 1, C), np.float32)
    raw = np.zeros((1, 1, 1, C), np.uint16)
    ctx = _ctx(geom, thr, ped, gain)
    pd.pd_set_tuning(ctx, kernels=kernels)
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = _oracle(geom, thr, ped, gain, raw, want_corrected=True)
    _compare(ctx, out, ref, 1)
    exp = np.zeros(1296, np.uint64)
    for _, b in vals:
        exp[b] += 1
    np.testing.assert_array_equal(pd.pd_get_summary(ctx)[1], exp)
