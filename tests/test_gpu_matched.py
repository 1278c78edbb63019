"""Matched-filter charge summing on the GPU (pd_set_filter_bank) against the
CPU oracle, bit for bit: hits, corrected frames, common mode and summaries,
with the example six-feature bank and with random banks (arbitrary signs
and magnitudes, sparse and dense taps, thresholds that make features
always or never valid), on row units, banks, ragged geometries and the
stacked mean common mode; entry points, batches, tuning and bank changes."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import filters, pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def random_bank(seed, n_features=6):
    rng = np.random.default_rng(seed)
    shape = (n_features, 4, 5)
    dense = rng.random(shape) < 0.35
    f1 = np.where(dense, rng.choice([1.0, 1.0, 0.5, 2.0, -0.25], shape), 0.0)
    f0 = np.where(rng.random(shape) < 0.2, rng.choice([1.0, 0.3, -1.0], shape), 0.0)
    fdx = np.where(f1 != 0, rng.uniform(-2, 2, shape), 0.0)
    fdy = np.where(rng.random(shape) < 0.4, rng.uniform(-2, 2, shape), 0.0)
    nmin = rng.choice([-1.0, 0.0, 1.0, 2.0, 2.5, 1e9], n_features)
    return dict(f0=f0, f1=f1, f1_dx=fdx, f1_dy=fdy, f1_nmin=nmin)


def binary_bank(seed, n_features=7):
    """Footprints of ones and positive rings (the table path: validity is a
    function of the window mask), thresholds fractional, never or always met."""
    rng = np.random.default_rng(seed)
    shape = (n_features, 4, 5)
    f1 = np.where(rng.random(shape) < 0.3, 1.0, 0.0)
    f0 = np.where((f1 == 0) & (rng.random(shape) < 0.3), rng.choice([0.3, 1.0, 2.0], shape), 0.0)
    fdx = np.where(f1 != 0, rng.uniform(-2, 2, shape), 0.0)
    fdy = np.where(f1 != 0, rng.uniform(-2, 2, shape), 0.0)
    nmin = np.resize(np.array([1.0, -1.0, 0.0, 2.5, 1e9, 3.0, 2.0]), n_features)
    return dict(f0=f0, f1=f1, f1_dx=fdx, f1_dy=fdy, f1_nmin=nmin)


BANKS = {"example": filters.example_bank(), "random1": random_bank(1),
         "random2_3f": random_bank(2, 3), "random3_8f": random_bank(3, 8),
         "binary4_7f": binary_bank(4)}

WORKLOADS = {
    "asic_rows_x8": (synth.asic_352x384(cloud_sigma=0.35), 8),
    "cspad_banks_x2": (synth.cspad_2p2m(n_modules=2, occupancy=0.01), 2),
    "epix_x1": (synth.epix_704x768(occupancy=0.02), 1),
    "ragged_37x45": (synth.Detector(n_modules=3, rows=37, cols=45, unit_rows=37,
                                    unit_cols=15, occupancy=0.03, cloud_sigma=0.4), 3),
    "tiny_3x5": (synth.Detector(n_modules=2, rows=3, cols=5, unit_rows=3, unit_cols=5,
                                occupancy=0.2), 4),
}


def _run(det, n, bank, cm_mode=0, tuning=None, ped=None, gain=None, raw=None):
    if ped is None:
        ped, gain = synth.maps(det)
        raw, _ = synth.frames(det, ped, gain, 0, n, truth=False)
    geom = dict(det.geometry(), cm_mode=cm_mode)
    thr = det.thresholds()
    ctx = pd.pd_create(geom, ped, gain, thr)
    if bank is not None:
        pd.pd_set_filter_bank(ctx, **bank)
    if tuning:
        pd.pd_set_tuning(ctx, **tuning)
    # every pixel can hold a hit when some feature is always valid
    cap = n * det.pixels_per_frame
    out = pd.process(ctx, pd.frames_to_device(raw), hit_capacity=cap, corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         want_corrected=True, hit_capacity=cap,
                         filters=None if bank is None else oracle.filters(**bank))
    return ctx, out, ref


def _compare(ctx, out, ref, n):
    hits, nh = out.hits_host()
    assert nh == ref.n_hits and len(hits) == nh and len(ref.hits) == nh
    assert sort_hits(hits).tobytes() == sort_hits(ref.hits).tobytes()
    assert out.cm.cpu().numpy().tobytes() == ref.cm.reshape(n, -1).tobytes()
    assert out.corrected.cpu().numpy().tobytes() == ref.corrected.reshape(n, -1).tobytes()
    for got, exp in zip(pd.pd_get_summary(ctx), (ref.count_map, ref.hist_pix, ref.hist_hit)):
        np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("bank", list(BANKS))
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_workloads_bit_exact(name, bank):
    det, n = WORKLOADS[name]
    ctx, out, ref = _run(det, n, BANKS[bank])
    if bank == "example" and name != "tiny_3x5":
        assert ref.n_hits > 0
    _compare(ctx, out, ref, n)


# Shapes of the band form (columns a multiple of 4, single gain): ragged last
# bands, modules of one and two rows, the widest and narrowest rows, units
# two columns wide (a four-pixel chunk meets two units), and signal dense
# enough that a band's candidate list overflows and every pixel is tested.
D = synth.Detector
BAND_SHAPES = {
    "one_row_modules": (D(n_modules=3, rows=1, cols=96, unit_rows=1, unit_cols=48,
                          occupancy=0.1), 4),
    "two_row_modules": (D(n_modules=2, rows=2, cols=388, unit_rows=2, unit_cols=194,
                          occupancy=0.05), 3),
    "ragged_bands_100x128": (D(n_modules=2, rows=100, cols=128, unit_rows=25, unit_cols=64,
                               occupancy=0.03), 3),
    "wide_2048": (D(n_modules=1, rows=20, cols=2048, unit_rows=20, unit_cols=512,
                    occupancy=0.01), 2),
    "narrow_4": (D(n_modules=2, rows=700, cols=4, unit_rows=100, unit_cols=4,
                   occupancy=0.05), 2),
    "two_column_units": (D(n_modules=1, rows=24, cols=64, unit_rows=24, unit_cols=2,
                           occupancy=0.03), 3),
    "dense_overflow": (D(n_modules=2, rows=40, cols=388, unit_rows=40, unit_cols=194,
                         occupancy=0.5, cloud_sigma=0.5), 2),
}


@pytest.mark.parametrize("bank", ["example", "random1"])
@pytest.mark.parametrize("name", list(BAND_SHAPES))
def test_band_shapes_bit_exact(name, bank):
    det, n = BAND_SHAPES[name]
    ctx, out, ref = _run(det, n, BANKS[bank])
    if bank == "example":
        assert ref.n_hits > 0
    _compare(ctx, out, ref, n)


@pytest.mark.parametrize("name", ["ragged_bands_100x128", "dense_overflow"])
def test_band_shapes_stacked_mean(name):
    det, n = BAND_SHAPES[name]
    ctx, out, ref = _run(det, n, filters.example_bank(), cm_mode=pd.PD_CM_MEAN_STACKED)
    assert ref.n_hits > 0
    _compare(ctx, out, ref, n)


def test_with_stacked_mean_common_mode():
    det = synth.cspad_2p2m(n_modules=2, occupancy=0.01)
    ctx, out, ref = _run(det, 3, filters.example_bank(), cm_mode=pd.PD_CM_MEAN_STACKED)
    assert ref.n_hits > 0
    _compare(ctx, out, ref, 3)


def test_bank_change_and_reset_to_local_maximum():
    det = synth.asic_352x384(rows=48)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 3, truth=False)
    ctx, out, ref = _run(det, 3, BANKS["random1"], ped=ped, gain=gain, raw=raw)
    _compare(ctx, out, ref, 3)
    for bank in (filters.example_bank(), None):
        pd.pd_reset_summary(ctx)
        if bank is None:
            pd.pd_set_filter_bank(ctx)
        else:
            pd.pd_set_filter_bank(ctx, **bank)
        out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
        torch.cuda.synchronize()
        ref = oracle.process(oracle.geometry(**det.geometry()),
                             oracle.thresholds(**det.thresholds()), ped, gain, raw,
                             want_corrected=True,
                             filters=None if bank is None else oracle.filters(**bank))
        _compare(ctx, out, ref, 3)


@pytest.mark.parametrize("tuning", [dict(chunk_frames=1, overlap=1, two_pass=0),
                                    dict(chunk_frames=2, overlap=0, band_rows=5)])
def test_tuning_does_not_change_results(tuning):
    det = synth.cspad_2p2m(n_modules=3, occupancy=0.01)
    ctx, out, ref = _run(det, 5, filters.example_bank(), tuning=tuning)
    assert pd.pd_get_tuning(ctx)["two_pass"] == 1
    _compare(ctx, out, ref, 5)


def test_entries_and_batches():
    det = synth.cspad_2p2m(n_modules=2, occupancy=0.01)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 4, truth=False)
    bank = filters.example_bank()
    ref = oracle.process(oracle.geometry(**det.geometry()), oracle.thresholds(**det.thresholds()),
                         ped, gain, raw, filters=oracle.filters(**bank))
    exp = sort_hits(ref.hits).tobytes()
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    pd.pd_set_filter_bank(ctx, **bank)
    hits, n = pd.pd_process_host(ctx, raw)
    assert n == ref.n_hits and sort_hits(hits).tobytes() == exp
    dev = pd.frames_to_device(raw)
    out = pd.Outputs(ctx, 4, 4 * n + 64)
    pd.pd_process_noalloc(ctx, dev.data_ptr(), 4, 0, **out.ptrs())
    torch.cuda.synchronize()
    hits, n2 = out.hits_host()
    assert n2 == n and sort_hits(hits).tobytes() == exp
    batch = pd.pd_batch_create(4)
    outs = [pd.Outputs(ctx, 2, 4 * n + 64) for _ in range(2)]
    half = 2 * det.pixels_per_frame * 2
    pd.pd_batch_process(batch, [(ctx, dev.data_ptr(), 2, 0, outs[0]),
                                (ctx, dev.data_ptr() + half, 2, 2, outs[1])])
    torch.cuda.synchronize()
    got = np.concatenate([o.hits_host()[0] for o in outs])
    assert sort_hits(got).tobytes() == exp
    pd.pd_batch_set_mixed(batch, True)
    with pytest.raises(pd.PdError) as ei:
        pd.pd_batch_process(batch, [(ctx, dev.data_ptr(), 2, 0, outs[0])])
    assert ei.value.code == pd.PD_ENOTSUP


def test_invalid_banks_rejected():
    det = synth.asic_352x384(rows=16)
    ped, gain = synth.maps(det)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    bank = filters.example_bank()
    bad = dict(bank, f0=np.where(bank["f0"] > 0, np.nan, 0))
    for b in (bad, dict(bank, f1_nmin=[np.nan] * 6)):
        with pytest.raises(pd.PdError) as ei:
            pd.pd_set_filter_bank(ctx, **b)
        assert ei.value.code == pd.PD_EINVAL
    with pytest.raises(ValueError):
        pd.pd_set_filter_bank(ctx, **random_bank(0, 9))
