"""The paper's processing order (gain before common mode, cm_after_gain = 1)
on the GPU against the CPU oracle, bit for bit: hits, common mode,
corrected frames and summaries with the median, the paper's mean and the
stacked stages, masked pixels, the matched filters and the entry points."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import filters, pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = {"median": pd.PD_CM_MEDIAN, "mean": pd.PD_CM_MEAN, "stacked": pd.PD_CM_MEAN_STACKED,
         "none": pd.PD_CM_NONE}
WORKLOADS = {
    "asic_rows_x8": (synth.asic_352x384(), 8),
    "cspad_banks_x3": (synth.cspad_2p2m(n_modules=2), 3),
    "ragged_37x45": (synth.Detector(n_modules=3, rows=37, cols=45, unit_rows=37, unit_cols=15,
                                    occupancy=0.03), 4),
}


def _run(det, n, mode, bank=None, mask=True):
    ped, gain = synth.maps(det)
    if mask:
        gain.reshape(-1)[::53] = 0.0
        gain.reshape(-1)[7] = -2.0
    raw, _ = synth.frames(det, ped, gain, 0, n, truth=False)
    geom = dict(det.geometry(), cm_mode=mode, cm_after_gain=1)
    thr = det.thresholds()
    ctx = pd.pd_create(geom, ped, gain, thr)
    if bank is not None:
        pd.pd_set_filter_bank(ctx, **bank)
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


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_workloads_bit_exact(name, mode):
    det, n = WORKLOADS[name]
    ctx, out, ref = _run(det, n, MODES[mode])
    assert ref.n_hits > 0
    _compare(ctx, out, ref, n)


def test_matched_filters_in_the_paper_order():
    det = synth.cspad_2p2m(n_modules=2, occupancy=0.01)
    ctx, out, ref = _run(det, 2, pd.PD_CM_MEAN_STACKED, bank=filters.example_bank())
    assert ref.n_hits > 0
    _compare(ctx, out, ref, 2)


def test_entries_and_rejections():
    det = synth.asic_352x384(rows=64)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 3, truth=False)
    geom = dict(det.geometry(), cm_after_gain=1)
    thr = det.thresholds()
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw)
    ctx = pd.pd_create(geom, ped, gain, thr)
    hits, n = pd.pd_process_host(ctx, raw)
    assert n == ref.n_hits and sort_hits(hits).tobytes() == sort_hits(ref.hits).tobytes()
    dev = pd.frames_to_device(raw)
    out = pd.Outputs(ctx, 3, 4 * n + 64)
    pd.pd_process_noalloc(ctx, dev.data_ptr(), 3, 0, **out.ptrs())
    torch.cuda.synchronize()
    h2, n2 = out.hits_host()
    assert n2 == n and sort_hits(h2).tobytes() == sort_hits(ref.hits).tobytes()
    for bad in (dict(geom, cm_after_gain=2),):
        with pytest.raises(pd.PdError):
            pd.pd_create(bad, ped, gain, thr)
    with pytest.raises(pd.PdError):
        pd.pd_create(geom, ped, gain, dict(thr, cm_cut_kev=float("nan")))
    mped, mgain = synth.multigain_maps(det, 2)
    with pytest.raises(pd.PdError):
        pd.pd_create(geom, mped, mgain, thr, n_gains=2, gain_shift=14)
