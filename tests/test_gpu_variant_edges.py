"""Edge cases of the variant modes on the GPU (paper mean, stacked stages,
matched filters, auto-ranging words, the paper's order): empty calls, hit
capacity overflow with the true count kept, frame offsets and summaries
accumulated over several calls, each against the CPU oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import filters, pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = {
    "mean": dict(geom=dict(cm_mode=pd.PD_CM_MEAN)),
    "stacked": dict(geom=dict(cm_mode=pd.PD_CM_MEAN_STACKED)),
    "matched": dict(bank=True),
    "after_gain_stacked": dict(geom=dict(cm_mode=pd.PD_CM_MEAN_STACKED, cm_after_gain=1)),
    "multigain": dict(gains=3),
}


def _setup(name, det, n, first=0):
    v = VARIANTS[name]
    geom = dict(det.geometry(), **v.get("geom", {}))
    thr = det.thresholds()
    if v.get("gains"):
        ped, gain = synth.multigain_maps(det, v["gains"])
        raw, _ = synth.multigain_frames(det, ped, gain, first, n)
        ctx = pd.pd_create(geom, ped, gain, thr, n_gains=v["gains"], gain_shift=14)
        okw = dict(n_gains=v["gains"], gain_shift=14)
    else:
        ped, gain = synth.maps(det)
        raw, _ = synth.frames(det, ped, gain, first, n, truth=False)
        ctx = pd.pd_create(geom, ped, gain, thr)
        okw = {}
    bank = filters.example_bank() if v.get("bank") else None
    if bank is not None:
        pd.pd_set_filter_bank(ctx, **bank)
        okw["filters"] = oracle.filters(**bank)
    return ctx, geom, thr, ped, gain, raw, okw


@pytest.mark.parametrize("name", list(VARIANTS))
def test_empty_call_and_overflow(name):
    det = synth.cspad_2p2m(n_modules=2, occupancy=0.01)
    ctx, geom, thr, ped, gain, raw, okw = _setup(name, det, 2)
    out = pd.Outputs(ctx, 0, 8)
    dummy = torch.zeros(8, dtype=torch.int16, device="cuda")
    pd.pd_process(ctx, dummy.data_ptr(), 0, 0, **out.ptrs())
    torch.cuda.synchronize()
    assert out.hits_host()[1] == 0
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         **okw)
    cap = max(1, ref.n_hits // 3)
    out = pd.process(ctx, pd.frames_to_device(raw), hit_capacity=cap)
    torch.cuda.synchronize()
    hits, n = out.hits_host()
    assert n == ref.n_hits and len(hits) == cap
    # the records kept are a subset of the oracle's
    exp = {h.tobytes() for h in ref.hits}
    assert all(h.tobytes() in exp for h in hits)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_frame_base_and_accumulation_over_calls(name):
    det = synth.asic_352x384(rows=96, occupancy=0.02)
    ctx, geom, thr, ped, gain, raw, okw = _setup(name, det, 5)
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         frame_base=100, **okw)
    got = []
    for a, b in ((0, 2), (2, 5)):
        out = pd.process(ctx, pd.frames_to_device(raw[a:b]), frame_base=100 + a)
        torch.cuda.synchronize()
        hits, n = out.hits_host()
        assert len(hits) == n
        got.append(hits)
    got = np.concatenate(got)
    assert sort_hits(got).tobytes() == sort_hits(ref.hits).tobytes()
    for g_, e_ in zip(pd.pd_get_summary(ctx), (ref.count_map, ref.hist_pix, ref.hist_hit)):
        np.testing.assert_array_equal(g_, e_)
