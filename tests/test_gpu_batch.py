"""Batched launches over mixed geometries, CUDA-graph replay, and the
autotuner, checked against single-context processing and the oracle.

The mix follows the batched workload: ePix100-like 704x768 modules at 6 keV,
CSPAD-like 185x388 sensors at 8 keV and 352x384 ASICs at 12 keV, interleaved,
with per-frame occupancy log-uniform in [0.1 %, 10 %] (sizes reduced so the
oracle runs in seconds).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX = [synth.epix_704x768(rows=96, occupancy=0.001, occupancy_hi=0.1, seed=21),
       synth.cspad_2p2m(n_modules=3, occupancy=0.001, occupancy_hi=0.1, seed=22),
       synth.asic16_352x384(n_modules=2, rows=64, occupancy=0.001, occupancy_hi=0.1,
                            seed=23)]
FRAMES = [5, 4, 6]


# the same with four CSPAD-like sensors: frames of a whole number of 16-byte
# groups, so the bank median's tensor copies and the work-queue launch apply
MIX_BANK = [MIX[0], synth.cspad_2p2m(n_modules=4, occupancy=0.001, occupancy_hi=0.1, seed=22),
            MIX[2]]


def _setup(mix=MIX):
    data = []
    for det, n in zip(mix, FRAMES):
        ped, gain = synth.maps(det)
        raw, _ = synth.frames(det, ped, gain, 0, n)
        data.append((det, ped, gain, raw))
    return data


def _ctxs(data):
    return [pd.pd_create(d.geometry(), ped, gain, d.thresholds()) for d, ped, gain, _ in data]


def _individual(data):
    res = []
    for (det, ped, gain, raw), ctx in zip(data, _ctxs(data)):
        out = pd.process(ctx, pd.frames_to_device(raw), cm=True)
        torch.cuda.synchronize()
        res.append((out.hits_host(), out.cm.cpu().numpy(), pd.pd_get_summary(ctx)))
    return res


def _outputs(ctxs, data):
    outs = []
    for ctx, (det, ped, gain, raw) in zip(ctxs, data):
        outs.append(pd.Outputs(ctx, len(raw), len(raw) * det.pixels_per_frame // 4, cm=True))
    return outs


def _check(ctxs, outs, ref):
    for ctx, out, ((rh, rn), rcm, rsum) in zip(ctxs, outs, ref):
        hits, n = out.hits_host()
        assert n == rn and len(hits) == n
        assert sort_hits(hits).tobytes() == sort_hits(rh).tobytes()
        assert out.cm.cpu().numpy().tobytes() == rcm.tobytes()
        for a, b in zip(pd.pd_get_summary(ctx), rsum):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_equals_single_context_processing_and_oracle(mixed):
    data = _setup()
    ref = _individual(data)
    # the single-context path itself against the oracle on the mix
    for (det, ped, gain, raw), ((rh, rn), rcm, rsum) in zip(data, ref):
        o = oracle.process(oracle.geometry(**det.geometry()),
                           oracle.thresholds(**det.thresholds()), ped, gain, raw)
        assert o.n_hits == rn
        assert sort_hits(o.hits).tobytes() == sort_hits(rh).tobytes()
    ctxs = _ctxs(data)
    devs = [pd.frames_to_device(raw) for *_, raw in data]
    outs = _outputs(ctxs, data)
    batch = pd.pd_batch_create(8)
    pd.pd_batch_set_mixed(batch, mixed)
    pd.pd_batch_process(batch, [(c, d.data_ptr(), len(r[3]), 0, o)
                                for c, d, r, o in zip(ctxs, devs, data, outs)])
    torch.cuda.synchronize()
    _check(ctxs, outs, ref)


@pytest.mark.parametrize("mixed,kernels", [(False, 0), (True, 0), (False, 3)],
                         ids=["per_item", "mixed", "per_item_work_queue"])
def test_batch_graph_replays_on_new_frame_contents(mixed, kernels):
    data = _setup(MIX_BANK if kernels == 3 else MIX)
    ctxs = _ctxs(data)
    if kernels:
        # the CSPAD-like context runs the work-queue launch inside the graph
        for c in ctxs:
            pd.pd_set_tuning(c, kernels=kernels)
        assert pd.pd_get_tuning(ctxs[1])["kernels"] == kernels
    devs = [pd.frames_to_device(raw) for *_, raw in data]
    outs = _outputs(ctxs, data)
    batch = pd.pd_batch_create(8)
    pd.pd_batch_set_mixed(batch, mixed)
    stream = torch.cuda.Stream()
    items = [(c, d.data_ptr(), len(r[3]), 0, o) for c, d, r, o in zip(ctxs, devs, data, outs)]
    with torch.cuda.stream(stream):
        pd.pd_batch_capture(batch, items, stream)
    stream.synchronize()
    for k in range(2):
        # new frames written into the same device buffers, then one replay
        new = []
        for (det, ped, gain, raw), dev in zip(data, devs):
            fresh, _ = synth.frames(det, ped, gain, 100 * (k + 1), len(raw))
            dev.copy_(torch.from_numpy(fresh.view(np.int16).reshape(dev.shape)))
            new.append((det, ped, gain, fresh))
        torch.cuda.synchronize()
        for ctx in ctxs:
            pd.pd_reset_summary(ctx)
        torch.cuda.synchronize()
        pd.pd_batch_replay(batch, stream)
        stream.synchronize()
        _check(ctxs, outs, _individual(new))


def test_autotune_keeps_results_and_summaries():
    det = synth.cspad_2p2m(n_modules=4)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 12)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    dev = pd.frames_to_device(raw)
    a = pd.process(ctx, dev)
    torch.cuda.synchronize()
    before = pd.pd_get_summary(ctx)
    tuning, us = pd.pd_autotune(ctx, dev.data_ptr(), 12)
    assert us > 0 and tuning["chunk_frames"] >= 1
    assert pd.pd_get_tuning(ctx) == tuning
    for x, y in zip(pd.pd_get_summary(ctx), before):
        np.testing.assert_array_equal(x, y)
    b = pd.process(ctx, dev)
    torch.cuda.synchronize()
    ha, na = a.hits_host()
    hb, nb = b.hits_host()
    assert na == nb and sort_hits(ha).tobytes() == sort_hits(hb).tobytes()
