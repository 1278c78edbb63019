"""The lean pair as one work-queue launch (pd_tuning.kernels = 3) against the
oracle, bit for bit.

The queue interleaves the bank medians of K frames with the stencil tiles
of the K frames before them (K = 4 for the 2.2 Mpx sensor), so the cases
cover one partial superstep, several supersteps with a ragged last one,
results equal to the kernel pair's, accumulation over calls, and the
full 1024-frame batch on sampled frames.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle(geom, thr, ped, gain, raw, **kw):
    return oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                          **kw)


def _queue_ctx(det, ped, gain):
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    pd.pd_set_tuning(ctx, kernels=3)
    assert pd.pd_get_tuning(ctx)["kernels"] == 3, "the work-queue launch does not apply"
    return ctx


def _compare(ctx, out, ref, n):
    hits, nh = out.hits_host()
    assert nh == ref.n_hits == len(hits) == len(ref.hits)
    assert sort_hits(hits).tobytes() == sort_hits(ref.hits).tobytes()
    assert out.cm.cpu().numpy().tobytes() == ref.cm.reshape(n, -1).tobytes()
    cmap, hp, hh = pd.pd_get_summary(ctx)
    np.testing.assert_array_equal(cmap, ref.count_map)
    np.testing.assert_array_equal(hp, ref.hist_pix)
    np.testing.assert_array_equal(hh, ref.hist_hit)


@pytest.mark.parametrize("n", [1, 3, 11], ids=["one_frame", "partial_superstep",
                                               "four_supersteps_ragged"])
def test_queue_launch_bit_exact(n):
    det = synth.cspad_2p2m(occupancy=0.01)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, n)
    ctx = _queue_ctx(det, ped, gain)
    out = pd.process(ctx, pd.frames_to_device(raw), cm=True, hit_capacity=n * 65536)
    torch.cuda.synchronize()
    ref = _oracle(det.geometry(), det.thresholds(), ped, gain, raw)
    assert ref.n_hits > 0
    _compare(ctx, out, ref, n)


def test_queue_equals_kernel_pair_and_accumulates():
    """Two calls with frame offsets through the queue give the pair's hits,
    common mode and summed summaries."""
    det = synth.cspad_2p2m(n_modules=32, occupancy=0.02)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 9)
    dev = pd.frames_to_device(raw)
    res = {}
    for k in (1, 3):
        ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
        pd.pd_set_tuning(ctx, kernels=k)
        parts = []
        for lo, hi in ((0, 5), (5, 9)):
            out = pd.process(ctx, dev[lo:hi], frame_base=lo, cm=True, hit_capacity=(hi - lo) * 65536)
            torch.cuda.synchronize()
            h, nh = out.hits_host()
            assert nh == len(h)
            parts.append((h, out.cm.cpu().numpy()))
        res[k] = (sort_hits(np.concatenate([p[0] for p in parts])),
                  np.concatenate([p[1] for p in parts]), pd.pd_get_summary(ctx))
    assert res[1][0].tobytes() == res[3][0].tobytes()
    assert res[1][1].tobytes() == res[3][1].tobytes()
    for a, b in zip(res[1][2], res[3][2]):
        np.testing.assert_array_equal(a, b)


def test_queue_full_batch_sampled():
    """The benchmark's 1024 frames in one queue launch: sampled frames equal
    the oracle, and the summaries obey size-independent identities."""
    det = synth.cspad_2p2m()
    ped, gain = synth.maps(det)
    n = 1024
    raw, _ = synth.frames(det, ped, gain, 0, n, truth=False)
    ctx = _queue_ctx(det, ped, gain)
    out = pd.process(ctx, pd.frames_to_device(raw), hit_capacity=n * 16384, cm=True)
    torch.cuda.synchronize()
    hits, nh = out.hits_host()
    assert nh == len(hits) > 0
    cm_all = out.cm.cpu().numpy()
    cmap, hp, hh = pd.pd_get_summary(ctx)
    assert hp.sum() == n * det.pixels_per_frame
    assert hh.sum() >= nh
    assert int(cmap.astype(np.int64).sum()) == int(hits["count"].astype(np.int64).sum())
    geom, thr = det.geometry(), det.thresholds()
    for f in (0, 3, 4, 517, n - 1):
        ref = _oracle(geom, thr, ped, gain, raw[f:f + 1])
        mine = hits[hits["frame"] == f].copy()
        mine["frame"] = 0
        assert sort_hits(mine).tobytes() == sort_hits(ref.hits).tobytes()
        assert cm_all[f].tobytes() == ref.cm.reshape(-1).tobytes()


def test_queue_not_used_for_corrected_frames():
    """Corrected frames fall back to the kernel pair (same results)."""
    det = synth.cspad_2p2m(n_modules=2)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 3)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    pd.pd_set_tuning(ctx, kernels=3)
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = _oracle(det.geometry(), det.thresholds(), ped, gain, raw, want_corrected=True)
    _compare(ctx, out, ref, 3)
    assert out.corrected.cpu().numpy().tobytes() == ref.corrected.reshape(3, -1).tobytes()
