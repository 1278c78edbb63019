"""The streaming server: frames of two geometries (ePix100-sized 704x768 and
the 2.2 Mpx CSPAD) committed to page-locked rings, continuously batched onto
the GPU.  Each frame's hit list in the mix must equal, bit for bit, the hit
list of pd_process on that frame alone, whatever batch it landed in; the
running count map and histograms must equal those of processing every frame
once.  Also: back-pressure on a full ring, admission by the device budget,
and the Poisson replay producer."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# occupancy log-uniform in [0.1 %, 2 %] per frame, as in the serving mix
DETS = [synth.epix_704x768(occupancy=0.001, occupancy_hi=0.02, seed=31),
        synth.cspad_2p2m(occupancy=0.001, occupancy_hi=0.02, seed=32)]
N = [40, 10]


@pytest.fixture(scope="module")
def data():
    out = []
    for det, n in zip(DETS, N):
        ped, gain = synth.maps(det)
        raw, _ = synth.frames(det, ped, gain, 0, n, truth=False)
        out.append((det, ped, gain, raw.reshape(n, -1)))
    return out


def _ctx(d):
    det, ped, gain, _ = d
    return pd.pd_create(det.geometry(), ped, gain, det.thresholds())


@pytest.fixture(scope="module")
def alone(data):
    """Per geometry: hits of each frame processed on its own, and the
    summaries of processing every frame once."""
    res = []
    for d in data:
        ctx = _ctx(d)
        per = []
        for k in range(len(d[3])):
            out = pd.process(ctx, pd.frames_to_device(d[3][k:k + 1]))
            hits, n = out.hits_host()
            assert len(hits) == n
            per.append(sort_hits(hits))
        torch.cuda.synchronize()
        res.append((per, pd.pd_get_summary(ctx)))
    return res


def _with_id(hits, fid):
    h = hits.copy()
    h["frame"] = fid
    return h


def _push(sv, g, frame, fid, timeout=30.0):
    t_end = time.monotonic() + timeout
    while True:
        got = sv.acquire(g)
        if got is not None:
            break
        assert time.monotonic() < t_end, "ring never freed"
        time.sleep(1e-4)
    slot, view = got
    view[:] = frame
    sv.commit(g, slot, fid)


def test_alone_matches_oracle(data, alone):
    for d, (per, _) in zip(data, alone):
        det, ped, gain, raw = d
        for k in (0, len(raw) - 1):
            o = oracle.process(oracle.geometry(**det.geometry()),
                               oracle.thresholds(**det.thresholds()), ped, gain,
                               raw[k:k + 1].reshape((1,) + det.frame_shape))
            assert sort_hits(o.hits).tobytes() == per[k].tobytes()


def test_mix_equals_alone(data, alone):
    ctxs = [_ctx(d) for d in data]
    sv = pd.Server(ctxs, n_slots=3, max_batch_frames=8, ring_frames=16,
                   hits_per_frame=1 << 15, keep_hits=True)
    assert sv.slots() == 3
    ids = {}
    fid = 1000
    # a held burst: the first batch is guaranteed to mix both geometries
    sv.hold(True)
    order = [(0, k) for k in range(6)] + [(1, k) for k in range(2)]
    for g, k in order:
        _push(sv, g, data[g][3][k], fid)
        ids[fid] = (g, k)
        fid += 1
    sv.hold(False)
    # the rest interleaved as fast as the rings accept them
    rest = [(0, k) for k in range(6, N[0])] + [(1, k) for k in range(2, N[1])]
    rng = np.random.default_rng(5)
    rng.shuffle(rest)
    for g, k in rest:
        _push(sv, g, data[g][3][k], fid)
        ids[fid] = (g, k)
        fid += 1
    sv.drain(120.0)
    st = sv.stats()
    assert st["frames_done"] == st["frames_committed"] == sum(N)
    assert st["max_batch_frames"] >= 8
    assert st["batches"] >= 2
    total = 0
    for f, (g, k) in ids.items():
        hits, lat = sv.frame_hits(f)
        assert lat > 0
        assert sort_hits(hits).tobytes() == _with_id(alone[g][0][k], f).tobytes(), (f, g, k)
        total += len(hits)
        if f % 7 == 0:   # the compact stream decodes to the same photon list
            back = pd.pd_decompress_hits(sv.frame_stream(f), frame=f)
            sh = sort_hits(hits)
            assert np.array_equal(back["pixel"], sh["pixel"])
            assert np.array_equal(back["count"], sh["count"])
            assert np.max(np.abs(back["energy_kev"] - sh["energy_kev"]), initial=0) <= 1 / 512
    assert st["hits"] == total
    assert st["raw_bytes"] == sum(n * d.pixels_per_frame * 2 for d, n in zip(DETS, N))
    assert st["compressed_bytes"] < st["raw_bytes"]
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    # the running summaries are those of processing every frame once
    torch.cuda.synchronize()
    for ctx, (_, rsum) in zip(ctxs, alone):
        for a, b in zip(pd.pd_get_summary(ctx), rsum):
            np.testing.assert_array_equal(a, b)
    sv.close()


def test_backpressure_on_a_full_ring(data):
    ctxs = [_ctx(d) for d in data]
    sv = pd.Server(ctxs, n_slots=1, max_batch_frames=4, ring_frames=4,
                   hits_per_frame=1 << 15, keep_hits=True)
    sv.hold(True)
    slots = [sv.acquire(0) for _ in range(4)]
    assert all(s is not None for s in slots)
    assert sv.acquire(0) is None                 # full: PD_EBUSY
    assert sv.stats()["frames_rejected"] == 1
    # a slot that was not handed out cannot be committed
    with pytest.raises(pd.PdError) as e:
        sv.commit(1, 0, 99)
    assert e.value.code == pd.PD_EINVAL
    for i, (slot, view) in enumerate(slots):
        view[:] = data[0][3][i]
        sv.commit(0, slot, i)
    sv.hold(False)
    sv.drain(60.0)
    assert sv.stats()["frames_done"] == 4
    assert sv.acquire(0) is not None             # freed again
    sv.close()


def test_admission_by_device_budget(data):
    ctxs = [_ctx(d) for d in data]
    with pytest.raises(pd.PdError) as e:
        pd.Server(ctxs, n_slots=4, max_batch_frames=8, ring_frames=8, hits_per_frame=4096,
                  device_budget=1 << 20)
    assert e.value.code == pd.PD_EBUSY
    # one slot's worth: frames + hits + common-mode values per geometry
    per_slot = sum(8 * (c.pixels_per_frame * 2 + 4096 * pd.HIT_DTYPE.itemsize +
                        c.units_per_frame * 4) for c in ctxs)
    sv = pd.Server(ctxs, n_slots=4, max_batch_frames=8, ring_frames=8, hits_per_frame=4096,
                   device_budget=per_slot)
    assert sv.slots() == 1
    sv.close()
    sv = pd.Server(ctxs, n_slots=4, max_batch_frames=8, ring_frames=8, hits_per_frame=4096,
                   device_budget=3 * per_slot + 1)
    assert sv.slots() == 3
    sv.close()


def test_poisson_replay(data, alone):
    """The built-in producer: ePix frames at 20 kHz for 0.25 s from a
    pre-filled ring; the k-th accepted frame uses ring slot k mod ring_frames."""
    ctxs = [_ctx(d) for d in data]
    cap = 32
    sv = pd.Server(ctxs, n_slots=4, max_batch_frames=16, ring_frames=cap,
                   hits_per_frame=1 << 14, keep_hits=True)
    for s in range(cap):
        sv.ring_frame(0, s)[:] = data[0][3][s % N[0]]
    sv.replay(20000.0, 0.25, mix=[1.0, 0.0], seed=3, first_id=0)
    sv.drain(60.0)
    st = sv.stats()
    assert st["frames_done"] == st["frames_committed"]
    assert st["frames_committed"] + st["frames_rejected"] > 3000
    assert st["frames_done"] > 0
    for f in range(0, st["frames_done"], 97):
        hits, _ = sv.frame_hits(f)
        k = (f % cap) % N[0]
        assert sort_hits(hits).tobytes() == _with_id(alone[0][0][k], f).tobytes()
    assert st["compressed_bytes"] * 10 < st["raw_bytes"]
    sv.close()
