"""The paper's mean common mode (Fig. c) and its three stacked stages on the
GPU against the CPU oracle, bit for bit: hits, every common-mode term,
corrected frames and summaries, on row units, banks, units too tall for a
warp, ragged geometries, separable offsets, empty background sets and
values far off the sum's grid; through pd_process, the host entry, the
no-allocation entry, batches, the 5x5 patch gather and any tuning."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = {"mean": pd.PD_CM_MEAN, "stacked": pd.PD_CM_MEAN_STACKED}

WORKLOADS = {
    "asic_rows_x16": (synth.asic_352x384(), 16),
    "cspad_banks_x4": (synth.cspad_2p2m(n_modules=2), 4),
    "epix_rows_x2": (synth.epix_704x768(occupancy=0.02), 2),
    "ragged_37x48_banks": (synth.Detector(n_modules=3, rows=37, cols=48, unit_rows=37,
                                          unit_cols=16, occupancy=0.03), 5),
    "ragged_rows_19x104": (synth.Detector(n_modules=1, rows=19, cols=104, unit_rows=1,
                                          unit_cols=52, occupancy=0.05), 7),
    "short_units_5x33": (synth.Detector(n_modules=2, rows=20, cols=99, unit_rows=5,
                                        unit_cols=33, occupancy=0.02), 3),
    "big_unit_256x256": (synth.Detector(n_modules=1, rows=256, cols=256, unit_rows=256,
                                        unit_cols=256, occupancy=0.01), 2),
}


def _run(det, n, mode, ped=None, gain=None, raw=None, thr_over=None, tuning=None):
    if ped is None:
        ped, gain = synth.maps(det)
    if raw is None:
        raw, _ = synth.frames(det, ped, gain, 0, n, truth=False)
    geom = dict(det.geometry(), cm_mode=mode)
    thr = dict(det.thresholds(), **(thr_over or {}))
    ctx = pd.pd_create(geom, ped, gain, thr)
    if tuning:
        pd.pd_set_tuning(ctx, **tuning)
    out = pd.process(ctx, pd.frames_to_device(raw), corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         want_corrected=True)
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
    assert ctx.cm_values_per_frame == oracle.cm_values_per_frame(
        oracle.geometry(**dict(det.geometry(), cm_mode=MODES[mode])))
    assert ref.n_hits > 0
    _compare(ctx, out, ref, n)


@pytest.mark.parametrize("mode", list(MODES))
def test_separable_offsets_noise_free(mode):
    R, C, ur, uc = 16, 72, 16, 24
    rng = np.random.default_rng(3)
    b = rng.integers(-6, 7, R)
    b[-1] -= b.sum()
    c = np.zeros(C, np.int64)
    for j in range(C // uc):
        cc = rng.integers(-6, 7, uc)
        cc[-1] -= cc.sum()
        c[j * uc:(j + 1) * uc] = cc
    a = rng.integers(-20, 21, (R // ur, C // uc))
    off = np.repeat(np.repeat(a, ur, 0), uc, 1) + b[:, None] + c[None, :]
    det = synth.Detector(n_modules=1, rows=R, cols=C, unit_rows=ur, unit_cols=uc)
    ped = np.full((1, R, C), 1000.0, np.float32)
    gain = np.ones((1, R, C), np.float32)
    raw = np.stack([(1000 + off + k).astype(np.uint16)[None] for k in range(3)])
    ctx, out, ref = _run(det, 3, MODES[mode], ped, gain, raw)
    _compare(ctx, out, ref, 3)
    if mode == "stacked":
        assert not out.corrected.cpu().numpy().any()


def test_background_sets_empty_partial_and_off_grid():
    # a 6 x 40 module of row units: row 0 all above the cut (N0 = 0), row 1
    # with one background pixel (the sqrt(40) guard), row 2 mixing values
    # of very different magnitude: d = 3 - 2^-12 and 3, one d = -2000 that
    # sets the sum's grid to 2^-28, one d = -3 * 2^-32 below that grid
    # (it rounds to 0) and one photon above the cut; rows 3-5 ordinary
    det = synth.Detector(n_modules=1, rows=6, cols=40, unit_rows=1, unit_cols=40)
    ped = np.full((1, 6, 40), 2000.0, np.float32)
    ped[0, 2, :20] = np.float32(2000.000244140625)
    ped[0, 2, 20] = np.float32(1.5)
    ped[0, 2, 22] = np.float32(3 * 2.0 ** -32)
    gain = np.ones((1, 6, 40), np.float32)
    raw = np.full((2, 1, 6, 40), 2003, np.uint16)
    raw[:, 0, 0, :] = 2500
    raw[:, 0, 1, 1:] = 2500
    raw[:, 0, 2, 20] = 60000
    raw[:, 0, 2, 21:23] = 0
    raw[1, 0, 4, ::3] = 1990
    for mode in MODES.values():
        ctx, out, ref = _run(det, 2, mode, ped, gain, raw, thr_over=dict(cm_cut_adu=300.0))
        _compare(ctx, out, ref, 2)
        assert ref.cm[0, 0] == 0.0


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("tuning", [dict(chunk_frames=1, overlap=1),
                                    dict(chunk_frames=3, overlap=0, band_rows=5)])
def test_results_independent_of_tuning(mode, tuning):
    det = synth.cspad_2p2m(n_modules=3, occupancy=0.01)
    ctx, out, ref = _run(det, 7, MODES[mode], tuning=tuning)
    _compare(ctx, out, ref, 7)


def test_host_noalloc_and_batch_entries_stacked():
    det = synth.cspad_2p2m(n_modules=2)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 6, truth=False)
    geom = dict(det.geometry(), cm_mode=pd.PD_CM_MEAN_STACKED)
    thr = det.thresholds()
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw)
    exp = sort_hits(ref.hits).tobytes()
    ctx = pd.pd_create(geom, ped, gain, thr)
    hits, n = pd.pd_process_host(ctx, raw)
    assert n == ref.n_hits and sort_hits(hits).tobytes() == exp
    dev = pd.frames_to_device(raw)
    out = pd.Outputs(ctx, 6, 4 * ref.n_hits + 64)
    pd.pd_process_noalloc(ctx, dev.data_ptr(), 6, 0, **out.ptrs())
    torch.cuda.synchronize()
    hits, n = out.hits_host()
    assert n == ref.n_hits and sort_hits(hits).tobytes() == exp
    batch = pd.pd_batch_create(4)
    outs = [pd.Outputs(ctx, 3, 4 * ref.n_hits + 64, cm=True) for _ in range(2)]
    half = 3 * det.pixels_per_frame * 2
    pd.pd_batch_process(batch, [(ctx, dev.data_ptr(), 3, 0, outs[0]),
                                (ctx, dev.data_ptr() + half, 3, 3, outs[1])])
    torch.cuda.synchronize()
    got = np.concatenate([o.hits_host()[0] for o in outs])
    assert sort_hits(got).tobytes() == exp
    cm = np.concatenate([o.cm.cpu().numpy() for o in outs])
    assert cm.tobytes() == ref.cm.tobytes()
    pd.pd_batch_set_mixed(batch, True)
    with pytest.raises(pd.PdError) as ei:
        pd.pd_batch_process(batch, [(ctx, dev.data_ptr(), 3, 0, outs[0])])
    assert ei.value.code == pd.PD_ENOTSUP


def test_patch_gather_applies_every_stage():
    det = synth.cspad_2p2m(n_modules=2, occupancy=0.01)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 2, truth=False)
    geom = dict(det.geometry(), cm_mode=pd.PD_CM_MEAN_STACKED)
    thr = det.thresholds()
    ctx = pd.pd_create(geom, ped, gain, thr)
    dev = pd.frames_to_device(raw)
    out = pd.process(ctx, dev, cm=True)
    torch.cuda.synchronize()
    hits, n = out.hits_host()
    patches = torch.empty((n, 25), dtype=torch.float32, device="cuda")
    pd.pd_net_gather(ctx, dev.data_ptr(), 0, out.cm.data_ptr(), out.hits.data_ptr(), n,
                     patches.data_ptr())
    torch.cuda.synchronize()
    got = patches.cpu().numpy()
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         want_corrected=True)
    e = ref.corrected.reshape(2, det.n_modules, det.rows, det.cols)
    dev_hits = out.hits[:n].cpu().numpy().view(pd.HIT_DTYPE).reshape(-1)
    for i in range(0, n, max(1, n // 200)):
        h = dev_hits[i]
        m, w = divmod(int(h["pixel"]), det.rows * det.cols)
        r0, c0 = divmod(w, det.cols)
        exp = np.zeros(25, np.float32)
        for k in range(25):
            r, c = r0 + k // 5 - 2, c0 + k % 5 - 2
            if 0 <= r < det.rows and 0 <= c < det.cols:
                exp[k] = e[h["frame"], m, r, c] / np.float32(thr["photon_kev"])
        assert got[i].tobytes() == exp.tobytes()


def test_oversized_units_rejected():
    det = synth.Detector(n_modules=1, rows=4096, cols=4096, unit_rows=4096, unit_cols=4096)
    ped = np.zeros((1, 4096, 4096), np.float32)
    with pytest.raises(pd.PdError) as ei:
        pd.pd_create(dict(det.geometry(), cm_mode=pd.PD_CM_MEAN), ped, ped + 1,
                     det.thresholds())
    assert ei.value.code == pd.PD_EINVAL
