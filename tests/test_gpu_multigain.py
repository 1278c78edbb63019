"""Auto-ranging multi-gain contexts (pd_create_multigain) on the GPU against
the CPU oracle, bit for bit: hits, corrected frames, common mode and
summaries, with 2 to 4 gain stages, corrupt stage bits, bright spots that
switch stages, the median and no common mode, the matched filters, units
too large for shared memory, the entry points, batches and the patch
gather."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import filters, pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKLOADS = {
    "asic_rows_3g_x4": (synth.asic_352x384(rows=128), 4, 3, 14),
    "cspad_banks_3g_x2": (synth.cspad_2p2m(n_modules=3), 2, 3, 14),
    "asic16_2g_x1": (synth.asic16_352x384(n_modules=4), 1, 2, 15),
    "ragged_37x45_4g": (synth.Detector(n_modules=2, rows=37, cols=45, unit_rows=37,
                                       unit_cols=15, occupancy=0.03), 3, 4, 13),
    "big_unit_256x256_3g": (synth.Detector(n_modules=1, rows=256, cols=256, unit_rows=256,
                                           unit_cols=256, occupancy=0.01), 2, 3, 14),
    # banks of odd width (one pixel per load in the bank median), and units
    # two columns wide (a four-pixel chunk of the band stencil meets two)
    "odd_banks_64x198_3g": (synth.Detector(n_modules=2, rows=64, cols=198, unit_rows=64,
                                           unit_cols=99, occupancy=0.02), 2, 3, 14),
    "two_column_units_2g": (synth.Detector(n_modules=1, rows=24, cols=64, unit_rows=24,
                                           unit_cols=2, occupancy=0.03), 3, 2, 15),
}


def _data(det, n, n_gains, shift):
    ratios = (1.0, 1 / 3, 1 / 20, 1 / 100)[:n_gains]
    offs = (0.0, -300.0, -600.0, -800.0)[:n_gains]
    ped, gain = synth.multigain_maps(det, n_gains, ratios, offs)
    raw, _ = synth.multigain_frames(det, ped, gain, 0, n, gain_shift=shift,
                                    blob_kev=4000.0, bad_frac=2e-4)
    return ped, gain, raw


def _run(det, n, n_gains, shift, ped, gain, raw, mode=0, bank=None):
    geom = dict(det.geometry(), cm_mode=mode)
    thr = det.thresholds()
    ctx = pd.pd_create(geom, ped, gain, thr, n_gains=n_gains, gain_shift=shift)
    if bank is not None:
        pd.pd_set_filter_bank(ctx, **bank)
    cap = n * det.pixels_per_frame
    out = pd.process(ctx, pd.frames_to_device(raw), hit_capacity=cap, corrected=True, cm=True)
    torch.cuda.synchronize()
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         want_corrected=True, hit_capacity=cap, n_gains=n_gains,
                         gain_shift=shift,
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


@pytest.mark.parametrize("mode", ["median", "none"])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_workloads_bit_exact(name, mode):
    det, n, n_gains, shift = WORKLOADS[name]
    ped, gain, raw = _data(det, n, n_gains, shift)
    stage = raw >> shift
    assert (stage == 1).any() and (stage == n_gains - 1).any()
    m = pd.PD_CM_MEDIAN if mode == "median" else pd.PD_CM_NONE
    ctx, out, ref = _run(det, n, n_gains, shift, ped, gain, raw, mode=m)
    assert ref.n_hits > 0
    _compare(ctx, out, ref, n)


def test_bank_median_below_window_uses_whole_unit_select():
    # stage-0 d about -400 ADU, below the bank median's window [cut - 512,
    # cut) = [-312, 200): the whole-unit selection, which must skip the words
    # of the other stages too
    det = synth.cspad_2p2m(n_modules=2)
    ped, gain, raw = _data(det, 2, 3, 14)
    ped_ctx = ped.copy()
    ped_ctx[0] += np.float32(400.0)
    ctx, out, ref = _run(det, 2, 3, 14, ped_ctx, gain, raw)
    assert float(ref.cm.max()) < -312.0
    _compare(ctx, out, ref, 2)


def test_with_matched_filters():
    det, n, n_gains, shift = WORKLOADS["cspad_banks_3g_x2"]
    ped, gain, raw = _data(det, n, n_gains, shift)
    ctx, out, ref = _run(det, n, n_gains, shift, ped, gain, raw, bank=filters.example_bank())
    assert ref.n_hits > 0
    _compare(ctx, out, ref, n)


def test_one_stage_equals_the_single_gain_context():
    det = synth.cspad_2p2m(n_modules=2)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 3, truth=False)
    single = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    multi = pd.pd_create(det.geometry(), ped[None], gain[None], det.thresholds(), n_gains=1,
                         gain_shift=15)
    dev = pd.frames_to_device(raw)
    a = pd.process(single, dev, corrected=True, cm=True)
    b = pd.process(multi, dev, corrected=True, cm=True)
    torch.cuda.synchronize()
    ha, na = a.hits_host()
    hb, nb = b.hits_host()
    assert na == nb and sort_hits(ha).tobytes() == sort_hits(hb).tobytes()
    assert a.corrected.cpu().numpy().tobytes() == b.corrected.cpu().numpy().tobytes()
    assert a.cm.cpu().numpy().tobytes() == b.cm.cpu().numpy().tobytes()


def test_entries_batches_and_gather():
    det, n, n_gains, shift = WORKLOADS["asic_rows_3g_x4"]
    ped, gain, raw = _data(det, n, n_gains, shift)
    geom, thr = det.geometry(), det.thresholds()
    ref = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         want_corrected=True, n_gains=n_gains, gain_shift=shift)
    exp = sort_hits(ref.hits).tobytes()
    ctx = pd.pd_create(geom, ped, gain, thr, n_gains=n_gains, gain_shift=shift)
    hits, nh = pd.pd_process_host(ctx, raw)
    assert nh == ref.n_hits and sort_hits(hits).tobytes() == exp
    dev = pd.frames_to_device(raw)
    out = pd.Outputs(ctx, n, 4 * nh + 64, cm=True)
    pd.pd_process_noalloc(ctx, dev.data_ptr(), n, 0, **out.ptrs())
    torch.cuda.synchronize()
    hits, nh2 = out.hits_host()
    assert nh2 == nh and sort_hits(hits).tobytes() == exp
    batch = pd.pd_batch_create(4)
    outs = [pd.Outputs(ctx, 2, 4 * nh + 64) for _ in range(2)]
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
    # 5x5 patches of e / photon_kev around the hits, from the stage maps
    patches = torch.empty((nh, 25), dtype=torch.float32, device="cuda")
    pd.pd_net_gather(ctx, dev.data_ptr(), 0, out.cm.data_ptr(), out.hits.data_ptr(), nh,
                     patches.data_ptr())
    torch.cuda.synchronize()
    got = patches.cpu().numpy()
    e = ref.corrected.reshape(n, det.rows, det.cols)
    dh = out.hits[:nh].cpu().numpy().view(pd.HIT_DTYPE).reshape(-1)
    for i in range(0, nh, max(1, nh // 300)):
        r0, c0 = divmod(int(dh[i]["pixel"]), det.cols)
        want = np.zeros(25, np.float32)
        for k in range(25):
            r, c = r0 + k // 5 - 2, c0 + k % 5 - 2
            if 0 <= r < det.rows and 0 <= c < det.cols:
                want[k] = e[dh[i]["frame"], r, c] / np.float32(thr["photon_kev"])
        assert got[i].tobytes() == want.tobytes()


def test_invalid_arguments():
    det = synth.asic_352x384(rows=8)
    ped, gain = synth.multigain_maps(det, 2)
    thr = det.thresholds()
    for kw in (dict(n_gains=5, gain_shift=14), dict(n_gains=2, gain_shift=16),
               dict(n_gains=2, gain_shift=0)):
        with pytest.raises((pd.PdError, ValueError)):
            p5 = np.concatenate([ped] * 3)[:kw["n_gains"]]
            g5 = np.concatenate([gain] * 3)[:kw["n_gains"]]
            pd.pd_create(det.geometry(), p5, g5, thr, **kw)
    with pytest.raises(pd.PdError) as ei:
        pd.pd_create(dict(det.geometry(), cm_mode=pd.PD_CM_MEAN), ped, gain, thr, n_gains=2,
                     gain_shift=14)
    assert ei.value.code == pd.PD_EINVAL
