"""pd_process_noalloc against pd_process, through the C ABI.

pd_process_noalloc serves callers that may not allocate device memory while
processing (a real-time acquisition thread, or a process whose device memory
belongs to another allocator): it keeps its common-mode scratch in a fixed
array inside the library instead of growing a buffer with cudaMalloc.  Its
results must be those of pd_process bit for bit (the tolerance of every
parity test of the plain chain), on two calls in a row, since the second
call finds the first call's values left in the shared array; and a call on a
warm context must leave the device's free memory unchanged.

This file is named so pytest collects it last.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1903_06838_gb300 import pd, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sorted(h):
    return np.sort(h, order=["frame", "pixel"])


def _case(name):
    """(detector, frames per call, geometry overrides, n_gains, gain_shift)"""
    if name == "bank_units":
        return synth.cspad_2p2m(n_modules=2), 6, {}, 0, 0
    if name == "row_units":
        return synth.asic_352x384(rows=96), 5, {}, 0, 0
    if name == "stacked_mean":
        # one value per unit, module row and module column per frame
        return synth.cspad_2p2m(n_modules=2), 4, {"cm_mode": pd.PD_CM_MEAN_STACKED}, 0, 0
    if name == "multigain":
        det = synth.Detector(n_modules=2, rows=64, cols=128, unit_rows=64, unit_cols=64,
                             occupancy=0.01)
        return det, 5, {}, 3, 14
    raise KeyError(name)


def _data(det, n_gains, shift, first, n):
    if n_gains:
        ped, gain = synth.multigain_maps(det, n_gains, (1.0, 1 / 3, 1 / 100)[:n_gains],
                                         (0.0, -300.0, -700.0)[:n_gains])
        raw, _ = synth.multigain_frames(det, ped, gain, first, n, gain_shift=shift,
                                        blob_kev=4000.0, bad_frac=2e-4)
    else:
        ped, gain = synth.maps(det)
        raw, _ = synth.frames(det, ped, gain, first, n)
    return ped, gain, raw


@pytest.mark.parametrize("name", ["bank_units", "row_units", "stacked_mean", "multigain"])
def test_noalloc_matches_pd_process_on_two_calls(name):
    det, n, over, n_gains, shift = _case(name)
    ped, gain, raw_a = _data(det, n_gains, shift, 0, n)
    _, _, raw_b = _data(det, n_gains, shift, n, n)
    ctx = pd.pd_create(dict(det.geometry(), **over), ped, gain, det.thresholds(),
                       n_gains=n_gains, gain_shift=shift)
    cap = n * det.pixels_per_frame // 4

    refs = []
    for raw, base in ((raw_a, 0), (raw_b, n)):
        out = pd.process(ctx, pd.frames_to_device(raw), hit_capacity=cap,
                         frame_base=base, corrected=True)
        torch.cuda.synchronize()
        refs.append((out.hits_host(), out.corrected.cpu().numpy()))
    ref_summary = pd.pd_get_summary(ctx)
    pd.pd_reset_summary(ctx)

    # two calls in a row through the no-allocation entry point
    for (raw, base), ((ref_hits, ref_n), ref_corr) in zip(((raw_a, 0), (raw_b, n)), refs):
        dev = pd.frames_to_device(raw)
        out = pd.Outputs(ctx, n, cap, corrected=True)
        pd.pd_process_noalloc(ctx, dev.data_ptr(), n, base, **out.ptrs())
        torch.cuda.synchronize()
        hits, nh = out.hits_host()
        assert nh == ref_n and len(hits) == nh
        assert _sorted(hits).tobytes() == _sorted(ref_hits).tobytes()
        assert out.corrected.cpu().numpy().tobytes() == ref_corr.tobytes()
    for got, exp in zip(pd.pd_get_summary(ctx), ref_summary):
        np.testing.assert_array_equal(got, exp)
    pd.pd_destroy(ctx)


def test_noalloc_warm_call_leaves_free_memory_unchanged():
    det, n, over, _, _ = _case("bank_units")
    ped, gain, raw = _data(det, 0, 0, 0, n)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    dev = pd.frames_to_device(raw)
    out = pd.Outputs(ctx, n, n * det.pixels_per_frame // 4)
    pd.pd_process_noalloc(ctx, dev.data_ptr(), n, 0, **out.ptrs())  # warm: kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        pd.pd_process_noalloc(ctx, dev.data_ptr(), n, 0, **out.ptrs())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    pd.pd_destroy(ctx)


@pytest.mark.parametrize("name", ["bank_units", "stacked_mean"])
def test_noalloc_rejects_requests_beyond_its_scratch(name):
    det = synth.cspad_2p2m(n_modules=1)
    over = _case(name)[2]
    ped, gain = synth.maps(det)
    ctx = pd.pd_create(dict(det.geometry(), **over), ped, gain, det.thresholds())
    # the bound counts every common-mode value of a frame (units, and for the
    # stacked mean also module rows and columns), not units alone
    too_many = pd.PD_NOALLOC_MAX_CM // ctx.cm_values_per_frame + 1
    if name == "stacked_mean":
        assert ctx.cm_values_per_frame > ctx.units_per_frame
        assert too_many * ctx.units_per_frame <= pd.PD_NOALLOC_MAX_CM
    out = pd.Outputs(ctx, 0, 8)
    dummy = torch.zeros(8, dtype=torch.int16, device="cuda")
    with pytest.raises(pd.PdError) as ei:
        pd.pd_process_noalloc(ctx, dummy.data_ptr(), too_many, 0, **out.ptrs())
    assert ei.value.code == pd.PD_EINVAL
    assert "PD_NOALLOC_MAX_CM" in str(ei.value)
    pd.pd_destroy(ctx)


def test_noalloc_one_kernel_chain_has_no_scratch_limit():
    # the one-kernel chain keeps the common mode on chip: a call beyond the
    # scratch's frame count is accepted (dark frames: no hits)
    det = synth.Detector(n_modules=1, rows=8, cols=8, unit_rows=8, unit_cols=8)
    ped, gain = synth.maps(det)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    pd.pd_set_tuning(ctx, two_pass=0)
    if pd.pd_get_tuning(ctx)["two_pass"] != 0:
        pytest.skip("one-kernel chain not available for this geometry")
    n = pd.PD_NOALLOC_MAX_CM // ctx.cm_values_per_frame + 1
    frames = torch.from_numpy(np.broadcast_to(
        np.rint(ped).astype(np.int16).reshape(1, -1), (n, det.pixels_per_frame)).copy()).cuda()
    out = pd.Outputs(ctx, 0, 1024)
    pd.pd_process_noalloc(ctx, frames.data_ptr(), n, 0, **out.ptrs())
    torch.cuda.synchronize()
    assert out.hits_host()[1] == 0
    pd.pd_destroy(ctx)
