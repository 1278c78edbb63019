"""pd_process_noalloc against pd_process, through the C ABI.

pd_process_noalloc serves callers that may not allocate device memory while
processing (a real-time acquisition thread, or a process whose device memory
belongs to another allocator): it keeps its common-mode scratch in a fixed
array inside the library instead of growing a buffer with cudaMalloc.  Its
results must be those of pd_process bit for bit (the tolerance of every
parity test of the plain chain), on two calls in a row, since the second
call finds the first call's values left in the shared array.

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


@pytest.mark.parametrize("det,n", [(synth.cspad_2p2m(n_modules=2), 6),
                                   (synth.asic_352x384(rows=96), 5)],
                         ids=["bank_units", "row_units"])
def test_noalloc_matches_pd_process_on_two_calls(det, n):
    ped, gain = synth.maps(det)
    raw_a, _ = synth.frames(det, ped, gain, 0, n)
    raw_b, _ = synth.frames(det, ped, gain, n, n)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
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


def test_noalloc_rejects_requests_beyond_its_scratch():
    det = synth.cspad_2p2m(n_modules=1)
    ped, gain = synth.maps(det)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    too_many = pd.PD_NOALLOC_MAX_CM // ctx.units_per_frame + 1
    out = pd.Outputs(ctx, 0, 8)
    dummy = torch.zeros(8, dtype=torch.int16, device="cuda")
    with pytest.raises(pd.PdError) as ei:
        pd.pd_process_noalloc(ctx, dummy.data_ptr(), too_many, 0, **out.ptrs())
    assert ei.value.code == pd.PD_EINVAL
    assert "PD_NOALLOC_MAX_CM" in str(ei.value)
    pd.pd_destroy(ctx)
