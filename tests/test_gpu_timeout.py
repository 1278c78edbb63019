"""Bounded device waits: a wait that gives up is reported, and the context
stays usable.

pd_set_wait_limit(ctx, 1) lets the first poll of a staged copy's mbarrier
(the bank median) or of a tile's dependency (the work-queue launch) give
up.  No fault is involved: the kernel that gives up still waits out its
own copies in flight with the default bound before it stops, so every
launch completes.  The call's results are not valid, pd_get_summary
returns PD_ETIMEDOUT, and after pd_reset_summary with the default bound
the same context gives results equal to the oracle's.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import pd, synth
from tests._cases import sort_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle(det, ped, gain, raw):
    return oracle.process(oracle.geometry(**det.geometry()), oracle.thresholds(**det.thresholds()),
                          ped, gain, raw)


@pytest.mark.parametrize("kernels", [1, 3], ids=["kernel_pair", "work_queue"])
def test_wait_timeout_is_reported_and_context_recovers(kernels):
    det = synth.cspad_2p2m(n_modules=4, occupancy=0.01)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 3)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    pd.pd_set_tuning(ctx, kernels=kernels)
    assert pd.pd_get_tuning(ctx)["kernels"] == kernels
    dev = pd.frames_to_device(raw)

    pd.pd_set_wait_limit(ctx, 1)
    pd.process(ctx, dev, cm=True, hit_capacity=3 * 65536)
    torch.cuda.synchronize()
    with pytest.raises(pd.PdError) as err:
        pd.pd_get_summary(ctx)
    assert err.value.code == pd.PD_ETIMEDOUT

    pd.pd_set_wait_limit(ctx, 0)
    pd.pd_reset_summary(ctx)
    out = pd.process(ctx, dev, cm=True, hit_capacity=3 * 65536)
    torch.cuda.synchronize()
    ref = _oracle(det, ped, gain, raw)
    hits, n = out.hits_host()
    assert n == ref.n_hits == len(hits)
    assert sort_hits(hits).tobytes() == sort_hits(ref.hits).tobytes()
    assert out.cm.cpu().numpy().tobytes() == ref.cm.reshape(3, -1).tobytes()
    cmap, hp, hh = pd.pd_get_summary(ctx)
    np.testing.assert_array_equal(cmap, ref.count_map)
    np.testing.assert_array_equal(hp, ref.hist_pix)
    np.testing.assert_array_equal(hh, ref.hist_hit)
