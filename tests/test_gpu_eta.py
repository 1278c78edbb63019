"""Centroid linearisation on the GPU (pd_eta_*) against the CPU oracle
(oracle/eta.py): histograms exactly, linearised offsets and flags bit for
bit, on hits with mixed counts, non-finite and out-of-range centroids."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import eta as oeta
from paper_1903_06838_gb300 import pd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _hits(rng, n):
    h = np.zeros(n, pd.HIT_DTYPE)
    u = rng.uniform(-0.5, 0.5, (n, 2))
    d = np.sin(np.pi * u) + rng.normal(0, 0.02, (n, 2))
    h["dx"], h["dy"] = d[:, 0], d[:, 1]
    h["count"] = rng.choice([0, 1, 1, 1, 2, 3], n)
    h["flags"] = rng.integers(0, 8, n)
    h["frame"] = rng.integers(0, 100, n)
    h["pixel"] = rng.integers(0, 388 * 185, n)
    h["energy_kev"] = rng.uniform(1, 30, n)
    h["npix"] = rng.integers(1, 10, n)
    if n > 16:
        h["dx"][3] = np.nan
        h["dy"][5] = np.inf
        h["dx"][7] = 1.0      # the top edge of the range
        h["dy"][9] = -1.0     # the bottom edge
        h["dx"][11] = 1.7     # beyond the range: clipped to the end bins
        h["dy"][13] = -3.0
    return h


def _dev(h):
    return torch.from_numpy(h.view(np.uint8).copy()).cuda()


@pytest.mark.parametrize("bins,n", [(1, 1000), (255, 300_001), (4095, 70_000)])
def test_histogram_and_apply_match_oracle(bins, n):
    rng = np.random.default_rng(bins + n)
    cal = _hits(rng, n)
    test = _hits(rng, n // 3 + 17)
    e = pd.pd_eta_create(bins)
    dcal = _dev(cal)
    half = (n // 2) * pd.HIT_DTYPE.itemsize
    pd.pd_eta_accumulate(e, dcal.data_ptr(), n // 2)              # in two calls
    pd.pd_eta_accumulate(e, dcal.data_ptr() + half, n - n // 2)
    pd.pd_eta_finalize(e)
    ref_hist = oeta.accumulate(np.zeros((2, bins), np.uint32), cal, bins)
    assert np.array_equal(pd.pd_eta_get_histogram(e), ref_hist)

    dtest = _dev(test)
    out = torch.empty_like(dtest)
    pd.pd_eta_apply(e, dtest.data_ptr(), len(test), out.data_ptr())
    got = out.cpu().numpy().view(pd.HIT_DTYPE)
    ref = oeta.apply(ref_hist, test, bins)
    assert got.tobytes() == ref.tobytes()

    pd.pd_eta_apply(e, dtest.data_ptr(), len(test), dtest.data_ptr())  # in place
    assert dtest.cpu().numpy().tobytes() == ref.tobytes()


def test_empty_and_reset_leave_centroids_unchanged():
    rng = np.random.default_rng(5)
    e = pd.pd_eta_create(63)
    pd.pd_eta_accumulate(e, 0, 0)
    pd.pd_eta_finalize(e)
    test = _hits(rng, 500)
    d = _dev(test)
    out = torch.empty_like(d)
    pd.pd_eta_apply(e, d.data_ptr(), len(test), out.data_ptr())
    got = out.cpu().numpy().view(pd.HIT_DTYPE)
    ref = oeta.apply(np.zeros((2, 63), np.uint32), test, 63)
    assert got.tobytes() == ref.tobytes()
    # accumulate, then reset: back to the identity
    pd.pd_eta_accumulate(e, d.data_ptr(), len(test))
    pd.pd_eta_reset(e)
    pd.pd_eta_finalize(e)
    assert pd.pd_eta_get_histogram(e).sum() == 0
    pd.pd_eta_apply(e, d.data_ptr(), len(test), out.data_ptr())
    assert out.cpu().numpy().tobytes() == ref.tobytes()
    pd.pd_eta_apply(e, 0, 0, 0)


def test_invalid_bins_are_rejected():
    for bins in (0, 2, 256, int(pd.PD_MAX_ETA_BINS) + 2):
        with pytest.raises(pd.PdError):
            pd.pd_eta_create(bins)
