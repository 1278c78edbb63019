"""The compact hit stream of the streaming server (pd_compress_hits /
pd_decompress_hits): host code, no GPU needed.  Pixel index and count
round-trip exactly; energy is kept to 1/256 keV and the subpixel offsets to
1/128 pixel (clipped to +-127/128), so a frame's photon list survives the
encoding with the precision the centroid has (sections "Photon Subpixel
Resolution" and "Performance")."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1903_06838_gb300 import pd


def _hits(rng, n, n_px=2_000_000):
    h = np.zeros(n, pd.HIT_DTYPE)
    h["frame"] = 7
    h["pixel"] = rng.choice(n_px, size=n, replace=False)
    h["energy_kev"] = rng.uniform(0.0, 60.0, n).astype(np.float32)
    h["dx"] = rng.uniform(-1.0, 1.0, n).astype(np.float32)
    h["dy"] = rng.uniform(-1.0, 1.0, n).astype(np.float32)
    h["count"] = rng.integers(0, 256, n)
    return h


def test_round_trip_keeps_pixels_and_counts_exactly():
    rng = np.random.default_rng(0)
    h = _hits(rng, 3000)
    blob = pd.pd_compress_hits(h)
    back = pd.pd_decompress_hits(blob, frame=7)
    order = np.argsort(h["pixel"], kind="stable")
    ref = h[order]
    assert len(back) == len(h)
    assert np.array_equal(back["pixel"], ref["pixel"])
    assert np.array_equal(back["count"], ref["count"])
    assert np.all(back["frame"] == 7)
    # quantisation: energy to 1/256 keV (nearest), offsets to 1/128 px
    assert np.max(np.abs(back["energy_kev"] - ref["energy_kev"])) <= 0.5 / 256 + 1e-6
    for k in ("dx", "dy"):
        want = np.clip(np.round(ref[k].astype(np.float64) * 128), -127, 127) / 128
        assert np.array_equal(back[k].astype(np.float64), want)


def test_size_matches_the_format():
    # one hit: count varint (1 byte) + pixel varint + 5 bytes of payload
    for pixel, nbytes in ((0, 1), (127, 1), (128, 2), (16383, 2), (16384, 3),
                          (2_200_000, 4)):
        h = np.zeros(1, pd.HIT_DTYPE)
        h["pixel"] = pixel
        assert len(pd.pd_compress_hits(h)) == 1 + nbytes + 5
    # deltas, not absolute indices: 200 neighbours at stride 3 -> 1 byte each
    h = np.zeros(200, pd.HIT_DTYPE)
    h["pixel"] = 1_000_000 + 3 * np.arange(200)
    assert len(pd.pd_compress_hits(h)) == 2 + 3 + 199 * 1 + 200 * 5


def test_empty_and_clipping():
    assert pd.pd_compress_hits(np.zeros(0, pd.HIT_DTYPE)) == b"\x00"
    assert len(pd.pd_decompress_hits(b"\x00")) == 0
    h = np.zeros(2, pd.HIT_DTYPE)
    h["pixel"] = [5, 9]
    h["energy_kev"] = [-3.0, 1e6]       # below 0 and above 65535/256 keV
    h["dx"] = [2.0, -2.0]
    back = pd.pd_decompress_hits(pd.pd_compress_hits(h))
    assert list(back["energy_kev"]) == [0.0, 65535 / 256]
    assert list(back["dx"]) == [127 / 128, -127 / 128]


def test_truncated_stream_is_an_error():
    rng = np.random.default_rng(1)
    blob = pd.pd_compress_hits(_hits(rng, 10))
    with pytest.raises(pd.PdError) as e:
        pd.pd_decompress_hits(blob[:-1])
    assert e.value.code == pd.PD_EINVAL


def test_output_buffer_too_small_is_an_overflow():
    import ctypes
    h = _hits(np.random.default_rng(2), 4)
    need = ctypes.c_size_t()
    lib = pd.load()
    assert lib.pd_compress_hits(h.ctypes.data, 4, None, 0, ctypes.byref(need)) == pd.PD_OK
    buf = (ctypes.c_uint8 * 8)()
    assert lib.pd_compress_hits(h.ctypes.data, 4, buf, 8, ctypes.byref(need)) == pd.PD_EOVERFLOW
