"""Helpers shared by the tests: golden-case loading and exact FP32 rounding."""
from __future__ import annotations

import json
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "cases.json")


def f32_of(fr) -> np.float32:
    """The binary32 value nearest to the rational fr (ties to even)."""
    fr = Fraction(fr)
    x = np.float32(float(fr))
    cands = [np.nextafter(x, np.float32(-np.inf)), x,
             np.nextafter(x, np.float32(np.inf))]

    def key(c):
        return (abs(Fraction(float(c)) - fr), int(c.view(np.uint32)) & 1)
    return np.float32(min(cands, key=key))


def _grid(spec, shape):
    if isinstance(spec, str) and spec.startswith("fill:"):
        return np.full(shape, np.float32(float(spec[5:])), np.float32)
    a = np.array(spec, np.float32)
    assert a.shape == shape, (a.shape, shape)
    return a


def load_cases():
    with open(GOLDEN) as f:
        doc = json.load(f)
    out = []
    for c in doc["cases"]:
        g = c["geometry"]
        shape = (g["n_modules"], g["rows"], g["cols"])
        case = dict(c)
        case["ped_arr"] = _grid(c["ped"], shape)
        case["gain_arr"] = _grid(c["gain"], shape)
        case["raw_arr"] = np.array(c["raw"], np.uint16)
        assert case["raw_arr"].shape[1:] == shape
        out.append(case)
    return out


def expected_hits(case):
    """Expected hits as a sorted structured array (dtype of the hit record)."""
    dt = np.dtype([("frame", "<u4"), ("pixel", "<u4"), ("energy_kev", "<f4"),
                   ("dx", "<f4"), ("dy", "<f4"), ("count", "u1"),
                   ("npix", "u1"), ("flags", "<u2")])
    hs = case["expect"]["hits"]
    a = np.zeros(len(hs), dt)
    for i, h in enumerate(hs):
        a[i] = (h["frame"], h["pixel"], f32_of(h["energy_kev"]),
                f32_of(h["dx"]), f32_of(h["dy"]), h["count"], h["npix"],
                h["flags"])
    return np.sort(a, order=["frame", "pixel"])


def sparse_to_dense(d, n, dtype=np.uint64):
    a = np.zeros(n, dtype)
    for k, v in d.items():
        a[int(k)] = v
    return a


def expected_cm(case):
    return np.array([[f32_of(v) for v in row] for row in case["expect"]["cm"]],
                    np.float32)


def sort_hits(h):
    return np.sort(h, order=["frame", "pixel"])
