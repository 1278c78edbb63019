"""Pins of the CPU oracle to facts outside itself.

Each test checks the oracle against something the paper or the mathematics
fixes — hand-derived worked examples (tests/golden/cases.json), closed forms
with exact rational arithmetic, invariants (dark frames, symmetry, totals),
special cases that reduce to a library routine (the lower median against
numpy's sort) — chosen so that a dropped term, a wrong sign, index or
threshold comparison, or a transposed operand fails at least one of them.
No GPU is needed.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1903_06838_gb300 import synth
from tests._cases import (expected_cm, expected_hits, f32_of, load_cases,
                          sort_hits, sparse_to_dense)

CASES = load_cases()


def _geom(**g):
    return oracle.geometry(**g)


def _thr(*a, **t):
    return oracle.thresholds(*a, **t)


# --------------------------------------------------------------------------
# hand-derived worked examples
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_golden_case(case):
    g = _geom(**case["geometry"])
    t = _thr(**case["thresholds"])
    r = oracle.process(g, t, case["ped_arr"], case["gain_arr"],
                       case["raw_arr"])
    exp = expected_hits(case)
    got = sort_hits(r.hits)
    assert r.n_hits == len(exp)
    assert got.tobytes() == exp.tobytes(), (got, exp)
    assert r.n_seeds == case["expect"]["n_seeds"]
    np.testing.assert_array_equal(r.cm, expected_cm(case))
    bins = case["thresholds"]["hist_bins"]
    np.testing.assert_array_equal(
        r.hist_pix, sparse_to_dense(case["expect"]["hist_pix"], bins))
    np.testing.assert_array_equal(
        r.hist_hit, sparse_to_dense(case["expect"]["hist_hit"], bins))
    npx = case["raw_arr"][0].size
    np.testing.assert_array_equal(
        r.count_map, sparse_to_dense(case["expect"]["count_map"], npx,
                                     np.uint32))


# --------------------------------------------------------------------------
# common mode: the lower median is numpy's sort at rank floor((n-1)/2)
def _np_lower_median(v):
    s = np.sort(np.asarray(v, np.float32))
    return s[(s.size - 1) // 2]


@pytest.mark.parametrize("seed", range(6))
def test_lower_median_matches_sort(seed):
    rng = np.random.default_rng(seed)
    for n in (1, 2, 3, 4, 5, 10, 31, 32, 33, 384, 1001):
        for kind in ("normal", "ties", "ints", "const", "neg"):
            if kind == "normal":
                v = rng.normal(0, 4, n)
            elif kind == "ties":
                v = rng.integers(-3, 3, n) * 0.5
            elif kind == "ints":
                v = rng.integers(-1000, 1000, n)
            elif kind == "const":
                v = np.full(n, 7.25)
            else:
                v = -np.abs(rng.normal(0, 100, n))
            v = v.astype(np.float32)
            assert oracle.lower_median(v) == _np_lower_median(v)


def test_lower_median_even_count_takes_lower():
    # {1, 2, 3, 4}: the lower median is 2 (rank 1), not 3 or 2.5.
    assert oracle.lower_median([4, 1, 3, 2]) == np.float32(2)
    assert oracle.lower_median([2, 1]) == np.float32(1)


@pytest.mark.parametrize("seed", range(4))
def test_cm_per_unit_matches_sort(seed):
    """Common mode of every unit equals numpy's lower median of the unit's
    d = raw - ped below the cut, or 0 when fewer than n_min pixels."""
    rng = np.random.default_rng(100 + seed)
    for (R, C, ur, uc) in ((6, 16, 1, 8), (8, 12, 4, 6), (5, 20, 5, 20)):
        ped = rng.normal(50, 3, (2, R, C)).astype(np.float32)
        gain = np.ones((2, R, C), np.float32)
        raw = np.clip(np.rint(rng.normal(60, 20, (3, 2, R, C))), 0, 65535) \
            .astype(np.uint16)
        cut = 15.0
        n_min = int(rng.integers(1, ur * uc))
        g = _geom(n_modules=2, rows=R, cols=C, unit_rows=ur, unit_cols=uc)
        t = _thr(cut, 0.5, 0.5, 8.0, cm_min_count=n_min)
        res = oracle.process(g, t, ped, gain, raw)
        d = raw.astype(np.float32) - ped[None]
        exp = []
        for f in range(3):
            for m in range(2):
                for a in range(R // ur):
                    for b in range(C // uc):
                        blk = d[f, m, a * ur:(a + 1) * ur, b * uc:(b + 1) * uc]
                        sel = blk[blk < np.float32(cut)]
                        exp.append(_np_lower_median(sel) if sel.size >= n_min
                                   else np.float32(0))
        np.testing.assert_array_equal(res.cm.reshape(-1),
                                      np.array(exp, np.float32))


def test_cm_default_min_count_is_ceil_sqrt():
    for n, k in ((1, 1), (2, 2), (4, 2), (5, 3), (384, 20), (35890, 190),
                 (35721, 189), (35722, 190)):
        assert oracle.default_min_count(n) == k


# --------------------------------------------------------------------------
# invariants on generated data
SMALL = {
    "asic": synth.asic_352x384(rows=48, cols=384),
    "cspad": synth.cspad_2p2m(n_modules=2),
    "epix": synth.epix_704x768(rows=32),
}


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("seed", (1, 2, 3))
def test_dark_frames_give_no_hits(name, seed):
    det = SMALL[name].replace(occupancy=0.0, seed=seed)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 4)
    r = oracle.process(_geom(**det.geometry()), _thr(**det.thresholds()),
                       ped, gain, raw)
    assert r.n_hits == 0
    assert r.count_map.sum() == 0


@pytest.mark.parametrize("name", list(SMALL))
def test_noise_free_dark_is_exactly_zero(name):
    """Integer pedestals, no noise: d is the injected offset rounded, so the
    common mode equals it exactly and every corrected pixel is exactly 0."""
    det = SMALL[name].replace(occupancy=0.0, noise_sigma=0.0, seed=7)
    ped, gain = synth.maps(det)
    ped = np.rint(ped).astype(np.float32)
    raw, _, cm_true = synth.frames(det, ped, gain, 0, 3, cm_truth=True)
    r = oracle.process(_geom(**det.geometry()), _thr(**det.thresholds()),
                       ped, gain, raw, want_corrected=True)
    np.testing.assert_array_equal(r.cm, np.rint(cm_true).astype(np.float32))
    assert not np.any(r.corrected)
    assert r.n_hits == 0


@pytest.mark.parametrize("name", list(SMALL))
def test_common_mode_tracks_injected_offset(name):
    """With noise sigma the median of n pixels has standard error about
    1.2533 sigma / sqrt(n); photons (above the cut or sparse) barely move it.
    Fixed seeds make this deterministic; the bound is 6 standard errors."""
    det = SMALL[name].replace(seed=11)
    ped, gain = synth.maps(det)
    raw, _, cm_true = synth.frames(det, ped, gain, 0, 4, cm_truth=True)
    r = oracle.process(_geom(**det.geometry()), _thr(**det.thresholds()),
                       ped, gain, raw)
    n = det.unit_rows * det.unit_cols
    bound = 6 * 1.2533 * det.noise_sigma / math.sqrt(n) + 0.5
    assert np.max(np.abs(r.cm - cm_true)) < bound


# --------------------------------------------------------------------------
# closed forms: isolated photons with exact integer arithmetic
def _embed(R, C, r0, c0, pat):
    raw = np.zeros((1, 1, R, C), np.uint16)
    for dy in range(3):
        for dx in range(3):
            rr, cc = r0 + dy - 1, c0 + dx - 1
            if 0 <= rr < R and 0 <= cc < C:
                raw[0, 0, rr, cc] = pat[dy, dx]
    return raw


@pytest.mark.parametrize("seed", range(8))
def test_isolated_photon_closed_form(seed):
    """E is the exact integer sum of the in-module 3x3; dx, dy are the
    correctly rounded quotients of the exact first moments; n = rint(E/ph)."""
    rng = np.random.default_rng(seed)
    R = C = 9
    g = _geom(n_modules=1, rows=R, cols=C, unit_rows=R, unit_cols=C)
    for _ in range(40):
        pat = rng.integers(0, 60, (3, 3))
        pat[1, 1] = pat.max() + rng.integers(1, 50)
        r0, c0 = int(rng.integers(0, R)), int(rng.integers(0, C))
        raw = _embed(R, C, r0, c0, pat)
        ph = float(rng.choice([5.0, 7.0, 13.0, 64.0]))
        t = _thr(0.5, 0.5, 0.5, ph, cm_min_count=1, hist_lo_kev=0.0,
                 hist_bin_kev=1.0, hist_bins=4096)
        r = oracle.process(g, t, np.zeros((1, R, C), np.float32),
                           np.ones((1, R, C), np.float32), raw)
        E = Mx = My = npix = 0
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                rr, cc = r0 + dy, c0 + dx
                if 0 <= rr < R and 0 <= cc < C:
                    v = int(pat[dy + 1, dx + 1])
                    E += v
                    Mx += v * dx
                    My += v * dy
                    npix += v > 0
        n = round(Fraction(E) / Fraction(ph))  # Python round: ties to even
        if n == 0:
            assert r.n_hits == 0
            continue
        assert r.n_hits == 1
        h = r.hits[0]
        assert h["pixel"] == r0 * C + c0
        assert h["energy_kev"] == np.float32(E)
        assert h["dx"] == f32_of(Fraction(Mx, E))
        assert h["dy"] == f32_of(Fraction(My, E))
        assert h["count"] == min(n, 255) and h["npix"] == npix
        edge = r0 in (0, R - 1) or c0 in (0, C - 1)
        assert h["flags"] == (oracle.HIT_EDGE if edge else 0)


def test_thresholds_are_strict():
    """A neighbour exactly at zero_thr is zeroed; a pixel exactly at
    seed_thr is not a seed (both comparisons are strict, Fig. e)."""
    R = C = 5
    g = _geom(n_modules=1, rows=R, cols=C, unit_rows=R, unit_cols=C)
    t = _thr(0.5, 2.0, 3.0, 1.0, cm_min_count=1)
    ones = np.ones((1, R, C), np.float32)
    zeros = np.zeros((1, R, C), np.float32)
    pat = np.array([[0, 0, 0], [2, 9, 3], [0, 0, 0]])
    r = oracle.process(g, t, zeros, ones, _embed(R, C, 2, 2, pat))
    assert r.n_hits == 1 and r.hits[0]["energy_kev"] == np.float32(12)
    assert r.hits[0]["npix"] == 2
    pat = np.array([[0, 0, 0], [0, 3, 0], [0, 0, 0]])
    r = oracle.process(g, t, zeros, ones, _embed(R, C, 2, 2, pat))
    assert r.n_seeds == 0 and r.n_hits == 0


@pytest.mark.parametrize("seed", range(5))
def test_centroid_matches_charge_cloud(seed):
    """Noise-free isolated photons from the generator: dx, dy equal the
    centre of mass of the renormalised 3x3 Gaussian fractions (closed form
    from erf) up to the ADU quantisation of the deposits."""
    rng = np.random.default_rng(seed)
    det = synth.asic_352x384(rows=16, cols=16, unit_rows=1, unit_cols=16,
                             noise_sigma=0.0, cm_sigma=0.0, occupancy=0.0,
                             photon_kev=1000.0, cloud_sigma=0.3, seed=seed + 1,
                             ped_sigma=0.0, gain_sigma=0.0)
    ped, gain = synth.maps(det)
    t = _thr(10.0, 0.02, 0.02, 1000.0, cm_min_count=1)
    g = _geom(**det.geometry())
    for _ in range(20):
        x = 7 + rng.uniform(0.1, 0.9)
        y = 8 + rng.uniform(0.1, 0.9)
        s = 0.3
        fx = [0.5 * (math.erf((7 + k + 1 - x) / (s * math.sqrt(2))) -
                     math.erf((7 + k - x) / (s * math.sqrt(2))))
              for k in (-1, 0, 1)]
        fy = [0.5 * (math.erf((8 + k + 1 - y) / (s * math.sqrt(2))) -
                     math.erf((8 + k - y) / (s * math.sqrt(2))))
              for k in (-1, 0, 1)]
        fx = np.array(fx) / sum(fx)
        fy = np.array(fy) / sum(fy)
        acc = np.full((16, 16), 1500.0)
        acc[7:10, 6:9] += 1000.0 * 25.0 * np.outer(fy, fx)
        raw = np.rint(acc).astype(np.uint16)[None, None]
        r = oracle.process(g, t, ped, gain, raw)
        assert r.n_hits == 1
        h = r.hits[0]
        assert h["pixel"] == 8 * 16 + 7
        cx = float(fx[2] - fx[0])
        cy = float(fy[2] - fy[0])
        assert abs(h["dx"] - cx) < 2e-4 and abs(h["dy"] - cy) < 2e-4
        assert abs(h["energy_kev"] - 1000.0) < 0.1
        assert h["count"] == 1


def _blob_frame(rng, R, C, n_blobs):
    """Sparse blobs with all-distinct positive integer values (no ties)."""
    raw = np.zeros((R, C), np.int64)
    vals = rng.permutation(np.arange(1, 40 * n_blobs + 1))[:9 * n_blobs]
    k = 0
    for _ in range(n_blobs):
        r0, c0 = int(rng.integers(0, R)), int(rng.integers(0, C))
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                rr, cc = r0 + dy, c0 + dx
                if 0 <= rr < R and 0 <= cc < C and raw[rr, cc] == 0:
                    raw[rr, cc] = vals[k] + 1000 * (dy == 0 and dx == 0)
                k += 1
    return raw.astype(np.uint16)


@pytest.mark.parametrize("seed", range(4))
def test_mirror_and_transpose_symmetry(seed):
    """Reflecting a frame left-right negates dx and mirrors the column;
    transposing a square module swaps (row, col) and (dx, dy).  Integer data
    without ties makes every sum exact, so equality is exact."""
    rng = np.random.default_rng(seed)
    N = 24
    t = _thr(0.5, 0.5, 0.5, 200.0, cm_min_count=1)
    g = _geom(n_modules=1, rows=N, cols=N, unit_rows=N, unit_cols=N)
    z = np.zeros((1, N, N), np.float32)
    o = np.ones((1, N, N), np.float32)
    raw = _blob_frame(rng, N, N, 12)
    base = oracle.process(g, t, z, o, raw[None, None])
    assert base.n_hits > 0

    def key(h, f):
        r, c = divmod(int(h["pixel"]), N)
        return f(r, c, h)

    ref = sorted(key(h, lambda r, c, h: (r, c, float(h["energy_kev"]),
                                         float(h["dx"]), float(h["dy"]),
                                         int(h["count"]), int(h["npix"])))
                 for h in base.hits)
    mir = oracle.process(g, t, z, o, raw[:, ::-1].copy()[None, None])
    got = sorted(key(h, lambda r, c, h: (r, N - 1 - c, float(h["energy_kev"]),
                                         -float(h["dx"]), float(h["dy"]),
                                         int(h["count"]), int(h["npix"])))
                 for h in mir.hits)
    assert got == ref
    tr = oracle.process(g, t, z, o, raw.T.copy()[None, None])
    got = sorted(key(h, lambda r, c, h: (c, r, float(h["energy_kev"]),
                                         float(h["dy"]), float(h["dx"]),
                                         int(h["count"]), int(h["npix"])))
                 for h in tr.hits)
    assert got == ref


@pytest.mark.parametrize("seed", range(10))
def test_seed_tie_properties(seed):
    """With heavy ties (values in 0..3): no two neighbouring pixels are both
    seeds; a pixel strictly above all neighbours is a seed; a pixel with a
    strictly larger neighbour is not; in every connected plateau of equal
    value whose outside neighbours are all lower, the first pixel in raster
    order is a seed, and a plateau of two pixels has no other seed."""
    rng = np.random.default_rng(seed)
    R, C = 12, 13
    raw = rng.integers(0, 4, (R, C)).astype(np.uint16)
    g = _geom(n_modules=1, rows=R, cols=C, unit_rows=R, unit_cols=C,
              cm_mode=oracle.CM_NONE)
    t = _thr(0.5, 0.5, 0.5, 0.001, hist_lo_kev=0.0, hist_bin_kev=1.0)
    r = oracle.process(g, t, np.zeros((1, R, C), np.float32),
                       np.ones((1, R, C), np.float32), raw[None, None])
    seeds = np.zeros((R, C), bool)
    for h in r.hits:
        seeds[divmod(int(h["pixel"]), C)] = True
    assert r.n_seeds == seeds.sum()
    v = raw.astype(int)

    def nbrs(a, b):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dy or dx) and 0 <= a + dy < R and 0 <= b + dx < C:
                    yield a + dy, b + dx

    for a in range(R):
        for b in range(C):
            ns = list(nbrs(a, b))
            if seeds[a, b]:
                assert not any(seeds[q] for q in ns)
            if v[a, b] >= 1 and all(v[a, b] > v[q] for q in ns):
                assert seeds[a, b]
            if any(v[q] > v[a, b] for q in ns):
                assert not seeds[a, b]
    seen = np.zeros((R, C), bool)
    for a in range(R):
        for b in range(C):
            if seen[a, b] or v[a, b] < 1:
                continue
            comp, stack = [], [(a, b)]
            seen[a, b] = True
            while stack:
                p = stack.pop()
                comp.append(p)
                for q in nbrs(*p):
                    if not seen[q] and v[q] == v[a, b]:
                        seen[q] = True
                        stack.append(q)
            outside = {q for p in comp for q in nbrs(*p)} - set(comp)
            if all(v[q] < v[a, b] for q in outside):
                assert seeds[min(comp)]
                if len(comp) <= 2:
                    assert [p for p in comp if seeds[p]] == [min(comp)]


def test_pileup_counts():
    """k photons landing together deposit k times the energy; with no noise
    and a low zeroing threshold rint(E / E_ph) recovers k (away from the
    module border, where part of the 3x3 footprint falls outside)."""
    det = synth.asic_352x384(rows=64, cols=64, unit_rows=1, unit_cols=64,
                             noise_sigma=0.0, cm_sigma=0.0, occupancy=0.0005,
                             multi_frac=1.0, cloud_sigma=0.25, seed=5)
    ped, gain = synth.maps(det)
    raw, ph = synth.frames(det, ped, gain, 0, 40)
    t = _thr(200.0, 0.05, 0.05, 8.0, cm_min_count=1)
    r = oracle.process(_geom(**det.geometry()), t, ped, gain, raw)
    sites = {}
    for p in ph:
        key = (int(p["frame"]), float(p["x"]), float(p["y"]))
        sites[key] = sites.get(key, 0) + 1
    by_frame = {}
    for (f, x, y), k in sites.items():
        by_frame.setdefault(f, []).append((x, y, k))
    checked = 0
    for h in r.hits:
        f = int(h["frame"])
        row, col = divmod(int(h["pixel"]), 64)
        near = [s for s in by_frame.get(f, [])
                if abs(s[0] - (col + 0.5)) < 1.5 and abs(s[1] - (row + 0.5)) < 1.5]
        far = [s for s in by_frame.get(f, [])
               if abs(s[0] - (col + 0.5)) < 4 and abs(s[1] - (row + 0.5)) < 4]
        inside = all(1 <= int(v) <= 62 for v in near[0][:2]) if near else False
        if len(near) == 1 and len(far) == 1 and inside:
            assert h["count"] == near[0][2]
            checked += 1
    assert checked > 20
    assert {k for k in sites.values()} >= {2, 3, 4}


@pytest.mark.parametrize("name", list(SMALL))
def test_summary_totals(name):
    det = SMALL[name].replace(seed=3)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 3)
    r = oracle.process(_geom(**det.geometry()), _thr(**det.thresholds()),
                       ped, gain, raw)
    assert r.hist_pix.sum() == raw.size
    assert r.hist_hit.sum() == r.n_seeds
    assert r.count_map.sum() == r.hits["count"].astype(np.int64).sum()
    assert r.n_hits <= r.n_seeds


def test_histogram_bins_and_clipping():
    """bin(v) = floor(fma(v, 1/width, -lo/width)), end bins clipped (here all
    operands are dyadic, so t = 2e + 4 exactly)."""
    C = 8
    g = _geom(n_modules=1, rows=1, cols=C, unit_rows=1, unit_cols=C,
              cm_mode=oracle.CM_NONE)
    t = _thr(0.5, 100.0, 100.0, 1.0, hist_lo_kev=-2.0, hist_bin_kev=0.5,
             hist_bins=10)
    # e values: -3 (below lo), -2 (edge of bin 0), -1.75, 0, 0.5, 2.49,
    # 2.5 (edge of bin 9), 40 (above)
    ped = np.array([3, 2, 1.75, 0, -0.5, -2.49, -2.5, -40], np.float32)
    raw = np.zeros((1, 1, 1, C), np.uint16)
    r = oracle.process(g, t, ped.reshape(1, 1, C), np.ones((1, 1, C), np.float32),
                       raw)
    exp = np.zeros(10, np.uint64)
    inv_w = np.float32(1) / np.float32(0.5)
    for e in (-3, -2, -1.75, 0, 0.5, 2.49, 2.5, 40):
        tt = float(np.float32(e)) * float(inv_w) + 4.0
        exp[int(min(max(math.floor(tt), 0), 9))] += 1
    np.testing.assert_array_equal(r.hist_pix, exp)
    assert list(np.nonzero(r.hist_pix)[0]) == [0, 4, 5, 8, 9]
    assert list(r.hist_pix[[0, 4, 5, 8, 9]]) == [3, 1, 1, 1, 2]


def _rn32(x: Fraction) -> Fraction:
    """x rounded to the nearest binary32 value (ties to even), exactly."""
    if x == 0:
        return Fraction(0)
    sign, a = (-1 if x < 0 else 1), abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while a >= Fraction(2) ** (e + 1):
        e += 1
    while a < Fraction(2) ** e:
        e -= 1
    m = a / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    q = math.floor(m)
    r = m - q
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and q % 2):
        q += 1
    return sign * q * Fraction(2) ** (e - 23)


# e values next to bin edges of 0.05 keV bins from -4 keV, with the bin the
# fused form gives and the bin the division form would give
NON_DYADIC = [(0.20000001788139343, 84, 83), (-0.9000000953674316, 62, 61),
              (0.44999998807907104, 89, 88), (0.5499998927116394, 91, 90),
              (-1.0000001192092896, 59, 60), (-0.9500001072883606, 60, 61)]


def test_histogram_bins_non_dyadic_width():
    """The summaries' bin with a width that is not dyadic (0.05 keV, lo = -4
    keV): bin(v) = floor(fma(v, 1/w, -lo * (1/w))), 1/w and lo * (1/w) each
    rounded to binary32 once and the fused product-sum rounded once.  Worked
    in exact rationals here: w rounds to 0.05000000074505806, 1/w to 20
    exactly and -lo/w to 80, so bin(v) = floor(RN(20 v + 80)).  At each value
    below the division form floor(RN(RN(v - lo) / w)) gives the neighbouring
    bin, so the pin tells the two readings apart."""
    w = Fraction(float(np.float32(0.05)))
    lo = Fraction(-4)
    inv_w = _rn32(1 / w)
    lo_s = _rn32(lo * inv_w)
    assert inv_w == 20 and lo_s == -80
    for v, fused, division in NON_DYADIC:
        vf = Fraction(float(np.float32(v)))
        assert math.floor(_rn32(vf * inv_w - lo_s)) == fused
        assert math.floor(_rn32(_rn32(vf - lo) / w)) == division
    C = len(NON_DYADIC)
    g = _geom(n_modules=1, rows=1, cols=C, unit_rows=1, unit_cols=C, cm_mode=oracle.CM_NONE)
    t = _thr(0.5, 100.0, 100.0, 1.0, hist_lo_kev=-4.0, hist_bin_kev=0.05, hist_bins=1296)
    # raw 0, unit gain: e = -pedestal exactly
    ped = np.array([-v for v, _, _ in NON_DYADIC], np.float32).reshape(1, 1, C)
    r = oracle.process(g, t, ped, np.ones((1, 1, C), np.float32), np.zeros((1, 1, 1, C), np.uint16))
    exp = np.zeros(1296, np.uint64)
    for _, fused, _ in NON_DYADIC:
        exp[fused] += 1
    np.testing.assert_array_equal(r.hist_pix, exp)


def test_split_calls_accumulate_like_one():
    det = SMALL["asic"].replace(seed=9)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 6)
    g, t = _geom(**det.geometry()), _thr(**det.thresholds())
    one = oracle.process(g, t, ped, gain, raw)
    a = oracle.process(g, t, ped, gain, raw[:2])
    b = oracle.process(g, t, ped, gain, raw[2:], frame_base=2,
                       count_map=a.count_map.copy(), hist_pix=a.hist_pix.copy(),
                       hist_hit=a.hist_hit.copy())
    hits = np.concatenate([a.hits, b.hits])
    assert hits.tobytes() == one.hits.tobytes()
    np.testing.assert_array_equal(b.count_map, one.count_map)
    np.testing.assert_array_equal(b.hist_pix, one.hist_pix)
    np.testing.assert_array_equal(b.hist_hit, one.hist_hit)


def test_invalid_thresholds_rejected():
    g = _geom(n_modules=1, rows=4, cols=4, unit_rows=4, unit_cols=4)
    raw = np.zeros((1, 1, 4, 4), np.uint16)
    z = np.zeros((1, 4, 4), np.float32)
    for bad in (_thr(1.0, 2.0, 1.0, 1.0), _thr(1.0, -1.0, 1.0, 1.0),
                _thr(1.0, 0.5, 1.0, 0.0), _thr(1.0, 0.5, 1.0, 1.0, hist_bins=0)):
        with pytest.raises(ValueError):
            oracle.process(g, bad, z, z, raw)
    with pytest.raises(ValueError):
        oracle.process(_geom(n_modules=1, rows=4, cols=4, unit_rows=3,
                             unit_cols=4), _thr(1.0, 0.5, 1.0, 1.0), z, z, raw)
