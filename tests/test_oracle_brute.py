"""The C oracle against an independent restatement of the whole chain.

The restatement below is written from the paper's steps as this library reads
them ("Dark and Gain" and Fig. b: d = raw - pedestal, e = (d - cm) / gain;
"Common Mode", Fig. c, with the lower median over d < cut; "Photon Charge
Summing", Fig. e: zeroing, 3x3 local maximum with the raster tie rule, the
3x3 sum and the count; "Photon Subpixel Resolution", Fig. f: centre of mass;
"Summarization", Fig. g: count map and the two histograms), in plain Python
and numpy float32 scalars: a sort for the median, explicit neighbour loops,
exact rational arithmetic for the fused multiply-add of the histogram bins.
It shares no code and no structure with pd_oracle.c.  Small random noisy
frames (8 x 8 modules and smaller, several modules and units each), and
frames made of small integers, where ties in the common-mode set and between
neighbours are everywhere, must give the same hits, common mode, corrected
frames, count map and histograms bit for bit.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

F32 = np.float32


def _rn32(x: Fraction) -> float:
    """x rounded to binary32, ties to even (x within the normal range)."""
    if x == 0:
        return 0.0
    sign, a = (-1 if x < 0 else 1), abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while a >= Fraction(2) ** (e + 1):
        e += 1
    while a < Fraction(2) ** e:
        e -= 1
    m = a / Fraction(2) ** (e - 23)
    q = math.floor(m)
    r = m - q
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and q % 2):
        q += 1
    return float(sign * q * Fraction(2) ** (e - 23))


def _bin(v, lo, w, bins):
    """floor(fma(v, 1/w, -lo/w)) clipped to [0, bins - 1], 1/w and lo/w each
    rounded to binary32 once, the fused product-sum rounded once."""
    inv_w = F32(1.0) / F32(w)
    nl = -(F32(lo) * inv_w)
    t = _rn32(Fraction(float(F32(v))) * Fraction(float(inv_w)) + Fraction(float(nl)))
    return int(min(max(math.floor(t), 0), bins - 1))


def restated_chain(geom, thr, ped, gain, raw):
    """Returns (hits as a set of tuples, cm [n][units], corrected [n][px],
    count map, hist_pix, hist_hit) for frames raw [n][modules][rows][cols]."""
    M, R, C = geom["n_modules"], geom["rows"], geom["cols"]
    UR, UC = geom["unit_rows"], geom["unit_cols"]
    cut, z, seed_t, ph = (F32(thr[k]) for k in ("cm_cut_adu", "zero_thr_kev",
                                                  "seed_thr_kev", "photon_kev"))
    lo, w, bins = thr["hist_lo_kev"], thr["hist_bin_kev"], thr["hist_bins"]
    n_min = thr.get("cm_min_count", 0) or math.isqrt(UR * UC - 1) + 1
    ped = np.asarray(ped, F32).reshape(M, R, C)
    gain = np.asarray(gain, F32).reshape(M, R, C)
    inv = np.zeros_like(gain)
    for idx in np.ndindex(gain.shape):
        g = gain[idx]
        inv[idx] = F32(1.0) / g if (g > 0 and math.isfinite(g)) else F32(0.0)
    raw = np.asarray(raw).reshape(-1, M, R, C)
    n = raw.shape[0]
    units_per_module = (R // UR) * (C // UC)
    cm_all = np.zeros((n, M * units_per_module), F32)
    corr = np.zeros((n, M * R * C), F32)
    cmap = np.zeros(M * R * C, np.uint64)
    hp = np.zeros(bins, np.uint64)
    hh = np.zeros(bins, np.uint64)
    hits = set()
    for f in range(n):
        for m in range(M):
            d = [[F32(float(raw[f, m, r, c])) - ped[m, r, c] for c in range(C)]
                 for r in range(R)]
            e = [[F32(0.0)] * C for _ in range(R)]
            for ur in range(R // UR):
                for uc in range(C // UC):
                    vals = [d[r][c] for r in range(ur * UR, (ur + 1) * UR)
                            for c in range(uc * UC, (uc + 1) * UC) if d[r][c] < cut]
                    cm = F32(0.0)
                    if vals and len(vals) >= n_min:
                        cm = sorted(vals)[(len(vals) - 1) // 2]
                    cm_all[f, m * units_per_module + ur * (C // UC) + uc] = cm
                    for r in range(ur * UR, (ur + 1) * UR):
                        for c in range(uc * UC, (uc + 1) * UC):
                            e[r][c] = (d[r][c] - cm) * inv[m, r, c]
            s = [[e[r][c] if e[r][c] > z else F32(0.0) for c in range(C)] for r in range(R)]
            for r in range(R):
                for c in range(C):
                    px = (m * R + r) * C + c
                    corr[f, px] = e[r][c]
                    hp[_bin(e[r][c], lo, w, bins)] += 1
            for r in range(R):
                for c in range(C):
                    sp = s[r][c]
                    if not sp > seed_t:
                        continue
                    nb, ok = [], True
                    for dr in (-1, 0, 1):
                        for dc in (-1, 0, 1):
                            rr, cc = r + dr, c + dc
                            q = s[rr][cc] if 0 <= rr < R and 0 <= cc < C else F32(0.0)
                            nb.append((dr, dc, q))
                            if (dr, dc) == (0, 0):
                                continue
                            earlier = dr < 0 or (dr == 0 and dc < 0)
                            if (earlier and not sp > q) or (not earlier and not sp >= q):
                                ok = False
                    if not ok:
                        continue
                    E = Mx = My = F32(0.0)
                    npix = 0
                    for dr, dc, q in nb:
                        E = E + q
                        Mx = Mx + q * F32(dc)
                        My = My + q * F32(dr)
                        npix += q > 0
                    hh[_bin(E, lo, w, bins)] += 1
                    qr = np.rint(E / ph)
                    flags = 0
                    if not qr >= 0:
                        cnt = 0
                    elif qr > 255:
                        cnt, flags = 255, flags | oracle.HIT_SATURATED
                    else:
                        cnt = int(qr)
                    if cnt < 1:
                        continue
                    if r in (0, R - 1) or c in (0, C - 1):
                        flags |= oracle.HIT_EDGE
                    px = (m * R + r) * C + c
                    cmap[px] += cnt
                    hits.add((f, px, F32(E).tobytes(), F32(Mx / E).tobytes(),
                              F32(My / E).tobytes(), cnt, npix, flags))
    return hits, cm_all, corr, cmap, hp, hh


def _oracle_set(res):
    return {(int(h["frame"]), int(h["pixel"]), F32(h["energy_kev"]).tobytes(),
             F32(h["dx"]).tobytes(), F32(h["dy"]).tobytes(), int(h["count"]),
             int(h["npix"]), int(h["flags"])) for h in res.hits[:res.n_hits]}


def _frames(rng, geom, n, integer):
    """ped, gain, raw for n frames: noisy pedestals with common-mode offsets
    per unit and frame and a few photons (charge over a 2 x 2 or 3 x 3 spot);
    integer=True: small integers throughout and unit gains (ties)."""
    M, R, C = geom["n_modules"], geom["rows"], geom["cols"]
    UR, UC = geom["unit_rows"], geom["unit_cols"]
    if integer:
        ped = rng.integers(95, 106, (M, R, C)).astype(F32)
        gain = np.ones((M, R, C), F32)
    else:
        ped = (1500 + 40 * rng.standard_normal((M, R, C))).astype(F32)
        gain = (25 * (1 + 0.03 * rng.standard_normal((M, R, C)))).astype(F32)
        gain.reshape(-1)[rng.integers(0, gain.size)] = 0.0  # a masked pixel
    raw = np.zeros((n, M, R, C), np.float64)
    for f in range(n):
        off = np.zeros((M, R, C))
        for ur in range(R // UR):
            for uc in range(C // UC):
                off[:, ur * UR:(ur + 1) * UR, uc * UC:(uc + 1) * UC] = (
                    rng.integers(-4, 5, (M, 1, 1)) if integer else 15 * rng.standard_normal((M, 1, 1)))
        noise = rng.integers(-1, 2, (M, R, C)) if integer else 4 * rng.standard_normal((M, R, C))
        sig = np.zeros((M, R, C))
        for _ in range(rng.integers(1, 4) * M):
            m, r, c = rng.integers(0, M), rng.integers(0, R), rng.integers(0, C)
            k = int(rng.integers(2, 4))
            amp = rng.integers(3, 9) if integer else 25 * 8 * rng.uniform(0.5, 3.0)
            sig[m, r:r + k, c:c + k] += amp if integer else amp / (k * k) * rng.uniform(0.2, 1.8, sig[m, r:r + k, c:c + k].shape)
        raw[f] = ped + off + noise + sig
    return ped, gain, np.clip(np.rint(raw), 0, 65535).astype(np.uint16)


GEOMS = {
    "two_modules_banks_8x4": dict(n_modules=2, rows=8, cols=8, unit_rows=8, unit_cols=4),
    "rows_of_8": dict(n_modules=1, rows=8, cols=8, unit_rows=1, unit_cols=8),
    "three_modules_2x4_units": dict(n_modules=3, rows=4, cols=8, unit_rows=2, unit_cols=4),
    "one_unit_8x8": dict(n_modules=1, rows=8, cols=8, unit_rows=8, unit_cols=8),
}


@pytest.mark.parametrize("integer", [False, True], ids=["noisy", "integer_ties"])
@pytest.mark.parametrize("name", list(GEOMS))
def test_restated_chain_equals_oracle(name, integer):
    geom = GEOMS[name]
    rng = np.random.default_rng(abs(hash((name, integer))) % (2 ** 32))
    if integer:
        thr = dict(cm_cut_adu=6.0, zero_thr_kev=1.0, seed_thr_kev=2.0, photon_kev=4.0,
                   hist_lo_kev=-16.0, hist_bin_kev=0.5, hist_bins=96)
    else:
        thr = dict(cm_cut_adu=200.0, zero_thr_kev=0.8, seed_thr_kev=0.8, photon_kev=8.0,
                   hist_lo_kev=-4.0, hist_bin_kev=0.05, hist_bins=1296)
    n_frames = 13  # 13 frames x 4 geometries x 2 kinds: over a hundred frames
    ped, gain, raw = _frames(rng, geom, n_frames, integer)
    hits, cm, corr, cmap, hp, hh = restated_chain(geom, thr, ped, gain, raw)
    res = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         want_corrected=True)
    assert len(hits) > 0
    assert _oracle_set(res) == hits
    assert res.n_hits == len(hits)
    assert res.cm.reshape(n_frames, -1).tobytes() == cm.tobytes()
    assert res.corrected.reshape(n_frames, -1).tobytes() == corr.tobytes()
    np.testing.assert_array_equal(res.count_map, cmap.astype(np.uint32))
    np.testing.assert_array_equal(res.hist_pix, hp)
    np.testing.assert_array_equal(res.hist_hit, hh)


def test_restated_chain_catches_a_planted_tie_rule_mistake():
    """The comparison above would see a tie rule with >= for earlier
    neighbours: on integer frames it accepts extra seeds."""
    geom = GEOMS["one_unit_8x8"]
    rng = np.random.default_rng(7)
    thr = dict(cm_cut_adu=6.0, zero_thr_kev=1.0, seed_thr_kev=2.0, photon_kev=4.0,
               hist_lo_kev=-16.0, hist_bin_kev=0.5, hist_bins=96)
    ped, gain, raw = _frames(rng, geom, 13, True)
    res = oracle.process(oracle.geometry(**geom), oracle.thresholds(**thr), ped, gain, raw,
                         want_corrected=True)
    # count tied local maxima: with a symmetric rule both of a tied pair seed
    corr = res.corrected.reshape(13, 8, 8)
    s = np.where(corr > F32(1.0), corr, F32(0.0))
    sym = 0
    for f in range(13):
        for r in range(8):
            for c in range(8):
                sp = s[f, r, c]
                if not sp > F32(2.0):
                    continue
                nb = [s[f, rr, cc] for rr in range(max(r - 1, 0), min(r + 2, 8))
                      for cc in range(max(c - 1, 0), min(c + 2, 8)) if (rr, cc) != (r, c)]
                sym += all(sp >= q for q in nb)
    assert sym > res.n_seeds  # ties exist, so the two rules differ on these frames
