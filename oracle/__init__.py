"""CPU oracle of the pixel-detector chain — TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  It shares no
code with the CUDA library (``paper_1903_06838_gb300``) and never imports it.

``pd_oracle.c`` states each step of the chain with its section of the paper
(Blaj, Chang, Kenney, AIP Conf. Proc. 2054, 060077, 2019); this module
compiles it with ``gcc -O2 -ffp-contract=off`` (IEEE binary32, no FMA
contraction) and wraps it with ctypes.  Parity pins: ``tests/test_oracle_*``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_LIB = os.path.join(_HERE, "libpdoracle.so")
_lock = threading.Lock()
_lib = None

HIT_DTYPE = np.dtype([("frame", "<u4"), ("pixel", "<u4"), ("energy_kev", "<f4"),
                      ("dx", "<f4"), ("dy", "<f4"), ("count", "u1"),
                      ("npix", "u1"), ("flags", "<u2")])
assert HIT_DTYPE.itemsize == 24

CM_MEDIAN, CM_NONE, CM_MEAN, CM_MEAN_STACKED = 0, 1, 2, 3
HIT_EDGE, HIT_SATURATED = 1, 2


MAX_FEATURES = 8


class Filters(ctypes.Structure):
    """Matched-filter bank: per feature 4 x 5 filters F0, F1, F1dx, F1dy and
    the threshold F1Nmin (Figs. d-f)."""
    _fields_ = [("n_features", ctypes.c_uint32),
                ("f0", ctypes.c_float * 20 * MAX_FEATURES),
                ("f1", ctypes.c_float * 20 * MAX_FEATURES),
                ("f1_dx", ctypes.c_float * 20 * MAX_FEATURES),
                ("f1_dy", ctypes.c_float * 20 * MAX_FEATURES),
                ("f1_nmin", ctypes.c_float * MAX_FEATURES)]


def filters(f0, f1, f1_dx, f1_dy, f1_nmin) -> Filters:
    """Bank from arrays [F][4][5] (and [F] thresholds)."""
    f0, f1, fdx, fdy = (np.asarray(a, np.float32).reshape(-1, 4, 5)
                        for a in (f0, f1, f1_dx, f1_dy))
    nmin = np.asarray(f1_nmin, np.float32).reshape(-1)
    nf = f1.shape[0]
    fb = Filters()
    fb.n_features = nf
    for name, a in (("f0", f0), ("f1", f1), ("f1_dx", fdx), ("f1_dy", fdy)):
        dst = np.zeros((MAX_FEATURES, 20), np.float32)
        dst[:nf] = a.reshape(nf, 20)
        ctypes.memmove(getattr(fb, name), dst.ctypes.data, dst.nbytes)
    dst = np.zeros(MAX_FEATURES, np.float32)
    dst[:nf] = nmin
    ctypes.memmove(fb.f1_nmin, dst.ctypes.data, dst.nbytes)
    return fb


class Geometry(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("n_modules", "rows", "cols", "unit_rows", "unit_cols",
                 "cm_mode", "cm_after_gain")]


class Thresholds(ctypes.Structure):
    _fields_ = [("cm_cut_adu", ctypes.c_float), ("zero_thr_kev", ctypes.c_float),
                ("seed_thr_kev", ctypes.c_float), ("photon_kev", ctypes.c_float),
                ("cm_min_count", ctypes.c_uint32),
                ("hist_lo_kev", ctypes.c_float), ("hist_bin_kev", ctypes.c_float),
                ("hist_bins", ctypes.c_uint32), ("cm_cut_kev", ctypes.c_float)]


def build(force: bool = False) -> str:
    """Compile libpdoracle.so next to its source."""
    with _lock:
        if force or not os.path.exists(_LIB) or \
                os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared",
                                   "-ffp-contract=off", "-fno-fast-math",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.oracle_process.argtypes = [
            ctypes.POINTER(Geometry), ctypes.POINTER(Thresholds), vp, vp, vp,
            ctypes.c_uint32, ctypes.c_uint32, vp, ctypes.c_uint32, vp, vp, vp,
            vp, vp, vp, vp]
        lib.oracle_process.restype = ctypes.c_int
        lib.oracle_process_matched.argtypes = [
            ctypes.POINTER(Geometry), ctypes.POINTER(Thresholds), ctypes.POINTER(Filters),
            vp, vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp, ctypes.c_uint32, vp, vp, vp,
            vp, vp, vp, vp]
        lib.oracle_process_matched.restype = ctypes.c_int
        lib.oracle_process_ext.argtypes = [
            ctypes.POINTER(Geometry), ctypes.POINTER(Thresholds), ctypes.POINTER(Filters),
            ctypes.c_uint32, ctypes.c_uint32,
            vp, vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp, ctypes.c_uint32, vp, vp, vp,
            vp, vp, vp, vp]
        lib.oracle_process_ext.restype = ctypes.c_int
        lib.oracle_lower_median.argtypes = [vp, ctypes.c_uint32]
        lib.oracle_lower_median.restype = ctypes.c_float
        lib.oracle_default_min_count.argtypes = [ctypes.c_uint32]
        lib.oracle_default_min_count.restype = ctypes.c_uint32
        lib.oracle_paper_mean.argtypes = [vp, ctypes.c_uint32, ctypes.c_float]
        lib.oracle_paper_mean.restype = ctypes.c_float
        lib.oracle_cm_values_per_frame.argtypes = [ctypes.POINTER(Geometry)]
        lib.oracle_cm_values_per_frame.restype = ctypes.c_uint32
        _lib = lib
    return _lib


def geometry(n_modules, rows, cols, unit_rows, unit_cols, cm_mode=CM_MEDIAN,
             cm_after_gain=0):
    """cm_after_gain = 1: the paper's order, gain before common mode."""
    return Geometry(n_modules, rows, cols, unit_rows, unit_cols, cm_mode, cm_after_gain)


def thresholds(cm_cut_adu, zero_thr_kev, seed_thr_kev, photon_kev,
               cm_min_count=0, hist_lo_kev=-4.0, hist_bin_kev=0.05,
               hist_bins=1296, cm_cut_kev=None):
    """cm_cut_kev: the common-mode cut in the paper's order (default: the
    photon energy, as cm_cut_adu defaults to it in ADU)."""
    return Thresholds(cm_cut_adu, zero_thr_kev, seed_thr_kev, photon_kev,
                      cm_min_count, hist_lo_kev, hist_bin_kev, hist_bins,
                      photon_kev if cm_cut_kev is None else cm_cut_kev)


def lower_median(values) -> np.float32:
    v = np.array(values, np.float32)
    if v.size == 0:
        raise ValueError("empty set")
    return np.float32(_load().oracle_lower_median(v.ctypes.data, v.size))


def default_min_count(unit_pixels: int) -> int:
    return int(_load().oracle_default_min_count(unit_pixels))


def paper_mean(values, cut) -> np.float32:
    """The paper's common-mode estimator (Fig. c) over one group of values."""
    v = np.ascontiguousarray(values, np.float32)
    return np.float32(_load().oracle_paper_mean(v.ctypes.data, v.size, np.float32(cut)))


def cm_values_per_frame(geom: Geometry) -> int:
    """Common-mode values per frame: units, then (stacked) module rows and
    module columns."""
    return int(_load().oracle_cm_values_per_frame(ctypes.byref(geom)))


class Result:
    """Outputs of one oracle run (hits in frame, module, row, col order)."""

    def __init__(self, hits, n_hits, n_seeds, count_map, hist_pix, hist_hit,
                 corrected, cm):
        self.hits, self.n_hits, self.n_seeds = hits, n_hits, n_seeds
        self.count_map, self.hist_pix, self.hist_hit = count_map, hist_pix, hist_hit
        self.corrected, self.cm = corrected, cm


def process(geom: Geometry, thr: Thresholds, ped, gain, raw, *, frame_base=0,
            want_corrected=False, want_cm=True, hit_capacity=None,
            count_map=None, hist_pix=None, hist_hit=None, filters=None,
            n_gains=0, gain_shift=0) -> Result:
    """Run the oracle.  raw: uint16 [n, modules, rows, cols] (or flat).
    filters: a Filters bank selects the matched-filter charge summing.
    n_gains > 0: auto-ranging words (stage = raw >> gain_shift) with ped and
    gain holding one map per stage, [n_gains, modules, rows, cols]."""
    lib = _load()
    ped = np.ascontiguousarray(ped, np.float32).reshape(-1)
    gain = np.ascontiguousarray(gain, np.float32).reshape(-1)
    fpx = geom.n_modules * geom.rows * geom.cols
    raw = np.ascontiguousarray(raw, np.uint16).reshape(-1)
    stages = n_gains or 1
    assert raw.size % fpx == 0 and ped.size == stages * fpx and gain.size == stages * fpx
    n = raw.size // fpx
    upf = cm_values_per_frame(geom)
    cap = hit_capacity if hit_capacity is not None else max(1024, n * fpx // 8)
    hits = np.zeros(cap, HIT_DTYPE)
    nh = ctypes.c_uint32(0)
    ns = ctypes.c_uint64(0)
    cmap = count_map if count_map is not None else np.zeros(fpx, np.uint32)
    hp = hist_pix if hist_pix is not None else np.zeros(thr.hist_bins, np.uint64)
    hh = hist_hit if hist_hit is not None else np.zeros(thr.hist_bins, np.uint64)
    corr = np.zeros((n, fpx), np.float32) if want_corrected else None
    cm = np.zeros((n, upf), np.float32) if want_cm else None
    rest = (ped.ctypes.data, gain.ctypes.data, raw.ctypes.data, n, frame_base,
            hits.ctypes.data, cap, ctypes.byref(nh), cmap.ctypes.data, hp.ctypes.data,
            hh.ctypes.data, corr.ctypes.data if corr is not None else None,
            cm.ctypes.data if cm is not None else None, ctypes.byref(ns))
    if n_gains:
        rc = lib.oracle_process_ext(ctypes.byref(geom), ctypes.byref(thr),
                                    ctypes.byref(filters) if filters is not None else None,
                                    n_gains, gain_shift, *rest)
    elif filters is None:
        rc = lib.oracle_process(ctypes.byref(geom), ctypes.byref(thr), *rest)
    else:
        rc = lib.oracle_process_matched(ctypes.byref(geom), ctypes.byref(thr),
                                        ctypes.byref(filters), *rest)
    if rc:
        raise ValueError("oracle rejected the geometry or thresholds")
    k = min(nh.value, cap)
    return Result(hits[:k].copy(), nh.value, ns.value, cmap, hp, hh, corr, cm)
