"""Seeded synthetic detector frames with ground truth (input generator).

This module models what a detector records — pedestal, per-unit common-mode
offset, Gaussian noise and photons whose charge cloud spreads over a 3x3
neighbourhood — and nothing of the correction chain.  The CPU oracle and the
CUDA path both take their inputs from here.  The C source (``synth.c``) holds
the generator; this file compiles it with gcc and wraps it with ctypes.

Workload recipes (see ``PRESETS``) follow the detector shapes the paper
names: an ePix100 module of 704x768 pixels (section "Methods"), the 2.2
Mpixel CSPAD (section "Introduction"), laid out as 32 sensors of 185x388 with
common mode per 185x194 bank, and a single 352x384 ASIC.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libpdsynth.so")
_lock = threading.Lock()
_lib = None


class PsConfig(ctypes.Structure):
    _fields_ = [
        ("n_modules", ctypes.c_uint32), ("rows", ctypes.c_uint32),
        ("cols", ctypes.c_uint32), ("unit_rows", ctypes.c_uint32),
        ("unit_cols", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
        ("ped_mean", ctypes.c_double), ("ped_sigma", ctypes.c_double),
        ("gain_mean", ctypes.c_double), ("gain_sigma", ctypes.c_double),
        ("adu_per_kev", ctypes.c_double), ("noise_sigma", ctypes.c_double),
        ("cm_sigma", ctypes.c_double), ("occ_lo", ctypes.c_double),
        ("occ_hi", ctypes.c_double), ("photon_kev", ctypes.c_double),
        ("cloud_lo", ctypes.c_double), ("cloud_hi", ctypes.c_double),
        ("multi_frac", ctypes.c_double), ("seed", ctypes.c_uint64),
    ]


PHOTON_DTYPE = np.dtype([("frame", "<u4"), ("module", "<u4"), ("x", "<f4"),
                         ("y", "<f4"), ("kev", "<f4"), ("sigma", "<f4")])


def build(force: bool = False) -> str:
    """Compile libpdsynth.so next to its source (gcc, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or \
                os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared",
                                   "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.ps_maps.argtypes = [ctypes.POINTER(PsConfig), ctypes.c_void_p,
                                ctypes.c_void_p]
        lib.ps_maps.restype = ctypes.c_int
        lib.ps_frames.argtypes = [ctypes.POINTER(PsConfig), ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_longlong]
        lib.ps_frames.restype = ctypes.c_longlong
        lib.ps_frame_occupancy.argtypes = [ctypes.POINTER(PsConfig),
                                           ctypes.c_uint32]
        lib.ps_frame_occupancy.restype = ctypes.c_double
        _lib = lib
    return _lib


@dataclasses.dataclass
class Detector:
    """A synthetic workload: geometry plus the physics of the recorded data."""
    n_modules: int = 1
    rows: int = 352
    cols: int = 384
    unit_rows: int = 1
    unit_cols: int = 384
    ped_mean: float = 1500.0
    ped_sigma: float = 40.0
    gain_mean: float = 1.0
    gain_sigma: float = 0.03
    adu_per_kev: float = 25.0
    noise_sigma: float = 4.0
    cm_sigma: float = 15.0
    occupancy: float = 0.01
    occupancy_hi: float = 0.0     # > occupancy: log-uniform per frame
    photon_kev: float = 8.0
    cloud_sigma: float = 0.3
    cloud_sigma_hi: float = 0.0   # > cloud_sigma: uniform per photon
    multi_frac: float = 0.0
    seed: int = 1

    @property
    def pixels_per_frame(self) -> int:
        return self.n_modules * self.rows * self.cols

    @property
    def units_per_frame(self) -> int:
        return self.n_modules * (self.rows // self.unit_rows) * \
            (self.cols // self.unit_cols)

    @property
    def frame_shape(self):
        return (self.n_modules, self.rows, self.cols)

    def replace(self, **kw) -> "Detector":
        return dataclasses.replace(self, **kw)

    def _c(self) -> PsConfig:
        c = PsConfig()
        c.n_modules, c.rows, c.cols = self.n_modules, self.rows, self.cols
        c.unit_rows, c.unit_cols = self.unit_rows, self.unit_cols
        c.ped_mean, c.ped_sigma = self.ped_mean, self.ped_sigma
        c.gain_mean, c.gain_sigma = self.gain_mean, self.gain_sigma
        c.adu_per_kev, c.noise_sigma = self.adu_per_kev, self.noise_sigma
        c.cm_sigma = self.cm_sigma
        c.occ_lo, c.occ_hi = self.occupancy, self.occupancy_hi
        c.photon_kev = self.photon_kev
        c.cloud_lo, c.cloud_hi = self.cloud_sigma, self.cloud_sigma_hi
        c.multi_frac = self.multi_frac
        c.seed = self.seed
        return c

    # ---- default processing parameters for this workload -----------------
    def thresholds(self, n_sigma: float = 5.0) -> dict:
        """Thresholds in the units the chain uses (keV after gain)."""
        thr = n_sigma * self.noise_sigma / self.adu_per_kev
        return dict(cm_cut_adu=self.photon_kev * self.adu_per_kev,
                    zero_thr_kev=thr, seed_thr_kev=thr,
                    photon_kev=self.photon_kev, cm_min_count=0,
                    hist_lo_kev=-4.0, hist_bin_kev=0.05, hist_bins=1296,
                    cm_cut_kev=self.photon_kev)

    def geometry(self) -> dict:
        return dict(n_modules=self.n_modules, rows=self.rows, cols=self.cols,
                    unit_rows=self.unit_rows, unit_cols=self.unit_cols,
                    cm_mode=0, cm_after_gain=0)


def maps(det: Detector):
    """(pedestal ADU, gain ADU/keV) float32 maps [modules, rows, cols]."""
    lib = _load()
    ped = np.empty(det.frame_shape, np.float32)
    gain = np.empty(det.frame_shape, np.float32)
    c = det._c()
    if lib.ps_maps(ctypes.byref(c), ped.ctypes.data, gain.ctypes.data):
        raise ValueError("invalid detector geometry")
    return ped, gain


def frame_occupancy(det: Detector, frame: int) -> float:
    c = det._c()
    return float(_load().ps_frame_occupancy(ctypes.byref(c), frame))


def frames(det: Detector, ped: np.ndarray, gain: np.ndarray, first: int,
           n: int, *, truth: bool = True, cm_truth: bool = False,
           threads: int = 0, out: np.ndarray | None = None):
    """Raw frames uint16 [n, modules, rows, cols] for absolute frame indices
    first..first+n-1, the photons (structured array, PHOTON_DTYPE) and, if
    cm_truth, the injected common-mode offsets float64 [n, units].

    Generation runs in ``threads`` host threads (0 = all cores); each frame's
    content depends only on (seed, frame index)."""
    lib = _load()
    ped = np.ascontiguousarray(ped, np.float32)
    gain = np.ascontiguousarray(gain, np.float32)
    raw = out if out is not None else np.empty((n,) + det.frame_shape, np.uint16)
    assert raw.shape == (n,) + det.frame_shape and raw.dtype == np.uint16
    assert raw.flags["C_CONTIGUOUS"]
    cmo = np.empty((n, det.units_per_frame), np.float64) if cm_truth else None
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, n)) if n else 1
    bounds = np.linspace(0, n, threads + 1).astype(int)
    c = det._c()
    fpx = det.pixels_per_frame
    occ_max = max(det.occupancy, det.occupancy_hi)

    def work(i):
        a, b = int(bounds[i]), int(bounds[i + 1])
        if b <= a:
            return np.empty(0, PHOTON_DTYPE)
        cap = 0
        tr = None
        if truth:
            cap = int((b - a) * fpx * occ_max * 1.5 + 64 * (b - a) + 1024)
            if det.multi_frac > 0:
                cap *= 3
            tr = np.empty(cap, PHOTON_DTYPE)
        rawp = raw.ctypes.data + a * fpx * 2
        cmp_ = cmo.ctypes.data + a * det.units_per_frame * 8 if cm_truth else None
        cnt = lib.ps_frames(ctypes.byref(c), ped.ctypes.data, gain.ctypes.data,
                            first + a, b - a, rawp, cmp_,
                            tr.ctypes.data if truth else None, cap)
        if cnt < 0:
            raise ValueError("invalid detector geometry")
        if truth and cnt > cap:
            tr = np.empty(cnt, PHOTON_DTYPE)
            lib.ps_frames(ctypes.byref(c), ped.ctypes.data, gain.ctypes.data,
                          first + a, b - a, rawp, cmp_, tr.ctypes.data, cnt)
            return tr
        return tr[:cnt] if truth else None

    if threads == 1:
        parts = [work(0)]
    else:
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(work, range(threads)))
    ph = np.concatenate([p for p in parts if p is not None]) if truth else None
    if cm_truth:
        return raw, ph, cmo
    return raw, ph


# ---- workload presets: detector shapes of the paper ----------------------
def asic_352x384(**kw) -> Detector:
    """One 352x384 ASIC, common mode per 384-pixel row, 8 keV, 1 % occupancy."""
    return Detector(n_modules=1, rows=352, cols=384, unit_rows=1,
                    unit_cols=384, occupancy=0.01, photon_kev=8.0).replace(**kw)


def cspad_2p2m(**kw) -> Detector:
    """2.2 Mpixel CSPAD-like: 32 sensors of 185x388, common mode per 185x194
    bank, 8 keV, 0.5 % occupancy."""
    return Detector(n_modules=32, rows=185, cols=388, unit_rows=185,
                    unit_cols=194, occupancy=0.005,
                    photon_kev=8.0).replace(**kw)


def epix_704x768(**kw) -> Detector:
    """ePix100-sized module of 704x768 (4 ASICs of 352x384), common mode per
    384-pixel ASIC row, 6 keV."""
    return Detector(n_modules=1, rows=704, cols=768, unit_rows=1,
                    unit_cols=384, occupancy=0.01,
                    photon_kev=6.0).replace(**kw)


def asic16_352x384(**kw) -> Detector:
    """16 ASICs of 352x384 as separate modules, row common mode, 12 keV."""
    return Detector(n_modules=16, rows=352, cols=384, unit_rows=1,
                    unit_cols=384, occupancy=0.01,
                    photon_kev=12.0).replace(**kw)


PRESETS = {
    "asic_352x384": asic_352x384,
    "cspad_2p2m": cspad_2p2m,
    "epix_704x768": epix_704x768,
    "asic16_352x384": asic16_352x384,
}


# ---- auto-ranging detectors ---------------------------------------------
def multigain_maps(det: Detector, n_gains: int = 3,
                   ratios=(1.0, 1.0 / 3.0, 1.0 / 100.0),
                   ped_offsets=(0.0, -300.0, -700.0)):
    """Pedestal and gain maps of each gain stage, float32 [n_gains, modules,
    rows, cols]: stage 0 is ``maps(det)``; stage g has gain ratios[g] times
    stage 0's and its pedestal shifted by ped_offsets[g] ADU."""
    ped0, gain0 = maps(det)
    ped = np.stack([ped0 + np.float32(ped_offsets[g]) for g in range(n_gains)])
    gain = np.stack([gain0 * np.float32(ratios[g]) for g in range(n_gains)])
    return ped.astype(np.float32), gain.astype(np.float32)


def multigain_frames(det: Detector, ped: np.ndarray, gain: np.ndarray, first: int, n: int,
                     gain_shift: int = 14, blobs: int = 3, blob_kev: float = 3000.0,
                     bad_frac: float = 1e-4):
    """Raw words of an auto-ranging detector, uint16 [n, modules, rows, cols]:
    stage = word >> gain_shift, ADC value = word & (2^gain_shift - 1).

    Each frame is ``frames`` (noise, common mode, photons) at stage 0 plus
    ``blobs`` bright Gaussian spots per module of up to ``blob_kev`` keV per
    pixel.  A pixel whose stage-0 reading would pass 90 % of the ADC range
    switches to the next stage, which reads the same charge at its own gain
    and pedestal, with its own noise and no common mode; a few pixels carry
    an invalid stage (n_gains) to model corrupt words.  Returns (raw, the
    bright spots' deposited energy in keV per pixel as float32)."""
    n_gains = ped.shape[0]
    full = (1 << gain_shift) - 1
    raw0, _, cm = frames(det, ped[0], gain[0], first, n, truth=True, cm_truth=True)
    rng = np.random.default_rng((det.seed, first, n, 7))
    shape = raw0.shape
    R, C = det.rows, det.cols
    yy, xx = np.mgrid[0:R, 0:C]
    blob = np.zeros(shape, np.float64)
    for f in range(n):
        for m in range(det.n_modules):
            for _ in range(blobs):
                cy, cx = rng.uniform(0, R), rng.uniform(0, C)
                w = rng.uniform(1.5, 6.0)
                amp = rng.uniform(0.05, 1.0) * blob_kev
                blob[f, m] += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * w * w))
    # common mode per pixel from its unit
    upr = C // det.unit_cols
    cm_px = np.repeat(np.repeat(cm.reshape(n, det.n_modules, R // det.unit_rows, upr),
                                det.unit_rows, 2), det.unit_cols, 3)
    a0 = raw0.astype(np.float64) + blob * gain[0][None].astype(np.float64)
    # stage-0 signal in ADU without pedestal and common mode (noise included)
    sig0 = a0 - ped[0][None] - cm_px
    stage = np.zeros(shape, np.int64)
    val = a0
    limit = 0.9 * full
    for g in range(1, n_gains):
        up = val > limit
        if not up.any():
            break
        ag = ped[g][None] + sig0 * (gain[g] / gain[0])[None] + \
            rng.normal(0.0, det.noise_sigma, shape)
        stage = np.where(up, g, stage)
        val = np.where(up, ag, val)
    raw = (stage << gain_shift) | np.clip(np.rint(val), 0, full).astype(np.int64)
    if (n_gains << gain_shift) <= 0xFFFF:
        bad = rng.random(shape) < bad_frac
        raw = np.where(bad, (n_gains << gain_shift) | (raw & full), raw)
    return raw.astype(np.uint16), blob.astype(np.float32)
