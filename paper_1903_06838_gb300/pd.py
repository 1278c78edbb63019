"""Thin Python binding of libpd (include/pd.h), with the same entry names.

Only argument marshalling happens here: every step of the chain runs in the
CUDA kernels of ``csrc/``.  PyTorch supplies device memory and streams.  If
the compiled library cannot be loaded the binding raises; there is no CPU
path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(_PKG, "libpd.so")
SOURCES = ["pd_api.cu", "pd_chain.cu", "pd_cm_mean.cu", "pd_eta.cu", "pd_fast.cu",
           "pd_fused.cu", "pd_lean.cu", "pd_matched.cu", "pd_noalloc.cu", "pd_net.cu", "pd_net_tc.cu",
           "pd_serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--fmad=false",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "-Xptxas", "-warn-spills"]

_lock = threading.Lock()
_lib = None

# ---- public constants (mirror include/pd.h) -------------------------------
PD_OK, PD_EINVAL, PD_EALIGN, PD_ENOMEM, PD_EOVERFLOW = 0, 1, 2, 3, 4
PD_ETIMEDOUT, PD_ECUDA, PD_ENOTSUP, PD_EBUSY = 5, 6, 7, 8
PD_CM_MEDIAN, PD_CM_NONE, PD_CM_MEAN, PD_CM_MEAN_STACKED = 0, 1, 2, 3
PD_HIT_EDGE, PD_HIT_SATURATED, PD_HIT_LEARNED, PD_HIT_LINEARISED = 1, 2, 4, 8
PD_MAX_ETA_BINS = 4095
PD_MAX_HIST_BINS = 4096

HIT_DTYPE = np.dtype([("frame", "<u4"), ("pixel", "<u4"), ("energy_kev", "<f4"),
                      ("dx", "<f4"), ("dy", "<f4"), ("count", "u1"),
                      ("npix", "u1"), ("flags", "<u2")])
assert HIT_DTYPE.itemsize == 24


PD_MAX_FEATURES = 8
PD_MAX_GAINS = 4


class PdFilterBank(ctypes.Structure):
    _fields_ = [("n_features", ctypes.c_uint32),
                ("f0", ctypes.c_float * 20 * PD_MAX_FEATURES),
                ("f1", ctypes.c_float * 20 * PD_MAX_FEATURES),
                ("f1_dx", ctypes.c_float * 20 * PD_MAX_FEATURES),
                ("f1_dy", ctypes.c_float * 20 * PD_MAX_FEATURES),
                ("f1_nmin", ctypes.c_float * PD_MAX_FEATURES)]


class PdGeometry(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("n_modules", "rows", "cols", "unit_rows", "unit_cols",
                 "cm_mode", "cm_after_gain")]


class PdThresholds(ctypes.Structure):
    _fields_ = [("cm_cut_adu", ctypes.c_float), ("zero_thr_kev", ctypes.c_float),
                ("seed_thr_kev", ctypes.c_float), ("photon_kev", ctypes.c_float),
                ("cm_min_count", ctypes.c_uint32),
                ("hist_lo_kev", ctypes.c_float), ("hist_bin_kev", ctypes.c_float),
                ("hist_bins", ctypes.c_uint32), ("cm_cut_kev", ctypes.c_float)]


class PdOutputs(ctypes.Structure):
    _fields_ = [("hits", ctypes.c_void_p), ("hit_capacity", ctypes.c_uint32),
                ("n_hits", ctypes.c_void_p), ("corrected", ctypes.c_void_p),
                ("cm", ctypes.c_void_p)]


class PdInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("pixels_per_frame", "units_per_frame", "unit_pixels",
                 "cm_min_count", "hist_bins", "masked_pixels", "cm_values_per_frame")]


class PdProfile(ctypes.Structure):
    _fields_ = [("n_kernels", ctypes.c_uint32),
                ("name", (ctypes.c_char * 32) * 8),
                ("launches", ctypes.c_uint32 * 8),
                ("total_ms", ctypes.c_double * 8)]


class PdTuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("chunk_frames", "band_rows", "overlap", "two_pass", "kernels")]


class PdBatchItem(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("frames", ctypes.c_void_p),
                ("n_frames", ctypes.c_uint32), ("frame_base", ctypes.c_uint32),
                ("out", PdOutputs)]


class PdServeConfig(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_uint32), ("max_batch_frames", ctypes.c_uint32),
                ("ring_frames", ctypes.c_uint32), ("hits_per_frame", ctypes.c_uint32),
                ("device_budget", ctypes.c_uint64), ("keep_hits", ctypes.c_uint32),
                ("encode_threads", ctypes.c_uint32), ("max_uploading", ctypes.c_uint32),
                ("cpu_pin", ctypes.c_uint32)]


class PdServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("frames_committed", "frames_done", "frames_rejected", "batches",
                 "max_batch_frames", "raw_bytes", "compressed_bytes", "hits")] + \
               [(n, ctypes.c_double) for n in
                ("elapsed_s", "p50_us", "p99_us", "max_us", "mean_us", "wait_mean_us",
                 "wait_p99_us", "device_mean_us", "device_p99_us", "fetch_mean_us",
                 "encode_mean_us")] + \
               [("replay_late", ctypes.c_uint64)] + \
               [(n, ctypes.c_double) for n in
                ("replay_late_max_us", "upload_mean_us", "run_mean_us")]


class PdError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        lib = _lib
        detail = lib.pd_last_error().decode() if lib is not None else ""
        name = lib.pd_strerror(code).decode() if lib is not None else str(code)
        super().__init__(f"{where}: {name} ({code}): {detail}")


# ---- build & load ----------------------------------------------------------
def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC)]
    deps += [os.path.join(_INCLUDE, f) for f in os.listdir(_INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libpd.so in-tree for sm_103a (translation units in parallel)."""
    with _lock:
        if not force and not _stale():
            return LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        procs, objs = [], []
        for src in SOURCES:
            obj = os.path.join(_BUILD, src.replace(".cu", ".o"))
            objs.append(obj)
            cmd = ["nvcc", *ARCH, *NVCC_FLAGS, "-I", _INCLUDE, "-I", _CSRC,
                   "-c", os.path.join(_CSRC, src), "-o", obj]
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT)))
        for cmd, pr in procs:
            out, _ = pr.communicate()
            if pr.returncode:
                raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" +
                                   out.decode(errors="replace"))
            if verbose and out:
                print(out.decode(errors="replace"))
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["nvcc", *ARCH, "-shared", "-o", tmp, *objs,
                               "-lcudart"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _declare(lib):
    vp, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
    sig = {
        "pd_create": ([ctypes.POINTER(PdGeometry), vp, vp,
                       ctypes.POINTER(PdThresholds), ctypes.POINTER(vp)], i32),
        "pd_create_multigain": ([ctypes.POINTER(PdGeometry), u32, u32, vp, vp,
                                 ctypes.POINTER(PdThresholds), ctypes.POINTER(vp)], i32),
        "pd_query": ([vp, ctypes.POINTER(PdInfo)], i32),
        "pd_process": ([vp, vp, u32, u32, ctypes.POINTER(PdOutputs), vp], i32),
        "pd_process_noalloc": ([vp, vp, u32, u32, ctypes.POINTER(PdOutputs), vp], i32),
        "pd_process_host": ([vp, vp, u32, u32, vp, u32,
                             ctypes.POINTER(u32)], i32),
        "pd_get_summary": ([vp, vp, vp, vp, vp], i32),
        "pd_reset_summary": ([vp, vp], i32),
        "pd_set_filter_bank": ([vp, vp], i32),
        "pd_destroy": ([vp], None),
        "pd_set_profiling": ([vp, i32], i32),
        "pd_autotune": ([vp, vp, u32, ctypes.POINTER(PdTuning),
                         ctypes.POINTER(ctypes.c_float)], i32),
        "pd_batch_create": ([u32, ctypes.c_uint64, ctypes.POINTER(vp)], i32),
        "pd_batch_process": ([vp, ctypes.POINTER(PdBatchItem), u32, vp], i32),
        "pd_batch_capture": ([vp, ctypes.POINTER(PdBatchItem), u32, vp], i32),
        "pd_batch_replay": ([vp, vp], i32),
        "pd_batch_set_mixed": ([vp, i32], i32),
        "pd_batch_destroy": ([vp], None),
        "pd_server_create": ([ctypes.POINTER(vp), u32, ctypes.POINTER(PdServeConfig),
                              ctypes.POINTER(vp)], i32),
        "pd_server_slots": ([vp, ctypes.POINTER(u32)], i32),
        "pd_server_hold": ([vp, i32], i32),
        "pd_server_ring_frame": ([vp, u32, u32, ctypes.POINTER(vp)], i32),
        "pd_server_acquire": ([vp, u32, ctypes.POINTER(vp), ctypes.POINTER(u32)], i32),
        "pd_server_commit": ([vp, u32, u32, ctypes.c_uint64], i32),
        "pd_server_replay": ([vp, ctypes.c_double, ctypes.c_double, vp, ctypes.c_uint64,
                              ctypes.c_uint64], i32),
        "pd_server_drain": ([vp, ctypes.c_double], i32),
        "pd_server_stats": ([vp, ctypes.POINTER(PdServeStats)], i32),
        "pd_server_reset_stats": ([vp], i32),
        "pd_server_frame_hits": ([vp, ctypes.c_uint64, vp, u32, ctypes.POINTER(u32),
                                  ctypes.POINTER(ctypes.c_float)], i32),
        "pd_server_frame_stream": ([vp, ctypes.c_uint64, vp, ctypes.c_size_t,
                                    ctypes.POINTER(ctypes.c_size_t)], i32),
        "pd_server_destroy": ([vp], None),
        "pd_compress_hits": ([vp, u32, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], i32),
        "pd_decompress_hits": ([vp, ctypes.c_size_t, u32, vp, u32, ctypes.POINTER(u32)], i32),
        "pd_eta_create": ([u32, ctypes.POINTER(vp)], i32),
        "pd_eta_accumulate": ([vp, vp, u32, vp], i32),
        "pd_eta_finalize": ([vp, vp], i32),
        "pd_eta_apply": ([vp, vp, u32, vp, vp], i32),
        "pd_eta_get_histogram": ([vp, vp], i32),
        "pd_eta_reset": ([vp, vp], i32),
        "pd_eta_destroy": ([vp], None),
        "pd_net_num_params": ([], u32),
        "pd_net_create": ([u32, ctypes.c_uint64, ctypes.POINTER(vp)], i32),
        "pd_net_set_params": ([vp, vp, u32], i32),
        "pd_net_get_params": ([vp, vp, u32], i32),
        "pd_net_gather": ([vp, vp, u32, vp, vp, u32, vp, vp], i32),
        "pd_net_forward": ([vp, vp, u32, vp, vp], i32),
        "pd_net_gradients": ([vp, vp, vp, vp, vp, u32, ctypes.c_float, ctypes.c_float, vp, vp,
                              vp], i32),
        "pd_net_take": ([vp, vp, vp, vp, vp, u32, vp, vp, vp, vp, vp], i32),
        "pd_net_train_step": ([vp, vp, vp, vp, vp, u32, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, vp, vp], i32),
        "pd_net_refine": ([vp, vp, u32, ctypes.c_float, ctypes.c_float, vp, vp], i32),
        "pd_net_destroy": ([vp], None),
        "pd_get_tuning": ([vp, ctypes.POINTER(PdTuning)], i32),
        "pd_set_tuning": ([vp, ctypes.POINTER(PdTuning)], i32),
        "pd_set_wait_limit": ([vp, u32], i32),
        "pd_read_profile": ([vp, ctypes.POINTER(PdProfile)], i32),
        "pd_strerror": ([i32], ctypes.c_char_p),
        "pd_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


def load(build_if_missing: bool = True):
    """Load libpd.so (building it first if needed).  Raises if unavailable."""
    global _lib
    if _lib is None:
        with _lock:
            pass
        if build_if_missing:
            build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpd is not built ({LIB_PATH})")
        lib = ctypes.CDLL(LIB_PATH)
        _declare(lib)
        _lib = lib
    return _lib


def exported_symbols():
    """Names the shared object exports (read from its dynamic symbol table)."""
    out = subprocess.check_output(["nm", "-D", "--defined-only", LIB_PATH])
    return {ln.split()[-1] for ln in out.decode().splitlines() if ln.strip()}


def _check(rc, where):
    if rc != PD_OK:
        raise PdError(rc, where)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- context ----------------------------------------------------------------
class Context:
    """Owns one pd_ctx (device maps and summaries)."""

    def __init__(self, handle, geometry: PdGeometry, thresholds: PdThresholds):
        self.handle = handle
        self.geometry = geometry
        self.thresholds = thresholds
        self.info = pd_query(self)

    @property
    def pixels_per_frame(self) -> int:
        return self.info.pixels_per_frame

    @property
    def units_per_frame(self) -> int:
        return self.info.units_per_frame

    @property
    def cm_values_per_frame(self) -> int:
        return self.info.cm_values_per_frame

    def close(self):
        if self.handle:
            pd_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_geometry(n_modules, rows, cols, unit_rows, unit_cols,
                  cm_mode=PD_CM_MEDIAN, cm_after_gain=0) -> PdGeometry:
    """cm_after_gain = 1: the paper's order, gain before common mode."""
    return PdGeometry(n_modules, rows, cols, unit_rows, unit_cols, cm_mode, cm_after_gain)


def make_thresholds(cm_cut_adu, zero_thr_kev, seed_thr_kev, photon_kev,
                    cm_min_count=0, hist_lo_kev=-4.0, hist_bin_kev=0.05,
                    hist_bins=1296, cm_cut_kev=None) -> PdThresholds:
    """cm_cut_kev: the common-mode cut in the paper's order (default: the
    photon energy)."""
    return PdThresholds(cm_cut_adu, zero_thr_kev, seed_thr_kev, photon_kev,
                        cm_min_count, hist_lo_kev, hist_bin_kev, hist_bins,
                        photon_kev if cm_cut_kev is None else cm_cut_kev)


def pd_create(geometry, pedestal, gain, thresholds, n_gains: int = 0,
              gain_shift: int = 0) -> Context:
    """geometry / thresholds: PdGeometry / PdThresholds or dicts of fields.
    n_gains > 0: an auto-ranging context (pd_create_multigain) whose
    pedestal and gain hold one map per stage."""
    lib = load()
    if isinstance(geometry, dict):
        geometry = make_geometry(**geometry)
    if isinstance(thresholds, dict):
        thresholds = make_thresholds(**thresholds)
    ped = np.ascontiguousarray(pedestal, np.float32).reshape(-1)
    gain = np.ascontiguousarray(gain, np.float32).reshape(-1)
    npx = geometry.n_modules * geometry.rows * geometry.cols * max(1, n_gains)
    if ped.size != npx or gain.size != npx:
        raise ValueError("pedestal/gain size does not match the geometry")
    h = ctypes.c_void_p()
    if n_gains:
        _check(lib.pd_create_multigain(ctypes.byref(geometry), n_gains, gain_shift,
                                       ped.ctypes.data, gain.ctypes.data,
                                       ctypes.byref(thresholds), ctypes.byref(h)),
               "pd_create_multigain")
        return Context(h.value, geometry, thresholds)
    _check(lib.pd_create(ctypes.byref(geometry), ped.ctypes.data,
                         gain.ctypes.data, ctypes.byref(thresholds),
                         ctypes.byref(h)), "pd_create")
    return Context(h.value, geometry, thresholds)


def pd_query(ctx: Context) -> PdInfo:
    info = PdInfo()
    _check(load().pd_query(ctx.handle, ctypes.byref(info)), "pd_query")
    return info


def pd_process(ctx: Context, frames_ptr: int, n_frames: int, frame_base: int,
               hits_ptr: int, hit_capacity: int, n_hits_ptr: int,
               corrected_ptr: int | None = None, cm_ptr: int | None = None,
               stream=None) -> None:
    """Enqueue the chain on device frames (raw device pointers)."""
    out = PdOutputs(hits_ptr, hit_capacity, n_hits_ptr, corrected_ptr, cm_ptr)
    _check(load().pd_process(ctx.handle, frames_ptr, n_frames, frame_base,
                             ctypes.byref(out), _stream_handle(stream)),
           "pd_process")


PD_NOALLOC_MAX_CM = 1 << 20


def pd_process_noalloc(ctx: Context, frames_ptr: int, n_frames: int, frame_base: int,
                       hits_ptr: int, hit_capacity: int, n_hits_ptr: int,
                       corrected_ptr: int | None = None, cm_ptr: int | None = None,
                       stream=None) -> None:
    """pd_process without device allocation (fixed in-library scratch)."""
    out = PdOutputs(hits_ptr, hit_capacity, n_hits_ptr, corrected_ptr, cm_ptr)
    _check(load().pd_process_noalloc(ctx.handle, frames_ptr, n_frames, frame_base,
                                     ctypes.byref(out), _stream_handle(stream)),
           "pd_process_noalloc")


def pd_process_host(ctx: Context, frames: np.ndarray, frame_base: int = 0,
                    hit_capacity: int | None = None, out: np.ndarray | None = None):
    """Chain on host frames (uint16 [n, ...]); returns (hits, n_hits).
    PD_EOVERFLOW is reported through n_hits > len(hits), not raised."""
    lib = load()
    fr = np.ascontiguousarray(frames)
    assert fr.dtype == np.uint16
    n = fr.size // ctx.pixels_per_frame
    assert n * ctx.pixels_per_frame == fr.size
    if out is None:
        cap = hit_capacity if hit_capacity is not None else \
            max(1024, n * ctx.pixels_per_frame // 16)
        out = np.empty(cap, HIT_DTYPE)
    nh = ctypes.c_uint32(0)
    rc = lib.pd_process_host(ctx.handle, fr.ctypes.data, n, frame_base,
                             out.ctypes.data, len(out), ctypes.byref(nh))
    if rc not in (PD_OK, PD_EOVERFLOW):
        raise PdError(rc, "pd_process_host")
    return out[:min(nh.value, len(out))], nh.value


def pd_get_summary(ctx: Context, stream=None):
    """(count_map u32 [pixels], hist_pix u64 [bins], hist_hit u64 [bins])."""
    cm = np.empty(ctx.pixels_per_frame, np.uint32)
    hp = np.empty(ctx.info.hist_bins, np.uint64)
    hh = np.empty(ctx.info.hist_bins, np.uint64)
    _check(load().pd_get_summary(ctx.handle, cm.ctypes.data, hp.ctypes.data,
                                 hh.ctypes.data, _stream_handle(stream)),
           "pd_get_summary")
    return cm, hp, hh


def pd_set_filter_bank(ctx: Context, f0=None, f1=None, f1_dx=None, f1_dy=None,
                       f1_nmin=None) -> None:
    """Matched-filter charge summing with the bank of arrays [F][4][5] (and
    [F] thresholds); with no arrays the default 3x3 local maximum."""
    if f1 is None:
        _check(load().pd_set_filter_bank(ctx.handle, None), "pd_set_filter_bank")
        return
    arrs = [np.asarray(a, np.float32).reshape(-1, 4, 5) for a in (f0, f1, f1_dx, f1_dy)]
    nmin = np.asarray(f1_nmin, np.float32).reshape(-1)
    nf = arrs[1].shape[0]
    if nf > PD_MAX_FEATURES or any(a.shape[0] != nf for a in arrs) or nmin.size != nf:
        raise ValueError("filter bank arrays disagree in their feature count")
    fb = PdFilterBank()
    fb.n_features = nf
    for name, a in zip(("f0", "f1", "f1_dx", "f1_dy"), arrs):
        dst = np.zeros((PD_MAX_FEATURES, 20), np.float32)
        dst[:nf] = a.reshape(nf, 20)
        ctypes.memmove(getattr(fb, name), dst.ctypes.data, dst.nbytes)
    dst = np.zeros(PD_MAX_FEATURES, np.float32)
    dst[:nf] = nmin
    ctypes.memmove(fb.f1_nmin, dst.ctypes.data, dst.nbytes)
    _check(load().pd_set_filter_bank(ctx.handle, ctypes.byref(fb)), "pd_set_filter_bank")


def pd_reset_summary(ctx: Context, stream=None) -> None:
    _check(load().pd_reset_summary(ctx.handle, _stream_handle(stream)),
           "pd_reset_summary")


def pd_destroy(ctx: Context) -> None:
    if ctx.handle:
        load().pd_destroy(ctx.handle)
        ctx.handle = None


def pd_get_tuning(ctx: Context) -> dict:
    t = PdTuning()
    _check(load().pd_get_tuning(ctx.handle, ctypes.byref(t)), "pd_get_tuning")
    return dict(chunk_frames=t.chunk_frames, band_rows=t.band_rows,
                overlap=t.overlap, two_pass=t.two_pass, kernels=t.kernels)


def pd_set_wait_limit(ctx: Context, polls: int) -> None:
    """Polls of a bounded device wait before it gives up (0: the default)."""
    _check(load().pd_set_wait_limit(ctx.handle, polls), "pd_set_wait_limit")


def pd_set_tuning(ctx: Context, chunk_frames=0, band_rows=0, overlap=None,
                  two_pass=None, kernels=0) -> None:
    """Zero chunk_frames / band_rows / kernels and None overlap / two_pass
    keep the context's current values."""
    cur = pd_get_tuning(ctx)
    t = PdTuning(chunk_frames, band_rows, cur["overlap"] if overlap is None else overlap,
                 cur["two_pass"] if two_pass is None else two_pass, kernels)
    _check(load().pd_set_tuning(ctx.handle, ctypes.byref(t)), "pd_set_tuning")


def pd_set_profiling(ctx: Context, enable: bool) -> None:
    _check(load().pd_set_profiling(ctx.handle, int(bool(enable))),
           "pd_set_profiling")


def pd_read_profile(ctx: Context) -> dict:
    """{kernel name: (launches, total device ms)} since the last read."""
    pr = PdProfile()
    _check(load().pd_read_profile(ctx.handle, ctypes.byref(pr)),
           "pd_read_profile")
    return {pr.name[k].value.decode(): (pr.launches[k], pr.total_ms[k])
            for k in range(pr.n_kernels) if pr.launches[k]}


def pd_autotune(ctx: Context, frames_ptr: int, n_frames: int):
    """Time candidate tunings on device frames; apply and return the best
    as (tuning dict, microseconds per frame)."""
    t = PdTuning()
    us = ctypes.c_float(0)
    _check(load().pd_autotune(ctx.handle, frames_ptr, n_frames, ctypes.byref(t),
                              ctypes.byref(us)), "pd_autotune")
    return (dict(chunk_frames=t.chunk_frames, band_rows=t.band_rows,
                 overlap=t.overlap, two_pass=t.two_pass, kernels=t.kernels),
            float(us.value))


class Batch:
    """A pd_batch (device item table + scratch, optional captured graph)."""

    def __init__(self, max_items: int, max_cm_values: int = 1 << 22):
        h = ctypes.c_void_p()
        _check(load().pd_batch_create(max_items, max_cm_values, ctypes.byref(h)),
               "pd_batch_create")
        self.handle = h.value
        self._keep = None

    def close(self):
        if self.handle:
            load().pd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_items(items):
    """items: sequence of (ctx, frames_ptr, n_frames, frame_base, Outputs)."""
    arr = (PdBatchItem * len(items))()
    for k, (ctx, fptr, n, base, out) in enumerate(items):
        o = out.ptrs()
        arr[k] = PdBatchItem(ctx.handle, fptr, n, base,
                             PdOutputs(o["hits_ptr"], o["hit_capacity"], o["n_hits_ptr"],
                                       o["corrected_ptr"], o["cm_ptr"]))
    return arr


def pd_batch_create(max_items: int, max_cm_values: int = 1 << 22) -> Batch:
    return Batch(max_items, max_cm_values)


def pd_batch_process(batch: Batch, items, stream=None) -> None:
    arr = _batch_items(items)
    _check(load().pd_batch_process(batch.handle, arr, len(items), _stream_handle(stream)),
           "pd_batch_process")


def pd_batch_capture(batch: Batch, items, stream) -> None:
    arr = _batch_items(items)
    batch._keep = arr
    _check(load().pd_batch_capture(batch.handle, arr, len(items), _stream_handle(stream)),
           "pd_batch_capture")


def pd_batch_set_mixed(batch: Batch, mixed: bool) -> None:
    _check(load().pd_batch_set_mixed(batch.handle, int(bool(mixed))), "pd_batch_set_mixed")


def pd_batch_replay(batch: Batch, stream=None) -> None:
    _check(load().pd_batch_replay(batch.handle, _stream_handle(stream)), "pd_batch_replay")


def pd_batch_destroy(batch: Batch) -> None:
    batch.close()


# ---- learned refinement (device pointers; torch tensors for convenience) ----
class Net:
    def __init__(self, max_batch: int = 8192, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().pd_net_create(max_batch, seed, ctypes.byref(h)), "pd_net_create")
        self.handle = h.value
        self.max_batch = max_batch

    def close(self):
        if self.handle:
            load().pd_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_net_num_params() -> int:
    return int(load().pd_net_num_params())


def pd_net_create(max_batch: int = 8192, seed: int = 0) -> Net:
    return Net(max_batch, seed)


def pd_net_set_params(net: Net, params: np.ndarray) -> None:
    a = np.ascontiguousarray(params, np.float32)
    _check(load().pd_net_set_params(net.handle, a.ctypes.data, a.size), "pd_net_set_params")


def pd_net_get_params(net: Net) -> np.ndarray:
    a = np.empty(pd_net_num_params(), np.float32)
    _check(load().pd_net_get_params(net.handle, a.ctypes.data, a.size), "pd_net_get_params")
    return a


def pd_net_gather(ctx: Context, frames_ptr: int, frame_base: int, cm_ptr: int, hits_ptr: int,
                  n_hits: int, patches_ptr: int, stream=None) -> None:
    _check(load().pd_net_gather(ctx.handle, frames_ptr, frame_base, cm_ptr, hits_ptr, n_hits,
                                patches_ptr, _stream_handle(stream)), "pd_net_gather")


def pd_net_forward(net: Net, patches_ptr: int, n: int, out_ptr: int, stream=None) -> None:
    _check(load().pd_net_forward(net.handle, patches_ptr, n, out_ptr, _stream_handle(stream)),
           "pd_net_forward")


def pd_net_take(patches_ptr, counts_ptr, targets_ptr, mask_ptr, idx_ptr, n, p_out, c_out,
                t_out, m_out, stream=None) -> None:
    _check(load().pd_net_take(patches_ptr, counts_ptr, targets_ptr, mask_ptr, idx_ptr, n,
                              p_out, c_out, t_out, m_out, _stream_handle(stream)),
           "pd_net_take")


def pd_net_gradients(net: Net, patches_ptr, counts_ptr, targets_ptr, mask_ptr, n, n_reg,
                     lam, grads_ptr, loss_ptr, stream=None) -> None:
    _check(load().pd_net_gradients(net.handle, patches_ptr, counts_ptr, targets_ptr, mask_ptr,
                                   n, n_reg, lam, grads_ptr, loss_ptr,
                                   _stream_handle(stream)), "pd_net_gradients")


def pd_net_train_step(net: Net, patches_ptr, counts_ptr, targets_ptr, mask_ptr, n, n_reg,
                      lam, lr, loss_ptr, stream=None) -> None:
    _check(load().pd_net_train_step(net.handle, patches_ptr, counts_ptr, targets_ptr,
                                    mask_ptr, n, n_reg, lam, lr, loss_ptr,
                                    _stream_handle(stream)), "pd_net_train_step")


def pd_net_refine(out_ptr: int, hits_in_ptr: int, n: int, conf: float, count_conf: float,
                  hits_out_ptr: int, stream=None) -> None:
    _check(load().pd_net_refine(out_ptr, hits_in_ptr, n, conf, count_conf, hits_out_ptr,
                                _stream_handle(stream)), "pd_net_refine")


def pd_net_destroy(net: Net) -> None:
    net.close()


# ---- streaming server --------------------------------------------------------
class Server:
    def __init__(self, ctxs, n_slots=4, max_batch_frames=32, ring_frames=256,
                 hits_per_frame=16384, device_budget=0, keep_hits=False, encode_threads=0,
                 max_uploading=0, cpu_pin=0):
        arr = (ctypes.c_void_p * len(ctxs))(*[c.handle for c in ctxs])
        cfg = PdServeConfig(n_slots, max_batch_frames, ring_frames, hits_per_frame,
                            device_budget, int(keep_hits), encode_threads, max_uploading,
                            cpu_pin)
        h = ctypes.c_void_p()
        _check(load().pd_server_create(arr, len(ctxs), ctypes.byref(cfg), ctypes.byref(h)),
               "pd_server_create")
        self.handle = h.value
        self.ctxs = list(ctxs)
        self.ring_frames = ring_frames

    def slots(self) -> int:
        n = ctypes.c_uint32()
        _check(load().pd_server_slots(self.handle, ctypes.byref(n)), "pd_server_slots")
        return n.value

    def hold(self, on: bool = True) -> None:
        _check(load().pd_server_hold(self.handle, int(bool(on))), "pd_server_hold")

    def ring_frame(self, geometry: int, slot: int) -> np.ndarray:
        """numpy view (uint16 [pixels]) of a ring slot's page-locked memory."""
        p = ctypes.c_void_p()
        _check(load().pd_server_ring_frame(self.handle, geometry, slot, ctypes.byref(p)),
               "pd_server_ring_frame")
        n = self.ctxs[geometry].pixels_per_frame
        return np.ctypeslib.as_array((ctypes.c_uint16 * n).from_address(p.value))

    def acquire(self, geometry: int):
        p = ctypes.c_void_p()
        slot = ctypes.c_uint32()
        rc = load().pd_server_acquire(self.handle, geometry, ctypes.byref(p), ctypes.byref(slot))
        if rc == PD_EBUSY:
            return None
        _check(rc, "pd_server_acquire")
        n = self.ctxs[geometry].pixels_per_frame
        return slot.value, np.ctypeslib.as_array((ctypes.c_uint16 * n).from_address(p.value))

    def commit(self, geometry: int, slot: int, frame_id: int) -> None:
        _check(load().pd_server_commit(self.handle, geometry, slot, frame_id), "pd_server_commit")

    def replay(self, rate_hz, duration_s, mix=None, seed=0, first_id=0) -> None:
        m = (ctypes.c_float * len(self.ctxs))(*mix) if mix is not None else None
        _check(load().pd_server_replay(self.handle, rate_hz, duration_s, m, seed, first_id),
               "pd_server_replay")

    def drain(self, timeout_s=60.0) -> None:
        _check(load().pd_server_drain(self.handle, timeout_s), "pd_server_drain")

    def stats(self) -> dict:
        st = PdServeStats()
        _check(load().pd_server_stats(self.handle, ctypes.byref(st)), "pd_server_stats")
        return {n: getattr(st, n) for n, _ in PdServeStats._fields_}

    def reset_stats(self) -> None:
        _check(load().pd_server_reset_stats(self.handle), "pd_server_reset_stats")

    def frame_hits(self, frame_id: int, cap: int = 1 << 20):
        out = np.empty(cap, HIT_DTYPE)
        n = ctypes.c_uint32()
        lat = ctypes.c_float()
        _check(load().pd_server_frame_hits(self.handle, frame_id, out.ctypes.data, cap,
                                           ctypes.byref(n), ctypes.byref(lat)),
               "pd_server_frame_hits")
        return out[:min(n.value, cap)], float(lat.value)

    def frame_stream(self, frame_id: int) -> bytes:
        n = ctypes.c_size_t()
        _check(load().pd_server_frame_stream(self.handle, frame_id, None, 0, ctypes.byref(n)),
               "pd_server_frame_stream")
        buf = (ctypes.c_uint8 * max(n.value, 1))()
        _check(load().pd_server_frame_stream(self.handle, frame_id, buf, n.value,
                                             ctypes.byref(n)), "pd_server_frame_stream")
        return bytes(buf[:n.value])

    def close(self):
        if self.handle:
            load().pd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_server_create(ctxs, **kw) -> Server:
    return Server(ctxs, **kw)


def pd_server_destroy(server: Server) -> None:
    server.close()


def pd_compress_hits(hits: np.ndarray) -> bytes:
    h = np.ascontiguousarray(hits, HIT_DTYPE)
    need = ctypes.c_size_t()
    _check(load().pd_compress_hits(h.ctypes.data, len(h), None, 0, ctypes.byref(need)),
           "pd_compress_hits")
    buf = (ctypes.c_uint8 * max(need.value, 1))()
    _check(load().pd_compress_hits(h.ctypes.data, len(h), buf, need.value, ctypes.byref(need)),
           "pd_compress_hits")
    return bytes(buf[:need.value])


def pd_decompress_hits(data: bytes, frame: int = 0) -> np.ndarray:
    src = (ctypes.c_uint8 * max(len(data), 1)).from_buffer_copy(data or b"\0")
    n = ctypes.c_uint32()
    _check(load().pd_decompress_hits(src, len(data), frame, None, 0, ctypes.byref(n)),
           "pd_decompress_hits")
    out = np.zeros(n.value, HIT_DTYPE)
    _check(load().pd_decompress_hits(src, len(data), frame, out.ctypes.data, n.value,
                                     ctypes.byref(n)), "pd_decompress_hits")
    return out


# ---- centroid linearisation -------------------------------------------------
class Eta:
    def __init__(self, bins: int = 255):
        h = ctypes.c_void_p()
        _check(load().pd_eta_create(bins, ctypes.byref(h)), "pd_eta_create")
        self.handle = h.value
        self.bins = bins

    def close(self):
        if self.handle:
            load().pd_eta_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_eta_create(bins: int = 255) -> Eta:
    return Eta(bins)


def pd_eta_accumulate(eta: Eta, hits_ptr: int, n: int, stream=None) -> None:
    _check(load().pd_eta_accumulate(eta.handle, hits_ptr, n, _stream_handle(stream)),
           "pd_eta_accumulate")


def pd_eta_finalize(eta: Eta, stream=None) -> None:
    _check(load().pd_eta_finalize(eta.handle, _stream_handle(stream)), "pd_eta_finalize")


def pd_eta_apply(eta: Eta, hits_in_ptr: int, n: int, hits_out_ptr: int, stream=None) -> None:
    _check(load().pd_eta_apply(eta.handle, hits_in_ptr, n, hits_out_ptr, _stream_handle(stream)),
           "pd_eta_apply")


def pd_eta_get_histogram(eta: Eta) -> np.ndarray:
    out = np.zeros((2, eta.bins), np.uint32)
    _check(load().pd_eta_get_histogram(eta.handle, out.ctypes.data), "pd_eta_get_histogram")
    return out


def pd_eta_reset(eta: Eta, stream=None) -> None:
    _check(load().pd_eta_reset(eta.handle, _stream_handle(stream)), "pd_eta_reset")


def pd_eta_destroy(eta: Eta) -> None:
    eta.close()


def pd_strerror(code: int) -> str:
    return load().pd_strerror(code).decode()


# ---- torch-side convenience (allocation only) --------------------------------
class Outputs:
    """Device output buffers of one pd_process call, allocated with torch."""

    def __init__(self, ctx: Context, n_frames: int, hit_capacity: int,
                 corrected: bool = False, cm: bool = False, device="cuda"):
        import torch
        self.hits = torch.empty((max(hit_capacity, 1), HIT_DTYPE.itemsize),
                                dtype=torch.uint8, device=device)
        self.hit_capacity = hit_capacity
        self.n_hits = torch.zeros(1, dtype=torch.int32, device=device)
        self.corrected = torch.empty((n_frames, ctx.pixels_per_frame),
                                     dtype=torch.float32, device=device) \
            if corrected else None
        self.cm = torch.empty((n_frames, ctx.cm_values_per_frame),
                              dtype=torch.float32, device=device) if cm else None

    def ptrs(self):
        return dict(hits_ptr=self.hits.data_ptr(), hit_capacity=self.hit_capacity,
                    n_hits_ptr=self.n_hits.data_ptr(),
                    corrected_ptr=self.corrected.data_ptr()
                    if self.corrected is not None else None,
                    cm_ptr=self.cm.data_ptr() if self.cm is not None else None)

    def hits_host(self):
        n = int(self.n_hits.item())
        k = min(n, self.hit_capacity)
        raw = self.hits[:k].cpu().numpy()
        return raw.view(HIT_DTYPE).reshape(-1), n


def frames_to_device(frames: np.ndarray, device="cuda"):
    """uint16 frames -> torch int16 tensor on the device (same bits)."""
    import torch
    a = np.ascontiguousarray(frames, np.uint16)
    return torch.from_numpy(a.view(np.int16)).to(device)


def process(ctx: Context, frames_dev, hit_capacity: int | None = None,
            frame_base: int = 0, corrected: bool = False, cm: bool = False,
            stream=None) -> Outputs:
    """pd_process on a device tensor of frames; returns the Outputs."""
    n = frames_dev.numel() // ctx.pixels_per_frame
    assert n * ctx.pixels_per_frame == frames_dev.numel()
    cap = hit_capacity if hit_capacity is not None else \
        max(1024, n * ctx.pixels_per_frame // 4)
    out = Outputs(ctx, n, cap, corrected, cm, device=frames_dev.device)
    pd_process(ctx, frames_dev.data_ptr(), n, frame_base, stream=stream,
               **out.ptrs())
    return out
