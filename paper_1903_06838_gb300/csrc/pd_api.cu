// pd_api.cu — host implementation of the C ABI declared in include/pd.h.
//
// A pd_ctx owns the device copies of the pedestal and inverse-gain maps,
// the accumulated summaries (photon-count map, two histograms) and the
// scratch it needs per call.  Compiled with -ffp-contract=off so the host
// reciprocal of the gain is the plain IEEE division.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "pd.h"
#include "pd_fast.cuh"
#include "pd_internal.cuh"
#include "pd_lean.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* what) {
    g_last_error = what;
    return code;
}

int fail_cuda(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return PD_ECUDA;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// pd_process_host: chunks between a chunk's processing and the download of
// its hits (the host waits for chunk k - kHitLag's count while chunks up to k
// are queued, so the device never runs dry)
constexpr uint32_t kHitLag = 2;

}  // namespace

struct pd_ctx {
    pd_geometry geom;
    pd_thresholds thr;
    pd::ChainParams params;
    pd::CmBigConfig cm_cfg;
    pd::BandConfig band_cfg;
    pd::FusedConfig fused_cfg;
    bool use_cm_big = false, use_cm_rows = false, use_band = false;
    bool use_fused = false;     // the geometry allows the one-kernel chain
    // the lean pair (pd_lean.cu): the integer-coded bank median and the
    // lean band stencil, where the context allows them
    bool use_bank = false, use_lean = false;
    pd::CodeMap cmap{};
    uint4* d_kmap = nullptr;
    pd::LeanConfig lean_cfg{};
    uint32_t kernels = 1;       // 1: the lean pair where available; 2: the earlier pair;
                                // 3: the lean pair as one work-queue launch
    bool use_queue = false;     // the lean pair can run as the work-queue launch
    uint32_t* d_qsync = nullptr;  // its queue counter and per-(frame, module) counts
    size_t qsync_cap = 0;         // words
    uint32_t* d_err = nullptr;  // bit 0: a bounded wait for staged copies gave up
    uint32_t wait_polls = 0;    // polls of a bounded device wait (0: the kernels' default)
    uint32_t two_pass = 1;      // 1: common-mode and stencil kernels (measured
                                // faster on GB300 so far); 0: the one-kernel chain
    bool multigain = false;     // auto-ranging words (pd_create_multigain)
    pd::MultiGain mg{};
    float* d_mg_ped = nullptr;  // [n_gains][pixels]
    float* d_mg_ig = nullptr;
    bool matched = false;       // matched-filter charge summing (pd_set_filter_bank)
    pd::MatchedBank* d_bank = nullptr;
    uint8_t* d_vtab = nullptr;  // valid-feature table of an all-binary bank
    uint32_t chunk_frames = 1;  // frames per common-mode/stencil launch pair
    uint32_t overlap = 1;       // common mode of chunk c+1 beside stencil of c
    cudaStream_t aux = nullptr; // second stream of the chunk pipeline
    cudaEvent_t ev_fork = nullptr, ev_cm[2] = {nullptr, nullptr};
    cudaEvent_t ev_st[2] = {nullptr, nullptr};
    int device = 0;
    uint32_t masked = 0;
    // device state
    float* d_ped = nullptr;
    float* d_nped = nullptr;
    float* d_inv_gain = nullptr;
    uint32_t* d_count_map = nullptr;
    unsigned long long* d_hist_pix = nullptr;
    unsigned long long* d_hist_hit = nullptr;
    // per-call scratch: common mode of each (frame, unit)
    float* d_cm = nullptr;
    size_t cm_cap = 0;  // floats
    // host-path staging (pd_process_host)
    uint16_t* d_stage[2] = {nullptr, nullptr};
    uint32_t stage_frames = 0;
    pd_hit* d_host_hits = nullptr;
    uint32_t host_hit_cap = 0;
    uint32_t* d_host_nhits = nullptr;
    cudaStream_t hstream[3] = {nullptr, nullptr, nullptr};  // process, upload, hit download
    cudaEvent_t hevent[4] = {nullptr, nullptr, nullptr, nullptr};
    // hit counts after each chunk, read back to page-locked slots
    uint32_t* h_counts = nullptr;
    cudaEvent_t hcount_ev[kHitLag + 1] = {};
    // kernel timing (pd_set_profiling)
    bool profiling = false;
    struct Mark { int kernel; cudaEvent_t a, b; };
    std::vector<Mark> marks;        // recorded since the last read
    std::vector<cudaEvent_t> spare; // event pool
};

namespace {

const char* const kKernelNames[] = {"common_mode", "stencil", "fused_chain", "chain_queue"};
constexpr int kNumKernelNames = 4;

cudaEvent_t take_event(pd_ctx* c) {
    if (!c->spare.empty()) {
        cudaEvent_t e = c->spare.back();
        c->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one launch with events when profiling is on.
struct ProfileScope {
    pd_ctx* c;
    int kernel;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    ProfileScope(pd_ctx* c_, int k, cudaStream_t s_) : c(c_), kernel(k), s(s_) {
        if (c->profiling) {
            a = take_event(c);
            cudaEventRecord(a, s);
        }
    }
    ~ProfileScope() {
        if (a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, s);
            c->marks.push_back({kernel, a, b});
        }
    }
};

}  // namespace

namespace pd {

int device_sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

}  // namespace pd

namespace {

int check_geometry(const pd_geometry* g) {
    if (!g) return fail(PD_EINVAL, "geometry is NULL");
    if (!g->n_modules || !g->rows || !g->cols || !g->unit_rows || !g->unit_cols)
        return fail(PD_EINVAL, "geometry sizes must be > 0");
    if (g->rows % g->unit_rows || g->cols % g->unit_cols)
        return fail(PD_EINVAL, "common-mode units must tile each module");
    if (g->cm_mode > PD_CM_MEAN_STACKED) return fail(PD_EINVAL, "unknown cm_mode");
    if (g->cm_after_gain > 1) return fail(PD_EINVAL, "cm_after_gain is 0 or 1");
    if (g->cm_mode >= PD_CM_MEAN && (uint64_t)g->unit_rows * g->unit_cols >= (1u << 24))
        return fail(PD_EINVAL, "the mean common mode needs units of fewer than 2^24 pixels");
    const unsigned long long fpx =
        (unsigned long long)g->n_modules * g->rows * g->cols;
    if (fpx >= (1ull << 31)) return fail(PD_EINVAL, "frame too large");
    if (g->rows > 65535 || g->cols > 65535) return fail(PD_EINVAL, "module too large");
    return PD_OK;
}

int check_thresholds(const pd_thresholds* t) {
    if (!t) return fail(PD_EINVAL, "thresholds is NULL");
    if (!(t->zero_thr_kev >= 0.0f) || !(t->seed_thr_kev >= t->zero_thr_kev) ||
        !isfinite(t->seed_thr_kev))
        return fail(PD_EINVAL, "need 0 <= zero_thr_kev <= seed_thr_kev, finite");
    if (!(t->photon_kev > 0.0f) || !isfinite(t->photon_kev))
        return fail(PD_EINVAL, "photon_kev must be finite and > 0");
    if (!(t->hist_bin_kev > 0.0f) || !isfinite(t->hist_bin_kev) ||
        !isfinite(t->hist_lo_kev))
        return fail(PD_EINVAL, "histogram lo and bin width must be finite, width > 0");
    if (t->hist_bins < 1 || t->hist_bins > PD_MAX_HIST_BINS)
        return fail(PD_EINVAL, "hist_bins must be in [1, PD_MAX_HIST_BINS]");
    if (isnan(t->cm_cut_adu)) return fail(PD_EINVAL, "cm_cut_adu is NaN");
    return PD_OK;
}

uint32_t ceil_sqrt_u32(uint32_t n) {
    uint32_t k = (uint32_t)sqrt((double)n);
    while ((uint64_t)k * k < n) k++;
    while (k && (uint64_t)(k - 1) * (k - 1) >= n) k--;
    return k;
}

void free_ctx(pd_ctx* c) {
    if (!c) return;
    cudaFree(c->d_ped);
    cudaFree(c->d_nped);
    cudaFree(c->d_inv_gain);
    cudaFree(c->d_count_map);
    cudaFree(c->d_hist_pix);
    cudaFree(c->d_hist_hit);
    cudaFree(c->d_cm);
    cudaFree(c->d_bank);
    cudaFree(c->d_vtab);
    cudaFree(c->d_mg_ped);
    cudaFree(c->d_mg_ig);
    cudaFree(c->d_kmap);
    cudaFree(c->d_qsync);
    cudaFree(c->d_err);
    cudaFree(c->d_stage[0]);
    cudaFree(c->d_stage[1]);
    cudaFree(c->d_host_hits);
    cudaFree(c->d_host_nhits);
    for (int i = 0; i < 3; i++)
        if (c->hstream[i]) cudaStreamDestroy(c->hstream[i]);
    for (int i = 0; i < 4; i++)
        if (c->hevent[i]) cudaEventDestroy(c->hevent[i]);
    for (uint32_t i = 0; i <= kHitLag; i++)
        if (c->hcount_ev[i]) cudaEventDestroy(c->hcount_ev[i]);
    if (c->h_counts) cudaFreeHost(c->h_counts);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (int i = 0; i < 2; i++) {
        if (c->ev_cm[i]) cudaEventDestroy(c->ev_cm[i]);
        if (c->ev_st[i]) cudaEventDestroy(c->ev_st[i]);
    }
    for (auto& m : c->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : c->spare) cudaEventDestroy(e);
    delete c;
}

// The one-kernel chain replaces the kernel pair.
bool fused_on(const pd_ctx* c) { return c->use_fused && !c->two_pass && !c->matched; }
// (use_fused and use_cm_rows are off for multi-gain contexts: those
// kernels read single-gain words)

// The charge-summing launch of a context (after its common mode).
cudaError_t launch_stencil_for(const pd_ctx* c, const uint16_t* fr, uint32_t nf,
                               uint32_t frame_base, const pd::CallOut& co, cudaStream_t s) {
    const pd::MultiGain* mg = c->multigain ? &c->mg : nullptr;
    if (c->matched)
        return pd::launch_matched(c->params, c->d_bank, fr, nf, frame_base, co, s, mg);
    if (c->use_lean && c->kernels == 1) {
        pd::LeanConfig lc = c->lean_cfg;
        lc.wait_polls = c->wait_polls;
        return pd::launch_stencil_lean(c->params, lc, fr, nf, frame_base, co, c->d_err, s);
    }
    return c->use_band
               ? pd::launch_stencil_band(c->params, c->band_cfg, fr, nf, frame_base, co, s, mg)
               : pd::launch_stencil(c->params, fr, nf, frame_base, co, s, mg);
}

// The common-mode launch(es) of a context for nf frames into cm.
cudaError_t launch_cm(const pd_ctx* c, const uint16_t* fr, uint32_t nf, float* cm,
                      cudaStream_t s) {
    if (pd::cm_kind(c->params) == PD_CM_MEAN || pd::cm_kind(c->params) == PD_CM_MEAN_STACKED)
        return pd::launch_cm_mean(c->params, fr, nf, cm, s);
    if (c->multigain)
        return c->use_cm_big ? pd::launch_cm_big(c->params, c->cm_cfg, fr, nf, cm, s,
                                                 ~c->mg.vmask & 0xFFFFu)
                             : pd::launch_cm_select(c->params, fr, nf, cm, s, &c->mg);
    if (c->use_bank && c->kernels == 1) {
        pd::CodeMap cmap = c->cmap;
        cmap.wait_polls = c->wait_polls;
        return pd::launch_cm_bank(c->params, c->cm_cfg, cmap, fr, nf, cm, c->d_err, s);
    }
    return c->use_cm_big    ? pd::launch_cm_big(c->params, c->cm_cfg, fr, nf, cm, s)
           : c->use_cm_rows ? pd::launch_cm_rows(c->params, fr, nf, cm, s)
                            : pd::launch_cm_select(c->params, fr, nf, cm, s);
}

int ensure_cm(pd_ctx* c, uint32_t n_frames) {
    const size_t need = (size_t)n_frames * pd::cm_per_frame(c->params);
    if (need <= c->cm_cap) return PD_OK;
    // growth reallocates: any work on the old buffer must be finished
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "synchronise before scratch growth");
    cudaFree(c->d_cm);
    c->d_cm = nullptr;
    c->cm_cap = 0;
    e = cudaMalloc(&c->d_cm, need * sizeof(float));
    if (e != cudaSuccess) return fail(PD_ENOMEM, "common-mode scratch allocation failed");
    c->cm_cap = need;
    return PD_OK;
}

// The work-queue launch applies (lean pair, column banks, no matched
// filters, no corrected frames).
bool queue_on(const pd_ctx* c, const pd_outputs* out) {
    return c->use_queue && c->kernels == 3 && !c->matched && !out->corrected &&
           pd::queue_supported(c->params, c->cmap, c->lean_cfg);
}

int ensure_qsync(pd_ctx* c, uint32_t n_frames) {
    const size_t need = pd::queue_sync_words(c->params, n_frames);
    if (need <= c->qsync_cap) return PD_OK;
    // growth reallocates: any work on the old buffer must be finished
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "synchronise before queue scratch growth");
    cudaFree(c->d_qsync);
    c->d_qsync = nullptr;
    c->qsync_cap = 0;
    if (cudaMalloc(&c->d_qsync, need * 4) != cudaSuccess)
        return fail(PD_ENOMEM, "queue scratch allocation failed");
    c->qsync_cap = need;
    return PD_OK;
}

int run_chain(pd_ctx* c, const uint16_t* frames, uint32_t n_frames, uint32_t frame_base,
              const pd_outputs* out, cudaStream_t s, bool zero = true) {
    cudaError_t e = cudaSuccess;
    if (zero && (e = cudaMemsetAsync(out->n_hits, 0, sizeof(uint32_t), s)) != cudaSuccess)
        return fail_cuda(e, "zero n_hits");
    if (n_frames == 0) return PD_OK;
    if (fused_on(c)) {
        pd::CallOut co{out->hits, out->hit_capacity, out->n_hits, out->corrected, out->cm};
        ProfileScope ps(c, 2, s);
        e = pd::launch_fused(c->params, c->fused_cfg, frames, n_frames, frame_base, co, s);
        return e == cudaSuccess ? PD_OK : fail_cuda(e, "chain kernel launch");
    }
    float* cm = out->cm;
    if (!cm) {
        int rc = ensure_cm(c, n_frames);
        if (rc) return rc;
        cm = c->d_cm;
    }
    if (queue_on(c, out)) {
        // every frame of the call in one work-queue launch
        int rc = ensure_qsync(c, n_frames);
        if (rc) return rc;
        pd::CallOut co{out->hits, out->hit_capacity, out->n_hits, nullptr, cm};
        ProfileScope ps(c, 3, s);
        pd::CodeMap cmap = c->cmap;
        pd::LeanConfig lc = c->lean_cfg;
        cmap.wait_polls = lc.wait_polls = c->wait_polls;
        e = pd::launch_chain_queue(c->params, c->cm_cfg, cmap, lc, frames, n_frames, frame_base, co,
                                   c->d_qsync, c->d_err, s);
        return e == cudaSuccess ? PD_OK : fail_cuda(e, "queue kernel launch");
    }
    // Frames go in chunks sized so raw stays resident in L2 between the
    // common-mode pass and the stencil pass that re-reads it.  With overlap,
    // the common mode of chunk c+1 runs on the auxiliary stream beside the
    // stencil of chunk c (and waits for the stencil of chunk c-1), so at most
    // two chunks are in flight.
    const bool two = c->overlap && n_frames > c->chunk_frames;
    cudaStream_t sc = s;
    if (two) {
        if ((e = cudaEventRecord(c->ev_fork, s)) || (e = cudaStreamWaitEvent(c->aux, c->ev_fork, 0)))
            return fail_cuda(e, "chunk pipeline fork");
        sc = c->aux;
    }
    uint32_t k = 0;
    for (uint32_t done = 0; done < n_frames; k++) {
        const uint32_t nf = std::min(c->chunk_frames, n_frames - done);
        const uint16_t* fr = frames + (size_t)done * c->params.frame_px;
        float* cmc = cm + (size_t)done * pd::cm_per_frame(c->params);
        if (two && k >= 2 && (e = cudaStreamWaitEvent(sc, c->ev_st[k & 1], 0)))
            return fail_cuda(e, "chunk pipeline wait");
        {
            ProfileScope ps(c, 0, sc);
            e = launch_cm(c, fr, nf, cmc, sc);
        }
        if (e != cudaSuccess) return fail_cuda(e, "common-mode kernel launch");
        if (two && ((e = cudaEventRecord(c->ev_cm[k & 1], sc)) ||
                    (e = cudaStreamWaitEvent(s, c->ev_cm[k & 1], 0))))
            return fail_cuda(e, "chunk pipeline join");
        pd::CallOut co{out->hits, out->hit_capacity, out->n_hits,
                       out->corrected ? out->corrected + (size_t)done * c->params.frame_px
                                      : nullptr,
                       cmc};
        {
            ProfileScope ps(c, 1, s);
            e = launch_stencil_for(c, fr, nf, frame_base + done, co, s);
        }
        if (e != cudaSuccess) return fail_cuda(e, "stencil kernel launch");
        if (two && (e = cudaEventRecord(c->ev_st[k & 1], s)))
            return fail_cuda(e, "chunk pipeline record");
        done += nf;
    }
    return PD_OK;
}

}  // namespace

namespace pd {

int internal_fail(int code, const char* why) { return fail(code, why ? why : "error"); }

uint32_t internal_cm_per_frame(const pd_ctx* c) { return pd::cm_per_frame(c->params); }

int internal_ctx_device(const pd_ctx* c) { return c->device; }

bool internal_uses_cm_scratch(const pd_ctx* c) { return !fused_on(c); }

int internal_check_process_args(const pd_ctx* c, const uint16_t* frames, uint32_t n_frames,
                                const pd_outputs* out, const char** why) {
    if (!c || !out) {
        *why = "NULL argument";
        return PD_EINVAL;
    }
    if (!out->n_hits || (!out->hits && out->hit_capacity)) {
        *why = "hits/n_hits are required";
        return PD_EINVAL;
    }
    if (n_frames && !frames) {
        *why = "frames are NULL";
        return PD_EINVAL;
    }
    if (!aligned(frames, 16) || !aligned(out->n_hits, 4) || !aligned(out->hits, 8) ||
        (out->corrected && !aligned(out->corrected, 16)) || (out->cm && !aligned(out->cm, 4))) {
        *why = "misaligned frames or output buffer";
        return PD_EALIGN;
    }
    return PD_OK;
}

int internal_run_sequential(pd_ctx* c, const uint16_t* frames, uint32_t n_frames,
                            uint32_t frame_base, const pd_outputs* out, float* cm,
                            cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out->n_hits, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return fail_cuda(e, "zero n_hits");
    if (fused_on(c)) {
        CallOut co{out->hits, out->hit_capacity, out->n_hits, out->corrected, out->cm};
        e = launch_fused(c->params, c->fused_cfg, frames, n_frames, frame_base, co, s);
        return e == cudaSuccess ? PD_OK : fail_cuda(e, "chain kernel launch");
    }
    for (uint32_t done = 0; done < n_frames;) {
        const uint32_t nf = std::min(c->chunk_frames, n_frames - done);
        const uint16_t* fr = frames + (size_t)done * c->params.frame_px;
        float* cmc = cm + (size_t)done * pd::cm_per_frame(c->params);
        e = launch_cm(c, fr, nf, cmc, s);
        if (e != cudaSuccess) return fail_cuda(e, "common-mode kernel launch");
        CallOut co{out->hits, out->hit_capacity, out->n_hits,
                   out->corrected ? out->corrected + (size_t)done * c->params.frame_px
                                  : nullptr,
                   cmc};
        e = launch_stencil_for(c, fr, nf, frame_base + done, co, s);
        if (e != cudaSuccess) return fail_cuda(e, "stencil kernel launch");
        done += nf;
    }
    return PD_OK;
}

}  // namespace pd

extern "C" {

const char* pd_strerror(int code) {
    switch (code) {
        case PD_OK: return "ok";
        case PD_EINVAL: return "invalid argument";
        case PD_EALIGN: return "misaligned pointer or size";
        case PD_ENOMEM: return "out of memory";
        case PD_EOVERFLOW: return "hit capacity exceeded";
        case PD_ETIMEDOUT: return "timed out";
        case PD_ECUDA: return "CUDA error";
        case PD_ENOTSUP: return "not supported";
        case PD_EBUSY: return "busy";
        default: return "unknown error";
    }
}

const char* pd_last_error(void) { return g_last_error.c_str(); }

namespace {
int create_impl(const pd_geometry* geometry, uint32_t n_gains, uint32_t gain_shift,
                const float* pedestal_host, const float* gain_host,
                const pd_thresholds* thresholds, pd_ctx** out);
}

int pd_create(const pd_geometry* geometry, const float* pedestal_host,
              const float* gain_host, const pd_thresholds* thresholds, pd_ctx** out) {
    return create_impl(geometry, 0, 0, pedestal_host, gain_host, thresholds, out);
}

int pd_create_multigain(const pd_geometry* geometry, uint32_t n_gains, uint32_t gain_shift,
                        const float* pedestal_host, const float* gain_host,
                        const pd_thresholds* thresholds, pd_ctx** out) {
    if (out) *out = nullptr;
    if (n_gains < 1 || n_gains > PD_MAX_GAINS || gain_shift < 1 || gain_shift > 15)
        return fail(PD_EINVAL, "multi-gain: 1..PD_MAX_GAINS stages, gain_shift in 1..15");
    if (geometry && geometry->cm_mode != PD_CM_MEDIAN && geometry->cm_mode != PD_CM_NONE)
        return fail(PD_EINVAL, "multi-gain: the median or no common mode");
    if (geometry && geometry->cm_after_gain)
        return fail(PD_EINVAL, "multi-gain: common mode before gain only");
    return create_impl(geometry, n_gains, gain_shift, pedestal_host, gain_host, thresholds, out);
}

namespace {
int create_impl(const pd_geometry* geometry, uint32_t n_gains, uint32_t gain_shift,
                const float* pedestal_host, const float* gain_host,
                const pd_thresholds* thresholds, pd_ctx** out) {
    if (!out) return fail(PD_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_geometry(geometry);
    if (rc) return rc;
    rc = check_thresholds(thresholds);
    if (rc) return rc;
    if (geometry->cm_after_gain && isnan(thresholds->cm_cut_kev))
        return fail(PD_EINVAL, "cm_cut_kev is NaN");
    if (!pedestal_host || !gain_host) return fail(PD_EINVAL, "maps are NULL");

    pd_ctx* c = new (std::nothrow) pd_ctx();
    if (!c) return fail(PD_ENOMEM, "host allocation failed");
    c->geom = *geometry;
    c->thr = *thresholds;
    cudaGetDevice(&c->device);
    const pd_geometry& g = *geometry;
    pd::ChainParams& p = c->params;
    p.n_modules = g.n_modules;
    p.rows = g.rows;
    p.cols = g.cols;
    p.unit_rows = g.unit_rows;
    p.unit_cols = g.unit_cols;
    p.units_per_row = g.cols / g.unit_cols;
    p.units_per_module = (g.rows / g.unit_rows) * p.units_per_row;
    p.unit_px = g.unit_rows * g.unit_cols;
    p.module_px = g.rows * g.cols;
    p.frame_px = g.n_modules * p.module_px;
    p.units_per_frame = g.n_modules * p.units_per_module;
    p.cm_mode = g.cm_mode | (g.cm_after_gain ? pd::kCmAfterGain : 0u);
    p.cm_min_count = thresholds->cm_min_count ? thresholds->cm_min_count
                                              : ceil_sqrt_u32(p.unit_px);
    p.cm_cut = g.cm_after_gain ? thresholds->cm_cut_kev : thresholds->cm_cut_adu;
    p.zero_thr = thresholds->zero_thr_kev;
    p.seed_thr = thresholds->seed_thr_kev;
    p.photon_kev = thresholds->photon_kev;
    p.hist_inv_w = 1.0f / thresholds->hist_bin_kev;
    p.hist_neg_lo_s = -(thresholds->hist_lo_kev * p.hist_inv_w);
    p.hist_bins = thresholds->hist_bins;

    c->cm_cfg = pd::make_cm_big_config(p);
    // the bank and row median kernels, the band stencil and the one-kernel
    // chain work on d in ADU: the paper's order uses the generic kernels
    const bool ag = g.cm_after_gain != 0;
    c->use_cm_big = !ag && g.cm_mode == PD_CM_MEDIAN && pd::cm_big_supported(p, c->cm_cfg);
    c->use_cm_rows = !ag && g.cm_mode == PD_CM_MEDIAN && !c->use_cm_big && pd::cm_rows_supported(p);
    c->band_cfg = pd::make_band_config(p);
    c->use_band = c->band_cfg.ok && !ag;
    c->fused_cfg = pd::make_fused_config(p);
    // the one-kernel chain computes the median (or nothing) itself
    c->use_fused = c->fused_cfg.ok && !ag && (g.cm_mode == PD_CM_MEDIAN || g.cm_mode == PD_CM_NONE);
    {
        const size_t fbytes = (size_t)p.frame_px * 2;
        // raw bytes per chunk: longer persistent launches leave fewer tails
        // (2.2 Mpx frames: 21 frames 122.8 k, 42 127.9 k, 128 132.7 k frames/s)
        const size_t target = 600u << 20;
        c->chunk_frames = (uint32_t)std::max<size_t>(1, target / fbytes);
    }

    const size_t fpx = p.frame_px;
    const size_t stages = n_gains ? n_gains : 1;
    for (size_t i = 0; i < stages * fpx; i++)
        if (!isfinite(pedestal_host[i])) {
            free_ctx(c);
            return fail(PD_EINVAL, "pedestal values must be finite");
        }
    std::vector<float> inv(fpx);
    uint32_t masked = 0;
    for (size_t i = 0; i < fpx; i++) {
        const float gv = gain_host[i];
        if (gv > 0.0f && isfinite(gv)) {
            inv[i] = 1.0f / gv;
        } else {
            inv[i] = 0.0f;
            masked++;
        }
    }
    c->masked = masked;
    cudaError_t e;
    std::vector<float> nped(fpx);
    for (size_t i = 0; i < fpx; i++) nped[i] = -pedestal_host[i];
    if ((e = cudaMalloc(&c->d_ped, fpx * 4)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_nped, fpx * 4)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_inv_gain, fpx * 4)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_count_map, fpx * 4)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_hist_pix, p.hist_bins * 8)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_hist_hit, p.hist_bins * 8)) != cudaSuccess ||
        (e = cudaMalloc(&c->d_err, 4)) != cudaSuccess) {
        free_ctx(c);
        return fail(PD_ENOMEM, "device allocation failed in pd_create");
    }
    if ((e = cudaMemcpy(c->d_ped, pedestal_host, fpx * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->d_nped, nped.data(), fpx * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->d_inv_gain, inv.data(), fpx * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(c->d_count_map, 0, fpx * 4)) ||
        (e = cudaMemset(c->d_hist_pix, 0, p.hist_bins * 8)) ||
        (e = cudaMemset(c->d_hist_hit, 0, p.hist_bins * 8)) ||
        (e = cudaMemset(c->d_err, 0, 4))) {
        free_ctx(c);
        return fail_cuda(e, "pd_create upload");
    }
    if ((e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&c->ev_cm[0], cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&c->ev_cm[1], cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&c->ev_st[0], cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&c->ev_st[1], cudaEventDisableTiming))) {
        free_ctx(c);
        return fail_cuda(e, "pd_create streams");
    }
    p.ped = c->d_ped;
    p.nped = c->d_nped;
    p.inv_gain = c->d_inv_gain;
    p.count_map = c->d_count_map;
    p.hist_pix = c->d_hist_pix;
    p.hist_hit = c->d_hist_hit;
    if (n_gains) {
        // all stages' maps; stage 0 is also the context's single-gain map above
        std::vector<float> ig(stages * fpx);
        for (size_t i = 0; i < stages * fpx; i++) {
            const float gv = gain_host[i];
            ig[i] = gv > 0.0f && isfinite(gv) ? 1.0f / gv : 0.0f;
        }
        if ((e = cudaMalloc(&c->d_mg_ped, stages * fpx * 4)) != cudaSuccess ||
            (e = cudaMalloc(&c->d_mg_ig, stages * fpx * 4)) != cudaSuccess) {
            free_ctx(c);
            return fail(PD_ENOMEM, "device allocation failed in pd_create_multigain");
        }
        if ((e = cudaMemcpy(c->d_mg_ped, pedestal_host, stages * fpx * 4,
                            cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(c->d_mg_ig, ig.data(), stages * fpx * 4, cudaMemcpyHostToDevice))) {
            free_ctx(c);
            return fail_cuda(e, "pd_create_multigain upload");
        }
        c->multigain = true;
        c->mg = pd::MultiGain{n_gains, gain_shift, (1u << gain_shift) - 1u, c->d_mg_ped,
                              c->d_mg_ig};
        // the bank median and the band stencil decode the stages (the
        // band stencil with four-pixel chunks only); the row-unit median
        // and the one-kernel chain read single-gain words
        c->use_cm_rows = c->use_fused = false;
        c->use_band = c->use_band && c->band_cfg.vec == 4;
    } else if (!ag) {
        // the lean pair: single-gain words, common mode before gain
        c->lean_cfg = pd::make_lean_config(p);
        c->use_lean = c->lean_cfg.ok &&
                      (g.cm_mode == PD_CM_MEDIAN || g.cm_mode == PD_CM_NONE || g.cm_mode == PD_CM_MEAN);
        std::vector<uint16_t> km;
        pd::CodeMap cmap{};
        if (c->use_cm_big && pd::build_code_map(p, pedestal_host, &km, &cmap) &&
            pd::cm_bank_supported(p, cmap)) {
            if ((e = cudaMalloc(&c->d_kmap, km.size() * 2)) != cudaSuccess) {
                free_ctx(c);
                return fail(PD_ENOMEM, "device allocation failed in pd_create");
            }
            if ((e = cudaMemcpy(c->d_kmap, km.data(), km.size() * 2, cudaMemcpyHostToDevice))) {
                free_ctx(c);
                return fail_cuda(e, "pd_create upload");
            }
            cmap.kmap = c->d_kmap;
            c->cmap = cmap;
            c->use_bank = true;
            c->use_queue = c->use_lean && pd::queue_supported(p, cmap, c->lean_cfg);
        }
    }
    pd::noalloc_prepare(c->device);
    *out = c;
    return PD_OK;
}
}  // namespace

int pd_query(const pd_ctx* c, pd_info* info) {
    if (!c || !info) return fail(PD_EINVAL, "NULL argument");
    info->pixels_per_frame = c->params.frame_px;
    info->units_per_frame = c->params.units_per_frame;
    info->cm_values_per_frame = pd::cm_per_frame(c->params);
    info->unit_pixels = c->params.unit_px;
    info->cm_min_count = c->params.cm_min_count;
    info->hist_bins = c->params.hist_bins;
    info->masked_pixels = c->masked;
    return PD_OK;
}

int pd_process(pd_ctx* c, const uint16_t* frames_dev, uint32_t n_frames,
               uint32_t frame_base, const pd_outputs* out, void* stream) {
    if (!c || !out) return fail(PD_EINVAL, "NULL argument");
    if (!out->n_hits || (!out->hits && out->hit_capacity))
        return fail(PD_EINVAL, "hits/n_hits are required");
    if (n_frames && !frames_dev) return fail(PD_EINVAL, "frames are NULL");
    if (!aligned(frames_dev, 16)) return fail(PD_EALIGN, "frames must be 16-byte aligned");
    if (!aligned(out->n_hits, 4) || !aligned(out->hits, 8))
        return fail(PD_EALIGN, "hit buffers misaligned");
    if ((out->corrected && !aligned(out->corrected, 16)) || (out->cm && !aligned(out->cm, 4)))
        return fail(PD_EALIGN, "corrected must be 16-byte and cm 4-byte aligned");
    return run_chain(c, frames_dev, n_frames, frame_base, out, (cudaStream_t)stream);
}

int pd_process_host(pd_ctx* c, const uint16_t* frames_host, uint32_t n_frames,
                    uint32_t frame_base, pd_hit* hits_host, uint32_t hit_capacity,
                    uint32_t* n_hits_host) {
    if (!c || !n_hits_host || (hit_capacity && !hits_host) || (n_frames && !frames_host))
        return fail(PD_EINVAL, "NULL argument");
    cudaError_t e;
    const size_t fbytes = (size_t)c->params.frame_px * sizeof(uint16_t);
    // chunk: about 64 MB of frames per stage buffer
    uint32_t chunk = (uint32_t)std::max<size_t>(1, (64u << 20) / fbytes);
    chunk = std::min<uint32_t>(chunk, std::max<uint32_t>(n_frames, 1));
    if (c->stage_frames < chunk) {
        cudaDeviceSynchronize();
        for (int i = 0; i < 2; i++) {
            cudaFree(c->d_stage[i]);
            c->d_stage[i] = nullptr;
        }
        c->stage_frames = 0;
        for (int i = 0; i < 2; i++)
            if (cudaMalloc(&c->d_stage[i], chunk * fbytes) != cudaSuccess)
                return fail(PD_ENOMEM, "staging allocation failed");
        c->stage_frames = chunk;
    }
    for (int i = 0; i < 3; i++)
        if (!c->hstream[i] &&
            (e = cudaStreamCreateWithFlags(&c->hstream[i], cudaStreamNonBlocking)))
            return fail_cuda(e, "stream create");
    for (int i = 0; i < 4; i++)
        if (!c->hevent[i] &&
            (e = cudaEventCreateWithFlags(&c->hevent[i], cudaEventDisableTiming)))
            return fail_cuda(e, "event create");
    for (uint32_t i = 0; i <= kHitLag; i++)
        if (!c->hcount_ev[i] &&
            (e = cudaEventCreateWithFlags(&c->hcount_ev[i], cudaEventDisableTiming)))
            return fail_cuda(e, "event create");
    if (!c->h_counts &&
        (e = cudaHostAlloc(reinterpret_cast<void**>(&c->h_counts), (kHitLag + 1) * sizeof(uint32_t),
                           cudaHostAllocDefault)))
        return fail_cuda(e, "page-locked count slots");
    const uint32_t cap = std::max<uint32_t>(hit_capacity, 1);
    if (c->host_hit_cap < cap) {
        cudaDeviceSynchronize();
        cudaFree(c->d_host_hits);
        c->d_host_hits = nullptr;
        c->host_hit_cap = 0;
        if (cudaMalloc(&c->d_host_hits, (size_t)cap * sizeof(pd_hit)) != cudaSuccess)
            return fail(PD_ENOMEM, "hit buffer allocation failed");
        c->host_hit_cap = cap;
    }
    if (!c->d_host_nhits && cudaMalloc(&c->d_host_nhits, sizeof(uint32_t)) != cudaSuccess)
        return fail(PD_ENOMEM, "counter allocation failed");
    int rc = ensure_cm(c, chunk);
    if (rc) return rc;

    // Copies run on hstream[1], processing on hstream[0]; chunk k uses
    // staging buffer k%2.  copy(k) waits for process(k-2) (same buffer),
    // process(k) waits for copy(k), so the upload of chunk k+1 overlaps the
    // processing of chunk k.  One device counter spans all chunks, so the
    // hit list is contiguous.  After each chunk the counter is copied to a
    // page-locked slot; once chunk k is queued the host waits for chunk
    // k - kHitLag's count and downloads the hits added up to it on
    // hstream[2], so the hit list comes back during the uploads (the link
    // carries both directions at once) instead of after the last chunk.
    cudaStream_t s0 = c->hstream[0], s1 = c->hstream[1], s2 = c->hstream[2];
    uint32_t downloaded = 0;
    auto download_upto = [&](uint32_t count) -> cudaError_t {
        const uint32_t upto = std::min(count, hit_capacity);
        if (upto <= downloaded) return cudaSuccess;
        const cudaError_t de =
            cudaMemcpyAsync(hits_host + downloaded, c->d_host_hits + downloaded,
                            (size_t)(upto - downloaded) * sizeof(pd_hit), cudaMemcpyDeviceToHost, s2);
        downloaded = upto;
        return de;
    };
    if ((e = cudaMemsetAsync(c->d_host_nhits, 0, sizeof(uint32_t), s0)))
        return fail_cuda(e, "zero counter");
    cudaEvent_t copied[2] = {c->hevent[0], c->hevent[1]};
    cudaEvent_t processed[2] = {c->hevent[2], c->hevent[3]};
    uint32_t done = 0, k = 0;
    // on a failure, the work already queued (uploads that read frames_host,
    // downloads that write hits_host) finishes before the call returns
    auto stop = [&](int code) -> int {
        for (cudaStream_t q : {s0, s1, s2}) cudaStreamSynchronize(q);
        return code;
    };
    while (done < n_frames) {
        const uint32_t nf = std::min(chunk, n_frames - done);
        const int b = k & 1;
        if (k >= 2) cudaStreamWaitEvent(s1, processed[b], 0);
        if ((e = cudaMemcpyAsync(c->d_stage[b], frames_host + (size_t)done * c->params.frame_px,
                                 nf * fbytes, cudaMemcpyHostToDevice, s1)))
            return stop(fail_cuda(e, "frame upload"));
        cudaEventRecord(copied[b], s1);
        cudaStreamWaitEvent(s0, copied[b], 0);
        pd_outputs o{};
        o.hit_capacity = hit_capacity;
        o.hits = c->d_host_hits;
        o.n_hits = c->d_host_nhits;
        rc = run_chain(c, c->d_stage[b], nf, frame_base + done, &o, s0, /*zero=*/false);
        if (rc) return stop(rc);
        cudaEventRecord(processed[b], s0);
        const uint32_t slot = k % (kHitLag + 1);
        if ((e = cudaMemcpyAsync(c->h_counts + slot, c->d_host_nhits, 4, cudaMemcpyDeviceToHost,
                                 s0)) ||
            (e = cudaEventRecord(c->hcount_ev[slot], s0)))
            return stop(fail_cuda(e, "hit count readback"));
        if (k >= kHitLag) {
            // chunk j = k - kHitLag is done once its count has arrived; its
            // slot is next written by chunk k + 1, queued after this read
            const uint32_t js = (k - kHitLag) % (kHitLag + 1);
            if ((e = cudaEventSynchronize(c->hcount_ev[js])) ||
                (e = download_upto(c->h_counts[js])))
                return stop(fail_cuda(e, "hit download"));
        }
        done += nf;
        k++;
    }
    uint32_t total = 0;
    if ((e = cudaMemcpyAsync(c->h_counts, c->d_host_nhits, 4, cudaMemcpyDeviceToHost, s0)) ||
        (e = cudaStreamSynchronize(s0)))
        return stop(fail_cuda(e, "hit count readback"));
    total = c->h_counts[0];
    if ((e = download_upto(total)) || (e = cudaStreamSynchronize(s2)))
        return stop(fail_cuda(e, "hit download"));
    if ((e = cudaStreamSynchronize(s1))) return fail_cuda(e, "host path synchronise");
    *n_hits_host = total;
    return total > hit_capacity ? fail(PD_EOVERFLOW, "hit capacity exceeded") : PD_OK;
}

int pd_get_summary(pd_ctx* c, uint32_t* count_map_host, uint64_t* hist_pix_host,
                   uint64_t* hist_hit_host, void* stream) {
    if (!c) return fail(PD_EINVAL, "NULL context");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (count_map_host && (e = cudaMemcpyAsync(count_map_host, c->d_count_map,
                                               (size_t)c->params.frame_px * 4,
                                               cudaMemcpyDeviceToHost, s)))
        return fail_cuda(e, "count map download");
    if (hist_pix_host && (e = cudaMemcpyAsync(hist_pix_host, c->d_hist_pix,
                                              (size_t)c->params.hist_bins * 8,
                                              cudaMemcpyDeviceToHost, s)))
        return fail_cuda(e, "histogram download");
    if (hist_hit_host && (e = cudaMemcpyAsync(hist_hit_host, c->d_hist_hit,
                                              (size_t)c->params.hist_bins * 8,
                                              cudaMemcpyDeviceToHost, s)))
        return fail_cuda(e, "histogram download");
    if ((e = cudaStreamSynchronize(s))) return fail_cuda(e, "summary synchronise");
    uint32_t err = 0;
    if ((e = cudaMemcpy(&err, c->d_err, 4, cudaMemcpyDeviceToHost)))
        return fail_cuda(e, "error word download");
    if (err) return fail(PD_ETIMEDOUT, "a bounded wait for staged raw copies gave up");
    return PD_OK;
}

int pd_set_filter_bank(pd_ctx* c, const pd_filter_bank* bank) {
    if (!c) return fail(PD_EINVAL, "NULL context");
    pd::MatchedBank mb{};
    if (bank && !pd::compile_bank(*bank, &mb))
        return fail(PD_EINVAL, "filter bank: 1..PD_MAX_FEATURES features, finite values");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "synchronise before a bank change");
    if (!bank) {
        c->matched = false;
        return PD_OK;
    }
    if (!c->d_bank && (e = cudaMalloc(&c->d_bank, sizeof(pd::MatchedBank))) != cudaSuccess) {
        c->d_bank = nullptr;
        return fail(PD_ENOMEM, "filter bank allocation failed");
    }
    if ((e = cudaMemcpy(c->d_bank, &mb, sizeof(mb), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail_cuda(e, "filter bank upload");
    if (mb.all_binary) {
        // the table is built from the uploaded bank, then the bank points at it
        if (!c->d_vtab && (e = cudaMalloc(&c->d_vtab, 1u << 20)) != cudaSuccess) {
            c->d_vtab = nullptr;
            return fail(PD_ENOMEM, "filter bank table allocation failed");
        }
        if ((e = pd::build_vtab(c->d_bank, c->d_vtab)) != cudaSuccess)
            return fail_cuda(e, "filter bank table");
        mb.vtab = c->d_vtab;
        if ((e = cudaMemcpy(c->d_bank, &mb, sizeof(mb), cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail_cuda(e, "filter bank upload");
    }
    c->matched = true;
    return PD_OK;
}

int pd_reset_summary(pd_ctx* c, void* stream) {
    if (!c) return fail(PD_EINVAL, "NULL context");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d_count_map, 0, (size_t)c->params.frame_px * 4, s)) ||
        (e = cudaMemsetAsync(c->d_hist_pix, 0, (size_t)c->params.hist_bins * 8, s)) ||
        (e = cudaMemsetAsync(c->d_hist_hit, 0, (size_t)c->params.hist_bins * 8, s)) ||
        (e = cudaMemsetAsync(c->d_err, 0, 4, s)))
        return fail_cuda(e, "summary reset");
    return PD_OK;
}

int pd_set_wait_limit(pd_ctx* c, uint32_t polls) {
    if (!c) return fail(PD_EINVAL, "NULL context");
    c->wait_polls = polls;
    return PD_OK;
}

int pd_get_tuning(const pd_ctx* c, pd_tuning* t) {
    if (!c || !t) return fail(PD_EINVAL, "NULL argument");
    t->chunk_frames = c->chunk_frames;
    const bool lean = c->use_lean && (c->kernels == 1 || c->kernels == 3) && !c->matched;
    t->band_rows = lean ? c->lean_cfg.rb : c->use_band ? c->band_cfg.rb : 0;
    t->overlap = c->overlap;
    t->two_pass = c->use_fused && !c->matched ? c->two_pass : 1;
    t->kernels = c->use_lean || c->use_bank ? (c->kernels == 3 && !c->use_queue ? 1u : c->kernels)
                                            : 2;
    return PD_OK;
}

int pd_set_tuning(pd_ctx* c, const pd_tuning* t) {
    if (!c || !t) return fail(PD_EINVAL, "NULL argument");
    if (t->chunk_frames) c->chunk_frames = t->chunk_frames;
    if (t->kernels > 3) return fail(PD_EINVAL, "kernels is 0, 1, 2 or 3");
    if (t->kernels) c->kernels = t->kernels;
    if (t->band_rows && c->use_lean) {
        const pd::LeanConfig lc = pd::make_lean_config(c->params, t->band_rows);
        if (!lc.ok || lc.rb != std::min(t->band_rows, c->params.rows))
            return fail(PD_EINVAL, "band too tall for shared memory");
        c->lean_cfg = lc;
    }
    if (t->band_rows && c->use_band) {
        const uint32_t rb = std::min(t->band_rows, c->params.rows);
        if (pd::band_smem_bytes(c->params, rb, c->band_cfg.pitch) > 200 * 1024)
            return fail(PD_EINVAL, "band too tall for shared memory");
        c->band_cfg.rb = rb;
        c->band_cfg.n_bands = (c->params.rows + rb - 1) / rb;
    }
    c->overlap = t->overlap ? 1 : 0;
    c->two_pass = t->two_pass ? 1 : 0;
    return PD_OK;
}

int pd_set_profiling(pd_ctx* c, int enable) {
    if (!c) return fail(PD_EINVAL, "NULL context");
    c->profiling = enable != 0;
    return PD_OK;
}

int pd_read_profile(pd_ctx* c, pd_profile* out) {
    if (!c || !out) return fail(PD_EINVAL, "NULL argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "profile synchronise");
    memset(out, 0, sizeof(*out));
    out->n_kernels = kNumKernelNames;
    for (int k = 0; k < kNumKernelNames; k++)
        snprintf(out->name[k], sizeof(out->name[k]), "%s", kKernelNames[k]);
    for (auto& m : c->marks) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            out->launches[m.kernel]++;
            out->total_ms[m.kernel] += ms;
        }
        c->spare.push_back(m.a);
        c->spare.push_back(m.b);
    }
    c->marks.clear();
    return PD_OK;
}

// ---------------------------------------------------------------------------
// Batched launches over contexts of different geometries.
struct pd_batch {
    uint32_t max_items = 0;
    uint64_t max_cm = 0;
    uint32_t table_cap[2] = {0, 0};                  // entries of each table
    uint32_t mixed = 0;  // 1: persistent kernels over all geometries of a chunk
    pd::BatchItem* d_table[2] = {nullptr, nullptr};  // [0] direct calls, [1] graph
    pd::BatchItem* h_table[2] = {nullptr, nullptr};  // page-locked staging
    cudaEvent_t copied = nullptr;                    // staging [0] free again
    bool copy_pending = false;
    float* d_cm = nullptr;  // common mode of items that pass out.cm == NULL
    cudaGraphExec_t exec = nullptr;
};

namespace {

void free_batch(pd_batch* b) {
    if (!b) return;
    for (int i = 0; i < 2; i++) {
        cudaFree(b->d_table[i]);
        cudaFreeHost(b->h_table[i]);
    }
    cudaFree(b->d_cm);
    if (b->copied) cudaEventDestroy(b->copied);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
}

// The frames of a batch go in chunks of about this many raw bytes, one
// common-mode + stencil launch pair each, so the stencil re-reads a chunk's
// raw frames from L2 (the chunk interleaves the items' geometries).
constexpr size_t kBatchChunkBytes = 96u << 20;

struct Piece {
    uint32_t item, first, count;
};

// Greedy split of the items' frames into chunks of about kBatchChunkBytes.
std::vector<std::vector<Piece>> plan_chunks(const pd_batch_item* items, uint32_t n) {
    std::vector<std::vector<Piece>> chunks;
    std::vector<Piece> cur;
    size_t cur_bytes = 0;
    for (uint32_t i = 0; i < n; i++) {
        const size_t fb = (size_t)items[i].ctx->params.frame_px * 2;
        uint32_t f = 0;
        while (f < items[i].n_frames) {
            size_t room = kBatchChunkBytes > cur_bytes ? kBatchChunkBytes - cur_bytes : 0;
            uint32_t take = (uint32_t)std::min<size_t>(room / fb, items[i].n_frames - f);
            if (take == 0) {
                if (cur.empty()) {
                    take = 1;  // a frame larger than a chunk
                } else {
                    chunks.push_back(cur);
                    cur.clear();
                    cur_bytes = 0;
                    continue;
                }
            }
            cur.push_back({i, f, take});
            cur_bytes += take * fb;
            f += take;
            if (cur_bytes >= kBatchChunkBytes) {
                chunks.push_back(cur);
                cur.clear();
                cur_bytes = 0;
            }
        }
    }
    if (!cur.empty()) chunks.push_back(cur);
    return chunks;
}

size_t plan_entries(const std::vector<std::vector<Piece>>& chunks) {
    size_t t = 0;
    for (const auto& c : chunks) t += c.size();
    return t;
}

// Table slot with room for `entries` sub-items (frees the old one; cudaFree
// waits for work that may still read it).
int ensure_table(pd_batch* b, int slot, size_t entries) {
    if (entries <= b->table_cap[slot]) return PD_OK;
    cudaFree(b->d_table[slot]);
    cudaFreeHost(b->h_table[slot]);
    b->d_table[slot] = nullptr;
    b->h_table[slot] = nullptr;
    b->table_cap[slot] = 0;
    if (cudaMalloc(&b->d_table[slot], entries * sizeof(pd::BatchItem)) != cudaSuccess ||
        cudaMallocHost(&b->h_table[slot], entries * sizeof(pd::BatchItem)) != cudaSuccess)
        return fail(PD_ENOMEM, "batch table allocation failed");
    b->table_cap[slot] = (uint32_t)entries;
    return PD_OK;
}

int batch_check_items(const pd_batch* b, const pd_batch_item* items, uint32_t n) {
    if (!items || n == 0 || n > b->max_items) return fail(PD_EINVAL, "batch: 1..max_items items");
    for (uint32_t i = 0; i < n; i++) {
        const pd_batch_item& it = items[i];
        const char* why = nullptr;
        int rc = pd::internal_check_process_args(it.ctx, it.frames, it.n_frames, &it.out, &why);
        if (rc) return fail(rc, why);
        if (b->mixed && !it.ctx->use_band)
            return fail(PD_ENOTSUP, "batch: the mixed launch needs the band stencil");
        if (b->mixed && it.ctx->multigain)
            return fail(PD_ENOTSUP, "batch: the mixed launch reads single-gain words");
        if (b->mixed && it.ctx->matched)
            return fail(PD_ENOTSUP, "batch: the mixed launch has no matched filters");
        if (b->mixed && pd::cm_kind(it.ctx->params) >= PD_CM_MEAN)
            return fail(PD_ENOTSUP, "batch: the mixed launch computes the median only");
    }
    return PD_OK;
}

int batch_enqueue(pd_batch* b, int slot, const pd_batch_item* items, uint32_t n,
                  cudaStream_t s) {
    int rc = batch_check_items(b, items, n);
    if (rc) return rc;
    if (slot == 0 && b->copy_pending) {
        cudaError_t e = cudaEventSynchronize(b->copied);
        if (e != cudaSuccess) return fail_cuda(e, "batch staging wait");
        b->copy_pending = false;
    }
    // per item: kernel configuration and its common-mode destination
    std::vector<pd::BatchItem> base(n);
    std::vector<float*> item_cm(n);
    uint64_t cm_used = 0;
    size_t cm_smem = 0, band_smem = 0;
    for (uint32_t i = 0; i < n; i++) {
        const pd_batch_item& it = items[i];
        pd_ctx* c = it.ctx;
        pd::BatchItem& d = base[i];
        d = pd::BatchItem{};
        d.p = c->params;
        d.cm_cfg = c->cm_cfg;
        d.band_cfg = c->band_cfg;
        const size_t gen_keys = (size_t)c->params.unit_px * 4;
        d.rows_magic = pd::cm_rows_magic(c->params);
        if (c->use_cm_big) {
            d.cm_kind = c->cm_cfg.vec == 2 ? 0u : 1u;
            cm_smem = std::max(cm_smem, pd::cm_big_smem_bytes(c->params));
        } else if (c->use_cm_rows) {
            d.cm_kind = 4;
        } else if (gen_keys <= pd::kCmBigMaxSmem) {
            d.cm_kind = 2;
            cm_smem = std::max(cm_smem, gen_keys);
        } else {
            d.cm_kind = 3;
        }
        d.band_vec = c->band_cfg.vec;
        band_smem = std::max(band_smem, pd::band_smem_bytes(c->params, c->band_cfg.rb,
                                                            c->band_cfg.pitch));
        const uint64_t ncm = (uint64_t)it.n_frames * pd::cm_per_frame(c->params);
        float* cm = it.out.cm;
        if (!cm) {
            if (cm_used + ncm > b->max_cm) return fail(PD_EINVAL, "batch: common-mode scratch too small");
            cm = b->d_cm + cm_used;
            cm_used += ncm;
        }
        item_cm[i] = cm;
    }
    cudaError_t e;
    for (uint32_t i = 0; i < n; i++)
        if ((e = cudaMemsetAsync(items[i].out.n_hits, 0, sizeof(uint32_t), s)))
            return fail_cuda(e, "zero n_hits");
    if (!b->mixed) {
        // each item as pd_process runs it (its context's chunks, band height
        // and two-stream overlap), its common mode in the batch's scratch
        for (uint32_t i = 0; i < n; i++) {
            pd_outputs o = items[i].out;
            o.cm = item_cm[i];
            const int r = run_chain(items[i].ctx, items[i].frames, items[i].n_frames,
                                    items[i].frame_base, &o, s, false);
            if (r) return r;
        }
        return PD_OK;
    }
    const auto chunks = plan_chunks(items, n);
    const size_t entries = plan_entries(chunks);
    if (entries > b->table_cap[slot]) {
        if (slot == 1) return fail(PD_EINVAL, "batch: table not sized before capture");
        if ((rc = ensure_table(b, slot, entries))) return rc;
    }
    pd::BatchItem* h = b->h_table[slot];
    struct Launch {
        size_t first;
        uint32_t count;
        unsigned long long cm_tasks;
    };
    std::vector<Launch> launches;
    size_t at = 0;
    for (const auto& ch : chunks) {
        Launch L{at, (uint32_t)ch.size(), 0};
        unsigned long long tiles = 0;
        for (const Piece& pc : ch) {
            const pd_batch_item& it = items[pc.item];
            const pd::ChainParams& cp = it.ctx->params;
            pd::BatchItem& d = h[at++];
            d = base[pc.item];
            d.raw = it.frames + (size_t)pc.first * cp.frame_px;
            d.n_frames = pc.count;
            d.frame_base = it.frame_base + pc.first;
            const uint64_t ncm = (uint64_t)pc.count * pd::cm_per_frame(cp);
            d.out = pd::CallOut{it.out.hits, it.out.hit_capacity, it.out.n_hits,
                                it.out.corrected ? it.out.corrected + (size_t)pc.first * cp.frame_px
                                                 : nullptr,
                                item_cm[pc.item] + (size_t)pc.first * pd::cm_per_frame(cp)};
            d.cm_first = L.cm_tasks;
            d.st_first = tiles;
            d.st_tiles = (unsigned long long)pc.count * cp.n_modules * d.band_cfg.n_bands;
            L.cm_tasks += d.cm_kind == 4 ? (ncm + 15) / 16 : ncm;
            tiles += d.st_tiles;
        }
        launches.push_back(L);
    }
    e = cudaMemcpyAsync(b->d_table[slot], h, entries * sizeof(pd::BatchItem),
                        cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_cuda(e, "batch table upload");
    if (slot == 0) {
        if ((e = cudaEventRecord(b->copied, s))) return fail_cuda(e, "batch event");
        b->copy_pending = true;
    }
    // kernels specialised to the kinds this batch holds
    bool all_kinds = false;
    int vec = -1;
    for (uint32_t i = 0; i < n; i++) {
        if (base[i].cm_kind != 0 && base[i].cm_kind != 4) all_kinds = true;
        const int v = (int)base[i].band_vec;
        vec = vec < 0 ? v : (vec == v ? v : 0);
    }
    for (const Launch& L : launches) {
        e = pd::launch_batch(b->d_table[slot] + L.first, L.count, L.cm_tasks, cm_smem, band_smem,
                             s, all_kinds, vec < 0 ? 0 : vec);
        if (e != cudaSuccess) return fail_cuda(e, "batch kernel launch");
    }
    return PD_OK;
}

}  // namespace

int pd_batch_create(uint32_t max_items, uint64_t max_cm_values, pd_batch** out) {
    if (!out || !max_items) return fail(PD_EINVAL, "batch: need out and max_items > 0");
    *out = nullptr;
    pd_batch* b = new (std::nothrow) pd_batch();
    if (!b) return fail(PD_ENOMEM, "host allocation failed");
    b->max_items = max_items;
    b->max_cm = max_cm_values;
    cudaError_t e;
    for (int i = 0; i < 2; i++)
        if (ensure_table(b, i, max_items) != PD_OK) {
            free_batch(b);
            return PD_ENOMEM;
        }
    if (max_cm_values && (e = cudaMalloc(&b->d_cm, max_cm_values * sizeof(float)))) {
        free_batch(b);
        return fail(PD_ENOMEM, "batch scratch allocation failed");
    }
    if ((e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming))) {
        free_batch(b);
        return fail_cuda(e, "batch event");
    }
    // kernel attributes and the SM count are set up here, outside any capture
    pd::device_sm_count();
    if ((e = pd::launch_batch(nullptr, 0, 0, 0, 0, nullptr)) != cudaSuccess) {
        free_batch(b);
        return fail_cuda(e, "batch kernel attributes");
    }
    *out = b;
    return PD_OK;
}

int pd_batch_set_mixed(pd_batch* b, int mixed) {
    if (!b) return fail(PD_EINVAL, "NULL batch");
    b->mixed = mixed ? 1u : 0u;
    return PD_OK;
}

int pd_batch_process(pd_batch* b, const pd_batch_item* items, uint32_t n_items, void* stream) {
    if (!b) return fail(PD_EINVAL, "NULL batch");
    return batch_enqueue(b, 0, items, n_items, (cudaStream_t)stream);
}

int pd_batch_capture(pd_batch* b, const pd_batch_item* items, uint32_t n_items, void* stream) {
    if (!b || !stream) return fail(PD_EINVAL, "batch capture needs a batch and a non-default stream");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);  // earlier replays may still read table [1]
    if (e != cudaSuccess) return fail_cuda(e, "batch capture synchronise");
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    // the table and the contexts' queue scratch are sized before the capture
    // (no allocation while capturing)
    int rc0 = batch_check_items(b, items, n_items);
    if (rc0) return rc0;
    if ((rc0 = ensure_table(b, 1, plan_entries(plan_chunks(items, n_items))))) return rc0;
    for (uint32_t i = 0; i < n_items; i++)
        if (queue_on(items[i].ctx, &items[i].out) &&
            (rc0 = ensure_qsync(items[i].ctx, items[i].n_frames)))
            return rc0;
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)))
        return fail_cuda(e, "begin capture");
    int rc = batch_enqueue(b, 1, items, n_items, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail_cuda(e, "end capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return fail_cuda(e, "graph instantiate");
    }
    return PD_OK;
}

int pd_batch_replay(pd_batch* b, void* stream) {
    if (!b || !b->exec) return fail(PD_EINVAL, "batch has no captured graph");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? PD_OK : fail_cuda(e, "graph launch");
}

void pd_batch_destroy(pd_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    free_batch(b);
}

// ---------------------------------------------------------------------------
// Autotuner: times candidate launch settings on the caller's frames.
int pd_autotune(pd_ctx* c, const uint16_t* frames_dev, uint32_t n_frames, pd_tuning* best,
                float* best_us_per_frame) {
    if (!c || !frames_dev || !n_frames) return fail(PD_EINVAL, "autotune needs frames");
    if (!aligned(frames_dev, 16)) return fail(PD_EALIGN, "frames must be 16-byte aligned");
    const pd::ChainParams& p = c->params;
    const size_t fpx = p.frame_px;
    const uint32_t cap = (uint32_t)std::min<uint64_t>((uint64_t)n_frames * fpx / 8 + 1024, 1u << 26);
    pd_hit* hits = nullptr;
    uint32_t* nh = nullptr;
    uint32_t* save_map = nullptr;
    unsigned long long* save_hist = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    int rc = PD_OK;
    // the summaries are saved and restored around the timing runs
    if ((e = cudaMalloc(&hits, (size_t)cap * sizeof(pd_hit))) ||
        (e = cudaMalloc(&nh, sizeof(uint32_t))) ||
        (e = cudaMalloc(&save_map, fpx * 4)) ||
        (e = cudaMalloc(&save_hist, 2 * (size_t)p.hist_bins * 8)) ||
        (e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) {
        rc = fail(PD_ENOMEM, "autotune allocation failed");
    }
    pd_tuning orig{};
    pd_get_tuning(c, &orig);
    pd_tuning best_t = orig;
    float best_ms = 1e30f;
    if (!rc) {
        cudaMemcpy(save_map, c->d_count_map, fpx * 4, cudaMemcpyDeviceToDevice);
        cudaMemcpy(save_hist, c->d_hist_pix, p.hist_bins * 8, cudaMemcpyDeviceToDevice);
        cudaMemcpy(save_hist + p.hist_bins, c->d_hist_hit, p.hist_bins * 8,
                   cudaMemcpyDeviceToDevice);
        const size_t fbytes = fpx * 2;
        std::vector<uint32_t> chunks;
        for (size_t mb : {96, 192, 384, 768}) {
            const uint32_t cf = (uint32_t)std::max<size_t>(1, ((size_t)mb << 20) / fbytes);
            if (std::find(chunks.begin(), chunks.end(), cf) == chunks.end()) chunks.push_back(cf);
        }
        // band heights around each stencil's default (explicit values, since
        // one band_rows setting applies to both stencils)
        auto band_set = [](uint32_t rb) {
            std::vector<uint32_t> v = {rb};
            for (uint32_t x : {rb / 2, rb * 3 / 2, rb * 2})
                if (x >= 2 && x != rb) v.push_back(x);
            return v;
        };
        const uint32_t lean_rb0 = c->lean_cfg.rb, band_rb0 = c->band_cfg.rb;
        pd_outputs o{};
        o.hits = hits;
        o.hit_capacity = cap;
        o.n_hits = nh;
        std::vector<pd_tuning> cands;
        if (c->use_fused && !c->matched)
            cands.push_back(pd_tuning{orig.chunk_frames, orig.band_rows, 1, 0, orig.kernels});
        std::vector<uint32_t> kopts = {orig.kernels};
        if ((c->use_lean || c->use_bank) && !c->matched) kopts = {1u, 2u};
        // the work-queue launch: one launch per call, so chunking, band
        // height and overlap are not varied
        if (c->use_queue && !c->matched) cands.push_back(pd_tuning{orig.chunk_frames, 0, 1, 1, 3});
        for (uint32_t k : kopts) {
            std::vector<uint32_t> bands = {0};
            if (!c->matched && k == 1 && c->use_lean) bands = band_set(lean_rb0);
            else if (!c->matched && c->use_band) bands = band_set(band_rb0);
            for (uint32_t cf : chunks)
                for (uint32_t bd : bands)
                    for (uint32_t ov : {1u, 0u}) cands.push_back(pd_tuning{cf, bd, ov, 1, k});
        }
        for (const pd_tuning& t : cands) {
                    if (pd_set_tuning(c, &t) != PD_OK) continue;
                    if (run_chain(c, frames_dev, n_frames, 0, &o, nullptr) != PD_OK) continue;
                    cudaEventRecord(e0, nullptr);
                    for (int k = 0; k < 2; k++) run_chain(c, frames_dev, n_frames, 0, &o, nullptr);
                    cudaEventRecord(e1, nullptr);
                    if ((e = cudaEventSynchronize(e1))) {
                        rc = fail_cuda(e, "autotune run");
                        break;
                    }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        pd_get_tuning(c, &best_t);
                    }
                }
        cudaMemcpy(c->d_count_map, save_map, fpx * 4, cudaMemcpyDeviceToDevice);
        cudaMemcpy(c->d_hist_pix, save_hist, p.hist_bins * 8, cudaMemcpyDeviceToDevice);
        cudaMemcpy(c->d_hist_hit, save_hist + p.hist_bins, p.hist_bins * 8,
                   cudaMemcpyDeviceToDevice);
    }
    pd_set_tuning(c, rc ? &orig : &best_t);
    cudaFree(hits);
    cudaFree(nh);
    cudaFree(save_map);
    cudaFree(save_hist);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    if (best) *best = best_t;
    if (best_us_per_frame) *best_us_per_frame = best_ms * 1e3f / (2.0f * n_frames);
    return best_ms < 1e30f ? PD_OK : fail(PD_ECUDA, "autotune: no candidate ran");
}

int pd_net_gather(pd_ctx* c, const uint16_t* frames_dev, uint32_t frame_base, const float* cm_dev,
                  const pd_hit* hits_dev, uint32_t n_hits, float* patches_dev, void* stream) {
    if (!c || (n_hits && (!frames_dev || !cm_dev || !hits_dev || !patches_dev)))
        return fail(PD_EINVAL, "pd_net_gather: NULL argument");
    cudaError_t e = pd::launch_gather(c->params, frames_dev, frame_base, cm_dev, hits_dev, n_hits,
                                      patches_dev, (cudaStream_t)stream,
                                      c->multigain ? &c->mg : nullptr);
    return e == cudaSuccess ? PD_OK : fail_cuda(e, "pd_net_gather");
}

void pd_destroy(pd_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    free_ctx(c);
}

}  // extern "C"
