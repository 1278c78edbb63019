// pd_serve.cu — streaming server: continuous batching of frames of several
// detector geometries from page-locked host rings, with latency statistics
// and compact hit lists.
//
// The paper times processing of frames already in memory and anticipates an
// online pipeline at LCLS-II rates (sections "Introduction", "Methods",
// "Conclusions"); this is that pipeline's host side.  A producer (a DAQ, or
// the built-in Poisson replay) writes frames into a per-geometry ring of
// page-locked slots and commits them with their arrival time.  A dispatcher
// thread keeps up to n_slots device batches in flight: whenever a slot is
// free it takes every committed frame (up to max_batch_frames per geometry),
// uploads them on the slot's stream, runs one batched launch (pd_batch) over
// all geometries, and copies the hit counts and then the hits back.  Frames
// that arrive while others are on the GPU join the next free slot, and the
// slots' copies and kernels overlap on the device.  Results are grouped per
// frame, encoded compactly, and timed from arrival to hits on the host.
#include <cuda_runtime.h>
#include <math.h>
#include <pthread.h>
#include <sched.h>
#include <sys/resource.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pd.h"
#include "pd_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch())
        .count();
}

// Pin a thread to the k-th CPU (modulo their number) of the CPUs this
// process may run on (a container's CPU set is often a subset of the online
// CPUs); false if the system refuses (the thread then keeps its mask).
bool pin_to_cpu(pthread_t th, uint32_t k) {
    cpu_set_t allowed;
    if (sched_getaffinity(0, sizeof(allowed), &allowed) != 0) return false;
    const int n = CPU_COUNT(&allowed);
    if (n <= 0) return false;
    int want = (int)(k % (uint32_t)n), cpu = -1;
    for (int c = 0; c < CPU_SETSIZE; c++)
        if (CPU_ISSET(c, &allowed) && want-- == 0) {
            cpu = c;
            break;
        }
    if (cpu < 0) return false;
    cpu_set_t set;
    CPU_ZERO(&set);
    CPU_SET(cpu, &set);
    return pthread_setaffinity_np(th, sizeof(set), &set) == 0;
}

enum : uint8_t { kFree = 0, kCommitted = 1, kInFlight = 2, kAcquired = 3 };

struct Ring {
    pd_ctx* ctx = nullptr;
    uint32_t frame_px = 0;
    uint32_t cap = 0;
    uint16_t* host = nullptr;  // page-locked, cap frames
    std::vector<uint8_t> state;
    std::vector<uint64_t> id;
    std::vector<int64_t> t_arrival;
    uint32_t head = 0;         // next slot to dispatch
    uint32_t fill = 0;         // next slot for the replay producer
};

struct Pending {  // one frame inside a device batch
    uint32_t geom, ring_slot;
    uint64_t id;
    int64_t t_arrival;
};

enum : int { kSlotFree = 0, kSlotRunning = 1, kSlotHits = 2, kSlotEncoding = 3 };

struct DevSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_up = nullptr, ev_counts = nullptr, ev_hits = nullptr;
    bool uploaded = false;            // the batch's frames are on the device (ring slots freed)
    pd_batch* batch = nullptr;
    std::vector<uint16_t*> d_frames;  // per geometry
    std::vector<pd_hit*> d_hits;
    std::vector<uint32_t*> d_nhits;
    uint32_t* h_nhits = nullptr;      // page-locked, one per geometry
    std::vector<pd_hit*> h_hits;      // page-locked
    std::atomic<int> state{kSlotFree};
    std::atomic<uint32_t> tasks_left{0};
    int64_t t_issue = 0, t_counts = 0, t_done = 0;  // issued, counts seen, hits on the host
    std::vector<std::vector<Pending>> frames;   // per geometry, batch order
};

// One geometry's hits of a finished batch, grouped by frame.  The encoders
// own it once it is built, so that the device slot is free again before
// the frames are encoded.
struct Job {
    uint32_t geom = 0;
    int64_t t_done = 0;                 // hits on the host
    std::vector<Pending> frames;        // batch order
    std::vector<pd_hit> grouped;        // hits by frame
    std::vector<uint32_t> offset;       // frames + 1
    std::atomic<uint32_t> ranges_left{0};
};

// Encoder work: group a slot's hits of one geometry (slot set), or sort and
// encode frames [first, last) of a job.
struct Task {
    DevSlot* slot = nullptr;
    std::shared_ptr<Job> job;
    uint32_t geom = 0, first = 0, last = 0;
};

constexpr uint32_t kEncodeRange = 8;  // frames per encode task

struct FrameResult {
    uint32_t geom = 0;
    uint32_t n_hits = 0;
    double latency_us = 0;
    std::vector<pd_hit> hits;     // sorted by pixel, when keep_hits
    std::vector<uint8_t> stream;  // compact encoding, when keep_hits
};

// Hits of one frame ordered by pixel: LSD radix sort of (pixel, index) in
// 11-bit digits, as many passes as the largest pixel index needs.
void sort_by_pixel(const pd_hit* h, uint32_t n, std::vector<uint64_t>& a,
                   std::vector<uint64_t>& tmp) {
    a.resize(n);
    uint32_t mx = 0;
    for (uint32_t i = 0; i < n; i++) {
        a[i] = ((uint64_t)h[i].pixel << 32) | i;
        mx = std::max(mx, h[i].pixel);
    }
    if (n < 64) {
        std::sort(a.begin(), a.end());
        return;
    }
    tmp.resize(n);
    uint32_t cnt[2048];
    for (int shift = 32; shift < 64 && (shift == 32 || (mx >> (shift - 32)) != 0); shift += 11) {
        memset(cnt, 0, sizeof(cnt));
        for (uint32_t i = 0; i < n; i++) cnt[(a[i] >> shift) & 2047]++;
        uint32_t sum = 0;
        for (int d = 0; d < 2048; d++) {
            const uint32_t c = cnt[d];
            cnt[d] = sum;
            sum += c;
        }
        for (uint32_t i = 0; i < n; i++) tmp[cnt[(a[i] >> shift) & 2047]++] = a[i];
        a.swap(tmp);
    }
}

// Compact encoding of one frame's hits in the given order (pixel ascending):
// varint hit count, then per hit the varint pixel delta, energy as u16 in
// 1/256 keV (nearest, clipped), dx and dy as i8 in 1/128 pixel (nearest,
// clipped to +-127), count u8.  Returns the bytes written (or needed).
size_t encode_sorted(const pd_hit* h, const uint64_t* order, uint32_t n, uint8_t* out,
                     size_t cap) {
    size_t o = 0;
    auto put = [&](uint8_t v) {
        if (out && o < cap) out[o] = v;
        o++;
    };
    auto varint = [&](uint32_t v) {
        do {
            put((uint8_t)((v & 0x7F) | (v > 0x7F ? 0x80 : 0)));
            v >>= 7;
        } while (v);
    };
    varint(n);
    uint32_t prev = 0;
    for (uint32_t i = 0; i < n; i++) {
        const pd_hit& x = h[(uint32_t)order[i]];
        varint(x.pixel - prev);
        prev = x.pixel;
        const float e = std::min(65535.0f, std::max(0.0f, rintf(x.energy_kev * 256.0f)));
        const uint16_t eq = (uint16_t)e;
        put((uint8_t)(eq & 0xFF));
        put((uint8_t)(eq >> 8));
        for (float q : {x.dx, x.dy}) {
            const float v = std::min(127.0f, std::max(-127.0f, rintf(q * 128.0f)));
            put((uint8_t)(int8_t)v);
        }
        put(x.count);
    }
    return o;
}

}  // namespace

struct pd_server {
    pd_serve_config cfg{};
    std::vector<Ring> rings;
    std::vector<std::unique_ptr<DevSlot>> slots;
    int device = 0;
    std::mutex mu;                    // rings, results, statistics
    std::thread dispatcher;
    std::vector<std::thread> encoders;
    std::mutex qmu;                   // encoder queue
    std::condition_variable qcv;
    std::deque<Task> queue;
    std::atomic<bool> stop{false};
    std::atomic<bool> hold{false};    // no new batches while set
    std::atomic<int> error{PD_OK};
    std::unordered_map<uint64_t, FrameResult> results;
    std::vector<double> latencies;
    std::vector<double> lat_wait, lat_device;  // per frame: ring queue, issue to counts
    double sum_fetch_us = 0, sum_encode_us = 0, replay_late_max_us = 0;
    double sum_upload_us = 0, sum_run_us = 0;  // per batch, device clock
    uint64_t encoded_batches = 0, replay_late = 0, timed_batches = 0;
    uint64_t committed = 0, done = 0, rejected = 0, raw_bytes = 0, comp_bytes = 0, hits = 0;
    uint64_t batches = 0, max_batch_seen = 0;
    int64_t t_first = 0, t_last = 0;
};

namespace {

void destroy_slot(DevSlot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    for (auto p : s.d_frames) cudaFree(p);
    for (auto p : s.d_hits) cudaFree(p);
    for (auto p : s.d_nhits) cudaFree(p);
    for (auto p : s.h_hits) cudaFreeHost(p);
    cudaFreeHost(s.h_nhits);
    if (s.batch) pd_batch_destroy(s.batch);
    if (s.ev_start) cudaEventDestroy(s.ev_start);
    if (s.ev_up) cudaEventDestroy(s.ev_up);
    if (s.ev_counts) cudaEventDestroy(s.ev_counts);
    if (s.ev_hits) cudaEventDestroy(s.ev_hits);
    if (s.stream) cudaStreamDestroy(s.stream);
}

// Issue one batch on a free slot from the committed frames (dispatcher
// thread).  Returns true if anything was issued.
bool issue(pd_server* sv, DevSlot& s) {
    const uint32_t G = (uint32_t)sv->rings.size();
    std::vector<std::pair<uint32_t, uint32_t>> take(G);  // (first ring slot, count)
    uint32_t total = 0;
    int64_t t_issue = 0;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        for (uint32_t g = 0; g < G; g++) {
            Ring& r = sv->rings[g];
            // committed slots form a run from head in fill order; take it up
            // to the ring's end (the next batch continues at slot 0)
            uint32_t n = 0;
            while (n < sv->cfg.max_batch_frames && r.head + n < r.cap &&
                   r.state[r.head + n] == kCommitted)
                n++;
            take[g] = {r.head, n};
            for (uint32_t k = 0; k < n; k++) r.state[r.head + k] = kInFlight;
            r.head = (r.head + n) % r.cap;
            total += n;
        }
        if (!total) return false;
        t_issue = now_ns();
        for (uint32_t g = 0; g < G; g++) {
            s.frames[g].clear();
            Ring& r = sv->rings[g];
            for (uint32_t k = 0; k < take[g].second; k++) {
                const uint32_t slot = take[g].first + k;
                s.frames[g].push_back({g, slot, r.id[slot], r.t_arrival[slot]});
            }
        }
        sv->max_batch_seen = std::max<uint64_t>(sv->max_batch_seen, total);
        sv->batches++;
    }
    std::vector<pd_batch_item> items;
    if (cudaEventRecord(s.ev_start, s.stream) != cudaSuccess) sv->error.store(PD_ECUDA);
    for (uint32_t g = 0; g < G; g++) {
        const uint32_t n = take[g].second;
        if (!n) continue;
        Ring& r = sv->rings[g];
        const size_t fb = (size_t)r.frame_px * 2;
        if (cudaMemcpyAsync(s.d_frames[g], r.host + (size_t)take[g].first * r.frame_px, n * fb,
                            cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
            sv->error.store(PD_ECUDA);
        pd_batch_item it{};
        it.ctx = r.ctx;
        it.frames = s.d_frames[g];
        it.n_frames = n;
        it.frame_base = 0;
        it.out.hits = s.d_hits[g];
        it.out.hit_capacity = sv->cfg.max_batch_frames * sv->cfg.hits_per_frame;
        it.out.n_hits = s.d_nhits[g];
        items.push_back(it);
    }
    if (cudaEventRecord(s.ev_up, s.stream) != cudaSuccess) sv->error.store(PD_ECUDA);
    s.uploaded = false;
    int rc = pd_batch_process(s.batch, items.data(), (uint32_t)items.size(), s.stream);
    if (rc) sv->error.store(rc);
    for (uint32_t g = 0; g < G; g++) {
        s.h_nhits[g] = 0;
        if (take[g].second && cudaMemcpyAsync(&s.h_nhits[g], s.d_nhits[g], 4,
                                              cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
            sv->error.store(PD_ECUDA);
    }
    if (cudaEventRecord(s.ev_counts, s.stream) != cudaSuccess) sv->error.store(PD_ECUDA);
    s.t_issue = t_issue;
    s.state.store(kSlotRunning);
    return true;
}

// Once the batch's upload has completed its frames are on the device, and
// their ring slots go back to the producer (the batch keeps their ids and
// arrival times); once only, so that a slot the producer has taken again is
// never released twice.
void frames_uploaded(pd_server* sv, DevSlot& s) {
    if (s.uploaded) return;
    s.uploaded = true;
    std::lock_guard<std::mutex> lock(sv->mu);
    for (uint32_t g = 0; g < (uint32_t)sv->rings.size(); g++)
        for (const Pending& p : s.frames[g]) sv->rings[g].state[p.ring_slot] = kFree;
}

// After the counts are on the host (the upload before them is complete):
// download exactly the hits.
void fetch_hits(pd_server* sv, DevSlot& s) {
    frames_uploaded(sv, s);
    const uint32_t cap = sv->cfg.max_batch_frames * sv->cfg.hits_per_frame;
    s.t_counts = now_ns();
    float up_ms = 0, run_ms = 0;
    cudaEventElapsedTime(&up_ms, s.ev_start, s.ev_up);
    cudaEventElapsedTime(&run_ms, s.ev_up, s.ev_counts);
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->sum_upload_us += up_ms * 1e3;
        sv->sum_run_us += run_ms * 1e3;
        sv->timed_batches++;
    }
    for (uint32_t g = 0; g < (uint32_t)sv->rings.size(); g++) {
        if (s.frames[g].empty()) continue;
        const uint32_t n = std::min(s.h_nhits[g], cap);
        if (n && cudaMemcpyAsync(s.h_hits[g], s.d_hits[g], (size_t)n * sizeof(pd_hit),
                                 cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
            sv->error.store(PD_ECUDA);
    }
    if (cudaEventRecord(s.ev_hits, s.stream) != cudaSuccess) sv->error.store(PD_ECUDA);
    s.state.store(kSlotHits);
}

void push_tasks(pd_server* sv, const std::vector<Task>& t) {
    {
        std::lock_guard<std::mutex> lock(sv->qmu);
        for (const Task& x : t) sv->queue.push_back(x);
    }
    if (t.size() == 1)
        sv->qcv.notify_one();
    else
        sv->qcv.notify_all();
}

// Hits are on the host: stamp every frame's latency and hand the slot to
// the encoders.
void hits_arrived(pd_server* sv, DevSlot& s) {
    const int64_t t_done = now_ns();
    const uint32_t G = (uint32_t)sv->rings.size();
    std::vector<Task> tasks;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        for (uint32_t g = 0; g < G; g++) {
            if (s.frames[g].empty()) continue;
            for (const Pending& p : s.frames[g]) {
                sv->latencies.push_back((t_done - p.t_arrival) / 1e3);
                sv->lat_wait.push_back((s.t_issue - p.t_arrival) / 1e3);
                sv->lat_device.push_back((s.t_counts - s.t_issue) / 1e3);
                sv->sum_fetch_us += (t_done - s.t_counts) / 1e3;
            }
            Task t;
            t.slot = &s;
            t.geom = g;
            tasks.push_back(t);
        }
        sv->t_last = t_done;
    }
    s.t_done = t_done;
    s.state.store(kSlotEncoding);
    s.tasks_left.store((uint32_t)tasks.size());
    push_tasks(sv, tasks);
}

// The last group task of a batch frees its slot.
void task_done(DevSlot& s) {
    if (s.tasks_left.fetch_sub(1) == 1) s.state.store(kSlotFree);
}

void group_task(pd_server* sv, DevSlot& s, uint32_t g) {
    const uint32_t cap = sv->cfg.max_batch_frames * sv->cfg.hits_per_frame;
    if (s.h_nhits[g] > cap) sv->error.store(PD_EOVERFLOW);
    const uint32_t n = std::min(s.h_nhits[g], cap);
    auto job = std::make_shared<Job>();
    job->geom = g;
    job->t_done = s.t_done;
    job->frames = s.frames[g];
    const uint32_t F = (uint32_t)job->frames.size();
    const pd_hit* h = s.h_hits[g];
    std::vector<uint32_t>& off = job->offset;
    off.assign(F + 1, 0);
    for (uint32_t i = 0; i < n; i++)
        if (h[i].frame < F) off[h[i].frame + 1]++;
    for (uint32_t k = 0; k < F; k++) off[k + 1] += off[k];
    std::vector<pd_hit>& out = job->grouped;
    out.resize(off[F]);
    std::vector<uint32_t> at(off.begin(), off.end() - 1);
    for (uint32_t i = 0; i < n; i++)
        if (h[i].frame < F) out[at[h[i].frame]++] = h[i];
    task_done(s);  // the slot's buffers are no longer read
    std::vector<Task> t;
    for (uint32_t k = 0; k < F; k += kEncodeRange) {
        Task x;
        x.job = job;
        x.geom = g;
        x.first = k;
        x.last = std::min(F, k + kEncodeRange);
        t.push_back(x);
    }
    job->ranges_left.store((uint32_t)t.size());
    push_tasks(sv, t);
}

void encode_task(pd_server* sv, Job& job, uint32_t first, uint32_t last) {
    thread_local std::vector<uint64_t> order, tmp;
    const uint32_t g = job.geom;
    size_t comp = 0;
    uint64_t hits = 0;
    std::vector<std::pair<uint64_t, FrameResult>> kept;
    for (uint32_t k = first; k < last; k++) {
        const pd_hit* h = job.grouped.data() + job.offset[k];
        const uint32_t n = job.offset[k + 1] - job.offset[k];
        sort_by_pixel(h, n, order, tmp);
        const size_t cb = encode_sorted(h, order.data(), n, nullptr, 0);
        comp += cb;
        hits += n;
        if (sv->cfg.keep_hits) {
            const Pending& p = job.frames[k];
            FrameResult res;
            res.geom = g;
            res.n_hits = n;
            res.stream.resize(cb);
            encode_sorted(h, order.data(), n, res.stream.data(), cb);
            res.hits.resize(n);
            for (uint32_t i = 0; i < n; i++) {
                res.hits[i] = h[(uint32_t)order[i]];
                res.hits[i].frame = (uint32_t)p.id;
            }
            res.latency_us = (job.t_done - p.t_arrival) / 1e3;
            kept.emplace_back(p.id, std::move(res));
        }
    }
    const bool last_range = job.ranges_left.fetch_sub(1) == 1;
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->comp_bytes += comp;
    sv->raw_bytes += (uint64_t)(last - first) * sv->rings[g].frame_px * 2;
    sv->hits += hits;
    sv->done += last - first;
    for (auto& kv : kept) sv->results[kv.first] = std::move(kv.second);
    if (last_range) {
        sv->sum_encode_us += (now_ns() - job.t_done) / 1e3;
        sv->encoded_batches++;
    }
}

void encoder_loop(pd_server* sv) {
    // encoding is off the latency path (a batch's slot frees before its
    // frames are encoded): on busy host cores the dispatcher and the
    // producer come first (Linux nice values are per thread)
    setpriority(PRIO_PROCESS, 0, 5);
    while (true) {
        Task t;
        {
            std::unique_lock<std::mutex> lock(sv->qmu);
            sv->qcv.wait(lock, [&] { return sv->stop.load() || !sv->queue.empty(); });
            if (sv->queue.empty()) return;  // stopping
            t = sv->queue.front();
            sv->queue.pop_front();
        }
        if (t.slot)
            group_task(sv, *t.slot, t.geom);
        else
            encode_task(sv, *t.job, t.first, t.last);
    }
}

// An event that reports an error (not cudaErrorNotReady) completes the slot
// with the error recorded, so that drain() ends.
bool event_done(pd_server* sv, cudaEvent_t ev) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaErrorNotReady) return false;
    if (e != cudaSuccess) sv->error.store(PD_ECUDA);
    return true;
}

// Admission: a free slot takes every committed frame, but only while fewer
// than max_uploading batches are still uploading, so frames queue in the
// host ring rather than behind a deep queue of copies on the link.
void dispatch_loop(pd_server* sv) {
    cudaSetDevice(sv->device);
    const uint32_t max_up = sv->cfg.max_uploading;
    while (!sv->stop.load(std::memory_order_relaxed)) {
        bool busy = false;
        uint32_t uploading = 0;
        for (auto& sp : sv->slots) {
            DevSlot& s = *sp;
            if (s.state.load() == kSlotRunning && !s.uploaded) {
                if (event_done(sv, s.ev_up))
                    frames_uploaded(sv, s);
                else
                    uploading++;
            }
            if (s.state.load() == kSlotRunning && event_done(sv, s.ev_counts)) {
                fetch_hits(sv, s);
                busy = true;
            }
            if (s.state.load() == kSlotHits && event_done(sv, s.ev_hits)) {
                hits_arrived(sv, s);
                busy = true;
            }
        }
        if (!sv->hold.load(std::memory_order_relaxed))
            for (auto& sp : sv->slots) {
                if (uploading >= max_up) break;
                if (sp->state.load() == kSlotFree && issue(sv, *sp)) {
                    busy = true;
                    uploading++;
                }
            }
        if (!busy) std::this_thread::yield();
    }
}

}  // namespace

extern "C" {

int pd_server_create(pd_ctx* const* ctxs, uint32_t n_geometries, const pd_serve_config* cfg,
                     pd_server** out) {
    if (!out || !ctxs || !n_geometries || !cfg || !cfg->max_batch_frames || !cfg->ring_frames ||
        !cfg->hits_per_frame || !cfg->n_slots ||
        (uint64_t)cfg->max_batch_frames * cfg->hits_per_frame > 0xFFFFFFFFull)
        return pd::internal_fail(PD_EINVAL, "pd_server_create: invalid arguments");
    *out = nullptr;
    pd_server* sv = new (std::nothrow) pd_server();
    if (!sv) return pd::internal_fail(PD_ENOMEM, "host allocation failed");
    sv->cfg = *cfg;
    cudaGetDevice(&sv->device);
    // admission: the device budget bounds the batches in flight
    size_t slot_bytes = 0;
    for (uint32_t g = 0; g < n_geometries; g++) {
        pd_info info{};
        if (pd_query(ctxs[g], &info)) {
            delete sv;
            return pd::internal_fail(PD_EINVAL, "pd_server_create: invalid context");
        }
        slot_bytes += (size_t)cfg->max_batch_frames *
                      ((size_t)info.pixels_per_frame * 2 + (size_t)cfg->hits_per_frame * sizeof(pd_hit) +
                       (size_t)info.cm_values_per_frame * 4);
    }
    // device_budget = 0: the free device memory now, less 1 GiB of headroom
    uint64_t budget = cfg->device_budget;
    if (!budget) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            delete sv;
            return pd::internal_fail(PD_ECUDA, "pd_server_create: cudaMemGetInfo failed");
        }
        budget = free_b > (1ull << 30) ? free_b - (1ull << 30) : 0;
    }
    uint32_t n_slots = (uint32_t)std::min<uint64_t>(cfg->n_slots, budget / slot_bytes);
    if (n_slots == 0) {
        delete sv;
        return pd::internal_fail(PD_EBUSY, "pd_server_create: device budget below one batch");
    }
    sv->cfg.n_slots = n_slots;
    if (!sv->cfg.max_uploading) sv->cfg.max_uploading = 1;
    int rc = PD_OK;
    for (uint32_t g = 0; g < n_geometries && !rc; g++) {
        Ring r;
        pd_info info{};
        pd_query(ctxs[g], &info);
        r.ctx = ctxs[g];
        r.frame_px = info.pixels_per_frame;
        r.cap = cfg->ring_frames;
        r.state.assign(r.cap, kFree);
        r.id.assign(r.cap, 0);
        r.t_arrival.assign(r.cap, 0);
        if (cudaMallocHost(&r.host, (size_t)r.cap * r.frame_px * 2) != cudaSuccess)
            rc = pd::internal_fail(PD_ENOMEM, "pd_server_create: host ring allocation failed");
        sv->rings.push_back(r);
    }
    for (uint32_t i = 0; i < n_slots && !rc; i++) {
        sv->slots.emplace_back(new (std::nothrow) DevSlot());
        if (!sv->slots.back()) {
            sv->slots.pop_back();
            rc = pd::internal_fail(PD_ENOMEM, "host allocation failed");
        }
    }
    const uint32_t cap = cfg->max_batch_frames * cfg->hits_per_frame;
    for (auto& sp : sv->slots) {
        if (rc) break;
        DevSlot& s = *sp;
        s.frames.resize(n_geometries);
        bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreate(&s.ev_start) == cudaSuccess &&
                  cudaEventCreate(&s.ev_up) == cudaSuccess &&
                  cudaEventCreate(&s.ev_counts) == cudaSuccess &&
                  cudaEventCreateWithFlags(&s.ev_hits, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMallocHost(&s.h_nhits, n_geometries * 4) == cudaSuccess;
        uint64_t cm_vals = 0;
        for (uint32_t g = 0; g < n_geometries && ok; g++) {
            pd_info info{};
            pd_query(ctxs[g], &info);
            cm_vals += (uint64_t)cfg->max_batch_frames * info.cm_values_per_frame;
            uint16_t* f = nullptr;
            pd_hit* dh = nullptr;
            uint32_t* dn = nullptr;
            pd_hit* hh = nullptr;
            ok = cudaMalloc(&f, (size_t)cfg->max_batch_frames * info.pixels_per_frame * 2) == cudaSuccess &&
                 cudaMalloc(&dh, (size_t)cap * sizeof(pd_hit)) == cudaSuccess &&
                 cudaMalloc(&dn, 4) == cudaSuccess &&
                 cudaMallocHost(&hh, (size_t)cap * sizeof(pd_hit)) == cudaSuccess;
            s.d_frames.push_back(f);
            s.d_hits.push_back(dh);
            s.d_nhits.push_back(dn);
            s.h_hits.push_back(hh);
        }
        if (!ok || pd_batch_create(n_geometries, cm_vals, &s.batch) != PD_OK)
            rc = pd::internal_fail(PD_ENOMEM, "pd_server_create: slot allocation failed");
    }
    if (rc) {
        for (auto& s : sv->slots) destroy_slot(*s);
        for (auto& r : sv->rings) cudaFreeHost(r.host);
        delete sv;
        return rc;
    }
    uint32_t n_enc = cfg->encode_threads;
    if (!n_enc) n_enc = std::max(1u, std::min(8u, std::thread::hardware_concurrency() / 2));
    for (uint32_t i = 0; i < n_enc; i++) sv->encoders.emplace_back(encoder_loop, sv);
    sv->dispatcher = std::thread(dispatch_loop, sv);
    if (cfg->cpu_pin) {
        // dedicated cores keep the dispatcher and encoders off the cores other
        // work of the host uses (latency tails came from sharing them)
        pin_to_cpu(sv->dispatcher.native_handle(), cfg->cpu_pin - 1);
        for (uint32_t i = 0; i < n_enc; i++)
            pin_to_cpu(sv->encoders[i].native_handle(), cfg->cpu_pin + i);
    }
    *out = sv;
    return PD_OK;
}

int pd_server_slots(const pd_server* sv, uint32_t* n_slots) {
    if (!sv || !n_slots) return pd::internal_fail(PD_EINVAL, "NULL argument");
    *n_slots = sv->cfg.n_slots;
    return PD_OK;
}

int pd_server_hold(pd_server* sv, int hold) {
    if (!sv) return pd::internal_fail(PD_EINVAL, "NULL server");
    sv->hold.store(hold != 0);
    return PD_OK;
}

int pd_server_ring_frame(pd_server* sv, uint32_t geom, uint32_t slot, uint16_t** frame_host) {
    if (!sv || !frame_host || geom >= sv->rings.size() || slot >= sv->rings[geom].cap)
        return pd::internal_fail(PD_EINVAL, "pd_server_ring_frame: geometry or slot out of range");
    *frame_host = sv->rings[geom].host + (size_t)slot * sv->rings[geom].frame_px;
    return PD_OK;
}

int pd_server_acquire(pd_server* sv, uint32_t geom, uint16_t** frame_host, uint32_t* slot) {
    if (!sv || !frame_host || !slot || geom >= sv->rings.size())
        return pd::internal_fail(PD_EINVAL, "pd_server_acquire: invalid arguments");
    std::lock_guard<std::mutex> lock(sv->mu);
    Ring& r = sv->rings[geom];
    if (r.state[r.fill] != kFree) {
        sv->rejected++;
        return PD_EBUSY;
    }
    r.state[r.fill] = kAcquired;
    *slot = r.fill;
    *frame_host = r.host + (size_t)r.fill * r.frame_px;
    r.fill = (r.fill + 1) % r.cap;
    return PD_OK;
}

namespace {
int commit_at(pd_server* sv, uint32_t geom, uint32_t slot, uint64_t frame_id, int64_t t_arrival) {
    std::lock_guard<std::mutex> lock(sv->mu);
    Ring& r = sv->rings[geom];
    if (r.state[slot] != kAcquired)
        return pd::internal_fail(PD_EINVAL, "pd_server_commit: slot not acquired");
    r.id[slot] = frame_id;
    r.t_arrival[slot] = t_arrival;
    r.state[slot] = kCommitted;
    if (!sv->t_first) sv->t_first = t_arrival;
    sv->committed++;
    return PD_OK;
}
}  // namespace

int pd_server_commit(pd_server* sv, uint32_t geom, uint32_t slot, uint64_t frame_id) {
    if (!sv || geom >= sv->rings.size() || slot >= sv->rings[geom].cap)
        return pd::internal_fail(PD_EINVAL, "pd_server_commit: invalid arguments");
    return commit_at(sv, geom, slot, frame_id, now_ns());
}

int pd_server_replay(pd_server* sv, double rate_hz, double duration_s, const float* mix,
                     uint64_t seed, uint64_t first_id) {
    if (!sv || !(rate_hz > 0) || !(duration_s > 0))
        return pd::internal_fail(PD_EINVAL, "pd_server_replay: invalid arguments");
    const uint32_t G = (uint32_t)sv->rings.size();
    std::vector<double> cdf(G);
    double tot = 0;
    for (uint32_t g = 0; g < G; g++) tot += mix ? std::max(0.0f, mix[g]) : 1.0;
    double acc = 0;
    for (uint32_t g = 0; g < G; g++) {
        acc += (mix ? std::max(0.0f, mix[g]) : 1.0) / tot;
        cdf[g] = acc;
    }
    // the replaying thread on its own core while it runs (mask put back after)
    cpu_set_t old_mask;
    const bool pinned = sv->cfg.cpu_pin &&
                        pthread_getaffinity_np(pthread_self(), sizeof(old_mask), &old_mask) == 0 &&
                        pin_to_cpu(pthread_self(),
                                   sv->cfg.cpu_pin + (uint32_t)sv->encoders.size());
    struct Restore {
        bool on;
        cpu_set_t* m;
        ~Restore() {
            if (on) pthread_setaffinity_np(pthread_self(), sizeof(*m), m);
        }
    } restore{pinned, &old_mask};
    std::mt19937_64 rng(seed);
    std::exponential_distribution<double> gap(rate_hz);
    std::uniform_real_distribution<double> pick(0.0, 1.0);
    const int64_t t0 = now_ns(), t_end = t0 + (int64_t)(duration_s * 1e9);
    double t = 0, late_max = 0;
    uint64_t id = first_id, n_late = 0;
    while (true) {
        t += gap(rng);
        const int64_t ta = t0 + (int64_t)(t * 1e9);
        if (ta >= t_end) break;
        const double u = pick(rng);
        uint32_t g = 0;
        while (g + 1 < G && u > cdf[g]) g++;
        int64_t tn;
        while ((tn = now_ns()) < ta) {
        }
        // arrivals the producer reached late (it was descheduled or held up)
        const double late_us = (tn - ta) / 1e3;
        if (late_us > 20.0) n_late++;
        late_max = std::max(late_max, late_us);
        uint16_t* ptr = nullptr;
        uint32_t slot = 0;
        if (pd_server_acquire(sv, g, &ptr, &slot) != PD_OK) continue;  // ring full: dropped
        commit_at(sv, g, slot, id++, ta);
    }
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->replay_late += n_late;
        sv->replay_late_max_us = std::max(sv->replay_late_max_us, late_max);
    }
    return sv->error.load();
}

int pd_server_drain(pd_server* sv, double timeout_s) {
    if (!sv) return pd::internal_fail(PD_EINVAL, "NULL server");
    const int64_t t_end = now_ns() + (int64_t)(timeout_s * 1e9);
    while (true) {
        {
            std::lock_guard<std::mutex> lock(sv->mu);
            if (sv->done >= sv->committed) break;
        }
        if (now_ns() > t_end) return pd::internal_fail(PD_ETIMEDOUT, "pd_server_drain: timed out");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    const int e = sv->error.load();
    return e ? pd::internal_fail(e, "pd_server: a batch failed") : PD_OK;
}

int pd_server_stats(pd_server* sv, pd_serve_stats* st) {
    if (!sv || !st) return pd::internal_fail(PD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    memset(st, 0, sizeof(*st));
    st->frames_committed = sv->committed;
    st->frames_done = sv->done;
    st->frames_rejected = sv->rejected;
    st->batches = sv->batches;
    st->max_batch_frames = sv->max_batch_seen;
    st->raw_bytes = sv->raw_bytes;
    st->compressed_bytes = sv->comp_bytes;
    st->hits = sv->hits;
    st->elapsed_s = sv->done ? (sv->t_last - sv->t_first) / 1e9 : 0.0;
    if (!sv->latencies.empty()) {
        std::vector<double> l = sv->latencies;
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
        st->p50_us = q(0.50);
        st->p99_us = q(0.99);
        st->max_us = l.back();
        double s = 0;
        for (double x : l) s += x;
        st->mean_us = s / l.size();
        for (int k = 0; k < 2; k++) {
            std::vector<double> v = k ? sv->lat_device : sv->lat_wait;
            std::sort(v.begin(), v.end());
            double m = 0;
            for (double x : v) m += x;
            const double p99 = v[std::min(v.size() - 1, (size_t)(0.99 * (v.size() - 1) + 0.5))];
            (k ? st->device_mean_us : st->wait_mean_us) = m / v.size();
            (k ? st->device_p99_us : st->wait_p99_us) = p99;
        }
        st->fetch_mean_us = sv->sum_fetch_us / l.size();
    }
    st->encode_mean_us = sv->encoded_batches ? sv->sum_encode_us / sv->encoded_batches : 0.0;
    if (sv->timed_batches) {
        st->upload_mean_us = sv->sum_upload_us / sv->timed_batches;
        st->run_mean_us = sv->sum_run_us / sv->timed_batches;
    }
    st->replay_late = sv->replay_late;
    st->replay_late_max_us = sv->replay_late_max_us;
    return PD_OK;
}

int pd_server_reset_stats(pd_server* sv) {
    if (!sv) return pd::internal_fail(PD_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->latencies.clear();
    sv->lat_wait.clear();
    sv->lat_device.clear();
    sv->sum_fetch_us = sv->sum_encode_us = sv->replay_late_max_us = 0;
    sv->sum_upload_us = sv->sum_run_us = 0;
    sv->encoded_batches = sv->replay_late = sv->timed_batches = 0;
    sv->results.clear();
    sv->committed -= sv->done;
    sv->done = 0;
    sv->t_first = sv->t_last = 0;
    sv->rejected = sv->raw_bytes = sv->comp_bytes = sv->hits = sv->batches = sv->max_batch_seen = 0;
    return PD_OK;
}

int pd_server_frame_hits(pd_server* sv, uint64_t frame_id, pd_hit* out, uint32_t cap,
                         uint32_t* n_hits, float* latency_us) {
    if (!sv || !n_hits) return pd::internal_fail(PD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->results.find(frame_id);
    if (it == sv->results.end()) return pd::internal_fail(PD_EINVAL, "frame not done or unknown");
    *n_hits = it->second.n_hits;
    if (latency_us) *latency_us = (float)it->second.latency_us;
    const uint32_t k = std::min<uint32_t>(cap, (uint32_t)it->second.hits.size());
    if (out && k) memcpy(out, it->second.hits.data(), k * sizeof(pd_hit));
    return PD_OK;
}

int pd_server_frame_stream(pd_server* sv, uint64_t frame_id, uint8_t* out, size_t cap,
                           size_t* len) {
    if (!sv || !len) return pd::internal_fail(PD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->results.find(frame_id);
    if (it == sv->results.end()) return pd::internal_fail(PD_EINVAL, "frame not done or unknown");
    const std::vector<uint8_t>& b = it->second.stream;
    *len = b.size();
    if (out && cap) memcpy(out, b.data(), std::min(cap, b.size()));
    return out && cap < b.size() ? pd::internal_fail(PD_EOVERFLOW, "output too small") : PD_OK;
}

int pd_compress_hits(const pd_hit* hits, uint32_t n, uint8_t* out, size_t cap, size_t* out_len) {
    if ((n && !hits) || !out_len) return pd::internal_fail(PD_EINVAL, "NULL argument");
    std::vector<uint64_t> order, tmp;
    sort_by_pixel(hits, n, order, tmp);
    *out_len = encode_sorted(hits, order.data(), n, out, cap);
    return *out_len > cap && out ? pd::internal_fail(PD_EOVERFLOW, "output too small") : PD_OK;
}

int pd_decompress_hits(const uint8_t* in, size_t len, uint32_t frame, pd_hit* out, uint32_t cap,
                       uint32_t* n_out) {
    if (!in || !n_out) return pd::internal_fail(PD_EINVAL, "NULL argument");
    size_t o = 0;
    auto varint = [&](uint32_t* v) -> bool {
        uint32_t x = 0;
        int sh = 0;
        while (o < len) {
            const uint8_t b = in[o++];
            x |= (uint32_t)(b & 0x7F) << sh;
            if (!(b & 0x80)) {
                *v = x;
                return true;
            }
            sh += 7;
            if (sh > 28) return false;
        }
        return false;
    };
    uint32_t n = 0;
    if (!varint(&n)) return pd::internal_fail(PD_EINVAL, "truncated hit stream");
    uint32_t pix = 0;
    for (uint32_t i = 0; i < n; i++) {
        uint32_t d = 0;
        if (!varint(&d) || o + 5 > len) return pd::internal_fail(PD_EINVAL, "truncated hit stream");
        pix += d;
        const uint16_t eq = (uint16_t)(in[o] | (in[o + 1] << 8));
        const int8_t qx = (int8_t)in[o + 2], qy = (int8_t)in[o + 3];
        const uint8_t cnt = in[o + 4];
        o += 5;
        if (out && i < cap) {
            pd_hit h{};
            h.frame = frame;
            h.pixel = pix;
            h.energy_kev = eq / 256.0f;
            h.dx = qx / 128.0f;
            h.dy = qy / 128.0f;
            h.count = cnt;
            out[i] = h;
        }
    }
    *n_out = n;
    return PD_OK;
}

void pd_server_destroy(pd_server* sv) {
    if (!sv) return;
    sv->stop.store(true);
    if (sv->dispatcher.joinable()) sv->dispatcher.join();
    {
        std::lock_guard<std::mutex> lock(sv->qmu);
        sv->queue.clear();
    }
    sv->qcv.notify_all();
    for (auto& t : sv->encoders) t.join();
    for (auto& s : sv->slots) destroy_slot(*s);
    for (auto& r : sv->rings) cudaFreeHost(r.host);
    delete sv;
}

}  // extern "C"
