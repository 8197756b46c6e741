// svt_serve.cu -- a trigger-style serving loop around the fused path.
//
// The paper measures the loop "data in -> GPU -> data out" of a trigger node
// (Sec. 3 and Sec. 4.2, where moving data to and from the GPU takes about a
// fifth of the total).  This is its single-GPU form with continuous
// batching:
//   * callers submit events by reference: a pointer to the event's words in
//     pinned host memory, which must stay valid until the event's result is
//     delivered (one copy of the data in host memory, as with GPUDirect);
//   * a dispatcher thread admits queued events into free device slots.  Each
//     slot owns device buffers for a batch of at most max_words words,
//     max_events events and max_roads roads (the device-memory budget); an
//     event is admitted when it fits what is left of the slot being filled;
//   * a slot's batch is one H2D copy per contiguous run of event words, one
//     H2D copy of its sizes and event offsets, a replay of the slot's
//     captured CUDA graph (the fused path of svt_run_sized) and one D2H copy
//     of its status, event table and records, all on the slot's own stream,
//     so batches in different slots overlap on the device;
//   * completion is polled with cudaEventQuery; every event gets its status,
//     its records and its arrival-to-delivery latency;
//   * a batch whose status reports a data error is re-run event by event, so
//     a corrupt event fails alone.
// No device memory is allocated here: the caller passes the device workspace
// (svt_server_sizes) and the library carves the slots out of it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "svt_kernels.cuh"

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Pending {
    const uint32_t *words;
    uint32_t n_words;
    uint32_t n_roads;
    uint64_t tag;
    int64_t t_arrive;
    uint32_t *dst;       // caller buffer for the records (may be null)
    bool single;         // re-run alone after a failed batch
};

// Bytes before the records in a slot's output block: the status word, then
// the event -> first road table, padded so the records start 256-aligned.
size_t out_header_bytes(uint64_t max_events) {
    return svt::align_up(16 + 4 * (max_events + 1), 256);
}

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t_start = nullptr, t_end = nullptr;   // device timestamps (tracing)
    bool traced = false;                              // this batch goes into the trace
    bool timed = false;                               // ... with device timestamps
    svt_graph graph = nullptr;
    svt_graph graph_small = nullptr;   // for batches of at most small_batch_events events
    bool busy = false;
    std::vector<Pending> events;
    uint64_t n_words = 0, n_roads = 0;
    int64_t t_dispatch = 0, t_enqueued = 0;
    uint32_t queued_after = 0;
    // device: the input block is {n_words, n_events, event offsets...} so that
    // one copy carries the sizes and the offsets; the output block is
    // {status, pad, event -> first road, pad, records} so that one copy
    // brings the whole result back
    uint32_t *d_words = nullptr;
    uint64_t *d_in = nullptr;        // 2 + max_events + 1
    uint64_t *d_sizes = nullptr;     // d_in
    uint64_t *d_off = nullptr;       // d_in + 2
    char *d_outblk = nullptr;
    uint64_t *d_status = nullptr;
    uint32_t *d_event_road = nullptr;
    uint32_t *d_out = nullptr;       // 6 * max_roads
    uint64_t *d_counts = nullptr;
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    // plain per-stage path (mode 1)
    uint32_t *d_road_word = nullptr, *d_road_nhit = nullptr, *d_road_flags = nullptr;
    uint64_t *d_comb_off = nullptr, *d_n_roads = nullptr, *d_n_combs = nullptr;
    uint32_t *d_comb_road = nullptr, *d_comb_hits = nullptr, *d_fit_chi2 = nullptr;
    int32_t *d_fit_par = nullptr;
    svt_best *d_best = nullptr;
    void *d_ws_unpack = nullptr, *d_ws_combine = nullptr;
    size_t ws_unpack = 0, ws_combine = 0;
    // pinned host mirrors of the two blocks (carved from the caller's pinned buffer)
    uint64_t *h_in = nullptr;
    char *h_outblk = nullptr;
    uint64_t *h_status = nullptr;
    uint32_t *h_event_road = nullptr;
    uint32_t *h_out = nullptr;
};

// Carves one slot's device buffers (base may be null to size them).
size_t carve_slot_device(void *base, const svt_server_config &c, const svt_schedule *sched,
                         Slot *s) {
    svt::Carver d(base);
    Slot t;
    Slot &o = s ? *s : t;
    const size_t hdr = out_header_bytes(c.max_events);
    o.d_words = d.take<uint32_t>(c.max_words + 4);
    o.d_in = d.take<uint64_t>(2 + c.max_events + 1);
    o.d_sizes = o.d_in;
    o.d_off = o.d_in ? o.d_in + 2 : nullptr;
    o.d_outblk = d.take<char>(hdr + 24 * c.max_roads);
    o.d_status = (uint64_t *)o.d_outblk;
    o.d_event_road = o.d_outblk ? (uint32_t *)(o.d_outblk + 16) : nullptr;
    o.d_out = o.d_outblk ? (uint32_t *)(o.d_outblk + hdr) : nullptr;
    o.d_counts = d.take<uint64_t>(4);
    if (c.mode == 0) {
        o.ws_bytes = svt_run_workspace_size(c.max_words, c.max_events, c.max_roads, sched);
        o.d_ws = d.take<char>(o.ws_bytes);
    } else {
        o.d_road_word = d.take<uint32_t>(c.max_roads);
        o.d_road_nhit = d.take<uint32_t>(c.max_roads);
        o.d_road_flags = d.take<uint32_t>(c.max_roads);
        o.d_comb_off = d.take<uint64_t>(c.max_roads + 1);
        o.d_n_roads = d.take<uint64_t>(1);
        o.d_n_combs = d.take<uint64_t>(1);
        o.d_comb_road = d.take<uint32_t>(c.max_combs);
        o.d_comb_hits = d.take<uint32_t>(c.max_combs);
        o.d_fit_chi2 = d.take<uint32_t>(c.max_combs);
        o.d_fit_par = d.take<int32_t>(3 * c.max_combs);
        o.d_best = d.take<svt_best>(c.max_roads);
        o.ws_unpack = svt_unpack_workspace_size(c.max_words);
        o.d_ws_unpack = d.take<char>(o.ws_unpack);
        o.ws_combine = svt_combine_workspace_size(c.max_roads);
        o.d_ws_combine = d.take<char>(o.ws_combine);
    }
    return d.size();
}

size_t carve_slot_host(void *base, const svt_server_config &c, Slot *s) {
    svt::Carver h(base);
    Slot t;
    Slot &o = s ? *s : t;
    const size_t hdr = out_header_bytes(c.max_events);
    o.h_in = h.take<uint64_t>(2 + c.max_events + 1);
    o.h_outblk = h.take<char>(hdr + 24 * c.max_roads);
    o.h_status = (uint64_t *)o.h_outblk;
    o.h_event_road = o.h_outblk ? (uint32_t *)(o.h_outblk + 16) : nullptr;
    o.h_out = o.h_outblk ? (uint32_t *)(o.h_outblk + hdr) : nullptr;
    return h.size();
}

}  // namespace

struct svt_server_s {
    svt_server_config c;
    svt_config cfg;
    svt_schedule sched;
    bool has_sched = false;
    const int16_t *F = nullptr, *q = nullptr;
    int device = 0;
    size_t out_hdr = 0;
    std::vector<Slot> slots;
    std::mutex mu;                     // pending, done
    std::condition_variable cv_work;   // the dispatcher: new events or stop
    std::condition_variable cv_done;   // pollers: new results
    std::deque<Pending> pending;
    std::deque<svt_event_result> done;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> queued_words{0};
    svt_server_stats stats{};
    std::mutex stats_mu;
    // per-batch trace (caller-owned buffer), written by the dispatcher
    std::mutex trace_mu;
    svt_batch_trace *trace = nullptr;
    uint64_t trace_cap = 0, trace_n = 0;
    cudaStream_t aux = nullptr;
    cudaEvent_t trace_base = nullptr;
    bool trace_on = false;
    bool trace_dev = false;   // also record device timestamps

    void run();
    bool launch(Slot &s);
    void finish(Slot &s);
    int submit_at(const uint32_t *h_words, uint32_t n_words, uint64_t tag, uint32_t *h_records,
                  int64_t t_arrive);
};

bool svt_server_s::launch(Slot &s) {
    // the caller holds no lock; s.events is filled
    const int64_t t0 = now_ns();
    const size_t E = s.events.size();
    uint64_t off = 0;
    uint64_t *h_off = s.h_in + 2;
    for (size_t e = 0; e < E; ++e) {
        h_off[e] = off;
        off += s.events[e].n_words;
    }
    h_off[E] = off;
    s.h_in[0] = off;   // sizes: n_words
    s.h_in[1] = E;     //        n_events
    s.n_words = off;
    cudaStream_t st = s.st;
    {
        std::lock_guard<std::mutex> g(trace_mu);
        s.traced = trace_on;
        s.timed = trace_on && trace_dev;
    }
    if (s.timed && cudaEventRecord(s.t_start, st) != cudaSuccess) return false;
    // one H2D per contiguous run of event words
    size_t e = 0;
    while (e < E) {
        const uint32_t *src = s.events[e].words;
        uint64_t n = s.events[e].n_words, dst = h_off[e];
        size_t f = e + 1;
        while (f < E && s.events[f].words == src + n) {
            n += s.events[f].n_words;
            ++f;
        }
        if (n && cudaMemcpyAsync(s.d_words + dst, src, n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return false;
        e = f;
    }
    if (cudaMemcpyAsync(s.d_in, s.h_in, (E + 3) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return false;
    if (c.mode == 0) {
        const bool small = s.graph_small && E <= c.small_batch_events;
        if (svt_graph_launch(small ? s.graph_small : s.graph, st) != SVT_OK) return false;
    } else {
        // the plain per-stage path, sized by the host-known batch
        const svt_config *fc = &cfg;
        if (svt_unpack(s.d_words, off, s.d_off, E, fc->n_sectors, fc->xft_pairs, c.max_roads,
                       s.d_road_word, s.d_road_nhit, s.d_event_road, s.d_n_roads, s.d_status,
                       s.d_ws_unpack, s.ws_unpack, st) != SVT_OK ||
            svt_combine(s.d_road_nhit, s.d_n_roads, c.max_roads, fc, c.max_combs, s.d_road_flags,
                        s.d_comb_off, s.d_comb_road, s.d_comb_hits, s.d_n_combs, s.d_status,
                        s.d_ws_combine, s.ws_combine, st) != SVT_OK ||
            svt_fit(s.d_words, s.d_road_word, s.d_road_nhit, s.d_comb_road, s.d_comb_hits,
                    s.d_n_combs, c.max_combs, F, q, fc, s.d_fit_chi2, s.d_fit_par, s.d_status,
                    st) != SVT_OK ||
            svt_select(s.d_fit_chi2, s.d_fit_par, c.max_combs, s.d_comb_off, s.d_road_flags,
                       s.d_n_roads, c.max_roads, fc, s.d_best, s.d_status, st) != SVT_OK ||
            svt_format(s.d_best, s.d_words, s.d_road_word, s.d_n_roads, c.max_roads, s.d_out,
                       s.d_status, st) != SVT_OK)
            return false;
    }
    // status, event table and records in one copy
    const size_t back = out_hdr + s.n_roads * 24;
    if (cudaMemcpyAsync(s.h_outblk, s.d_outblk, back, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return false;
    if (s.timed && cudaEventRecord(s.t_end, st) != cudaSuccess) return false;
    if (cudaEventRecord(s.done, st) != cudaSuccess) return false;
    s.busy = true;
    s.t_enqueued = now_ns();
    std::lock_guard<std::mutex> g(stats_mu);
    stats.batches += 1;
    stats.h2d_bytes += s.n_words * 4 + (E + 3) * 8;
    stats.d2h_bytes += back;
    stats.launch_ns += (uint64_t)(s.t_enqueued - t0);
    if (E > stats.max_batch_events) stats.max_batch_events = E;
    return true;
}

void svt_server_s::finish(Slot &s) {
    const int64_t t = now_ns();
    const uint64_t status = *s.h_status;
    const size_t E = s.events.size();
    if (s.traced) {
        std::lock_guard<std::mutex> g(trace_mu);
        if (trace_on && trace_n < trace_cap) {
            svt_batch_trace &b = trace[trace_n++];
            b.slot = (uint32_t)(&s - slots.data());
            b.n_events = (uint32_t)E;
            b.n_roads = (uint32_t)s.n_roads;
            b.queued_after = s.queued_after;
            int64_t first = s.events.empty() ? s.t_dispatch : s.events[0].t_arrive;
            for (const Pending &p : s.events) first = std::min(first, p.t_arrive);
            b.t_first_arrive_ns = first;
            b.t_dispatch_ns = s.t_dispatch;
            b.t_enqueued_ns = s.t_enqueued;
            b.t_done_ns = t;
            float a = -1e-3f, z = -1e-3f;
            if (s.timed && cudaEventElapsedTime(&a, trace_base, s.t_start) != cudaSuccess) a = -1e-3f;
            if (s.timed && cudaEventElapsedTime(&z, trace_base, s.t_end) != cudaSuccess) z = -1e-3f;
            b.dev_start_us = a * 1e3f;
            b.dev_end_us = z * 1e3f;
        }
    }
    if (status != SVT_STATUS_OK && E > 1) {
        // a data error somewhere in the batch: run its events one by one
        {
            std::lock_guard<std::mutex> g(mu);
            for (size_t e = E; e-- > 0;) {
                Pending p = s.events[e];
                p.single = true;
                pending.push_front(p);
                queued_words += p.n_words;
            }
        }
        std::lock_guard<std::mutex> g(stats_mu);
        stats.retried_batches += 1;
    } else {
        std::vector<svt_event_result> res(E);
        for (size_t e = 0; e < E; ++e) {
            const Pending &p = s.events[e];
            svt_event_result &r = res[e];
            r.tag = p.tag;
            r.status = status;
            r.n_roads = p.n_roads;
            r.t_arrive_ns = p.t_arrive;
            if (status == SVT_STATUS_OK && p.dst && p.n_roads) {
                const uint32_t r0 = s.h_event_road[e];
                std::memcpy(p.dst, s.h_out + (size_t)r0 * 6, (size_t)p.n_roads * 24);
            }
        }
        // the events are complete once their records are in the callers' buffers
        const int64_t t_out = now_ns();
        for (size_t e = 0; e < E; ++e) res[e].latency_ns = (uint64_t)(t_out - s.events[e].t_arrive);
        {
            std::lock_guard<std::mutex> g(mu);
            for (auto &r : res) done.push_back(r);
        }
        std::lock_guard<std::mutex> g(stats_mu);
        stats.events_done += E;
        if (status != SVT_STATUS_OK) stats.events_failed += E;
        stats.finish_ns += (uint64_t)(now_ns() - t);
    }
    s.events.clear();
    s.busy = false;
    cv_done.notify_all();
}

void svt_server_s::run() {
    cudaSetDevice(device);
    while (!stop.load(std::memory_order_acquire)) {
        bool progress = false;
        for (auto &s : slots) {
            if (s.busy && cudaEventQuery(s.done) == cudaSuccess) {
                finish(s);
                progress = true;
            }
        }
        for (auto &s : slots) {
            if (s.busy) continue;
            {
                std::unique_lock<std::mutex> g(mu);
                if (pending.empty()) break;
                const uint64_t depth = pending.size();
                uint64_t w = 0, r = 0;
                while (!pending.empty()) {
                    const Pending &p = pending.front();
                    if (p.single && !s.events.empty()) break;
                    if (s.events.size() + 1 > c.max_events || w + p.n_words > c.max_words ||
                        r + p.n_roads > c.max_roads)
                        break;
                    w += p.n_words;
                    r += p.n_roads;
                    s.events.push_back(p);
                    pending.pop_front();
                    if (s.events.back().single) break;
                }
                s.n_roads = r;
                s.queued_after = (uint32_t)pending.size();
                queued_words -= w;
                g.unlock();
                s.t_dispatch = now_ns();
                std::lock_guard<std::mutex> gs(stats_mu);
                if (depth > stats.max_queued) stats.max_queued = depth;
            }
            if (s.events.empty()) continue;
            if (!launch(s)) {
                // a CUDA failure: report every event of the batch as failed
                std::lock_guard<std::mutex> g(mu);
                for (auto &p : s.events) {
                    svt_event_result res{};
                    res.tag = p.tag;
                    res.status = ((uint64_t)0 << 8) | SVT_ERR_CUDA;
                    res.n_roads = p.n_roads;
                    res.latency_ns = (uint64_t)(now_ns() - p.t_arrive);
                    res.t_arrive_ns = p.t_arrive;
                    done.push_back(res);
                }
                {
                    std::lock_guard<std::mutex> gs(stats_mu);
                    stats.events_failed += s.events.size();
                }
                s.events.clear();
                cv_done.notify_all();
            }
            progress = true;
        }
        if (!progress) {
            bool any_busy = false;
            for (auto &s : slots) any_busy |= s.busy;
            if (!any_busy) {
                std::unique_lock<std::mutex> g(mu);
                if (pending.empty() && !stop.load())
                    cv_work.wait_for(g, std::chrono::microseconds(200));
            }
        }
    }
}

int svt_server_s::submit_at(const uint32_t *h_words, uint32_t n_words, uint64_t tag,
                            uint32_t *h_records, int64_t t_arrive) {
    if (!h_words || n_words < 1) return SVT_ERR_BAD_ARG;
    const uint32_t n_roads = h_words[0] & 0xFFFu;
    if (n_words > c.max_words || n_roads > c.max_roads) return SVT_ERR_OOM;
    if (c.max_queued_words &&
        queued_words.load(std::memory_order_relaxed) + n_words > c.max_queued_words) {
        std::lock_guard<std::mutex> g(stats_mu);
        stats.rejected += 1;
        return SVT_ERR_OOM;
    }
    Pending p{h_words, n_words, n_roads, tag, t_arrive, h_records, false};
    {
        std::lock_guard<std::mutex> g(mu);
        pending.push_back(p);
        queued_words += n_words;
    }
    cv_work.notify_one();
    return SVT_OK;
}

extern "C" {

int svt_server_sizes(const svt_server_config *c, const svt_schedule *sched, size_t *device_bytes,
                     size_t *pinned_bytes) {
    if (!c || !device_bytes || !pinned_bytes || c->n_slots < 1 || c->n_slots > 16 ||
        c->max_events < 1 || c->max_words < 1 || c->max_roads < 1 || c->mode > 1 ||
        (c->mode == 1 && c->max_combs < 1) || c->max_words >= (1ull << 32) ||
        c->max_events >= (1ull << 31) || c->max_roads >= (1ull << 31))
        return SVT_ERR_BAD_ARG;
    *device_bytes = carve_slot_device(nullptr, *c, sched, nullptr) * c->n_slots;
    *pinned_bytes = carve_slot_host(nullptr, *c, nullptr) * c->n_slots;
    return SVT_OK;
}

namespace {
void release_slots(svt_server srv) {
    for (auto &s : srv->slots) {
        if (s.graph) svt_graph_destroy(s.graph);
        if (s.graph_small) svt_graph_destroy(s.graph_small);
        if (s.done) cudaEventDestroy(s.done);
        if (s.t_start) cudaEventDestroy(s.t_start);
        if (s.t_end) cudaEventDestroy(s.t_end);
        if (s.st) cudaStreamDestroy(s.st);
    }
    if (srv->trace_base) cudaEventDestroy(srv->trace_base);
    if (srv->aux) cudaStreamDestroy(srv->aux);
}
}  // namespace

int svt_server_create(const svt_server_config *c, const int16_t *d_F, const int16_t *d_q,
                      const svt_config *cfg, const svt_schedule *sched, void *d_workspace,
                      size_t workspace_bytes, void *h_pinned, size_t pinned_bytes,
                      svt_server *out) {
    size_t need_d = 0, need_h = 0;
    if (!out || !d_F || !d_q || !cfg || !d_workspace || !h_pinned) return SVT_ERR_BAD_ARG;
    int rc = svt_server_sizes(c, sched, &need_d, &need_h);
    if (rc != SVT_OK) return rc;
    if (workspace_bytes < need_d || pinned_bytes < need_h) return SVT_ERR_BAD_ARG;
    if (c->device_budget && need_d > c->device_budget) return SVT_ERR_OOM;
    if (((uintptr_t)d_workspace & 255u) || ((uintptr_t)h_pinned & 255u)) return SVT_ERR_BAD_ARG;
    svt_server srv = new svt_server_s();
    srv->c = *c;
    srv->cfg = *cfg;
    if (sched) {
        srv->sched = *sched;
        srv->has_sched = true;
    }
    srv->F = d_F;
    srv->q = d_q;
    srv->out_hdr = out_header_bytes(c->max_events);
    cudaGetDevice(&srv->device);
    const size_t dev_slot = carve_slot_device(nullptr, *c, sched, nullptr);
    const size_t host_slot = carve_slot_host(nullptr, *c, nullptr);
    srv->slots.resize(c->n_slots);
    if (cudaStreamCreateWithFlags(&srv->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&srv->trace_base) != cudaSuccess)
        rc = SVT_ERR_CUDA;
    for (uint32_t i = 0; i < c->n_slots && rc == SVT_OK; ++i) {
        Slot &s = srv->slots[i];
        carve_slot_device((char *)d_workspace + dev_slot * i, *c, sched, &s);
        carve_slot_host((char *)h_pinned + host_slot * i, *c, &s);
        if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&s.t_start) != cudaSuccess || cudaEventCreate(&s.t_end) != cudaSuccess) {
            rc = SVT_ERR_CUDA;
            break;
        }
        if (c->mode == 0) {
            rc = svt_graph_create(s.d_words, c->max_words, s.d_off, c->max_events, s.d_sizes, d_F,
                                  d_q, cfg, c->max_roads, s.d_out, s.d_event_road, s.d_counts,
                                  s.d_status, s.d_ws, s.ws_bytes,
                                  srv->has_sched ? &srv->sched : nullptr, &s.graph);
            if (rc != SVT_OK) break;
            if (c->small_batch_events) {
                svt_schedule small = srv->has_sched ? srv->sched : svt_schedule{0, 0, 0, 0, 0, 0};
                small.blocks_per_sm = c->small_blocks_per_sm ? c->small_blocks_per_sm : 1u;
                rc = svt_graph_create(s.d_words, c->max_words, s.d_off, c->max_events, s.d_sizes,
                                      d_F, d_q, cfg, c->max_roads, s.d_out, s.d_event_road,
                                      s.d_counts, s.d_status, s.d_ws, s.ws_bytes, &small,
                                      &s.graph_small);
                if (rc != SVT_OK) break;
            }
        }
    }
    if (rc != SVT_OK) {
        release_slots(srv);
        delete srv;
        return rc;
    }
    srv->worker = std::thread([srv] { srv->run(); });
    *out = srv;
    return SVT_OK;
}

int svt_server_submit(svt_server srv, const uint32_t *h_words, uint32_t n_words, uint64_t tag,
                      uint32_t *h_records) {
    if (!srv) return SVT_ERR_BAD_ARG;
    return srv->submit_at(h_words, n_words, tag, h_records, now_ns());
}

int svt_server_poll(svt_server srv, svt_event_result *out, uint32_t max_results,
                    uint32_t *n_out, uint32_t wait_us) {
    if (!srv || !n_out || (max_results && !out)) return SVT_ERR_BAD_ARG;
    std::unique_lock<std::mutex> g(srv->mu);
    if (srv->done.empty() && wait_us)
        srv->cv_done.wait_for(g, std::chrono::microseconds(wait_us),
                              [srv] { return !srv->done.empty(); });
    uint32_t n = 0;
    while (n < max_results && !srv->done.empty()) {
        out[n++] = srv->done.front();
        srv->done.pop_front();
    }
    *n_out = n;
    return SVT_OK;
}

int svt_server_stats_get(svt_server srv, svt_server_stats *out) {
    if (!srv || !out) return SVT_ERR_BAD_ARG;
    {
        std::lock_guard<std::mutex> g(srv->stats_mu);
        *out = srv->stats;
    }
    std::lock_guard<std::mutex> g2(srv->mu);
    out->queued = srv->pending.size();
    return SVT_OK;
}

int svt_server_stats_reset(svt_server srv) {
    if (!srv) return SVT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> g(srv->stats_mu);
    srv->stats = svt_server_stats{};
    return SVT_OK;
}

int svt_server_trace(svt_server srv, svt_batch_trace *buf, uint64_t cap, uint32_t device_times) {
    if (!srv || (buf && !cap)) return SVT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> g(srv->trace_mu);
    if (buf && device_times) {
        // the time origin of the device timestamps: an event on an idle stream
        if (cudaEventRecord(srv->trace_base, srv->aux) != cudaSuccess ||
            cudaEventSynchronize(srv->trace_base) != cudaSuccess)
            return SVT_ERR_CUDA;
    }
    srv->trace = buf;
    srv->trace_cap = buf ? cap : 0;
    if (buf) srv->trace_n = 0;   // stopping keeps the count for svt_server_trace_count
    srv->trace_on = buf != nullptr;
    srv->trace_dev = buf != nullptr && device_times != 0;
    return SVT_OK;
}

int svt_server_trace_count(svt_server srv, uint64_t *n) {
    if (!srv || !n) return SVT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> g(srv->trace_mu);
    *n = srv->trace_n;
    return SVT_OK;
}

int svt_server_destroy(svt_server srv) {
    if (!srv) return SVT_ERR_BAD_ARG;
    srv->stop.store(true, std::memory_order_release);
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    for (auto &s : srv->slots)
        if (s.busy) cudaEventSynchronize(s.done);
    release_slots(srv);
    delete srv;
    return SVT_OK;
}

// Poisson arrivals (rate_hz) of n_events events taken in turn from a pool of
// events in pinned memory.  Arrival times come from a SplitMix64 stream (seed)
// turned into exponential gaps; an event's latency is counted from its
// scheduled arrival time, so a late submission counts against the server and
// not in its favour.  The submitting thread sleeps until shortly before an
// arrival that is more than 200 us away and spins for the rest.
int svt_server_bench_poisson(svt_server srv, const uint32_t *h_pool, const uint64_t *pool_off,
                             uint32_t n_pool, double rate_hz, uint64_t n_events, uint64_t seed,
                             uint32_t *h_records, const uint64_t *rec_off, uint64_t *lat_ns,
                             double *wall_s) {
    if (!srv || !h_pool || !pool_off || !n_pool || rate_hz <= 0 || !lat_ns || !wall_s ||
        (h_records && !rec_off))
        return SVT_ERR_BAD_ARG;
    std::atomic<uint64_t> got{0};
    int64_t t_first = 0, t_last = 0;
    std::thread consumer([&] {
        std::vector<svt_event_result> buf(4096);
        while (got.load() < n_events) {
            uint32_t n = 0;
            svt_server_poll(srv, buf.data(), (uint32_t)buf.size(), &n, 1000);
            for (uint32_t i = 0; i < n; ++i) {
                const svt_event_result &r = buf[i];
                if (r.tag < n_events)
                    lat_ns[r.tag] = r.status == SVT_STATUS_OK ? r.latency_ns : ~0ull;
            }
            if (n) t_last = now_ns();
            got += n;
        }
    });
    uint64_t x = seed;
    auto next_u = [&x]() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    int64_t t = now_ns();
    t_first = t;
    int rc = SVT_OK;
    for (uint64_t i = 0; i < n_events; ++i) {
        t += (int64_t)(-std::log(next_u()) / rate_hz * 1e9);
        int64_t ahead = t - now_ns();
        if (ahead > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(ahead - 100000));
        while (now_ns() < t) {
        }
        const uint32_t k = (uint32_t)(i % n_pool);
        const uint32_t *w = h_pool + pool_off[k];
        const uint32_t nw = (uint32_t)(pool_off[k + 1] - pool_off[k]);
        uint32_t *dst = h_records ? h_records + 6 * rec_off[i] : nullptr;
        int s;
        while ((s = srv->submit_at(w, nw, i, dst, t)) == SVT_ERR_OOM && srv->c.max_queued_words) {
            // back-pressure: the admission queue is full; retry shortly
            std::this_thread::yield();
        }
        if (s != SVT_OK) {
            rc = s;
            lat_ns[i] = ~0ull;
            got += 1;
        }
    }
    consumer.join();
    *wall_s = (double)(t_last - t_first) * 1e-9;
    return rc;
}

}  // extern "C"
