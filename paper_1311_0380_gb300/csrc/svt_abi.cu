// svt_abi.cu -- the extern "C" entry points of include/svt.h: argument checks,
// workspace carving and the launch sequence of each call.
#include <mutex>

#include "svt_kernels.cuh"

namespace svt {
size_t scan_u64_tile_count(uint64_t cap);
}

using namespace svt;

namespace {

constexpr int MAX_DEVICES = 64;
int g_sm_count[MAX_DEVICES];
std::once_flag g_sm_once[MAX_DEVICES];

int sm_count_of(int dev) {
    if (dev < 0 || dev >= MAX_DEVICES) return 0;
    std::call_once(g_sm_once[dev], [dev] {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 0;
        g_sm_count[dev] = n;
    });
    return g_sm_count[dev];
}

int current_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    return sm_count_of(dev);
}

bool config_ok(const svt_config *c) {
    if (!c) return false;
    if (c->oshift < 9 || c->oshift > 31) return false;
    if (c->qshift > 24) return false;
    if (c->max_comb < 1) return false;
    if (c->min_layers > 6) return false;
    if (c->n_sectors < 1 || c->n_sectors > 512) return false;
    if (c->xft_pairs > 1) return false;
    return true;
}

svt_schedule resolve(const svt_schedule *s) {
    svt_schedule r{8, 0, 16, 4, 4096, 0};
    if (s) {
        if (s->warps_per_block) r.warps_per_block = s->warps_per_block;
        if (s->blocks_per_sm) r.blocks_per_sm = s->blocks_per_sm;
        if (s->rows_per_item) r.rows_per_item = s->rows_per_item;
        if (s->roads_per_chunk) r.roads_per_chunk = s->roads_per_chunk;
        if (s->small_max) r.small_max = s->small_max;
        r.pair_small = s->pair_small;
    }
    return r;
}

bool schedule_ok(const svt_schedule &s) {
    return s.warps_per_block >= 1 && s.warps_per_block <= 16 && s.blocks_per_sm <= 32 &&
           s.rows_per_item >= 1 && s.rows_per_item <= 1024 && s.roads_per_chunk >= 1 &&
           s.roads_per_chunk <= 32 && s.small_max >= 1 && s.pair_small <= 3 &&
           (s.pair_small != 3 || s.warps_per_block <= 12);
}

// word tiles: up to 16 blocks of 128 threads per SM at once (grid-stride
// over the tiles beyond)
int tile_grid() {
    int sms = current_sm_count();
    return (sms > 0 ? sms : 1) * 16;
}

// warps' road grouping of the fit kernel for a schedule's pair_small
uint32_t fit_group(uint32_t pair_small) {
    return pair_small == 3 ? 32u : pair_small == 2 ? 4u : pair_small == 1 ? 2u : 1u;
}

int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SVT_OK : SVT_ERR_CUDA;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Workspace layout of svt_unpack.
struct UnpackWs {
    Dims *dims;
    unsigned long long *tile_state;   // road counts the tiles publish (look-back)
    uint32_t *tile_ticket;            // next tile to take
    uint32_t *first_ev;
    size_t bytes;
};
UnpackWs carve_unpack(void *base, uint64_t max_words) {
    Carver c(base);
    UnpackWs w;
    w.dims = c.take<Dims>(1);
    w.tile_state = c.take<unsigned long long>(n_tiles(max_words) + 1);
    w.tile_ticket = c.take<uint32_t>(1);
    w.first_ev = c.take<uint32_t>(n_tiles(max_words) + 1);
    w.bytes = c.size();
    return w;
}

// Workspace layout of svt_run.
struct RunWs {
    Dims *dims;
    uint64_t *counts;
    uint64_t *work;   // [0] split-road reservation, [1] the fit kernel's two queue counters
    unsigned long long *tile_state;   // road counts the tiles publish (look-back)
    uint32_t *tile_ticket, *first_ev;
    RoadDesc *desc;
    uint32_t *big_road, *big_item_off, *big_pending;
    unsigned long long *key;
    uint32_t *event_road;
    size_t bytes;
};
RunWs carve_run(void *base, uint64_t max_words, uint64_t max_events, uint64_t road_cap) {
    Carver c(base);
    RunWs w;
    const uint64_t T = n_tiles(max_words);
    w.dims = c.take<Dims>(1);
    w.counts = c.take<uint64_t>(4);
    w.work = c.take<uint64_t>(2);
    w.tile_state = c.take<unsigned long long>(T + 1);
    w.tile_ticket = c.take<uint32_t>(1);
    w.first_ev = c.take<uint32_t>(T + 1);
    w.desc = c.take<RoadDesc>(road_cap);
    w.big_road = c.take<uint32_t>(road_cap);
    w.big_item_off = c.take<uint32_t>(road_cap);
    w.big_pending = c.take<uint32_t>(road_cap);
    w.key = c.take<unsigned long long>(road_cap);
    w.event_road = c.take<uint32_t>(max_events + 1);
    w.bytes = c.size();
    return w;
}

// Sector index of the calibration tracks.
struct CalibIndex {
    uint32_t *counts;
    int32_t *sector_off, *sector_item, *item_sector, *item_start, *n_items;
    uint32_t max_items;
    size_t bytes;
};
CalibIndex carve_calib_index(const void *base, uint64_t n, uint32_t S) {
    Carver c(const_cast<void *>(base));
    CalibIndex x;
    x.max_items = calib_max_items(n, S);
    x.counts = c.take<uint32_t>((size_t)S * calib_tiles(n) + 1);
    x.sector_off = c.take<int32_t>(S + 1);
    x.sector_item = c.take<int32_t>(S + 1);
    x.item_sector = c.take<int32_t>(x.max_items);
    x.item_start = c.take<int32_t>(x.max_items);
    x.n_items = c.take<int32_t>(1);
    x.bytes = c.size();
    return x;
}
struct CalibWs {
    float *item_loss, *item_grad, *sector_loss, *loss;
    unsigned int *tickets;
    size_t bytes;
};
CalibWs carve_calib_ws(void *base, uint64_t n, uint32_t S) {
    Carver c(base);
    CalibWs w;
    const uint32_t mi = calib_max_items(n, S);
    w.item_loss = c.take<float>(mi);
    w.item_grad = c.take<float>((size_t)mi * 42);
    w.sector_loss = c.take<float>(S);
    w.loss = c.take<float>(1);
    w.tickets = c.take<unsigned int>(S + 2);   // per sector, the batch, a copy-wait flag
    w.bytes = c.size();
    return w;
}
bool calib_sizes_ok(uint64_t n, uint32_t S) { return n < (1ull << 31) && S >= 1 && S <= 512; }

}  // namespace

struct svt_timer_s {
    cudaEvent_t start, end;
    bool recorded;
};

extern "C" {

int svt_timer_create(svt_timer *out) {
    if (!out) return SVT_ERR_BAD_ARG;
    svt_timer t = new svt_timer_s();
    if (cudaEventCreate(&t->start) != cudaSuccess || cudaEventCreate(&t->end) != cudaSuccess) {
        delete t;
        return SVT_ERR_CUDA;
    }
    t->recorded = false;
    *out = t;
    return SVT_OK;
}

int svt_timer_destroy(svt_timer t) {
    if (!t) return SVT_ERR_BAD_ARG;
    cudaEventDestroy(t->start);
    cudaEventDestroy(t->end);
    delete t;
    return SVT_OK;
}

int svt_timer_fit_ms(svt_timer t, float *ms) {
    if (!t || !ms || !t->recorded) return SVT_ERR_BAD_ARG;
    if (cudaEventSynchronize(t->end) != cudaSuccess) return SVT_ERR_CUDA;
    return cudaEventElapsedTime(ms, t->start, t->end) == cudaSuccess ? SVT_OK : SVT_ERR_CUDA;
}

int svt_version(void) { return 10000; }

int svt_device_sm_count(int device) { return sm_count_of(device); }

size_t svt_unpack_workspace_size(uint64_t n_words) { return carve_unpack(nullptr, n_words).bytes; }

int svt_unpack(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
               uint64_t n_events, uint32_t n_sectors, uint32_t xft_pairs, uint64_t road_cap,
               uint32_t *d_road_word, uint32_t *d_road_nhit, uint32_t *d_event_road,
               uint64_t *d_n_roads, uint64_t *d_status, void *d_workspace,
               size_t workspace_bytes, void *stream) {
    const NvtxRange range("svt_unpack");
    if (!d_event_off || !d_event_road || !d_n_roads || !d_status || !d_workspace)
        return SVT_ERR_BAD_ARG;
    if (n_words > 0 && (!d_words || !aligned16(d_words))) return SVT_ERR_BAD_ARG;
    if (road_cap > 0 && (!d_road_word || !d_road_nhit)) return SVT_ERR_BAD_ARG;
    if (n_words >= (1ull << 32) || n_events >= (1ull << 31) || road_cap >= (1ull << 32))
        return SVT_ERR_BAD_ARG;
    if (n_sectors < 1 || n_sectors > 512 || xft_pairs > 1) return SVT_ERR_BAD_ARG;
    UnpackWs w = carve_unpack(d_workspace, n_words);
    if (workspace_bytes < w.bytes) return SVT_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *status = (unsigned long long *)d_status;
    const int grid = tile_grid();
    svt_config cfg{15, 15, 0, 1, 0, n_sectors, xft_pairs};
    launch_prologue(w.dims, n_words, n_events, nullptr, d_event_off, w.first_ev, status, d_n_roads,
                    1, nullptr, 0, w.tile_state, w.tile_ticket, grid, st);
    const FusedRoads none{nullptr, nullptr, BigList{}, 1, 0};
    launch_unpack_roads(d_words, d_event_off, w.dims, w.first_ev, n_words, w.tile_state,
                        w.tile_ticket, d_n_roads, road_cap, d_road_word, d_road_nhit, d_event_road,
                        cfg, none, nullptr, status, grid, st);
    launch_unpack_events(d_words, d_event_off, w.dims, n_events, d_event_road, status, grid, st);
    return launch_status();
}

size_t svt_combine_workspace_size(uint64_t road_cap) {
    return align_up(scan_u64_tile_count(road_cap + 1) * sizeof(uint64_t), 256);
}

int svt_combine(const uint32_t *d_road_nhit, const uint64_t *d_n_roads, uint64_t road_cap,
                const svt_config *cfg, uint64_t comb_cap, uint32_t *d_road_flags,
                uint64_t *d_comb_off, uint32_t *d_comb_road, uint32_t *d_comb_hits,
                uint64_t *d_n_combs, uint64_t *d_status, void *d_workspace,
                size_t workspace_bytes, void *stream) {
    const NvtxRange range("svt_combine");
    if (!config_ok(cfg)) return SVT_ERR_BAD_CONFIG;
    if (!d_n_roads || !d_comb_off || !d_n_combs || !d_status || !d_workspace) return SVT_ERR_BAD_ARG;
    if (road_cap > 0 && (!d_road_nhit || !d_road_flags)) return SVT_ERR_BAD_ARG;
    if (comb_cap > 0 && (!d_comb_road || !d_comb_hits)) return SVT_ERR_BAD_ARG;
    if (road_cap >= (1ull << 32)) return SVT_ERR_BAD_ARG;
    if (workspace_bytes < svt_combine_workspace_size(road_cap)) return SVT_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = tile_grid();
    unsigned long long *status = (unsigned long long *)d_status;
    launch_combine_count(d_road_nhit, d_n_roads, road_cap, *cfg, d_road_flags, d_comb_off, status,
                         grid, st);
    launch_scan_u64(d_comb_off, d_n_roads, road_cap, (uint64_t *)d_workspace, d_n_combs, status,
                    grid, st);
    launch_combine_write(d_road_nhit, d_n_roads, road_cap, d_comb_off, comb_cap, cfg->xft_pairs,
                         d_comb_road, d_comb_hits, status, grid, st);
    return launch_status();
}

int svt_fit(const uint32_t *d_words, const uint32_t *d_road_word, const uint32_t *d_road_nhit,
            const uint32_t *d_comb_road, const uint32_t *d_comb_hits, const uint64_t *d_n_combs,
            uint64_t comb_cap, const int16_t *d_F, const int16_t *d_q, const svt_config *cfg,
            uint32_t *d_fit_chi2, int32_t *d_fit_par, const uint64_t *d_status, void *stream) {
    const NvtxRange range("svt_fit");
    if (!config_ok(cfg)) return SVT_ERR_BAD_CONFIG;
    if (!d_n_combs || !d_F || !d_q || !d_status) return SVT_ERR_BAD_ARG;
    if (comb_cap > 0 && (!d_words || !d_road_word || !d_road_nhit || !d_comb_road ||
                         !d_comb_hits || !d_fit_chi2 || !d_fit_par))
        return SVT_ERR_BAD_ARG;
    launch_fit_plain(d_words, d_road_word, d_road_nhit, d_comb_road, d_comb_hits, d_n_combs,
                     comb_cap, d_F, d_q, *cfg, d_fit_chi2, d_fit_par,
                     (const unsigned long long *)d_status, current_sm_count() * 16,
                     (cudaStream_t)stream);
    return launch_status();
}

int svt_select(const uint32_t *d_fit_chi2, const int32_t *d_fit_par, uint64_t comb_cap,
               const uint64_t *d_comb_off, const uint32_t *d_road_flags,
               const uint64_t *d_n_roads, uint64_t road_cap, const svt_config *cfg,
               svt_best *d_best, const uint64_t *d_status, void *stream) {
    const NvtxRange range("svt_select");
    if (!config_ok(cfg)) return SVT_ERR_BAD_CONFIG;
    if (!d_comb_off || !d_n_roads || !d_status) return SVT_ERR_BAD_ARG;
    if (road_cap > 0 && (!d_road_flags || !d_best)) return SVT_ERR_BAD_ARG;
    if (comb_cap > 0 && (!d_fit_chi2 || !d_fit_par)) return SVT_ERR_BAD_ARG;
    launch_select(d_fit_chi2, d_fit_par, comb_cap, d_comb_off, d_road_flags, d_n_roads, road_cap,
                  *cfg, d_best, (const unsigned long long *)d_status, current_sm_count() * 16,
                  (cudaStream_t)stream);
    return launch_status();
}

int svt_format(const svt_best *d_best, const uint32_t *d_words, const uint32_t *d_road_word,
               const uint64_t *d_n_roads, uint64_t road_cap, uint32_t *d_out,
               const uint64_t *d_status, void *stream) {
    const NvtxRange range("svt_format");
    if (!d_n_roads || !d_status) return SVT_ERR_BAD_ARG;
    if (road_cap > 0 && (!d_best || !d_words || !d_road_word || !d_out)) return SVT_ERR_BAD_ARG;
    launch_format(d_best, d_words, d_road_word, d_n_roads, road_cap, d_out,
                  (const unsigned long long *)d_status, current_sm_count() * 8,
                  (cudaStream_t)stream);
    return launch_status();
}

size_t svt_run_workspace_size(uint64_t max_words, uint64_t max_events, uint64_t road_cap,
                              const svt_schedule *sched) {
    (void)sched;
    return carve_run(nullptr, max_words, max_events, road_cap).bytes;
}

}  // extern "C"

namespace {

// The fused launch sequence.  With d_sizes the batch sizes are read on the
// device (capacities n_words / n_events), which lets one captured graph serve
// batches of any size up to its capacities.
int run_impl(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
             uint64_t n_events, const uint64_t *d_sizes, const int16_t *d_F, const int16_t *d_q,
             const svt_config *cfg, uint64_t road_cap, uint32_t *d_out, uint32_t *d_event_road,
             uint64_t *d_counts, uint64_t *d_status, void *d_workspace, size_t workspace_bytes,
             const svt_schedule *sched, svt_timer timer, cudaStream_t st) {
    if (!config_ok(cfg)) return SVT_ERR_BAD_CONFIG;
    const svt_schedule sc = resolve(sched);
    if (!schedule_ok(sc)) return SVT_ERR_BAD_ARG;
    if (!d_event_off || !d_F || !d_q || !d_status || !d_workspace) return SVT_ERR_BAD_ARG;
    if (n_words > 0 && (!d_words || !aligned16(d_words))) return SVT_ERR_BAD_ARG;
    if (road_cap > 0 && !d_out) return SVT_ERR_BAD_ARG;
    if (n_words >= (1ull << 32) || n_events >= (1ull << 31) || road_cap >= (1ull << 31))
        return SVT_ERR_BAD_ARG;
    if ((uintptr_t)d_workspace & 255u) return SVT_ERR_BAD_ARG;
    // one road per lane reads the constants as 32-bit pairs
    if (fit_group(sc.pair_small) == 32 && (((uintptr_t)d_F | (uintptr_t)d_q) & 3u))
        return SVT_ERR_BAD_ARG;
    RunWs w = carve_run(d_workspace, n_words, n_events, road_cap);
    if (workspace_bytes < w.bytes) return SVT_ERR_BAD_ARG;
    unsigned long long *status = (unsigned long long *)d_status;
    uint64_t *counts = d_counts ? d_counts : w.counts;
    uint32_t *event_road = d_event_road ? d_event_road : w.event_road;
    const int grid = tile_grid();
    const int sms = current_sm_count();
    if (sms <= 0) return SVT_ERR_CUDA;
    const int occ =
        fit_persistent_blocks_per_sm((int)sc.warps_per_block, fit_group(sc.pair_small));
    if (occ <= 0) return SVT_ERR_CUDA;
    const int bps = (sc.blocks_per_sm == 0 || (int)sc.blocks_per_sm > occ) ? occ : (int)sc.blocks_per_sm;
    const BigList bl{w.big_road, w.big_item_off, w.big_pending, (unsigned long long *)w.work,
                     (uint32_t *)(w.work + 1)};
    const FusedRoads fr{w.desc, w.key, bl, sc.rows_per_item, sc.small_max};

    const NvtxRange range("svt_run");
    {
        const NvtxRange stage("svt_run: unpack");
        launch_prologue(w.dims, n_words, n_events, d_sizes, d_event_off, w.first_ev, status, counts, 4,
                        w.work, 2, w.tile_state, w.tile_ticket, grid, st);
        launch_unpack_roads(d_words, d_event_off, w.dims, w.first_ev, n_words, w.tile_state,
                            w.tile_ticket, counts + 0, road_cap, nullptr, nullptr, event_road,
                            *cfg, fr, counts, status, grid, st);
    }
    const NvtxRange fit_range("svt_run: combine, fit, cut, select, format");
    if (timer && cudaEventRecord(timer->start, st) != cudaSuccess) return SVT_ERR_CUDA;
    if (launch_fit_persistent(d_words, d_event_off, w.dims, event_road, w.desc, counts, road_cap,
                              d_F, d_q, *cfg, fr, sc.roads_per_chunk,
                              fit_group(sc.pair_small), d_out,
                              status, (int)sc.warps_per_block, sms * bps, st) != cudaSuccess)
        return SVT_ERR_CUDA;
    if (timer) {
        if (cudaEventRecord(timer->end, st) != cudaSuccess) return SVT_ERR_CUDA;
        timer->recorded = true;
    }
    return launch_status();
}

}  // namespace

struct svt_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

int svt_run(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
            uint64_t n_events, const int16_t *d_F, const int16_t *d_q, const svt_config *cfg,
            uint64_t road_cap, uint32_t *d_out, uint32_t *d_event_road, uint64_t *d_counts,
            uint64_t *d_status, void *d_workspace, size_t workspace_bytes,
            const svt_schedule *sched, svt_timer timer, void *stream) {
    return run_impl(d_words, n_words, d_event_off, n_events, nullptr, d_F, d_q, cfg, road_cap,
                    d_out, d_event_road, d_counts, d_status, d_workspace, workspace_bytes, sched,
                    timer, (cudaStream_t)stream);
}

int svt_run_sized(const uint32_t *d_words, uint64_t max_words, const uint64_t *d_event_off,
                  uint64_t max_events, const uint64_t *d_sizes, const int16_t *d_F,
                  const int16_t *d_q, const svt_config *cfg, uint64_t road_cap, uint32_t *d_out,
                  uint32_t *d_event_road, uint64_t *d_counts, uint64_t *d_status,
                  void *d_workspace, size_t workspace_bytes, const svt_schedule *sched,
                  void *stream) {
    if (!d_sizes) return SVT_ERR_BAD_ARG;
    return run_impl(d_words, max_words, d_event_off, max_events, d_sizes, d_F, d_q, cfg, road_cap,
                    d_out, d_event_road, d_counts, d_status, d_workspace, workspace_bytes, sched,
                    nullptr, (cudaStream_t)stream);
}

int svt_graph_create(const uint32_t *d_words, uint64_t max_words, const uint64_t *d_event_off,
                     uint64_t max_events, const uint64_t *d_sizes, const int16_t *d_F,
                     const int16_t *d_q, const svt_config *cfg, uint64_t road_cap,
                     uint32_t *d_out, uint32_t *d_event_road, uint64_t *d_counts,
                     uint64_t *d_status, void *d_workspace, size_t workspace_bytes,
                     const svt_schedule *sched, svt_graph *out) {
    if (!out || !d_sizes) return SVT_ERR_BAD_ARG;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return SVT_ERR_CUDA;
    int rc = SVT_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return SVT_ERR_CUDA;
    }
    rc = run_impl(d_words, max_words, d_event_off, max_events, d_sizes, d_F, d_q, cfg, road_cap,
                  d_out, d_event_road, d_counts, d_status, d_workspace, workspace_bytes, sched,
                  nullptr, cs);
    cudaError_t ce = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != SVT_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != SVT_OK ? rc : SVT_ERR_CUDA;
    }
    svt_graph h = new svt_graph_s();
    h->graph = g;
    if (cudaGraphInstantiate(&h->exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        delete h;
        return SVT_ERR_CUDA;
    }
    *out = h;
    return SVT_OK;
}

int svt_autotune(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
                 uint64_t n_events, const int16_t *d_F, const int16_t *d_q, const svt_config *cfg,
                 uint64_t road_cap, uint32_t *d_out, uint64_t *d_status, void *d_workspace,
                 size_t workspace_bytes, uint32_t reps, void *d_flush, size_t flush_bytes,
                 svt_schedule *best, float *best_ms, void *stream) {
    if (!best || !best_ms || reps < 1 || reps > 100 || (flush_bytes && !d_flush))
        return SVT_ERR_BAD_ARG;
    static const uint32_t kWarps[] = {4, 8, 16};
    static const uint32_t kRows[] = {8, 16, 32, 64};
    static const uint32_t kChunk[] = {1, 2, 4, 8};
    static const uint32_t kSmall[] = {1024, 4096, 16384};
    constexpr int kTop = 4;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SVT_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SVT_ERR_CUDA;
    }
    // the fastest schedules so far, fastest first
    svt_schedule top_s[kTop] = {};
    float top_t[kTop];
    for (float &t : top_t) t = 3.4e38f;
    int rc = SVT_OK;
    auto run = [&](const svt_schedule &sc) {
        return svt_run(d_words, n_words, d_event_off, n_events, d_F, d_q, cfg, road_cap, d_out,
                       nullptr, nullptr, d_status, d_workspace, workspace_bytes, &sc, nullptr,
                       stream);
    };
    // mean time per run of schedule sc over n runs after one warm-up.  With a
    // flush buffer every run is timed alone, after the buffer has been
    // overwritten (outside the timed region), so that no run finds the batch
    // or the previous run's results in L2; without one the runs go back to
    // back.
    auto time_runs = [&](const svt_schedule &sc, uint32_t n, float &ms) -> int {
        int r = run(sc);
        if (r != SVT_OK) return r;
        ms = 0.f;
        if (!flush_bytes && cudaEventRecord(e0, st) != cudaSuccess) return SVT_ERR_CUDA;
        for (uint32_t k = 0; k < n; ++k) {
            if (flush_bytes) {
                if (cudaMemsetAsync(d_flush, (int)(k & 0xFFu), flush_bytes, st) != cudaSuccess ||
                    cudaEventRecord(e0, st) != cudaSuccess)
                    return SVT_ERR_CUDA;
            }
            if ((r = run(sc)) != SVT_OK) return r;
            if (flush_bytes) {
                float one = 0.f;
                if (cudaEventRecord(e1, st) != cudaSuccess ||
                    cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&one, e0, e1) != cudaSuccess)
                    return SVT_ERR_CUDA;
                ms += one;
            }
        }
        if (!flush_bytes && (cudaEventRecord(e1, st) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            return SVT_ERR_CUDA;
        ms /= (float)n;
        return SVT_OK;
    };
    auto trial = [&](const svt_schedule &sc) -> int {
        float ms = 0.f;
        const int r = time_runs(sc, reps, ms);
        if (r != SVT_OK) return r;
        for (int i = 0; i < kTop; ++i)
            if (ms < top_t[i]) {
                for (int j = kTop - 1; j > i; --j) {
                    top_t[j] = top_t[j - 1];
                    top_s[j] = top_s[j - 1];
                }
                top_t[i] = ms;
                top_s[i] = sc;
                break;
            }
        return SVT_OK;
    };
    for (uint32_t w : kWarps)
        for (uint32_t r : kRows)
            for (uint32_t c : kChunk)
                for (uint32_t m : kSmall)
                    if ((rc = trial(svt_schedule{w, 0, r, c, m, 0})) != SVT_OK) goto done;
    {
        // longer items of split roads (each item repeats its road's set-up)
        const svt_schedule base = top_s[0];
        for (uint32_t f : {2u, 4u}) {
            svt_schedule sc = base;
            sc.rows_per_item = base.rows_per_item * f;
            if ((rc = trial(sc)) != SVT_OK) goto done;
        }
    }
    {
        const svt_schedule base = top_s[0];
        for (uint32_t g : {1u, 2u})
            for (uint32_t c : {2u, 4u, 8u})
                if ((rc = trial(svt_schedule{base.warps_per_block, 0, base.rows_per_item,
                                             g == 2 ? 2 * c : c, base.small_max, g})) != SVT_OK)
                    goto done;
        // tiny roads on 1, 2 or 4 lanes each: 32, 16 or 8 roads per chunk
        // (constants that are not 4-byte aligned rule it out)
        if (!(((uintptr_t)d_F | (uintptr_t)d_q) & 3u))
            for (uint32_t c : {8u, 16u, 32u})
                if ((rc = trial(svt_schedule{base.warps_per_block > 12 ? 8 : base.warps_per_block,
                                             0, base.rows_per_item, c, base.small_max, 3})) !=
                    SVT_OK)
                    goto done;
    }
    {
        // fewer resident blocks: small batches leave most warps idle and
        // finish sooner with less contention
        const svt_schedule base = top_s[0];
        for (uint32_t b : {1u, 2u}) {
            svt_schedule sc = base;
            sc.blocks_per_sm = b;
            if ((rc = trial(sc)) != SVT_OK) goto done;
        }
    }
    {
        // the few fastest again, with three times the runs: the first pass
        // over a hundred and fifty schedules favours a lucky measurement
        int pick = 0;
        float pick_t = 3.4e38f;
        for (int i = 0; i < kTop && top_t[i] < 3.4e38f; ++i) {
            float ms = 0.f;
            if ((rc = time_runs(top_s[i], 3 * reps, ms)) != SVT_OK) goto done;
            if (ms < pick_t) {
                pick_t = ms;
                pick = i;
            }
        }
        *best = top_s[pick];
        *best_ms = pick_t;
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"

namespace {

// Device buffers of svt_run_host: the batch's words and offsets, the status,
// the records, then svt_run's own workspace.
struct HostRunWs {
    uint32_t *words;
    uint64_t *off, *status;
    uint32_t *out;
    void *run;
    size_t run_bytes, bytes;
};
HostRunWs carve_host_run(void *base, uint64_t n_words, uint64_t n_events, uint64_t road_cap,
                         const svt_schedule *sched) {
    Carver c(base);
    HostRunWs w;
    w.words = c.take<uint32_t>(n_words + 4);
    w.off = c.take<uint64_t>(n_events + 1);
    w.status = c.take<uint64_t>(1);
    w.out = c.take<uint32_t>(6 * (road_cap ? road_cap : 1));
    w.run_bytes = svt_run_workspace_size(n_words, n_events, road_cap, sched);
    w.run = c.take<char>(w.run_bytes);
    w.bytes = c.size();
    return w;
}

}  // namespace

extern "C" {

size_t svt_run_host_workspace_size(uint64_t max_words, uint64_t max_events, uint64_t road_cap,
                                   const svt_schedule *sched) {
    return carve_host_run(nullptr, max_words, max_events, road_cap, sched).bytes;
}

int svt_run_host(const uint32_t *h_words, uint64_t n_words, const uint64_t *h_event_off,
                 uint64_t n_events, const int16_t *d_F, const int16_t *d_q, const svt_config *cfg,
                 uint64_t road_cap, uint32_t *h_out, uint64_t *h_status, uint64_t *n_records,
                 void *d_workspace, size_t workspace_bytes, const svt_schedule *sched,
                 void *stream) {
    if (!h_event_off || !h_status || !d_workspace || (n_words > 0 && !h_words) ||
        (road_cap > 0 && !h_out))
        return SVT_ERR_BAD_ARG;
    if (n_words >= (1ull << 32) || n_events >= (1ull << 31) || road_cap >= (1ull << 31))
        return SVT_ERR_BAD_ARG;
    if ((uintptr_t)d_workspace & 255u) return SVT_ERR_BAD_ARG;
    const HostRunWs w = carve_host_run(d_workspace, n_words, n_events, road_cap, sched);
    if (workspace_bytes < w.bytes) return SVT_ERR_BAD_ARG;
    // records to bring back: the road count the event headers state, at most
    // road_cap (for a valid batch this is R; for an invalid one the status
    // says so and the records are unspecified)
    uint64_t R = 0;
    for (uint64_t e = 0; e < n_events; ++e) {
        const uint64_t s = h_event_off[e];
        if (s < n_words) R += h_words[s] & 0xFFFu;
    }
    R = R < road_cap ? R : road_cap;
    if (n_records) *n_records = R;
    cudaStream_t st = (cudaStream_t)stream;
    if ((n_words && cudaMemcpyAsync(w.words, h_words, n_words * 4, cudaMemcpyHostToDevice, st) !=
                        cudaSuccess) ||
        cudaMemcpyAsync(w.off, h_event_off, (n_events + 1) * 8, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return SVT_ERR_CUDA;
    const int rc = svt_run(w.words, n_words, w.off, n_events, d_F, d_q, cfg, road_cap, w.out,
                           nullptr, nullptr, w.status, w.run, w.run_bytes, sched, nullptr, stream);
    if (rc != SVT_OK) return rc;
    if ((R && cudaMemcpyAsync(h_out, w.out, R * 24, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        cudaMemcpyAsync(h_status, w.status, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SVT_ERR_CUDA;
    return SVT_OK;
}

int svt_host_alloc(size_t bytes, void **host, void **device) {
    if (!host || !device || bytes == 0) return SVT_ERR_BAD_ARG;
    *host = nullptr;
    *device = nullptr;
    void *h = nullptr;
    if (cudaHostAlloc(&h, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
        return SVT_ERR_OOM;
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess || !d ||
        (((uintptr_t)h | (uintptr_t)d) & 255u)) {
        cudaFreeHost(h);
        return SVT_ERR_CUDA;
    }
    *host = h;
    *device = d;
    return SVT_OK;
}

int svt_host_free(void *host) {
    if (!host) return SVT_ERR_BAD_ARG;
    return cudaFreeHost(host) == cudaSuccess ? SVT_OK : SVT_ERR_CUDA;
}

int svt_graph_launch(svt_graph g, void *stream) {
    if (!g) return SVT_ERR_BAD_ARG;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? SVT_OK : SVT_ERR_CUDA;
}

int svt_graph_destroy(svt_graph g) {
    if (!g) return SVT_ERR_BAD_ARG;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return SVT_OK;
}

size_t svt_calib_index_size(uint64_t n_tracks, uint32_t n_sectors) {
    return carve_calib_index(nullptr, n_tracks, n_sectors).bytes;
}

int svt_calib_index(const int32_t *d_sector, uint64_t n_tracks, uint32_t n_sectors, void *d_index,
                    size_t index_bytes, int32_t *d_perm, uint64_t *d_status, void *stream) {
    if (!calib_sizes_ok(n_tracks, n_sectors) || !d_index || !d_status) return SVT_ERR_BAD_ARG;
    if (n_tracks > 0 && (!d_sector || !d_perm)) return SVT_ERR_BAD_ARG;
    CalibIndex x = carve_calib_index(d_index, n_tracks, n_sectors);
    if (index_bytes < x.bytes) return SVT_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *status = (unsigned long long *)d_status;
    launch_prologue(nullptr, 0, 0, nullptr, nullptr, nullptr, status, nullptr, 0, nullptr, 0,
                    nullptr, nullptr, 1, st);
    if (cudaMemsetAsync(x.sector_off, 0, sizeof(int32_t) * (n_sectors + 1), st) != cudaSuccess ||
        cudaMemsetAsync(x.sector_item, 0, sizeof(int32_t) * (n_sectors + 1), st) != cudaSuccess ||
        cudaMemsetAsync(x.n_items, 0, sizeof(int32_t), st) != cudaSuccess)
        return SVT_ERR_CUDA;
    launch_calib_sort(d_sector, n_tracks, n_sectors, x.counts, d_perm, x.sector_off,
                      x.sector_item, x.item_sector, x.item_start, x.n_items, status, tile_grid(),
                      st);
    return launch_status();
}

int svt_calib_gather(const float *d_src, uint32_t width, const int32_t *d_perm, uint64_t n,
                     float *d_dst, void *stream) {
    if (n == 0) return SVT_OK;
    if (!d_src || !d_perm || !d_dst || width == 0 || width > 64 || n >= (1ull << 31))
        return SVT_ERR_BAD_ARG;
    launch_calib_gather(d_src, width, d_perm, n, d_dst, tile_grid(), (cudaStream_t)stream);
    return launch_status();
}

size_t svt_calib_workspace_size(uint64_t n_tracks, uint32_t n_sectors) {
    return carve_calib_ws(nullptr, n_tracks, n_sectors).bytes;
}

int svt_calib_forward(const float *d_x, uint64_t n_tracks, uint32_t n_sectors,
                      const void *d_index, const float *d_F, const float *d_q, float *d_y,
                      void *stream) {
    if (!calib_sizes_ok(n_tracks, n_sectors) || !d_index || !d_F || !d_q) return SVT_ERR_BAD_ARG;
    if (n_tracks == 0) return SVT_OK;
    if (!d_x || !d_y || ((uintptr_t)d_x & 7u) || ((uintptr_t)d_y & 7u)) return SVT_ERR_BAD_ARG;
    CalibIndex x = carve_calib_index(d_index, n_tracks, n_sectors);
    launch_calib_forward(d_x, x.item_sector, x.item_start, x.sector_off, x.n_items, x.max_items,
                         d_F, d_q, d_y, tile_grid(), (cudaStream_t)stream);
    return launch_status();
}

int svt_calib_loss(const float *d_x, const float *d_theta, const float *d_w, uint64_t n_tracks,
                   uint32_t n_sectors, const void *d_index, const float *d_F, const float *d_q,
                   float *d_loss, void *d_workspace, size_t workspace_bytes, void *stream) {
    if (!calib_sizes_ok(n_tracks, n_sectors) || !d_index || !d_F || !d_q || !d_w || !d_loss ||
        !d_workspace)
        return SVT_ERR_BAD_ARG;
    if (n_tracks > 0 && (!d_x || !d_theta || ((uintptr_t)d_x & 7u))) return SVT_ERR_BAD_ARG;
    CalibWs w = carve_calib_ws(d_workspace, n_tracks, n_sectors);
    if (workspace_bytes < w.bytes) return SVT_ERR_BAD_ARG;
    CalibIndex x = carve_calib_index(d_index, n_tracks, n_sectors);
    launch_calib_loss(d_x, d_theta, x.item_sector, x.item_start, x.sector_off, x.sector_item,
                      x.n_items, x.max_items, n_sectors, n_tracks, d_F, d_q, d_w, w.item_loss,
                      w.tickets + n_sectors + 1, d_loss, current_sm_count(), tile_grid(),
                      (cudaStream_t)stream);
    return launch_status();
}

int svt_calib_loss_backward(const float *d_x, const float *d_theta, const float *d_w,
                            uint64_t n_tracks, uint32_t n_sectors, const void *d_index,
                            const float *d_F, const float *d_q, const float *d_grad_loss,
                            float *d_dF, float *d_dq, void *d_workspace, size_t workspace_bytes,
                            void *stream) {
    if (!calib_sizes_ok(n_tracks, n_sectors) || !d_index || !d_F || !d_q || !d_w || !d_dF ||
        !d_dq || !d_workspace)
        return SVT_ERR_BAD_ARG;
    if (n_tracks > 0 && (!d_x || !d_theta || ((uintptr_t)d_x & 7u))) return SVT_ERR_BAD_ARG;
    CalibWs w = carve_calib_ws(d_workspace, n_tracks, n_sectors);
    if (workspace_bytes < w.bytes) return SVT_ERR_BAD_ARG;
    CalibIndex x = carve_calib_index(d_index, n_tracks, n_sectors);
    // the fused pass, its loss kept in the workspace
    launch_calib_loss_grad(d_x, d_theta, x.item_sector, x.item_start, x.sector_off,
                           x.sector_item, x.n_items, n_sectors, n_tracks, d_F, d_q, d_w,
                           d_grad_loss, w.item_loss, w.item_grad, w.sector_loss, w.tickets,
                           w.loss, d_dF, d_dq, nullptr, current_sm_count(), (cudaStream_t)stream);
    return launch_status();
}

int svt_calib_loss_grad(const float *d_x, const float *d_theta, const float *d_w,
                        uint64_t n_tracks, uint32_t n_sectors, const void *d_index,
                        const float *d_F, const float *d_q, float *d_loss, float *d_dF,
                        float *d_dq, float *d_y, void *d_workspace, size_t workspace_bytes,
                        void *stream) {
    if (!calib_sizes_ok(n_tracks, n_sectors) || !d_index || !d_F || !d_q || !d_w || !d_loss ||
        !d_dF || !d_dq || !d_workspace)
        return SVT_ERR_BAD_ARG;
    if (n_tracks > 0 && (!d_x || !d_theta || ((uintptr_t)d_x & 7u) || ((uintptr_t)d_y & 7u)))
        return SVT_ERR_BAD_ARG;
    CalibWs w = carve_calib_ws(d_workspace, n_tracks, n_sectors);
    if (workspace_bytes < w.bytes) return SVT_ERR_BAD_ARG;
    CalibIndex x = carve_calib_index(d_index, n_tracks, n_sectors);
    launch_calib_loss_grad(d_x, d_theta, x.item_sector, x.item_start, x.sector_off,
                           x.sector_item, x.n_items, n_sectors, n_tracks, d_F, d_q, d_w, nullptr,
                           w.item_loss, w.item_grad, w.sector_loss, w.tickets, d_loss, d_dF, d_dq,
                           d_y, current_sm_count(), (cudaStream_t)stream);
    return launch_status();
}

int svt_calib_grad_scale(const float *d_scale, const float *d_dF, const float *d_dq,
                         uint32_t n_sectors, float *d_out_dF, float *d_out_dq, void *stream) {
    if (!d_scale || !d_dF || !d_dq || !d_out_dF || !d_out_dq || n_sectors < 1 || n_sectors > 512)
        return SVT_ERR_BAD_ARG;
    launch_calib_grad_scale(d_scale, d_dF, d_dq, n_sectors, d_out_dF, d_out_dq,
                            (cudaStream_t)stream);
    return launch_status();
}

int svt_calib_backward(const float *d_x, const float *d_grad_y, uint64_t n_tracks,
                       uint32_t n_sectors, const void *d_index, const float *d_F, float *d_dF,
                       float *d_dq, float *d_dx, void *d_workspace, size_t workspace_bytes,
                       void *stream) {
    if (!calib_sizes_ok(n_tracks, n_sectors) || !d_index || !d_F || !d_dF || !d_dq ||
        !d_workspace)
        return SVT_ERR_BAD_ARG;
    if (n_tracks > 0 && (!d_x || !d_grad_y || ((uintptr_t)d_x & 7u) || ((uintptr_t)d_grad_y & 7u) ||
                         ((uintptr_t)d_dx & 7u)))
        return SVT_ERR_BAD_ARG;
    CalibWs w = carve_calib_ws(d_workspace, n_tracks, n_sectors);
    if (workspace_bytes < w.bytes) return SVT_ERR_BAD_ARG;
    CalibIndex x = carve_calib_index(d_index, n_tracks, n_sectors);
    launch_calib_grad(d_x, d_grad_y, x.item_sector, x.item_start, x.sector_off, x.sector_item,
                      x.n_items, x.max_items, n_sectors, d_F, w.item_grad, d_dF, d_dq, d_dx,
                      tile_grid(), (cudaStream_t)stream);
    return launch_status();
}

}  // extern "C"
