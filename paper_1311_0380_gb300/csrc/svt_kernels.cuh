// svt_kernels.cuh -- declarations of the kernels and launch helpers that the
// C-ABI layer (svt_abi.cu) strings together.
#pragma once

#include "svt_internal.cuh"

namespace svt {

// Device-side view of a batch's sizes.  Every pipeline kernel reads the sizes
// through this so that one captured launch sequence serves batches of any
// size up to its capacities.
struct Dims {
    uint64_t n_words;
    uint64_t n_events;
};

// ---- programmatic dependent launch --------------------------------------------
// The kernels of a sequence after its first are launched with programmatic
// stream serialization (launch_after): once every block of the kernel before
// has started and called allow_next_grid, the next kernel's blocks may be
// scheduled as SMs free up, and each waits in wait_prior_grid
// (griddepcontrol.wait: the kernel before has completed and its writes are
// visible) before it touches anything.  Every kernel of a sequence calls
// wait_prior_grid first, in every block, so the completion of one kernel
// implies that of all kernels before it.  For a kernel launched without the
// attribute both calls return at once.
__device__ __forceinline__ void wait_prior_grid() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_next_grid() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_after(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t st, Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t c = {};
    c.gridDim = grid;
    c.blockDim = block;
    c.dynamicSmemBytes = smem;
    c.stream = st;
    c.attrs = attr;
    c.numAttrs = 1;
    cudaLaunchKernelEx(&c, kernel, args...);   // errors surface through cudaGetLastError
}

// Per-road descriptor of the fused path (32 bytes), built once by the road
// extraction:
//   a = {header word index, hits per layer (5 bits each), header word,
//        evaluated combinations C_eval}
//   b = {geo, NB, NA, 0} with the split c = a_row * NB + b_col (see road_split),
//       NA = ceil(C_eval / NB) rows, and geo bits [2:0] split, [7:3] NBp (columns
//       below the top suffix layer, NB = ntop * NBp), [12:8] ntop, [18:13] layer
//       mask, [25:19] total hits, [26] OVERFLOW, [27] BAD_PATTERN, [28] SMALL:
//       at most 8 hits on every layer, NBp <= 16 and NA <= 16, so that half a
//       warp can fit the road (the fit kernel pairs such roads).
struct RoadDesc {
    uint4 a, b;
};
// Estimated warp instructions of the fused fit for a road of C evaluated
// combinations whose suffix starts at layer l and has nb entries: about 20
// per row step of a lane (full passes of 32 columns, then the partial pass in
// lane groups of nb mod 32, each with its own rows), 45 per pass over the
// columns of a 64-row chunk, 15 per prefix layer and 32 rows of the row
// build, 15 per suffix-table layer.  Only ever compared with itself, so single
// precision with approximate quotients is ample.
__device__ __forceinline__ float split_cost(uint32_t C, uint32_t nb, uint32_t l) {
    const float na = ceilf(__fdividef((float)C, (float)nb));
    const uint32_t full = nb >> 5, w = nb & 31u;
    const float chunks = ceilf(na * (1.f / 64.f));
    // lane groups of the partial pass; 32 / w is either exact or at least
    // 1/31 above its floor, so the small bias keeps floorf exact
    const float groups = w ? floorf(__fdividef(32.f, (float)w) + 1e-3f) : 1.f;
    const float tail = w ? ceilf(__fdividef(na, groups)) + chunks : 0.f;
    return 20.f * ((float)full * na + tail) + 45.f * chunks * (float)(full + (w ? 1u : 0u)) +
           15.f * (float)l * (ceilf(na * (1.f / 32.f)) - 1.f);
}

__device__ __forceinline__ RoadDesc make_road_desc(uint32_t rw, uint32_t packed, uint32_t hw,
                                                   const svt_config &cfg) {
    const RoadShape s = road_shape(packed, cfg.xft_pairs);
    const bool bad = s.n_layers_hit < cfg.min_layers;
    const uint32_t C = (uint32_t)s.C;
    const uint32_t C_eval = bad ? 0u : (C > cfg.max_comb ? cfg.max_comb : C);
    uint32_t split, NB;
    road_split(s, split, NB);
    // The fit kernel takes one column per lane (the last, partial pass over
    // the columns in groups of lanes, each with a block of rows), so one layer
    // fewer in the suffix, under 32 columns, can cost less than the rule's
    // split: keep whichever of the two the estimate favours.
    // (The row of a combination must stay below 2^23 in the fit's 64-bit
    // keys: the shorter suffix is taken only while rows stay below 2^16.)
    if (C_eval > 0 && split + 1 < (uint32_t)N_LAYERS) {
        uint32_t nb1 = 1;
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l)
            if ((uint32_t)l > split) nb1 *= s.n[l];
        if (((uint64_t)nb1 << 16) >= C_eval &&
            split_cost(C_eval, nb1, split + 1) < split_cost(C_eval, NB, split)) {
            split += 1;
            NB = nb1;
        }
    }
    uint32_t NBp = 1, ntop = 1;
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) {
        if ((uint32_t)l > split) NBp *= s.n[l];
        if ((uint32_t)l == split) ntop = s.n[l];
    }
    const uint32_t NA = C_eval ? (C_eval + NB - 1) / NB : 0u;
    bool small = NBp <= 16u && NA <= 16u;
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) small = small && nhit_of(packed, l) <= 8u;
    const uint32_t geo = split | (NBp << 3) | (ntop << 8) | (s.mask << 13) | (s.total_hits << 19) |
                         ((!bad && C > cfg.max_comb) ? (1u << 26) : 0u) | (bad ? (1u << 27) : 0u) |
                         (small ? (1u << 28) : 0u);
    RoadDesc d;
    d.a = make_uint4(rw, packed, hw, C_eval);
    d.b = make_uint4(geo, NB, NA, 0u);
    return d;
}

// Split roads of the fused path.  The road extraction appends each tile's
// split roads with one 64-bit atomic on `reserve` ((items << 32) | roads), so
// road slots and item ranges are reserved together and item_off increases
// with the slot; the fit kernel's work queues are counters[0] (items) and
// counters[1] (roads).
struct BigList {
    uint32_t *road;                // split road of each slot
    uint32_t *item_off;            // its first work item
    uint32_t *pending;             // its items not yet finished
    unsigned long long *reserve;   // (items << 32) | roads appended so far
    uint32_t *counters;            // [0] items taken, [1] roads taken
};

// Fused-path outputs of the road extraction (desc == nullptr: plain path).
struct FusedRoads {
    RoadDesc *desc;            // per road
    unsigned long long *key;   // per split road: best key so far (UINT64_MAX:
                               // none passed), set by the road extraction and
                               // lowered by the road's items
    BigList bl;                // split roads
    uint32_t rows;             // rows per item
    uint32_t small_max;        // roads above this many combinations are split
};

// Work items of a road for the fused fit: roads with more than small_max
// evaluated combinations are split into items of `rows` rows of the
// (prefix x suffix) grid; smaller roads are fitted whole by one warp.
__device__ __forceinline__ uint32_t road_big_items(const RoadDesc &d, const FusedRoads &fr) {
    if (d.a.w <= fr.small_max) return 0;
    return (d.b.z + fr.rows - 1) / fr.rows;
}

// ---- unpack (svt_unpack.cu) --------------------------------------------------
// Prologue: batch sizes (from `sizes` on the device when given, bounded by
// n_words / n_events), status reset, counts[0..n_counts) and zero[0..n_zero)
// cleared and, when first_ev is given, first_ev[t] = the first event whose
// offset is at or after word tile t's start, for t = 0..T, and the tiles'
// published road counts (tile_state[0..T)) and the tile counter cleared.
// Only block 0 writes the sizes and the status; no block reports anything.
void launch_prologue(Dims *dims, uint64_t n_words, uint64_t n_events, const uint64_t *sizes,
                     const uint64_t *event_off, uint32_t *first_ev, unsigned long long *status,
                     uint64_t *counts, int n_counts, uint64_t *zero, int n_zero,
                     unsigned long long *tile_state, uint32_t *tile_ticket, int grid,
                     cudaStream_t st);
// The one pass over the word tiles: per-word validation (rules V1..V9),
// global road indices (block scan plus a look-back over the counts earlier
// tiles publish), road_word, road_nhit (either may be null), event_road of
// the events starting in each tile and of n_events (the road count R, also
// written to *total64); with fr.desc also the road descriptors, the split-road
// list and the evaluated combinations (counts[2]).
void launch_unpack_roads(const uint32_t *words, const uint64_t *event_off, const Dims *dims,
                         const uint32_t *first_ev, uint64_t max_words,
                         unsigned long long *tile_state, uint32_t *tile_ticket, uint64_t *total64,
                         uint64_t road_cap, uint32_t *road_word, uint32_t *road_nhit,
                         uint32_t *event_road, const svt_config cfg, const FusedRoads fr,
                         uint64_t *counts, unsigned long long *status, int grid, cudaStream_t st);
// Per-event rules of the plain path: offsets and V10.
void launch_unpack_events(const uint32_t *words, const uint64_t *event_off, const Dims *dims,
                          uint64_t max_events, const uint32_t *event_road,
                          unsigned long long *status, int grid, cudaStream_t st);

// Per-event rules shared by the plain path's event kernel and the fused fit
// kernel: the offsets (BAD_ARG) and V10.  `tid`/`stride` enumerate the calling
// threads.
__device__ __forceinline__ void check_events(const uint32_t *__restrict__ words,
                                             const uint64_t *__restrict__ event_off,
                                             uint64_t n_words, uint64_t n_events,
                                             const uint32_t *__restrict__ event_road,
                                             unsigned long long *status, uint64_t tid,
                                             uint64_t stride) {
    if (tid == 0) {
        if (__ldg(event_off) != 0 || __ldg(event_off + n_events) != n_words)
            report(status, 0, SVT_ERR_BAD_ARG);
    }
    for (uint64_t e = tid; e < n_events; e += stride) {
        const uint64_t s = __ldg(event_off + e), s1 = __ldg(event_off + e + 1);
        if (s1 <= s || s >= n_words) {
            report(status, 0, SVT_ERR_BAD_ARG);
            continue;
        }
        const uint32_t h = __ldg(words + s);
        // V1 is K1's; an event that starts with a non-header word has no count
        if (w_type(h) == TYPE_EVENT && ev_nroads(h) != event_road[e + 1] - event_road[e])
            report(status, s, SVT_ERR_NROADS_MISMATCH);                            // V10
    }
}

// ---- fused path (svt_fused.cu) -------------------------------------------------
// K4: the persistent fit over split-road items, then over chunks of roads.
// It first checks the per-event rules (check_events), then fits; counts[0]
// holds R on entry, counts[1] receives the number of work items.
cudaError_t launch_fit_persistent(const uint32_t *words, const uint64_t *event_off,
                                  const Dims *dims, const uint32_t *event_road,
                                  const RoadDesc *desc, uint64_t *counts, uint64_t road_cap,
                                  const int16_t *F, const int16_t *q, const svt_config cfg,
                                  const FusedRoads fr, uint32_t roads_per_chunk, bool pair_small,
                                  uint32_t *out, unsigned long long *status,
                                  int warps_per_block, int grid, cudaStream_t st);
int fit_persistent_blocks_per_sm(int warps_per_block);
size_t fit_smem_bytes(int warps_per_block);

// ---- plain path (svt_plain.cu) --------------------------------------------------
// Every plain-path kernel returns at once when *status already holds an error.
void launch_combine_count(const uint32_t *road_nhit, const uint64_t *n_roads, uint64_t road_cap,
                          const svt_config cfg, uint32_t *road_flags, uint64_t *comb_cnt,
                          const unsigned long long *status, int grid, cudaStream_t st);
void launch_scan_u64(uint64_t *a, const uint64_t *n_dev, uint64_t cap, uint64_t *tile_sums,
                     uint64_t *total, const unsigned long long *status, int grid, cudaStream_t st);
void launch_combine_write(const uint32_t *road_nhit, const uint64_t *n_roads, uint64_t road_cap,
                          const uint64_t *comb_off, uint64_t comb_cap, uint32_t xft_pairs,
                          uint32_t *comb_road, uint32_t *comb_hits, unsigned long long *status,
                          int grid, cudaStream_t st);
void launch_fit_plain(const uint32_t *words, const uint32_t *road_word, const uint32_t *road_nhit,
                      const uint32_t *comb_road, const uint32_t *comb_hits,
                      const uint64_t *n_combs, uint64_t comb_cap, const int16_t *F,
                      const int16_t *q, const svt_config cfg, uint32_t *fit_chi2,
                      int32_t *fit_par, const unsigned long long *status, int grid,
                      cudaStream_t st);
void launch_select(const uint32_t *fit_chi2, const int32_t *fit_par, uint64_t comb_cap,
                   const uint64_t *comb_off, const uint32_t *road_flags, const uint64_t *n_roads,
                   uint64_t road_cap, const svt_config cfg, svt_best *best,
                   const unsigned long long *status, int grid, cudaStream_t st);
void launch_format(const svt_best *best, const uint32_t *words, const uint32_t *road_word,
                   const uint64_t *n_roads, uint64_t road_cap, uint32_t *out,
                   const unsigned long long *status, int grid, cudaStream_t st);

// ---- calibration (svt_calib.cu) ------------------------------------------------
uint32_t calib_max_items(uint64_t n, uint32_t S);
uint32_t calib_tiles(uint64_t n);
void launch_calib_sort(const int32_t *sector, uint64_t n, uint32_t S, uint32_t *counts,
                       int32_t *perm, int32_t *sector_off, int32_t *sector_item,
                       int32_t *item_sector, int32_t *item_start, int32_t *n_items,
                       unsigned long long *status, int grid, cudaStream_t st);
void launch_calib_gather(const float *src, uint32_t width, const int32_t *perm, uint64_t n,
                         float *dst, int grid, cudaStream_t st);
void launch_calib_forward(const float *x, const int32_t *item_sector, const int32_t *item_start,
                          const int32_t *sector_off, const int32_t *n_items, uint32_t max_items,
                          const float *F, const float *q, float *y, int grid, cudaStream_t st);
void launch_calib_loss(const float *x, const float *theta, const int32_t *item_sector,
                       const int32_t *item_start, const int32_t *sector_off,
                       const int32_t *n_items, uint32_t max_items, uint64_t n, const float *F,
                       const float *q, const float *w, float *item_loss, float *loss, int grid,
                       cudaStream_t st);
void launch_calib_loss_grad(const float *x, const float *theta, const int32_t *item_sector,
                            const int32_t *item_start, const int32_t *sector_off,
                            const int32_t *sector_item, const int32_t *n_items, uint32_t S,
                            uint64_t n, const float *F, const float *q, const float *w,
                            const float *scale_dev, float *item_loss, float *item_grad,
                            float *sector_loss, unsigned int *tickets, float *loss, float *dF,
                            float *dq, float *y, int sms, cudaStream_t st);
void launch_calib_grad_scale(const float *g, const float *dF, const float *dq, uint32_t S,
                             float *out_F, float *out_q, cudaStream_t st);
void launch_calib_grad(const float *x, const float *grad_y, const int32_t *item_sector,
                       const int32_t *item_start, const int32_t *sector_off,
                       const int32_t *sector_item, const int32_t *n_items, uint32_t max_items,
                       uint32_t S, const float *F, float *item_grad, float *dF, float *dq,
                       float *dx, int grid, cudaStream_t st);

}  // namespace svt
