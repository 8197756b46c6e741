// svt_kernels.cuh -- declarations of the kernels and launch helpers that the
// C-ABI layer (svt_abi.cu) strings together.
#pragma once

#include "svt_internal.cuh"
#include "svt_roads.cuh"

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
                                  const FusedRoads fr, uint32_t roads_per_chunk, uint32_t group,
                                  uint32_t *out, unsigned long long *status,
                                  int warps_per_block, int grid, cudaStream_t st);
// persistent blocks of the fit kernel per SM for a block size and a road
// grouping (1, 2, 4 or 32; both chi2-cut instances of it)
int fit_persistent_blocks_per_sm(int warps_per_block, uint32_t group);
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
                       const int32_t *sector_item, const int32_t *n_items, uint32_t max_items,
                       uint32_t S, uint64_t n, const float *F, const float *q, const float *w,
                       float *item_loss, unsigned int *flag, float *loss, int sms, int grid,
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
