/*
 * svt.h -- C ABI of the GB300 (sm_103a) SVT linearised track-fit library.
 *
 * The method (Amerio et al., "Many-core applications to online track
 * reconstruction in HEP experiments", Sec. 2): inside every road (a coarse
 * track candidate), every combination of one hit per detector layer is fitted
 * with a linearised fit, p_i = f_i . x + q_i, using integer multiply/add and
 * constants looked up per road; the fit also yields a chi-square.  Sec. 2.1
 * splits the code into three stages -- unpack the input words, compute all
 * hit combinations of each road, fit each combination -- over three nested
 * loops (events, roads, combinations).  This library adds the chi-square cut,
 * the best combination per road and an output record.
 *
 * Fixed-point reading used throughout (the paper gives the form, not the
 * widths):
 *   x_l      unsigned 15-bit coordinate of the chosen hit of layer l (0..5),
 *            0 for a layer without hits;
 *   m        6-bit layer mask, bit l set iff layer l has at least one hit;
 *   acc_k    = q[s][m][k] * 2^qshift + sum_l F[s][m][k][l] * x_l   (exact int64)
 *   y_k      = floor(acc_k / 2^oshift)
 *   p_k      = (int32) y_k for k = 0,1,2   (d0, phi, curvature)
 *   chi2     = sum_{k=3..5} clamp(y_k, -32767, 32767)^2   (uint32)
 *   pass     iff chi2 <= chi2_cut; per road keep the passing combination with
 *            the smallest chi2, ties to the smallest combination index.
 * Combination index c: mixed radix over layers, layer 0 most significant,
 * layer 5 fastest, hits in order of appearance; n'_l = max(n_l, 1) and
 * C = prod n'_l.  A road with C > max_comb evaluates c < max_comb only and is
 * flagged OVERFLOW.  A road with fewer than min_layers layers hit is flagged
 * BAD_PATTERN and not fitted.
 * Track-trigger pairing (svt_config.xft_pairs = 1): layers 4 and 5 are the
 * two coordinates (phi, curvature) of one track-trigger track, so hit i of
 * layer 4 and hit i of layer 5 form one pair.  A road must then hold as many
 * layer-5 hits as layer-4 hits (else SVT_ERR_XFT_UNPAIRED at the road's last
 * hit word); the combination index runs over layers 0..4 only (layer 4 fastest,
 * C = prod_{l<5} n'_l) and layer 5 takes layer 4's hit index.
 *
 * Input words (uint32, type in bits [31:30]):
 *   event header (3): [29:12] event id, [11:0] number of roads (<= 4095)
 *   road header  (2): [29:21] sector (< n_sectors <= 512), [20:0] road id
 *   hit          (0): [29:27] layer (0..5), [26:15] reserved = 0, [14:0] coordinate
 *   type 1 is invalid.  An event is its header followed by its roads; a road
 *   is its header followed by its hits sorted by layer (at most 16 per layer).
 *   event_off[n_events + 1] (uint64) gives each event's first word;
 *   event_off[0] = 0, event_off[n_events] = n_words < 2^32.
 *
 * Output record, 6 x uint32 per road, roads in input order:
 *   w0 = road id [20:0] | flags << 24   (PASS 1, OVERFLOW 2, BAD_PATTERN 4, NO_HITS 8)
 *   w1 = best combination index (0xFFFFFFFF when nothing passes)
 *   w2 = chi2 of the best combination (0 when nothing passes)
 *   w3..w5 = p_0..p_2 as int32 bit patterns (0 when nothing passes)
 *
 * Constants: int16 F[n_sectors][64][6][6] (F[s][m][k][l]) and
 * q[n_sectors][64][6], row-major, little endian.
 *
 * Conventions for every entry point below:
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *     pointers; the library never allocates, frees or keeps device memory
 *     except where a function says otherwise (the serving loop).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     only enqueue work and return; nothing is synchronised unless stated.
 *   - The return value is a host-side status: SVT_OK, SVT_ERR_BAD_ARG for an
 *     argument the host can reject (null pointer, size over a limit, config
 *     out of range, workspace too small) or SVT_ERR_CUDA when a launch fails.
 *   - Problems found in the DATA are reported on the device in d_status, one
 *     uint64: UINT64_MAX when all is well, else (word_index << 8) | code, the
 *     smallest such key over all violated rules.  The outputs of a batch whose
 *     status is not UINT64_MAX are unspecified.  svt_unpack and svt_run reset
 *     d_status; the later plain stages read it, do no work when it already
 *     holds an error, and only ever lower it.
 */
#ifndef SVT_H
#define SVT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (host return values and the low 8 bits of d_status) ---- */
#define SVT_OK 0
#define SVT_ERR_BAD_ARG 1         /* bad argument; on the device: bad event offsets (word 0) */
#define SVT_ERR_BAD_TYPE 2        /* word type not allowed at this position            */
#define SVT_ERR_BAD_RESERVED 3    /* hit word with reserved bits set                    */
#define SVT_ERR_BAD_LAYER 4       /* hit layer > 5                                      */
#define SVT_ERR_UNSORTED 5        /* hit layer lower than the previous hit's            */
#define SVT_ERR_TOO_MANY_HITS 6   /* 17th hit of one layer in a road                    */
#define SVT_ERR_BAD_SECTOR 7      /* road sector >= n_sectors                           */
#define SVT_ERR_NROADS_MISMATCH 8 /* event header's road count differs from its roads   */
#define SVT_ERR_OOM 9             /* a caller-sized buffer is too small                 */
#define SVT_ERR_BAD_CONFIG 10     /* svt_config out of range                            */
#define SVT_ERR_TIMEOUT 11        /* a bounded device wait gave up                      */
#define SVT_ERR_XFT_UNPAIRED 12   /* paired layers 4 and 5 with different hit counts    */
#define SVT_ERR_CUDA 20           /* a CUDA call failed (host return value only)        */

#define SVT_STATUS_OK UINT64_MAX

/* ---- output flags (bits [31:24] of record word 0) ---- */
#define SVT_FLAG_PASS 1u
#define SVT_FLAG_OVERFLOW 2u
#define SVT_FLAG_BAD_PATTERN 4u
#define SVT_FLAG_NO_HITS 8u

/* Fit configuration.  Limits (else SVT_ERR_BAD_CONFIG): 9 <= oshift <= 31,
 * qshift <= 24, max_comb >= 1, min_layers <= 6, 1 <= n_sectors <= 512,
 * xft_pairs <= 1.  These limits keep |y_k| < 2^31 for every int16/uint15
 * input. */
typedef struct {
    uint32_t oshift;
    uint32_t qshift;
    uint32_t chi2_cut;
    uint32_t max_comb;
    uint32_t min_layers;
    uint32_t n_sectors;
    uint32_t xft_pairs;   /* 1: layers 4 and 5 come in track-trigger pairs (above) */
} svt_config;

/* Best combination of one road, as produced by svt_select (24 bytes). */
typedef struct {
    uint32_t flags;   /* SVT_FLAG_* */
    uint32_t comb;    /* best combination index, 0xFFFFFFFF if none passes */
    uint32_t chi2;
    int32_t p[3];
} svt_best;

/* Schedule of the fused path's persistent fit kernel.  Zero fields take the
 * defaults.
 *   warps_per_block  warps of one persistent block (1..16, default 8)
 *   blocks_per_sm    persistent blocks per SM (default: as many as fit)
 *   rows_per_item    rows of the (prefix x suffix) combination grid in one
 *                    work item of a split road (1..1024, default 16; each
 *                    item repeats its road's set-up, so longer items cost
 *                    less set-up and balance the work less finely)
 *   roads_per_chunk  consecutive roads a warp takes at once (1..32, default 4)
 *   small_max        roads with more evaluated combinations than this are
 *                    split into work items; the others are fitted whole by
 *                    one warp (default 4096)
 *   pair_small       1: two consecutive roads of a chunk that are both small
 *                    (at most 8 hits per layer, at most 16 rows and 16
 *                    suffix-table entries) and of the same split geometry are
 *                    fitted side by side by the two halves of one warp;
 *                    2: also four consecutive tiny roads (at most 2 hits per
 *                    layer, at most 8 rows and 16 suffix-table entries) of
 *                    the same geometry by the four quarters of one warp;
 *                    3: every tiny road of a chunk by lanes of its own (any
 *                    geometry): one lane a road with more than 16 roads per
 *                    chunk, two with 9..16, four with at most 8 (each lane
 *                    then takes every second or fourth row of the road's
 *                    combinations), then the chunk's other roads one per
 *                    warp; needs d_F and d_q 4-byte aligned and at most 12
 *                    warps per block (else BAD_ARG);
 *                    0 (default): one road per warp.  Grouping pays when most
 *                    roads are small and alike (the paper's fixed shape); on
 *                    mixed roads the warps keep switching between the code
 *                    paths and it costs. */
typedef struct {
    uint32_t warps_per_block;
    uint32_t blocks_per_sm;
    uint32_t rows_per_item;
    uint32_t roads_per_chunk;
    uint32_t small_max;
    uint32_t pair_small;
} svt_schedule;

/* Library version (major * 10000 + minor * 100 + patch). */
int svt_version(void);

/* Number of CUDA devices visible and the SM count of `device` (0 on error). */
int svt_device_sm_count(int device);

/* Arithmetic throughput of the current device, measured: every thread of a
 * full grid runs rings of eight dependent chains for 4 x iters steps (mode 0:
 * int32 3-input adds; 1: int32 multiply-adds; 2: both, as two independent
 * rings; 3: fp32 multiplies and fused multiply-adds, the fastest instruction
 * stream and so a measure of the schedulers' issue rate), timed with CUDA
 * events on `stream` after a warm-up launch.  *ops_per_s receives the
 * operations (lanes) per second, *seconds (may be NULL) the timed launch's
 * duration.  Context for the fused fit kernel's integer-ALU and issue
 * rooflines.  Synchronises the stream; allocates 1 KB of device memory for
 * the call.  Errors: SVT_ERR_BAD_ARG (mode > 3, iters = 0, null output),
 * SVT_ERR_CUDA. */
int svt_pipe_peak(uint32_t mode, uint32_t iters, double *ops_per_s, double *seconds,
                  void *stream);

/* ======================================================================
 * Plain path: one call per stage, one or more launches each, every
 * intermediate materialised in caller memory (the per-stage structure of the
 * paper's Sec. 2.1: unpack, combine, fit; then select and format).
 * ====================================================================== */

/* Workspace bytes svt_unpack needs for up to n_words words. */
size_t svt_unpack_workspace_size(uint64_t n_words);

/*
 * svt_unpack -- stage 1 of Sec. 2.1: unpack the input words into per-road
 * arrays and validate them.
 *   d_words[n_words], d_event_off[n_events+1]  input (see the word format)
 *   n_sectors      sectors of the constant table (road headers must be below)
 *   xft_pairs      1: check the layer-4/layer-5 pairing (SVT_ERR_XFT_UNPAIRED)
 *   road_cap       capacity of the road arrays
 *   d_road_word[road_cap]   out: word index of each road header, input order
 *   d_road_nhit[road_cap]   out: hits per layer, 5 bits each: n_l = (v >> 5l) & 31
 *   d_event_road[n_events+1] out: index of each event's first road; the last
 *                           entry is the road count R
 *   d_n_roads[1]   out: R (uint64)
 *   d_status[1]    out: reset, then the validation key (see above); R > road_cap
 *                  gives SVT_ERR_OOM at the first header that does not fit
 *   d_workspace    svt_unpack_workspace_size(n_words) bytes
 */
int svt_unpack(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
               uint64_t n_events, uint32_t n_sectors, uint32_t xft_pairs, uint64_t road_cap,
               uint32_t *d_road_word, uint32_t *d_road_nhit, uint32_t *d_event_road,
               uint64_t *d_n_roads,
               uint64_t *d_status, void *d_workspace, size_t workspace_bytes, void *stream);

/* Workspace bytes svt_combine needs for up to road_cap roads. */
size_t svt_combine_workspace_size(uint64_t road_cap);

/*
 * svt_combine -- stage 2 of Sec. 2.1: all combinations of one hit per layer
 * in every road, written out one record per combination.
 *   d_road_nhit, d_n_roads, road_cap   from svt_unpack
 *   cfg            host pointer to the fit configuration
 *   comb_cap       capacity of the combination arrays
 *   d_road_flags[road_cap]  out: OVERFLOW / BAD_PATTERN / NO_HITS per road
 *   d_comb_off[road_cap+1]  out: first combination of each road (uint64);
 *                           road r owns [d_comb_off[r], d_comb_off[r+1])
 *   d_comb_road[comb_cap]   out: road of each combination
 *   d_comb_hits[comb_cap]   out: hit index per layer, 4 bits each (layer l at
 *                           bits [4l+3:4l]); combinations of a road in
 *                           increasing index c
 *   d_n_combs[1]   out: total combinations (uint64)
 *   d_status       lowered to (0 << 8 | SVT_ERR_OOM) when the total exceeds comb_cap
 */
int svt_combine(const uint32_t *d_road_nhit, const uint64_t *d_n_roads, uint64_t road_cap,
                const svt_config *cfg, uint64_t comb_cap, uint32_t *d_road_flags,
                uint64_t *d_comb_off, uint32_t *d_comb_road, uint32_t *d_comb_hits,
                uint64_t *d_n_combs, uint64_t *d_status, void *d_workspace,
                size_t workspace_bytes, void *stream);

/*
 * svt_fit -- stage 3 of Sec. 2.1: the linearised fit of every combination
 * (one thread per combination; a block stages the constant rows and hit
 * coordinates of the roads of its tile of combinations in shared memory).
 *   d_words                       the input words (coordinates are read there)
 *   d_road_word, d_road_nhit      from svt_unpack
 *   d_comb_road, d_comb_hits, d_n_combs, comb_cap   from svt_combine
 *   d_F, d_q       constant table (int16, layout above), cfg->n_sectors sectors
 *   d_fit_chi2[comb_cap]    out: chi2 of each combination
 *   d_fit_par[3*comb_cap]   out: p_k of combination j at d_fit_par[k*comb_cap + j]
 */
int svt_fit(const uint32_t *d_words, const uint32_t *d_road_word, const uint32_t *d_road_nhit,
            const uint32_t *d_comb_road, const uint32_t *d_comb_hits, const uint64_t *d_n_combs,
            uint64_t comb_cap, const int16_t *d_F, const int16_t *d_q, const svt_config *cfg,
            uint32_t *d_fit_chi2, int32_t *d_fit_par, const uint64_t *d_status, void *stream);

/*
 * svt_select -- chi-square cut and best combination per road (one warp per
 * road, shuffle argmin; roads of more than 4096 combinations one block each,
 * in a second launch).
 *   d_fit_chi2, d_fit_par, comb_cap   from svt_fit
 *   d_comb_off, d_road_flags          from svt_combine
 *   d_best[road_cap]       out: per-road best (svt_best)
 */
int svt_select(const uint32_t *d_fit_chi2, const int32_t *d_fit_par, uint64_t comb_cap,
               const uint64_t *d_comb_off, const uint32_t *d_road_flags,
               const uint64_t *d_n_roads, uint64_t road_cap, const svt_config *cfg,
               svt_best *d_best, const uint64_t *d_status, void *stream);

/*
 * svt_format -- pack each road's result into the 6-word output record.
 *   d_best, d_n_roads, road_cap   from svt_select / svt_unpack
 *   d_words, d_road_word          to read each road id from its header
 *   d_out[6*road_cap]             out: records in input road order
 */
int svt_format(const svt_best *d_best, const uint32_t *d_words, const uint32_t *d_road_word,
               const uint64_t *d_n_roads, uint64_t road_cap, uint32_t *d_out,
               const uint64_t *d_status, void *stream);

/* ======================================================================
 * Kernel timer: a pair of CUDA events that svt_run records, on its stream,
 * right before and right after its persistent fit kernel (the events keep
 * that kernel from overlapping the one before it, so time whole runs without
 * a timer).  The timer is a
 * host object; create/destroy are the only calls that allocate (two events).
 * ====================================================================== */
typedef struct svt_timer_s *svt_timer;
int svt_timer_create(svt_timer *out);
int svt_timer_destroy(svt_timer timer);
/* Milliseconds of the last timed fit kernel; waits for its end event. */
int svt_timer_fit_ms(svt_timer timer, float *ms);

/* ======================================================================
 * Fused path: unpack, combine, fit, cut, select and format of a whole batch
 * of uneven events, with the combine, fit, cut, select and format in one
 * persistent kernel (dynamic work queue over warp-sized work items; each
 * warp writes the records of the roads it finished, one road per lane).
 * ====================================================================== */

/* Workspace bytes svt_run needs for batches of up to max_words words and
 * max_events events with up to road_cap roads.  sched may be NULL. */
size_t svt_run_workspace_size(uint64_t max_words, uint64_t max_events, uint64_t road_cap,
                              const svt_schedule *sched);

/*
 * svt_run -- the whole hot path of one batch.
 *   d_words[n_words], d_event_off[n_events+1]  input
 *   d_F, d_q, cfg      constant table and configuration
 *   road_cap           capacity of d_out (roads)
 *   d_out[6*road_cap]  out: one record per road, input order
 *   d_event_road[n_events+1]  out (may be NULL): first road of each event, then R
 *   d_counts[4]        out (may be NULL): R, work items of split roads, total
 *                      evaluated combinations, roads that passed
 *   d_status[1]        out: reset, then the validation key
 *   d_workspace        svt_run_workspace_size(n_words, n_events, road_cap, sched)
 *                      bytes, 256-byte aligned
 *   sched              schedule (NULL = defaults)
 *   timer              NULL, or a timer that records the fit kernel's events
 * Host-side limits: n_words < 2^32, n_events < 2^31, road_cap < 2^31.
 */
int svt_run(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
            uint64_t n_events, const int16_t *d_F, const int16_t *d_q, const svt_config *cfg,
            uint64_t road_cap, uint32_t *d_out, uint32_t *d_event_road, uint64_t *d_counts,
            uint64_t *d_status, void *d_workspace, size_t workspace_bytes,
            const svt_schedule *sched, svt_timer timer, void *stream);

/*
 * svt_run_sized -- svt_run with the batch sizes read on the device:
 * d_sizes[2] = {n_words, n_events} (device memory), at most max_words /
 * max_events, the capacities every buffer and the workspace are sized for
 * (svt_run_workspace_size(max_words, max_events, road_cap, sched)).  Sizes
 * above the capacities give status (0 << 8 | SVT_ERR_BAD_ARG) and no work.
 * This is the form a CUDA graph captures once and replays for every batch.
 */
int svt_run_sized(const uint32_t *d_words, uint64_t max_words, const uint64_t *d_event_off,
                  uint64_t max_events, const uint64_t *d_sizes, const int16_t *d_F,
                  const int16_t *d_q, const svt_config *cfg, uint64_t road_cap, uint32_t *d_out,
                  uint32_t *d_event_road, uint64_t *d_counts, uint64_t *d_status,
                  void *d_workspace, size_t workspace_bytes, const svt_schedule *sched,
                  void *stream);

/* Schedule autotuner: runs svt_run on one device-resident batch for every
 * schedule of {4, 8, 16} warps per block x {8, 16, 32, 64} rows per item x
 * {1, 2, 4, 8} roads per chunk x {1024, 4096, 16384} small_max (blocks per SM
 * as many as fit, no pairing), then the fastest of those with 2 and 4 times
 * its rows per item, then the fastest so far with pair_small = 1
 * and {2, 4, 8} roads per chunk, with pair_small = 2 and {4, 8, 16} roads
 * per chunk and (for 4-byte aligned d_F and d_q) with pair_small = 3 and
 * {8, 16, 32} roads per chunk (8 warps per block where the fastest had 16), then
 * the fastest so far with 1 and 2 blocks per SM, one warm-up and `reps` timed
 * runs each (CUDA events on `stream`);
 * finally the four fastest of all these once more with 3 * reps runs each,
 * and returns the fastest of that pass and its mean time per run.
 *   d_flush, flush_bytes  device scratch (may be NULL with flush_bytes 0):
 *                      when given, every timed run is preceded by a write of
 *                      flush_bytes to it outside the timed region and timed
 *                      alone, so that with flush_bytes above the L2 size no
 *                      run finds the batch in L2 (as for batches that arrive
 *                      one after another); without it the runs go back to back
 * Errors: SVT_ERR_BAD_ARG for reps outside [1, 100], a NULL best / best_ms or
 * flush_bytes > 0 with a NULL d_flush; else as svt_run.
 * Synchronises the stream.  Buffers as for svt_run; on return d_out and
 * d_status hold a valid result of the batch (every schedule gives the same
 * bits). */
int svt_autotune(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
                 uint64_t n_events, const int16_t *d_F, const int16_t *d_q, const svt_config *cfg,
                 uint64_t road_cap, uint32_t *d_out, uint64_t *d_status, void *d_workspace,
                 size_t workspace_bytes, uint32_t reps, void *d_flush, size_t flush_bytes,
                 svt_schedule *best, float *best_ms, void *stream);

/* CUDA graph of svt_run_sized's launch sequence, captured once on a private
 * stream (same arguments).  svt_graph_launch replays it on `stream`; every
 * replay reads the then-current device contents of d_sizes, d_words and
 * d_event_off.  create/destroy allocate and free the graph objects. */
typedef struct svt_graph_s *svt_graph;
int svt_graph_create(const uint32_t *d_words, uint64_t max_words, const uint64_t *d_event_off,
                     uint64_t max_events, const uint64_t *d_sizes, const int16_t *d_F,
                     const int16_t *d_q, const svt_config *cfg, uint64_t road_cap,
                     uint32_t *d_out, uint32_t *d_event_road, uint64_t *d_counts,
                     uint64_t *d_status, void *d_workspace, size_t workspace_bytes,
                     const svt_schedule *sched, svt_graph *out);
int svt_graph_launch(svt_graph graph, void *stream);
int svt_graph_destroy(svt_graph graph);

/* ======================================================================
 * End to end from host memory: the batch's words and offsets copied in, the
 * fused path, the records and the status copied out -- every step enqueued
 * on `stream`, in that order (the trigger node's "data in -> GPU -> data
 * out" loop of Sec. 3 and Sec. 4.2 as one call).
 *   h_words[n_words], h_event_off[n_events+1]  host input; pinned memory
 *                      makes the copies asynchronous (pageable memory is
 *                      copied before the call returns)
 *   d_F, d_q, cfg, road_cap, sched   as for svt_run
 *   h_out[6*road_cap]  host, out: the records (valid once the stream has
 *                      completed the call's work)
 *   h_status[1]        host, out: the validation key, likewise
 *   n_records          host, out (may be NULL): records written to h_out,
 *                      the road count the event headers state (read on the
 *                      host before the call returns), at most road_cap
 *   d_workspace        svt_run_host_workspace_size(n_words, n_events,
 *                      road_cap, sched) bytes of device memory, 256-byte
 *                      aligned; it holds the batch's device copies and
 *                      svt_run's workspace
 * The host buffers and the workspace must stay untouched until the stream
 * has completed the call.  To overlap one batch's copies with another's
 * compute, alternate two streams, each with its own workspace and host
 * buffers.  Errors: SVT_ERR_BAD_ARG (null pointers, sizes over the limits
 * of svt_run, a workspace too small or misaligned), else as svt_run.
 * ====================================================================== */
size_t svt_run_host_workspace_size(uint64_t max_words, uint64_t max_events, uint64_t road_cap,
                                   const svt_schedule *sched);
int svt_run_host(const uint32_t *h_words, uint64_t n_words, const uint64_t *h_event_off,
                 uint64_t n_events, const int16_t *d_F, const int16_t *d_q, const svt_config *cfg,
                 uint64_t road_cap, uint32_t *h_out, uint64_t *h_status, uint64_t *n_records,
                 void *d_workspace, size_t workspace_bytes, const svt_schedule *sched,
                 void *stream);

/* ======================================================================
 * svt_run without a workspace argument.  The paper has no counterpart: this
 * is for callers of this library that cannot allocate device memory at all
 * -- a front-end process that only receives device pointers from whatever
 * owns the GPU, a real-time loop whose rules forbid allocating (with its
 * latency and failure modes) once data taking has started, or a host program
 * linked without a device allocator of its own.
 *
 * The scratch is one fixed array inside the library, SVT_NOALLOC_SCRATCH_BYTES
 * (32 MiB) per GPU.  It is reserved on a GPU when the library's code is
 * loaded there -- under CUDA's default lazy module loading, at the first
 * svt_run_noalloc call on that GPU -- and held until the process exits.
 * A batch whose svt_run_workspace_size(n_words, n_events, road_cap, sched)
 * exceeds it is refused with SVT_ERR_OOM before anything is enqueued (32 MiB
 * covers, e.g., a 3000-event batch of 3.5 million words and 190 thousand
 * roads).  The first call on a device looks up the array's device address
 * (only a successful lookup is kept; a failed one returns SVT_ERR_CUDA and
 * is retried by the next call); make that first call before any stream
 * capture.  Every call on a device
 * shares the array and it keeps the last call's contents; each call
 * re-initialises everything it reads, but calls whose work overlaps on the
 * GPU (different streams, or different host threads) race on it: issue them
 * on one stream or otherwise one after another.  Nothing is allocated or
 * freed.  Arguments and results are those of svt_run.
 * ====================================================================== */
#define SVT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
size_t svt_run_noalloc_scratch_bytes(void);
int svt_run_noalloc(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
                    uint64_t n_events, const int16_t *d_F, const int16_t *d_q,
                    const svt_config *cfg, uint64_t road_cap, uint32_t *d_out,
                    uint32_t *d_event_road, uint64_t *d_counts, uint64_t *d_status,
                    const svt_schedule *sched, void *stream);

/* ======================================================================
 * Host memory the GPU reads and writes in place (zero-copy).  The paper's
 * Sec. 4.2 compares staging a packet through host buffers with delivering it
 * straight into GPU memory; on a GB300 node the Grace host memory is itself
 * reachable from the GPU over NVLink-C2C, so a batch can stay in host memory
 * and be read by the kernels directly.  svt_host_alloc returns `bytes` of
 * pinned host memory mapped into the device address space: *host for the
 * CPU, *device for kernels (both 256-byte aligned); any svt_* argument that
 * takes device memory may point into it (for example d_words, d_event_off or
 * d_out of svt_run).  Errors: BAD_ARG (null pointers, zero size), OOM (the
 * allocation failed), CUDA (no device mapping, or a mapping that is not
 * 256-byte aligned).  svt_host_free releases the
 * memory; no work that uses it may still be in flight.
 * ====================================================================== */
int svt_host_alloc(size_t bytes, void **host, void **device);
int svt_host_free(void *host);

/* ======================================================================
 * Serving loop (the single-GPU form of the paper's trigger-node loop,
 * Sec. 3 and Sec. 4.2: data in -> GPU -> data out), with continuous
 * batching.  Events are submitted by reference -- a pointer to the event's
 * words (its header first) in PINNED host memory that stays valid until the
 * event's result is delivered.  A dispatcher thread admits queued events into
 * free device slots (each slot holds a batch of at most max_words words,
 * max_events events and max_roads roads: this is the device-memory budget),
 * copies each contiguous run of event words with one H2D copy, replays the
 * slot's captured CUDA graph of svt_run_sized and copies the records back,
 * each slot on its own stream, so batches overlap on the device.  A batch
 * whose status reports a data error is re-run event by event, so a corrupt
 * event fails alone.  The library allocates no device or pinned memory here:
 * the caller passes both (svt_server_sizes).  Results carry the latency from
 * submission to the moment the event's records are in the caller's buffer.
 * Per batch the dispatcher issues one copy per contiguous run of event words,
 * one copy of the sizes and offsets, the graph replay and one copy back of
 * the status, the event table and the records.
 * ====================================================================== */
typedef struct {
    uint32_t n_slots;            /* batches in flight, 1..16 */
    uint32_t mode;               /* 0: fused path, one captured graph per slot;
                                    1: plain per-stage path (svt_unpack .. svt_format) */
    uint64_t max_words;          /* per batch */
    uint64_t max_events;         /* per batch */
    uint64_t max_roads;          /* per batch */
    uint64_t max_combs;          /* per batch, mode 1 only (combination records) */
    uint64_t device_budget;      /* bytes; 0 = no limit (else create fails with OOM) */
    uint64_t max_queued_words;   /* admission queue bound; 0 = unbounded */
    uint32_t small_batch_events; /* mode 0: batches of at most this many events replay a
                                    second graph whose fit launch has small_blocks_per_sm
                                    persistent blocks per SM (fewer resident warps suit
                                    small batches); 0 = one graph per slot */
    uint32_t small_blocks_per_sm;   /* 0 = 1 */
} svt_server_config;

typedef struct {
    uint64_t tag;                /* as submitted */
    uint64_t status;             /* SVT_STATUS_OK or the event's error key */
    uint32_t n_roads;
    uint32_t reserved;
    uint64_t latency_ns;         /* submission -> completion seen */
    int64_t t_arrive_ns;         /* steady-clock submission time */
} svt_event_result;

typedef struct {
    uint64_t batches, events_done, events_failed, retried_batches, rejected, queued;
    uint64_t h2d_bytes, d2h_bytes;
    uint64_t max_queued;        /* most events waiting when a batch was taken */
    uint64_t max_batch_events;  /* most events in one batch */
    uint64_t launch_ns;         /* dispatcher time spent enqueueing batches */
    uint64_t finish_ns;         /* dispatcher time spent delivering results */
} svt_server_stats;

/* One served batch, as recorded by svt_server_trace.  Host times are
 * steady-clock nanoseconds (the clock of svt_event_result.t_arrive_ns);
 * device times are microseconds since the trace started, from timing events
 * recorded on the slot's stream before its first copy and after its last
 * one (so two slots' intervals that overlap show batches in flight on the
 * device together). */
typedef struct {
    uint32_t slot, n_events;
    uint32_t n_roads, queued_after;   /* events still waiting once the batch was taken */
    int64_t t_first_arrive_ns;        /* earliest arrival among the batch's events */
    int64_t t_dispatch_ns;            /* the dispatcher took the events */
    int64_t t_enqueued_ns;            /* every copy and launch of the batch enqueued */
    int64_t t_done_ns;                /* the dispatcher saw the batch complete */
    float dev_start_us, dev_end_us;   /* -1 when a timestamp could not be read */
} svt_batch_trace;

typedef struct svt_server_s *svt_server;

/* Device workspace and pinned host bytes a server with this config needs. */
int svt_server_sizes(const svt_server_config *cfg, const svt_schedule *sched,
                     size_t *device_bytes, size_t *pinned_bytes);
/* Creates the slots (streams, events, one captured graph each) and starts the
 * dispatcher thread.  d_F, d_q, fit stay owned by the caller and must outlive
 * the server.  d_workspace and h_pinned must be 256-byte aligned. */
int svt_server_create(const svt_server_config *cfg, const int16_t *d_F, const int16_t *d_q,
                      const svt_config *fit, const svt_schedule *sched, void *d_workspace,
                      size_t workspace_bytes, void *h_pinned, size_t pinned_bytes,
                      svt_server *out);
/* Queues one event (thread safe).  h_records (may be NULL) receives the
 * event's records (6 x uint32 per road) before its result is delivered.
 * SVT_ERR_OOM: the event can never fit a slot, or the queue bound is reached. */
int svt_server_submit(svt_server server, const uint32_t *h_words, uint32_t n_words, uint64_t tag,
                      uint32_t *h_records);
/* Takes up to max_results delivered results; waits up to wait_us for one. */
int svt_server_poll(svt_server server, svt_event_result *out, uint32_t max_results,
                    uint32_t *n_out, uint32_t wait_us);
int svt_server_stats_get(svt_server server, svt_server_stats *out);
/* Zeroes the counters (the queue length is always the current one). */
int svt_server_stats_reset(svt_server server);
/* Starts recording one svt_batch_trace per completed batch into the caller's
 * host array buf[cap] (from its first entry; batches beyond cap are not
 * recorded); buf = NULL stops.  With device_times each batch also records
 * two timing events on its stream (a few microseconds of latency per batch);
 * without, dev_start_us and dev_end_us are -1.  Read the entries after
 * stopping the trace, or once the server is idle: svt_server_trace_count
 * gives how many were written. */
int svt_server_trace(svt_server server, svt_batch_trace *buf, uint64_t cap, uint32_t device_times);
int svt_server_trace_count(svt_server server, uint64_t *n);
/* Stops the dispatcher after the batches in flight; undelivered events are dropped. */
int svt_server_destroy(svt_server server);
/* Poisson arrivals at rate_hz of n_events events, event i being pool event
 * i mod n_pool (words h_pool in pinned memory, pool_off[n_pool + 1] word
 * offsets).  h_records (may be NULL): event i's records go to
 * h_records + 6 * rec_off[i] (rec_off[n_events] road offsets).  lat_ns[i] =
 * latency of event i from its scheduled arrival time to the delivery of its
 * result (UINT64_MAX if it failed); *wall_s = time from the first arrival to
 * the last completion. */
int svt_server_bench_poisson(svt_server server, const uint32_t *h_pool, const uint64_t *pool_off,
                             uint32_t n_pool, double rate_hz, uint64_t n_events, uint64_t seed,
                             uint32_t *h_records, const uint64_t *rec_off, uint64_t *lat_ns,
                             double *wall_s);

/* ======================================================================
 * FP32 calibration relaxation.  The fit of Sec. 2 without the integer shift
 * and clamp, per track t of sector s:
 *     y_t = F[s] x_t + q[s]        (F: float [S][6][6], q: float [S][6])
 *     L   = (1/N) sum_t [ sum_{k<3} w_k (y_tk - theta_tk)^2 + sum_{k>=3} y_tk^2 ]
 * with hand-written forward and backward kernels, for calibrating fit
 * constants on tracks whose true parameters theta are known.  Tracks are
 * used in sector order: svt_calib_index sorts them (stable counting sort on
 * the device) and svt_calib_gather permutes per-track arrays.  All sums run
 * in a fixed order, so repeated calls give identical bits.
 * Layouts: x float [N][6], theta float [N][3], w float [3], y float [N][6].
 * ====================================================================== */

/* Bytes of the sector index of n tracks in n_sectors sectors. */
size_t svt_calib_index_size(uint64_t n_tracks, uint32_t n_sectors);

/* Sector index: d_perm[i] = original index of the i-th track in sector order
 * (stable).  d_status: reset, then (track << 8 | SVT_ERR_BAD_SECTOR) of the
 * first track whose sector is outside [0, n_sectors).  n_tracks < 2^31,
 * n_sectors <= 512. */
int svt_calib_index(const int32_t *d_sector, uint64_t n_tracks, uint32_t n_sectors, void *d_index,
                    size_t index_bytes, int32_t *d_perm, uint64_t *d_status, void *stream);

/* d_dst[i][c] = d_src[d_perm[i]][c] for c < width. */
int svt_calib_gather(const float *d_src, uint32_t width, const int32_t *d_perm, uint64_t n,
                     float *d_dst, void *stream);

/* Workspace bytes of the loss and backward calls (zero-fill it once after
 * allocating it: see svt_calib_loss_grad). */
size_t svt_calib_workspace_size(uint64_t n_tracks, uint32_t n_sectors);

/* y = F[s] x + q[s] for sector-ordered tracks. */
int svt_calib_forward(const float *d_x, uint64_t n_tracks, uint32_t n_sectors,
                      const void *d_index, const float *d_F, const float *d_q, float *d_y,
                      void *stream);

/* d_loss[0] = L for sector-ordered tracks (staged in shared memory by bulk
 * copies, as in svt_calib_loss_grad, when d_x and d_theta start on 16-byte
 * boundaries). */
int svt_calib_loss(const float *d_x, const float *d_theta, const float *d_w, uint64_t n_tracks,
                   uint32_t n_sectors, const void *d_index, const float *d_F, const float *d_q,
                   float *d_loss, void *d_workspace, size_t workspace_bytes, void *stream);

/* d_dF = g dL/dF, d_dq = g dL/dq with g = *d_grad_loss (NULL: g = 1): the
 * pass of svt_calib_loss_grad with its loss kept in the workspace. */
int svt_calib_loss_backward(const float *d_x, const float *d_theta, const float *d_w,
                            uint64_t n_tracks, uint32_t n_sectors, const void *d_index,
                            const float *d_F, const float *d_q, const float *d_grad_loss,
                            float *d_dF, float *d_dq, void *d_workspace, size_t workspace_bytes,
                            void *stream);

/* The loss and its gradient in one pass over the tracks (x and theta read
 * once): d_loss[0] = L, d_dF = dL/dF, d_dq = dL/dq and, when d_y is not NULL,
 * d_y = F[s] x + q[s] as svt_calib_forward writes it.  Every sum runs in a
 * fixed order for a given device, so repeated calls give identical bits.
 * Sectors without tracks get zero gradients.  When d_x and d_theta start on
 * 16-byte boundaries, each item's tracks are staged in shared memory by
 * bulk copies (the bulk-copy unit's alignment rule) and the final sums are
 * made by a second kernel chained by programmatic dependent launch; a staged
 * copy that does not land within the pass's bounded wait makes *d_loss NaN.
 * Otherwise every lane loads its own tracks and the final sums are made by
 * the warps that complete each sector and the batch (atomic tickets in the
 * workspace; nothing waits).  Both give the same y.  The workspace must be
 * zero-filled once after it is allocated; every call of svt_calib_loss_grad
 * or svt_calib_loss_backward leaves its tickets and flag at zero again. */
int svt_calib_loss_grad(const float *d_x, const float *d_theta, const float *d_w,
                        uint64_t n_tracks, uint32_t n_sectors, const void *d_index,
                        const float *d_F, const float *d_q, float *d_loss, float *d_dF,
                        float *d_dq, float *d_y, void *d_workspace, size_t workspace_bytes,
                        void *stream);

/* d_out_dF = (*d_scale) d_dF and d_out_dq = (*d_scale) d_dq (n_sectors
 * sectors; the outputs may alias the inputs): the chain rule's last step when
 * the gradient of L was formed by svt_calib_loss_grad before the upstream
 * gradient was known. */
int svt_calib_grad_scale(const float *d_scale, const float *d_dF, const float *d_dq,
                         uint32_t n_sectors, float *d_out_dF, float *d_out_dq, void *stream);

/* Backward of y = F[s] x + q[s] from d_grad_y [N][6]: d_dF[s] = sum_t g_t x_t^T,
 * d_dq[s] = sum_t g_t and, when d_dx is not NULL, d_dx_t = F[s]^T g_t. */
int svt_calib_backward(const float *d_x, const float *d_grad_y, uint64_t n_tracks,
                       uint32_t n_sectors, const void *d_index, const float *d_F, float *d_dF,
                       float *d_dq, float *d_dx, void *d_workspace, size_t workspace_bytes,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SVT_H */
