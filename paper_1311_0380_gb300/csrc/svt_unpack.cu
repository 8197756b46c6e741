// svt_unpack.cu -- stage 1 of the paper's Sec. 2.1 for GB300: the input
// words are parsed and the per-road structures the later stages read are
// built.
//
// The batch is cut into tiles of 1024 words (128 threads x 8 words; smaller
// tiles than 2048 words of 256 threads take 1-2 % off the step, since the
// kernels are bound by each tile's chain of barriers and scans).  A prologue maps every tile to
// the first event that starts in it (one pass over the event offsets).  One
// pass over the tiles then validates every word against its left neighbour
// (rules V2..V7, V9 of include/svt.h's format), checks V1 for the events
// starting in the tile, gives every road header its global index (a block
// scan, plus the road count of the tiles before, found by looking back over
// the counts that earlier tiles publish), records where it sits, counts its
// hits (rule V8, hits per layer) and, for the fused path, sizes its work and
// appends split roads to the work list.  The offsets and V10 are checked per
// event afterwards.  Loads are vectorised (2 x 16 B per thread, coalesced
// across the warp).
#include "svt_kernels.cuh"

namespace svt {

namespace {

static_assert(TILE_PER_THREAD == 8, "load8 fills eight words per thread");
__device__ __forceinline__ void load8(const uint32_t *__restrict__ words, uint64_t base,
                                      uint64_t n_words, uint32_t (&w)[TILE_PER_THREAD]) {
    if (base + TILE_PER_THREAD <= n_words) {
        const uint4 *p = reinterpret_cast<const uint4 *>(words + base);
        uint4 a = __ldg(p), b = __ldg(p + 1);
        w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
        w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    } else {
#pragma unroll
        for (int j = 0; j < TILE_PER_THREAD; ++j)
            w[j] = (base + j < n_words) ? __ldg(words + base + j) : 0u;
    }
}

// First index e in [0, n) with off[e] >= v (off assumed non-decreasing),
// searched cooperatively by a warp (every lane gets the result): 32 probes per
// round, so log32(n) dependent loads instead of log2(n).
__device__ __forceinline__ uint64_t warp_lower_bound64(const uint64_t *__restrict__ off,
                                                       uint64_t n, uint64_t v, int lane) {
    uint64_t lo = 0, hi = n;
    while (hi > lo) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t p = lo + (uint64_t)lane * step;
        const bool lt = p < hi && __ldg(off + p) < v;
        const uint32_t k = __popc(__ballot_sync(0xffffffffu, lt));
        if (k == 0) {
            hi = lo;
        } else {
            const uint64_t pk = lo + (uint64_t)(k - 1) * step;
            hi = min(pk + step, hi);
            lo = pk + 1;
        }
    }
    return lo;
}

// Batch sizes for the launch sequence: the given values, or -- when `sizes`
// is set -- the device-resident pair {n_words, n_events}, which must not
// exceed the capacities the sequence was sized for (else BAD_ARG, empty batch).
// Every block derives the sizes itself; block 0 publishes them.
//
// first_ev[t] = lower_bound(event_off, t * TILE_WORDS) for t = 0..T: event e
// writes the tiles t with event_off[e-1] < t * TILE_WORDS <= event_off[e].
// With increasing offsets every entry is written once; otherwise the offsets
// are reported as BAD_ARG (the smallest key) by the per-event check, and the
// consumers clamp what they read to [0, n_events].
__global__ void k_prologue(Dims *dims, uint64_t n_words, uint64_t n_events,
                           const uint64_t *sizes, const uint64_t *__restrict__ event_off,
                           uint32_t *first_ev, unsigned long long *status, uint64_t *counts,
                           int n_counts, uint64_t *zero, int n_zero,
                           unsigned long long *tile_state, uint32_t *tile_ticket) {
    // first of its sequence: launched in stream order after whatever came
    // before, so only the next kernel is let in early
    allow_next_grid();
    bool bad = false;
    if (sizes) {
        const uint64_t w = sizes[0], e = sizes[1];
        bad = w > n_words || e > n_events;
        n_words = bad ? 0 : w;
        n_events = bad ? 0 : e;
    }
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        if (dims) {
            dims->n_words = n_words;
            dims->n_events = n_events;
        }
        if (status) *status = bad ? (unsigned long long)SVT_ERR_BAD_ARG : ~0ull;
    }
    if (counts && tid < (uint64_t)n_counts) counts[tid] = 0;
    if (zero && tid < (uint64_t)n_zero) zero[tid] = 0;
    if (!first_ev) return;
    const uint64_t T = n_tiles(n_words);
    // nothing published and no tile taken yet
    if (tile_ticket && tid == 0) *tile_ticket = 0;
    if (tile_state)
        for (uint64_t t = tid; t < T; t += stride) tile_state[t] = 0ull;
    for (uint64_t e = tid; e <= n_events; e += stride) {
        const uint64_t t0 = e > 0 ? min(__ldg(event_off + e - 1), n_words) / TILE_WORDS + 1 : 0;
        const uint64_t t1 = e < n_events ? min(__ldg(event_off + e), n_words) / TILE_WORDS : T;
        for (uint64_t t = t0; t <= min(t1, T); ++t) first_ev[t] = (uint32_t)e;
    }
}

// Events [e_lo, e_hi) that start in tile t, clamped to the batch.
__device__ __forceinline__ void tile_events(const uint32_t *__restrict__ first_ev, uint64_t t,
                                            uint64_t n_events, uint64_t &e_lo, uint64_t &e_hi) {
    e_lo = min((uint64_t)__ldg(first_ev + t), n_events);
    e_hi = max(e_lo, min((uint64_t)__ldg(first_ev + t + 1), n_events));
}

// ---- road indices across tiles: one pass with look-back --------------------------
// Every tile publishes its road count in tile_state[t] as soon as its block
// has counted (kind TILE_AGGREGATE), and its inclusive prefix -- the roads of
// tiles 0..t -- once it knows the tiles before it (kind TILE_INCLUSIVE; tile 0
// publishes that at once).  Words: kind in bits [63:62], count in [39:0];
// zero means nothing published yet.
constexpr unsigned long long TILE_AGGREGATE = 1, TILE_INCLUSIVE = 2;
constexpr unsigned long long TILE_COUNT_MASK = (1ull << 40) - 1;
constexpr uint32_t LOOK_BACK_SPINS = 1u << 20;   // bounded wait, then SVT_ERR_TIMEOUT

__device__ __forceinline__ void publish_tile(unsigned long long *p, unsigned long long kind,
                                             unsigned long long v) {
    const unsigned long long x = (kind << 62) | (v & TILE_COUNT_MASK);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(x) : "memory");
}
__device__ __forceinline__ unsigned long long peek_tile(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Roads in the tiles before tile t (t >= 1), by one warp: lane k reads tile
// hi - k of a window of 32 tiles, newest first; the sum runs over the window's
// tiles up to the newest one whose inclusive count is out (that one
// included), else over the whole window and on to the next.  A tile that has
// published nothing yet is re-read after a short sleep; it belongs to a block
// that took its tile earlier and is running, so it publishes soon.  After
// LOOK_BACK_SPINS rounds the wait gives up with SVT_ERR_TIMEOUT (the batch's
// status is then an error and its outputs are not used).
__device__ unsigned long long tiles_before(const unsigned long long *state, uint64_t t, int lane,
                                           unsigned long long *status) {
    unsigned long long excl = 0;
    uint32_t spins = 0;
    for (int64_t hi = (int64_t)t - 1; hi >= 0; hi -= 32) {
        const int64_t idx = hi - lane;
        // before tile 0 there is nothing: read as an inclusive count of zero
        unsigned long long v = idx >= 0 ? peek_tile(state + idx) : (TILE_INCLUSIVE << 62);
        for (;;) {
            const uint32_t incl = __ballot_sync(0xffffffffu, (v >> 62) == TILE_INCLUSIVE);
            const uint32_t stop = incl ? (uint32_t)(__ffs(incl) - 1) : 31u;
            const uint32_t need = stop == 31u ? 0xffffffffu : ((2u << stop) - 1u);
            const uint32_t missing = __ballot_sync(0xffffffffu, (v >> 62) == 0) & need;
            if (!missing) {
                unsigned long long x = (uint32_t)lane <= stop ? (v & TILE_COUNT_MASK) : 0ull;
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
                excl += x;
                if (incl) return excl;
                break;
            }
            if (++spins > LOOK_BACK_SPINS) {
                if (lane == 0) report(status, 0, SVT_ERR_TIMEOUT);
                return excl;
            }
            __nanosleep(64);
            if ((missing >> lane) & 1u) v = peek_tile(state + idx);
        }
    }
    return excl;
}

// Largest v over the lower threads of the block (-1 when there are none);
// `smem` holds TILE_THREADS / 32 entries.
__device__ __forceinline__ int block_exclusive_max(int v, int *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x = max(x, y);
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < n_warps ? smem[lane] : -1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t = max(t, y);
        }
        if (lane < n_warps) smem[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    int e = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) e = -1;
    const int res = max(e, warp > 0 ? smem[warp - 1] : -1);
    __syncthreads();
    return res;
}

// K2, data-parallel per tile:
//  * the tile is staged in shared memory with 16 words before it and 100
//    after it (a valid road has at most 96 hits, so a road that starts in the
//    tile ends in the staged range);
//  * a block scan gives every road header its index; each thread adds its hits
//    to its road's counters of their layers (one shared-memory atomic per run
//    of its words in one road, on the packed 5-bits-per-layer word; a field can
//    only overflow with more than 31 hits of one layer, which rule V8 already
//    rejects);
//  * rule V8: a hit whose 16 predecessors are hits of the same layer is the
//    17th (or later) of a contiguous block.  For the smallest status key this
//    matches counting over the run: the first out-of-order hit of a run is an
//    UNSORTED word that precedes any later, non-contiguous 17th hit.  Every
//    word gets one bit, "a hit of the same layer as the word before", in a
//    bitmap of the tile and its front halo; V8 fires where 16 set bits end;
//  * one thread per road then writes the road's outputs; for the fused path
//    the tile's split roads are appended to the work list at a range that
//    one atomic reserves for the whole tile.
// (40 registers, a few spilled, for 12 resident tiles per SM: 2-3 % faster
// than 56 registers and 9 tiles)
__global__ void __launch_bounds__(TILE_THREADS, 12)
    k_unpack_roads(const uint32_t *__restrict__ words, const uint64_t *__restrict__ event_off,
                   const Dims *__restrict__ dims, const uint32_t *__restrict__ first_ev,
                   unsigned long long *tile_state, uint32_t *tile_ticket, uint64_t *total64,
                   uint64_t road_cap, uint32_t *road_word, uint32_t *road_nhit,
                   uint32_t *event_road, const svt_config cfg, const FusedRoads fr,
                   uint64_t *counts, unsigned long long *status) {
    constexpr int FRONT = 16, BACK = 100;
    static_assert(TILE_THREADS >= BACK && TILE_THREADS > TILE_WORDS / 32,
                  "one pass of the block loads the halo and covers the V8 bitmap");
    constexpr uint32_t SENTINEL = 0xC0000000u;   // an event-header word: ends every run
    __shared__ uint32_t red[TILE_THREADS / 32 + 1];
    __shared__ unsigned long long red64[TILE_THREADS / 32 + 1];
    __shared__ int redi[TILE_THREADS / 32];
    __shared__ uint32_t sw[FRONT + TILE_WORDS + BACK];
    __shared__ uint32_t cnt[TILE_WORDS];              // per road of the tile: 5 bits per layer
    // V11 counts of each road's hit run: layer 4 [9:0], layer 5 [19:10], all
    // hits [31:20].  A field can only overflow in a run of more than 1023 hits,
    // which then also shows more than 96 hits and is not checked.
    __shared__ uint32_t cnt45[TILE_WORDS];
    __shared__ uint16_t hdr_pos[TILE_WORDS];          // tile position of each road header
    __shared__ int last_nonhit;
    __shared__ int v1_flag;   // a V1 failure in the tile (read after the header barrier)
    __shared__ unsigned long long big_base;
    __shared__ unsigned long long tile_comb;   // evaluated combinations of the tile
    __shared__ uint32_t same_bits[1 + TILE_WORDS / 32];   // V8 bitmap, see below
    __shared__ uint32_t tile_s;                            // the tile this block took
    __shared__ unsigned long long base_s;                  // roads before the tile
    wait_prior_grid();
    allow_next_grid();
    if (threadIdx.x == 0) tile_comb = 0;   // visible after the tile loop's first barrier
    const uint64_t n_words = dims->n_words, n_events = dims->n_events;
    const uint64_t T = n_tiles(n_words);
    // tiles are taken in increasing order from a counter, so the tiles before
    // the one a block holds belong to blocks that are already running
    // (the next tile is taken by thread 0 before the barrier that ends a tile)
    if (threadIdx.x == 0) tile_s = atomicAdd(tile_ticket, 1u);
    __syncthreads();
    for (;;) {
        const uint64_t t = tile_s;
        if (t >= T) break;
        const uint64_t tile_start = t * TILE_WORDS;
        const uint64_t tile_end = min(tile_start + TILE_WORDS, n_words);
        const int tile_len = (int)(tile_end - tile_start);
        const uint64_t base = tile_start + (uint64_t)threadIdx.x * TILE_PER_THREAD;
        if (threadIdx.x == 0) {
            last_nonhit = -1;
            v1_flag = 0;
        }
        uint32_t w[TILE_PER_THREAD];
        load8(words, base, n_words, w);
        // the events that start in the tile and the first offset of this
        // thread's first one, loaded while the block scans
        uint64_t e_lo, e_hi;
        tile_events(first_ev, t, n_events, e_lo, e_hi);
        const uint64_t s0_first =
            e_lo + threadIdx.x < e_hi ? __ldg(event_off + e_lo + threadIdx.x) : 0ull;
        uint32_t nh = 0;   // road headers (low 16 bits) and event headers (high 16 bits)
#pragma unroll
        for (int j = 0; j < TILE_PER_THREAD; ++j) {
            const int p = threadIdx.x * TILE_PER_THREAD + j;
            const bool in = p < tile_len;
            sw[FRONT + p] = in ? w[j] : SENTINEL;
            nh += (in && w_type(w[j]) == TYPE_ROAD) ? 1u : 0u;
            nh += (in && w_type(w[j]) == TYPE_EVENT) ? 1u << 16 : 0u;
        }
        if (threadIdx.x < FRONT) {
            const int64_t k = (int64_t)tile_start - FRONT + threadIdx.x;
            sw[threadIdx.x] = k >= 0 ? __ldg(words + k) : SENTINEL;
        }
        if (threadIdx.x < BACK) {
            const uint64_t k = tile_end + threadIdx.x;
            sw[FRONT + TILE_WORDS + threadIdx.x] = k < n_words ? __ldg(words + k) : SENTINEL;
        }
        uint32_t n_heads_tile;
        // (no closing barrier: `red` is next written by the split-road scan,
        // several barriers later)
        const uint32_t ex = block_exclusive_scan<uint32_t, false>(nh, red, &n_heads_tile) & 0xFFFFu;
        const uint32_t n_roads_tile = n_heads_tile & 0xFFFFu;
        // the tile's road count for the tiles after it, before anything else
        if (threadIdx.x == 0)
            publish_tile(tile_state + t, t == 0 ? TILE_INCLUSIVE : TILE_AGGREGATE, n_roads_tile);
        // per-word rules V3..V7 and V9 against the word before (the staged
        // front halo holds the previous tile's last word; tile 0 has none).
        // A branch-free filter first: a word is suspect when it is of the
        // reserved type, a road header of a sector past n_sectors, or a hit
        // with reserved bits, a layer above 5, an event header before it, or a
        // hit of a higher layer before it.  Only warps with a suspect word run
        // the rules one by one (which report the exact status keys).
        // Word types by value: hit < 2^30 <= reserved < 2^31 <= road < 3 2^30
        // <= event header; a valid hit is below layer 6 (x < 6 2^27) with no
        // reserved bit; the word before comes from registers (the first one
        // from the staged front halo).
        const uint32_t n_in = (uint32_t)max(0, min(TILE_PER_THREAD,
                                                   tile_len - (int)threadIdx.x * TILE_PER_THREAD));
        uint32_t suspect = 0;
        {
            uint32_t pw = sw[FRONT + threadIdx.x * TILE_PER_THREAD - 1];
#pragma unroll
            for (int j = 0; j < TILE_PER_THREAD; ++j) {
                const uint32_t x = w[j];
                const uint32_t hit_bad = (x >= (6u << 27)) | ((x & 0x07FF8000u) != 0u) |
                                         (pw >= (3u << 30)) |
                                         ((pw < (1u << 30)) & ((pw >> 27) > (x >> 27)));
                const uint32_t bad = x < (1u << 30)   ? hit_bad
                                     : x < (2u << 30) ? 1u
                                     : x < (3u << 30) ? (uint32_t)(rd_sector(x) >= cfg.n_sectors)
                                                      : 0u;
                suspect |= ((uint32_t)j < n_in ? bad : 0u);
                pw = x;
            }
        }
        if (__any_sync(0xffffffffu, suspect != 0u)) {
#pragma unroll
            for (int j = 0; j < TILE_PER_THREAD; ++j) {
                const int p = threadIdx.x * TILE_PER_THREAD + j;
                if (p >= tile_len) break;
                const uint64_t i = tile_start + p;
                const uint32_t x = w[j], pw = sw[FRONT + p - 1];
                const uint32_t ty = w_type(x);
                if (ty == TYPE_ROAD) {
                    if (rd_sector(x) >= cfg.n_sectors) report(status, i, SVT_ERR_BAD_SECTOR);   // V9
                } else if (ty == TYPE_BAD) {
                    report(status, i, SVT_ERR_BAD_TYPE);                                      // V3
                } else if (ty == TYPE_HIT) {
                    // V4 and V7 also fire on an event's first word, where V1 already
                    // reports the same word with the smallest code, so the key is unchanged.
                    if (i > 0 && w_type(pw) == TYPE_EVENT) report(status, i, SVT_ERR_BAD_TYPE);  // V4
                    if (hit_reserved(x) != 0) report(status, i, SVT_ERR_BAD_RESERVED);          // V5
                    if (hit_layer(x) > 5) report(status, i, SVT_ERR_BAD_LAYER);                 // V6
                    if (i > 0 && w_type(pw) == TYPE_HIT && hit_layer(pw) > hit_layer(x))
                        report(status, i, SVT_ERR_UNSORTED);                                    // V7
                }
            }
        }
        // V1: the events starting in this tile start with an event header
        // (their first words are staged; the outcome is read after the next
        // barrier)
        for (uint64_t e = e_lo + threadIdx.x; e < e_hi; e += TILE_THREADS) {
            const uint64_t s0 = e == e_lo + threadIdx.x ? s0_first : __ldg(event_off + e);
            if (s0 >= tile_start && s0 < tile_end &&
                w_type(sw[FRONT + (int)(s0 - tile_start)]) != TYPE_EVENT) {
                report(status, s0, SVT_ERR_BAD_TYPE);                                   // V1
                v1_flag = 1;
            }
        }
        // road headers: positions; counters cleared (a loop over the set bits
        // of this thread's header mask: headers are about one word in 18)
        {
            uint32_t hm = 0;
#pragma unroll
            for (int j = 0; j < TILE_PER_THREAD; ++j)
                hm |= (threadIdx.x * TILE_PER_THREAD + j < tile_len && w_type(w[j]) == TYPE_ROAD)
                          ? 1u << j : 0u;
            uint32_t r = ex;
            while (hm) {
                const int j = __ffs(hm) - 1;
                hm &= hm - 1;
                hdr_pos[r] = (uint16_t)(threadIdx.x * TILE_PER_THREAD + j);
                cnt[r] = 0u;
                cnt45[r] = 0u;
                r += 1;
            }
        }
        __syncthreads();
        // V2: every event-header word must sit at an event offset.  When the
        // tile holds as many headers as events start in it and all of those
        // start with a header (V1), the headers are exactly those starts;
        // otherwise every header of the tile is looked up.
        if ((n_heads_tile >> 16) != e_hi - e_lo || v1_flag) {   // (rare: the batch is invalid)
            const int lane = threadIdx.x & 31;
            for (int j = 0; j < TILE_PER_THREAD; ++j) {
                const bool ev = base + j < n_words && w_type(w[j]) == TYPE_EVENT;
                uint32_t bal = __ballot_sync(0xffffffffu, ev);
                while (bal) {
                    const int src = __ffs(bal) - 1;
                    const uint64_t i = __shfl_sync(0xffffffffu, base + j, src);
                    const uint64_t e = warp_lower_bound64(event_off, n_events, i, lane);
                    const bool start = e < n_events && __ldg(event_off + e) == i;
                    if (lane == src && !start) report(status, i, SVT_ERR_BAD_TYPE);
                    bal &= bal - 1;
                }
            }
        }
        // hits: count into their road (one shared atomic per run of the
        // thread's words that belongs to one road), note the tile's last
        // non-hit word, and mark "same layer as the word before" for V8
        {
            int r = (int)ex - 1;   // local road of the latest header before this thread's words
            int my_last_nonhit = -1;
            uint32_t acc = 0;      // hits of road r among this thread's words, 5 bits per layer
            uint32_t acc45 = 0;    // ... in cnt45's fields, within the road's run (pairing only)
            uint32_t same = 0;     // bit j: word j and the word before are hits of one layer
            uint32_t prev = sw[FRONT + threadIdx.x * TILE_PER_THREAD - 1];
            // pairing counts only hits inside a road's run (a road header and
            // the hits right after it): is this thread's first word inside
            // one, i.e. is the latest earlier non-hit word of the tile a road
            // header?  (Hits before the tile's first header are not counted:
            // the tile before takes them through its back halo.)
            bool in_run = true;
            if (cfg.xft_pairs) {
                int mine = -1;   // (position << 1) | is-road of this thread's last non-hit word
#pragma unroll
                for (int j = 0; j < TILE_PER_THREAD; ++j) {
                    const int p = threadIdx.x * TILE_PER_THREAD + j;
                    if (p < tile_len && w_type(w[j]) != TYPE_HIT)
                        mine = (p << 1) | (w_type(w[j]) == TYPE_ROAD ? 1 : 0);
                }
                const int before = block_exclusive_max(mine, redi);
                in_run = before >= 0 && (before & 1);
            }
            if (!cfg.xft_pairs) {
                // the same steps by word value (hit < 2^30, road in [2^31,
                // 3 2^30)), without the pairing counts
#pragma unroll
                for (int j = 0; j < TILE_PER_THREAD; ++j) {
                    const uint32_t x = w[j];
                    const bool in = (uint32_t)j < n_in;
                    const bool hit = in && x < (1u << 30);
                    // a hit whose predecessor has the same top five bits is a
                    // hit of the same layer
                    same |= (hit && ((prev ^ x) >> 27) == 0u) ? 1u << j : 0u;
                    prev = x;
                    if (in && x >= (2u << 30) && x < (3u << 30)) {
                        if (acc && r >= 0) atomicAdd(&cnt[r], acc);
                        acc = 0;
                        r += 1;
                    }
                    if (in && !hit) my_last_nonhit = (int)threadIdx.x * TILE_PER_THREAD + j;
                    acc += hit ? 1u << (5 * hit_layer(x)) : 0u;
                }
            } else {
#pragma unroll
                for (int j = 0; j < TILE_PER_THREAD; ++j) {
                    const int p = threadIdx.x * TILE_PER_THREAD + j;
                    const uint32_t x = w[j];
                    const bool in = p < tile_len;
                    const uint32_t ty = w_type(x);
                    if (in && ty == TYPE_HIT && w_type(prev) == TYPE_HIT && hit_layer(prev) == hit_layer(x))
                        same |= 1u << j;
                    prev = x;
                    if (!in) continue;
                    if (ty == TYPE_ROAD) {
                        if (acc && r >= 0) atomicAdd(&cnt[r], acc);
                        if (acc45 && r >= 0) atomicAdd(&cnt45[r], acc45);
                        acc = 0;
                        acc45 = 0;
                        r += 1;
                    }
                    if (ty != TYPE_HIT) {
                        my_last_nonhit = p;
                        in_run = ty == TYPE_ROAD;
                        continue;
                    }
                    acc += 1u << (5 * hit_layer(x));
                    if (in_run)
                        acc45 += (1u << 20) + (hit_layer(x) == 4 ? 1u : 0u) + (hit_layer(x) == 5 ? 1u << 10 : 0u);
                }
            }
            if (acc && r >= 0) atomicAdd(&cnt[r], acc);
            if (acc45 && r >= 0) atomicAdd(&cnt45[r], acc45);
            if (my_last_nonhit >= 0) atomicMax(&last_nonhit, my_last_nonhit);
            // same-layer bits of tile position q at bit q + 32 of the bitmap
            // (word 1 + q / 32); word 0 covers the front halo
            uint32_t v = same << (8 * (threadIdx.x & 3));
            v |= __shfl_xor_sync(0xffffffffu, v, 1);
            v |= __shfl_xor_sync(0xffffffffu, v, 2);
            if ((threadIdx.x & 3) == 0) same_bits[1 + threadIdx.x / 4] = v;
            if (threadIdx.x < 32) {
                const int q = (int)threadIdx.x - 32;   // halo position, -32..-1 (-15..-1 used)
                const uint32_t a = q >= -15 ? sw[FRONT + q] : 0u, b = q >= -15 ? sw[FRONT + q - 1] : 0u;
                const bool s_ = q >= -15 && w_type(a) == TYPE_HIT && w_type(b) == TYPE_HIT &&
                                hit_layer(a) == hit_layer(b);
                const uint32_t h = __ballot_sync(0xffffffffu, s_);
                if (threadIdx.x == 0) same_bits[0] = h;
            }
        }
        __syncthreads();
        // V8: a hit whose 16 predecessors are hits of its layer is the 17th (or
        // later) of a run, i.e. 16 consecutive "same" bits end at it.  Thread
        // k - 1 (the first warp) looks at bitmap words k - 1 and k: bit i of X
        // is position 32 (k - 2) + i, and after the four steps bit s of y says
        // bits s .. s + 15 of X are set.
        static_assert(TILE_WORDS / 32 == 32, "one warp covers the bitmap's words");
        if (threadIdx.x < TILE_WORDS / 32) {
            const int k = threadIdx.x + 1;
            const unsigned long long X =
                (unsigned long long)same_bits[k - 1] | ((unsigned long long)same_bits[k] << 32);
            unsigned long long y = X & (X >> 1);
            y &= y >> 2;
            y &= y >> 4;
            y &= y >> 8;
            const unsigned long long m = y & (0xFFFFFFFFull << 17);   // runs ending in word k
            if (m) {
                const int s_ = __ffsll((long long)m) - 1;
                report(status, tile_start + (uint64_t)(32 * (k - 2) + s_ + 15),
                       SVT_ERR_TOO_MANY_HITS);
            }
        }
        // hits after the tile that continue the tile's last road
        if (n_roads_tile > 0 && last_nonhit == (int)hdr_pos[n_roads_tile - 1]) {
            const int r = (int)n_roads_tile - 1;
            if (threadIdx.x < 32) {
                // length of the run of hit words at the start of the back halo
                int run = 0;
                for (int c0 = 0; c0 < BACK; c0 += 32) {
                    const int h = c0 + threadIdx.x;
                    const bool hit = h < BACK && w_type(sw[FRONT + tile_len + h]) == TYPE_HIT &&
                                     tile_len + h < FRONT + TILE_WORDS + BACK - FRONT;
                    const uint32_t nb = __ballot_sync(0xffffffffu, !hit);
                    if (nb) {
                        run = c0 + __ffs(nb) - 1;
                        break;
                    }
                    run = c0 + 32;
                }
                run = min(run, BACK);
                for (int h = threadIdx.x; h < run; h += 32) {
                    const uint32_t l = hit_layer(sw[FRONT + tile_len + h]);
                    atomicAdd(&cnt[r], 1u << (5 * l));
                    if (cfg.xft_pairs)
                        atomicAdd(&cnt45[r], (1u << 20) + (l == 4 ? 1u : 0u) + (l == 5 ? 1u << 10 : 0u));
                }
            }
        }
        // the roads of the tiles before this one (the last warp, while the
        // first may still be counting the hits past the tile's end); then the
        // tile's inclusive count for the tiles after it
        if (threadIdx.x >= TILE_THREADS - 32) {
            const int lane = threadIdx.x & 31;
            const unsigned long long before = t ? tiles_before(tile_state, t, lane, status) : 0ull;
            if (lane == 0) {
                if (t) publish_tile(tile_state + t, TILE_INCLUSIVE, before + n_roads_tile);
                base_s = before;
                if (t + 1 == T) {   // the last tile: the batch's road count
                    const unsigned long long R = before + n_roads_tile;
                    if (R > 0xFFFFFFFFull) report(status, 0, SVT_ERR_OOM);
                    if (total64) *total64 = R;
                    if (event_road) event_road[n_events] = (uint32_t)R;
                }
            }
        }
        __syncthreads();
        const uint64_t tile_base = base_s;
        // one thread per road of the tile; for the fused path cnt[rl] then
        // holds the road's work items (0 unless it is split)
        uint32_t items_sum = 0, big_sum = 0;
        unsigned long long comb_sum = 0;
        for (uint32_t rl = threadIdx.x; rl < n_roads_tile; rl += TILE_THREADS) {
            const uint64_t r = tile_base + rl;
            const int p = hdr_pos[rl];
            if (cfg.xft_pairs) {
                // V11, at the last word of the road's run.  A run of more than 96
                // hits (or one that goes past the back halo) breaks V6, V7 or V8
                // at one of its own words, which is then the smaller key.
                const uint32_t v = cnt45[rl], run = v >> 20;
                if (run <= 96u && (v & 1023u) != ((v >> 10) & 1023u))
                    report(status, tile_start + p + run, SVT_ERR_XFT_UNPAIRED);
            }
            if (r >= road_cap) {
                report(status, tile_start + p, SVT_ERR_OOM);
                cnt[rl] = 0;
                continue;
            }
            const uint32_t packed = cnt[rl];
            if (road_word) road_word[r] = (uint32_t)(tile_start + p);
            if (road_nhit) road_nhit[r] = packed;
            if (fr.desc) {
                const RoadDesc d = make_road_desc((uint32_t)(tile_start + p), packed, sw[FRONT + p], cfg);
                const uint32_t it = road_big_items(d, fr);
                fr.desc[r] = d;
                cnt[rl] = it;
                items_sum += it;
                big_sum += it ? 1u : 0u;
                comb_sum += d.a.w;
            }
        }
        // first road of every event that starts inside this tile: the number
        // of road headers before the event's first word
        for (uint64_t e = e_lo + threadIdx.x; e < e_hi; e += TILE_THREADS) {
            const uint64_t s0 = __ldg(event_off + e);
            if (s0 >= tile_start && s0 < tile_end) {
                // roads of the tile whose header lies before s0 (hdr_pos is increasing)
                const int ps = (int)(s0 - tile_start);
                uint32_t lo = 0, hi = n_roads_tile;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if ((int)hdr_pos[mid] < ps) lo = mid + 1; else hi = mid;
                }
                event_road[e] = (uint32_t)(tile_base + lo);
            }
        }
        if (fr.desc) {
            // this thread's split roads go to slots [base + big_ex, ...) with
            // items from [base_items + it_ex, ...), in the order it visited them
            // (most tiles hold no split road and skip both scans); the tile's
            // evaluated combinations are summed per warp into tile_comb, which
            // the barrier of __syncthreads_or orders before thread 0 reads it
            unsigned long long cw = comb_sum;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) cw += __shfl_xor_sync(0xffffffffu, cw, d);
            if ((threadIdx.x & 31) == 0 && cw) atomicAdd(&tile_comb, cw);
            uint32_t it_total = 0, big_total = 0, it_ex = 0, big_ex = 0;
            if (__syncthreads_or(big_sum != 0)) {
                // items and roads in one scan ((items << 32) | roads); its
                // shared entries are read before the barrier below
                unsigned long long tot64;
                const unsigned long long ex64 = block_exclusive_scan<unsigned long long, false>(
                    ((unsigned long long)items_sum << 32) | big_sum, red64, &tot64);
                it_ex = (uint32_t)(ex64 >> 32);
                big_ex = (uint32_t)ex64;
                it_total = (uint32_t)(tot64 >> 32);
                big_total = (uint32_t)tot64;
            }
            if (threadIdx.x == 0) {
                const unsigned long long c_total = tile_comb;
                tile_comb = 0;   // the next tile adds to it only after further barriers
                unsigned long long b = 0;
                if (big_total) {
                    b = atomicAdd(fr.bl.reserve,
                                  ((unsigned long long)it_total << 32) | big_total);
                    if ((b >> 32) + it_total > 0xFFFFFFFFull)
                        report(status, tile_start, SVT_ERR_OOM);   // item count needs 32 bits
                }
                big_base = b;
                if (counts && c_total) atomicAdd((unsigned long long *)(counts + 2), c_total);
            }
            __syncthreads();
            if (big_sum) {
                const uint32_t slot0 = (uint32_t)big_base, item0 = (uint32_t)(big_base >> 32);
                for (uint32_t rl = threadIdx.x; rl < n_roads_tile; rl += TILE_THREADS) {
                    const uint32_t it = cnt[rl];
                    if (!it) continue;
                    const uint32_t j = slot0 + big_ex;   // < R <= road_cap
                    fr.bl.road[j] = (uint32_t)(tile_base + rl);
                    fr.bl.item_off[j] = item0 + it_ex;
                    fr.key[tile_base + rl] = ~0ull;
                    fr.bl.pending[j] = it;
                    big_ex += 1;
                    it_ex += it;
                }
            }
        }
        if (threadIdx.x == 0) tile_s = atomicAdd(tile_ticket, 1u);   // every thread has read t
        __syncthreads();
    }
    // an empty batch has no last tile to write the road count of
    if (T == 0 && blockIdx.x == 0 && threadIdx.x == 0 && event_road) event_road[n_events] = 0;
}

__global__ void k_unpack_events(const uint32_t *__restrict__ words,
                                const uint64_t *__restrict__ event_off,
                                const Dims *__restrict__ dims,
                                const uint32_t *__restrict__ event_road,
                                unsigned long long *status) {
    wait_prior_grid();
    allow_next_grid();
    check_events(words, event_off, dims->n_words, dims->n_events, event_road, status,
                 (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (uint64_t)gridDim.x * blockDim.x);
}

}  // namespace

void launch_prologue(Dims *dims, uint64_t n_words, uint64_t n_events, const uint64_t *sizes,
                     const uint64_t *event_off, uint32_t *first_ev, unsigned long long *status,
                     uint64_t *counts, int n_counts, uint64_t *zero, int n_zero,
                     unsigned long long *tile_state, uint32_t *tile_ticket, int grid,
                     cudaStream_t st) {
    uint64_t g = first_ev ? (n_events + 1 + 255) / 256 : 1;
    const uint64_t gt = tile_state ? (n_tiles(n_words) + 255) / 256 : 1;
    if (gt > g) g = gt;
    if (g > (uint64_t)grid) g = (uint64_t)grid;
    if (g < 1) g = 1;
    k_prologue<<<(int)g, 256, 0, st>>>(dims, n_words, n_events, sizes, event_off, first_ev, status,
                                       counts, n_counts, zero, n_zero, tile_state, tile_ticket);
}

void launch_unpack_roads(const uint32_t *words, const uint64_t *event_off, const Dims *dims,
                         const uint32_t *first_ev, uint64_t max_words,
                         unsigned long long *tile_state, uint32_t *tile_ticket, uint64_t *total64,
                         uint64_t road_cap, uint32_t *road_word, uint32_t *road_nhit,
                         uint32_t *event_road, const svt_config cfg, const FusedRoads fr,
                         uint64_t *counts, unsigned long long *status, int grid, cudaStream_t st) {
    uint64_t T = n_tiles(max_words);
    int g = (int)(T < (uint64_t)grid ? T : (uint64_t)grid);
    if (g < 1) g = 1;   // an empty batch still writes its road count
    launch_after(k_unpack_roads, g, TILE_THREADS, 0, st, words, event_off, dims, first_ev,
                 tile_state, tile_ticket, total64, road_cap, road_word, road_nhit, event_road, cfg,
                 fr, counts, status);
}

void launch_unpack_events(const uint32_t *words, const uint64_t *event_off, const Dims *dims,
                          uint64_t max_events, const uint32_t *event_road,
                          unsigned long long *status, int grid, cudaStream_t st) {
    uint64_t blocks = (max_events + 255) / 256;
    if (blocks < 1) blocks = 1;
    int g = (int)(blocks < (uint64_t)grid ? blocks : (uint64_t)grid);
    launch_after(k_unpack_events, g, 256, 0, st, words, event_off, dims, event_road, status);
}

}  // namespace svt
