// svt_fused.cu -- combine + fit + chi-square cut + best-per-road + format of
// the paper's Sec. 2 / Sec. 2.1 in one persistent kernel.
//
// Design (GB300 first; the paper's Kepler port used one thread per
// combination and a separate kernel per stage):
//   * The fit is linear, so with the layers split into a prefix (rows, index
//     a) and a suffix (columns, index b) every accumulator is
//         acc_k(a, b) = A_k(a) + B_k(b),
//     A_k(a) = q_k 2^qshift + sum_{prefix l} F_kl x_l,  B_k(b) = sum_{suffix l} F_kl x_l,
//     exactly in int64.  A warp builds the per-hit terms F_kl x_l and up to 64
//     A rows in shared memory; each lane holds the B of one column in
//     registers.  One combination then costs three 64-bit adds, three funnel
//     shifts, the clamp, three multiply-adds and one compare.  Only the three
//     chi rows are evaluated in the loop; the parameters are recomputed once
//     for the winning combination.
//   * Work: roads with more than small_max evaluated combinations are split
//     into items of `rows` rows and handled first (items taken from an atomic
//     counter; the road of an item is found by a 32-way warp search of the
//     short list of split roads).  Then warps take chunks of consecutive
//     roads (one coalesced load of their 16-byte descriptors) and fit every
//     remaining road whole, one warp per road.
//   * Each lane visits its combinations in increasing c within a column (or
//     within its block of rows of a column), so a strict '<' keeps the
//     smallest index among equal chi2; across columns, row blocks, lanes and
//     items the (chi2, c) pairs are merged as 64-bit keys (warp
//     shuffles; atomicMin on the road's slot for split roads, whose record is
//     written by the warp that retires the road's last item).
#include "svt_kernels.cuh"

namespace svt {

namespace {

constexpr int ROWS_MAX = 64;

// All accumulator terms are kept multiplied by 2^(32 - oshift): the high word
// of a 64-bit sum of such terms is then exactly floor(sum / 2^oshift).
struct WarpSmem {
    longlong2 T[N_LAYERS * MAX_HITS][2];  // chi-row terms F[3+k][l] * x * 2^(32-oshift) of hit i of
                                          // layer l at [l*16+i]: (k=3, k=4), (k=5, -); 32-byte entries
                                          // so a lookup is one 16-byte and one 8-byte load
    longlong2 S01[32];                    // suffix sums below the top suffix layer, rows 3, 4 [b']
    long long S5[32];                     // ... row 5
    longlong2 A01[ROWS_MAX];              // prefix sums incl. q, rows 3, 4, per row of the chunk
    long long A5[ROWS_MAX];               // ... row 5
    uint32_t x[N_LAYERS * MAX_HITS];      // hit coordinates [l][i] (x = 0 for an empty layer)
    int32_t F[36];                        // F[s][m][k][l] at k*6+l
    int32_t q[6];
    uint32_t n[N_LAYERS];                 // n'_l = max(n_l, 1)
    uint32_t m[N_LAYERS];                 // division magic of n'_l
    uint32_t off[N_LAYERS];               // index of the first hit of layer l in the road
};

// largest j in [0, n) with off[j] <= it (off non-decreasing, off[0] = 0)
__device__ __forceinline__ uint32_t find_slot(const uint32_t *__restrict__ off, uint32_t n,
                                              uint32_t it, int lane) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t p = lo + (uint32_t)lane * step;
        const bool le = (p < hi) && (__ldg(off + p) <= it);
        const uint32_t bal = __ballot_sync(0xffffffffu, le);
        const uint32_t L = 31 - __clz(bal);
        lo = lo + L * step;
        hi = min(lo + step, hi);
    }
    return lo;
}

// Smallest 64-bit key over the warp: the smallest high word, then the
// smallest low word among the lanes that hold it.
__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
    const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
    const uint32_t m_hi = __reduce_min_sync(0xffffffffu, hi);
    const uint32_t m_lo = __reduce_min_sync(0xffffffffu, hi == m_hi ? lo : 0xFFFFFFFFu);
    return ((unsigned long long)m_hi << 32) | m_lo;
}

__device__ __forceinline__ int32_t clamp_chi(int32_t y) { return max(min(y, 32767), -32767); }


// Road geometry unpacked from its descriptor (warp-uniform values).
struct Geo {
    uint32_t split, NBp, NB, NA, C_eval, mask, total_hits;
};
__device__ __forceinline__ Geo geo_of(const RoadDesc &D) {
    Geo g;
    const uint32_t w = D.b.x;
    g.split = w & 7u;
    g.NBp = (w >> 3) & 31u;
    g.mask = (w >> 13) & 63u;
    g.total_hits = (w >> 19) & 127u;
    g.NB = D.b.y;
    g.NA = D.b.z;
    g.C_eval = D.a.w;
    return g;
}

// Constants, hit coordinates, per-hit chi terms and the suffix table of road D
// in the warp's slot.  Global loads are issued before any shared-memory work.
__device__ __forceinline__ void road_setup(WarpSmem &sm, const uint32_t *__restrict__ words,
                                           const RoadDesc &D, const Geo &g,
                                           const int16_t *__restrict__ F,
                                           const int16_t *__restrict__ q, uint32_t sh,
                                           uint32_t xft, long long bias, int lane) {
    const uint32_t rw = D.a.x, packed = D.a.y;
    const size_t cs = (size_t)rd_sector(D.a.z) * 64 + g.mask;
    const int32_t f0 = __ldg(F + cs * 36 + lane);
    int32_t f1 = 0;
    if (lane < 4) f1 = __ldg(F + cs * 36 + 32 + lane);
    else if (lane < 10) f1 = __ldg(q + cs * 6 + (lane - 4));
    uint32_t hv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const uint32_t h = (uint32_t)lane + 32u * j;
        hv[j] = h < g.total_hits ? __ldg(words + rw + 1 + h) : 0u;
    }
    sm.F[lane] = f0;
    if (lane < 4) sm.F[32 + lane] = f1;
    else if (lane < 10) sm.q[lane - 4] = f1;
    const uint32_t nl = lane < N_LAYERS ? nhit_of(packed, lane) : 0u;
    uint32_t incl = nl;   // inclusive prefix of the layer counts
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane < N_LAYERS) {
        // with track-trigger pairs layer 5 is no digit of its own (radix 1)
        const uint32_t np = (nl && !(xft && lane == N_LAYERS - 1)) ? nl : 1u;
        sm.n[lane] = np;
        sm.m[lane] = kDivMagic[np];
        sm.off[lane] = incl - nl;
        if (nl == 0) {   // a layer without hits contributes x = 0
            sm.x[lane * MAX_HITS] = 0;
            sm.T[lane * MAX_HITS][0] = make_longlong2(0, 0);
            sm.T[lane * MAX_HITS][1].x = 0;
        }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const uint32_t h = (uint32_t)lane + 32u * j;
        if (h < g.total_hits) {
            const uint32_t l = hit_layer(hv[j]);
            const uint32_t i = h - sm.off[l];   // hits are sorted by layer (validated)
            const uint32_t xc = hit_coord(hv[j]);
            sm.x[l * MAX_HITS + i] = xc;
            longlong2 *t = sm.T[l * MAX_HITS + i];
            t[0] = make_longlong2((long long)(sm.F[18 + l] * (int32_t)xc) << sh,
                                  (long long)(sm.F[24 + l] * (int32_t)xc) << sh);
            t[1].x = (long long)(sm.F[30 + l] * (int32_t)xc) << sh;
        }
    }
    __syncwarp();
    if (xft) {
        // pair i: layer 4's entry i carries both coordinates of track-trigger
        // track i (equal counts are validated); layer 5 then adds nothing
        const uint32_t n4 = nhit_of(packed, 4);
        if ((uint32_t)lane < n4) {
            longlong2 *t4 = sm.T[4 * MAX_HITS + lane];
            const longlong2 *t5 = sm.T[5 * MAX_HITS + lane];
            t4[0].x += t5[0].x;
            t4[0].y += t5[0].y;
            t4[1].x += t5[1].x;
        }
        __syncwarp();
        if (lane == 0) {
            sm.T[5 * MAX_HITS][0] = make_longlong2(0, 0);
            sm.T[5 * MAX_HITS][1].x = 0;
        }
    }
    __syncwarp();
    // S[b'] = bias + sum over the suffix layers below the top one, b' < NBp (< 32)
    if ((uint32_t)lane < g.NBp) {
        uint32_t rem = lane;
        long long S3 = bias, S4 = bias, S5 = bias;
#pragma unroll
        for (int l = N_LAYERS - 1; l >= 1; --l) {
            if ((uint32_t)l > g.split) {
                const uint32_t nl = sm.n[l];
                const uint32_t qd = div_by(rem, nl, sm.m[l]);
                const uint32_t i = rem - qd * nl;
                rem = qd;
                const longlong2 t01 = sm.T[l * MAX_HITS + i][0];
                S3 += t01.x;
                S4 += t01.y;
                S5 += sm.T[l * MAX_HITS + i][1].x;
            }
        }
        sm.S01[lane] = make_longlong2(S3, S4);
        sm.S5[lane] = S5;
    }
    __syncwarp();
}

__device__ __forceinline__ void build_row(WarpSmem &sm, uint32_t split, uint32_t a,
                                          uint32_t slot, uint32_t qsh) {
    uint32_t rem = a;
    long long A3 = (long long)sm.q[3] << qsh;
    long long A4 = (long long)sm.q[4] << qsh;
    long long A5 = (long long)sm.q[5] << qsh;
#pragma unroll
    for (int l = N_LAYERS - 1; l >= 0; --l) {
        if ((uint32_t)l < split) {
            const uint32_t nl = sm.n[l];
            const uint32_t qd = div_by(rem, nl, sm.m[l]);
            const uint32_t i = rem - qd * nl;
            rem = qd;
            const longlong2 t01 = sm.T[l * MAX_HITS + i][0];
            A3 += t01.x;
            A4 += t01.y;
            A5 += sm.T[l * MAX_HITS + i][1].x;
        }
    }
    sm.A01[slot] = make_longlong2(A3, A4);
    sm.A5[slot] = A5;
}

__device__ __forceinline__ int32_t hi_word(long long v) {
    return (int32_t)((unsigned long long)v >> 32);
}

// Bias carried by the column terms (in the suffix table): with GUARDED the
// high word of a sum is g_k = y_k + 32768 (mod 2^32) instead of y_k.
template <bool GUARDED>
constexpr long long kColBias = GUARDED ? (32768LL << 32) : 0LL;

// Best key over rows [a_lo, a_hi) of the road, reduced over the warp.  The key
// is (chi2 << 32) | (row << 9) | column; since columns < NB < 512 its low word
// orders exactly like the combination index c = row * NB + column.
// Each lane takes one column and runs down the rows of the chunk; in the last
// pass over the columns, when only w < 32 of them are left, the lanes form
// floor(32 / w) groups of w and each group takes one block of the rows.
// GUARDED (valid when chi2_cut < 32767^2): a combination with a chi component
// of magnitude 32767 or more cannot pass, clamped or not.  One range test keeps
// only combinations with -32768 <= y_k <= 32767 for all three components; for
// those the sum of the squares is below 3 * 2^30 < 2^32 and is formed exactly
// in 32 bits, and the clamp changes no square that could still pass.
// Pass/fail, chi2 of passing combinations and the argmin are unchanged.
template <bool GUARDED>
__device__ __forceinline__ unsigned long long eval_rows(WarpSmem &sm, const Geo &g, uint32_t a_lo,
                                                        uint32_t a_hi, uint32_t qsh,
                                                        uint32_t init_chi, int lane) {
    unsigned long long best = ~0ull;
    const uint32_t NB = g.NB, NA = g.NA, C_eval = g.C_eval, NBp = g.NBp, top = g.split;
    const uint32_t mp = kDivMagic[NBp];
    for (uint32_t ac = a_lo; ac < a_hi; ac += ROWS_MAX) {
        const uint32_t ae = min(ac + (uint32_t)ROWS_MAX, a_hi), rows = ae - ac;
#pragma unroll
        for (uint32_t r0 = 0; r0 < (uint32_t)ROWS_MAX; r0 += 32)
            if (r0 + lane < rows) build_row(sm, top, ac + r0 + lane, r0 + lane, qsh);
        __syncwarp();
        for (uint32_t b0 = 0; b0 < NB; b0 += 32) {
            uint32_t b = b0 + (uint32_t)lane, lo = ac, hi = ae;
            if (NB - b0 < 32u) {   // warp-uniform: the last, partial pass
                const uint32_t w = NB - b0, mw = kDivMagic[w];
                const uint32_t grp = div_by((uint32_t)lane, w, mw), n_grp = div_by(32u, w, mw);
                const uint32_t len = div_by(rows + n_grp - 1u, n_grp, kDivMagic[n_grp]);
                b -= grp * w;
                lo = min(ac + grp * len, ae);   // groups past the last row get none
                hi = min(lo + len, ae);
            }
            // column b = is * NBp + bp: hit `is` of the top suffix layer and
            // entry bp of the suffix table
            const uint32_t is = div_by(b, NBp, mp), bp = b - is * NBp;
            const longlong2 t01 = sm.T[top * MAX_HITS + is][0];
            const long long t5 = sm.T[top * MAX_HITS + is][1].x;
            const longlong2 s01 = sm.S01[bp];
            const long long s5 = sm.S5[bp];
            const long long B3 = t01.x + s01.x, B4 = t01.y + s01.y, B5 = t5 + s5;
            if (hi == NA && lo < hi && (NA - 1) * NB + b >= C_eval) hi -= 1;
            uint32_t bchi = init_chi, ba = 0;
#pragma unroll 4
            for (uint32_t a = lo; a < hi; ++a) {
                const longlong2 v01 = sm.A01[a - ac];
                const long long v5 = sm.A5[a - ac];
                const int32_t y3 = hi_word(v01.x + B3);
                const int32_t y4 = hi_word(v01.y + B4);
                const int32_t y5 = hi_word(v5 + B5);
                if (GUARDED) {
                    const uint32_t g3 = (uint32_t)y3, g4 = (uint32_t)y4, g5 = (uint32_t)y5;
                    // g_k < 2^16 for all three <=> -32768 <= y_k <= 32767; then
                    // sum (g_k - 32768)^2 = sum g_k^2 - 2^16 sum g_k + 3 * 2^30
                    // holds exactly in 32-bit arithmetic
                    const uint32_t range = g3 | g4 | g5;
                    const uint32_t chi2 = g3 * g3 + g4 * g4 + g5 * g5 + (3u << 30) -
                                          ((g3 + g4 + g5) << 16);
                    if (range < 65536u && chi2 < bchi) {
                        bchi = chi2;
                        ba = a;
                    }
                } else {
                    const int32_t c3 = clamp_chi(y3), c4 = clamp_chi(y4), c5 = clamp_chi(y5);
                    const uint32_t chi2 = (uint32_t)(c3 * c3) + (uint32_t)(c4 * c4) + (uint32_t)(c5 * c5);
                    if (chi2 < bchi) {
                        bchi = chi2;
                        ba = a;
                    }
                }
            }
            if (bchi != init_chi) {
                const unsigned long long key = ((unsigned long long)bchi << 32) | (ba << 9) | b;
                best = key < best ? key : best;
            }
        }
        __syncwarp();
    }
    return warp_min64(best);
}

// Record of a road from its best key (all lanes call; lanes 0..2 recompute the
// parameters from the warp's slot, which still holds this road; lanes 0..5
// store one word each).  Returns whether the road passed.
__device__ __forceinline__ bool format_road(WarpSmem &sm, const RoadDesc &D, const Geo &g,
                                            const svt_config &cfg, unsigned long long best,
                                            uint32_t *o, int lane) {
    const uint32_t geo = D.b.x;
    const bool pass = best != ~0ull;
    uint32_t flags = 0;
    if (g.total_hits == 0) flags |= SVT_FLAG_NO_HITS;
    if (geo & (1u << 27)) flags |= SVT_FLAG_BAD_PATTERN;
    if (geo & (1u << 26)) flags |= SVT_FLAG_OVERFLOW;
    if (pass) flags |= SVT_FLAG_PASS;
    const uint32_t low = (uint32_t)best;
    const uint32_t row = low >> 9, col = low & 511u;
    // parameters of the best combination: lane 8k + l (k < 3, l < 6) forms
    // F[k][l] x_l, the groups of eight lanes sum them, lane 8k adds q_k
    int32_t p = 0;
    if (pass) {
        const uint32_t k = (uint32_t)lane >> 3, lk = (uint32_t)lane & 7u;
        uint32_t rem = col, i_own = 0;
#pragma unroll
        for (int l = N_LAYERS - 1; l >= 0; --l) {
            if ((uint32_t)l + 1u == g.split) rem = row;   // the prefix layers take the row
            const uint32_t nl = sm.n[l];
            const uint32_t qd = div_by(rem, nl, sm.m[l]);
            if ((uint32_t)l == (cfg.xft_pairs && lk == 5u ? 4u : lk)) i_own = rem - qd * nl;
            rem = qd;
        }
        long long t = 0;
        if (k < 3 && lk < (uint32_t)N_LAYERS)
            t = (long long)sm.F[k * 6 + lk] * (long long)sm.x[lk * MAX_HITS + i_own];
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        if (k < 3 && lk == 0) {
            const long long acc = (long long)sm.q[k] * (1ll << cfg.qshift) + t;
            p = (int32_t)(acc >> cfg.oshift);   // arithmetic shift: floor
        }
    }
    const int32_t pk = __shfl_sync(0xffffffffu, p, ((lane + 29) & 31) << 3);   // lane 3 + k gets p_k
    const uint32_t w = lane == 0   ? (rd_id(D.a.z) | (flags << 24))
                       : lane == 1 ? (pass ? row * g.NB + col : 0xFFFFFFFFu)
                       : lane == 2 ? (pass ? (uint32_t)(best >> 32) : 0u)
                                   : (uint32_t)pk;
    if (lane < 6) o[lane] = w;
    return pass;
}

// K4: persistent fit / cut / select / format
template <bool GUARDED>
__global__ void __launch_bounds__(512, 2)
    k_fit_persistent(const uint32_t *__restrict__ words, const uint64_t *__restrict__ event_off,
                     const Dims *__restrict__ dims, const uint32_t *__restrict__ event_road,
                     const RoadDesc *__restrict__ desc, uint64_t *counts, uint64_t road_cap,
                     const int16_t *__restrict__ F, const int16_t *__restrict__ q,
                     const svt_config cfg, const FusedRoads fr, uint32_t roads_per_chunk,
                     uint32_t *out, unsigned long long *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem &sm = reinterpret_cast<WarpSmem *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    wait_prior_grid();   // road extraction has completed (see launch_after)
    // per-event rules first, whatever the status, so that the key stays the
    // smallest over all rules
    check_events(words, event_off, dims->n_words, dims->n_events, event_road, status,
                 (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (uint64_t)gridDim.x * blockDim.x);
    const BigList &bl = fr.bl;
    const unsigned long long rv = *(volatile unsigned long long *)bl.reserve;
    const uint32_t n_big = (uint32_t)rv, n_items = (uint32_t)(rv >> 32);
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[1] = n_items;
    if (!status_ok(status)) return;
    const uint64_t R64 = counts[0];
    if (R64 > road_cap || R64 == 0) return;
    const uint32_t R = (uint32_t)R64;
    const uint32_t sh = 32u - cfg.oshift, qsh = cfg.qshift + sh;
    const uint32_t init_chi = cfg.chi2_cut == 0xFFFFFFFFu ? 0xFFFFFFFFu : cfg.chi2_cut + 1u;
    uint32_t n_pass = 0;   // passing roads formatted by this warp, added to counts[3] once

    // phase 1: items of split roads
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(bl.counters + 0, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const uint32_t j = find_slot(bl.item_off, n_big, it, lane);
        const uint32_t r = __ldg(bl.road + j);
        const uint32_t k = it - __ldg(bl.item_off + j);
        RoadDesc D;
        D.a = __ldg(&desc[r].a);
        D.b = __ldg(&desc[r].b);
        const Geo g = geo_of(D);
        road_setup(sm, words, D, g, F, q, sh, cfg.xft_pairs, kColBias<GUARDED>, lane);
        const uint32_t a_lo = k * fr.rows;
        const uint32_t a_hi = min(a_lo + fr.rows, g.NA);
        const unsigned long long best = eval_rows<GUARDED>(sm, g, a_lo, a_hi, qsh, init_chi, lane);
        uint32_t last = 0;
        if (lane == 0) {
            if (best != ~0ull) atomicMin(bl.best + j, best);
            __threadfence();
            last = (atomicSub(bl.pending + j, 1u) == 1u) ? 1u : 0u;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            const unsigned long long fb = __ldcg(bl.best + j);
            n_pass += format_road(sm, D, g, cfg, fb, out + (size_t)r * 6, lane) ? 1u : 0u;
        }
        __syncwarp();
    }

    // phase 2: chunks of consecutive roads, each fitted whole by this warp
    for (;;) {
        uint32_t c0 = 0;
        if (lane == 0) c0 = atomicAdd(bl.counters + 1, roads_per_chunk);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if (c0 >= R) break;
        const uint32_t n = min(roads_per_chunk, R - c0);
        uint4 da = make_uint4(0, 0, 0, 0), db = make_uint4(0, 0, 0, 0);
        if ((uint32_t)lane < n) {
            da = __ldg(&desc[c0 + lane].a);
            db = __ldg(&desc[c0 + lane].b);
        }
        for (uint32_t jj = 0; jj < n; ++jj) {
            RoadDesc D;
            D.a.x = __shfl_sync(0xffffffffu, da.x, jj);
            D.a.y = __shfl_sync(0xffffffffu, da.y, jj);
            D.a.z = __shfl_sync(0xffffffffu, da.z, jj);
            D.a.w = __shfl_sync(0xffffffffu, da.w, jj);
            D.b.x = __shfl_sync(0xffffffffu, db.x, jj);
            D.b.y = __shfl_sync(0xffffffffu, db.y, jj);
            D.b.z = __shfl_sync(0xffffffffu, db.z, jj);
            D.b.w = 0;
            if (D.a.w > fr.small_max) continue;   // split road: done in phase 1
            const Geo g = geo_of(D);
            unsigned long long best = ~0ull;
            if (g.C_eval > 0) {
                road_setup(sm, words, D, g, F, q, sh, cfg.xft_pairs, kColBias<GUARDED>, lane);
                best = eval_rows<GUARDED>(sm, g, 0, g.NA, qsh, init_chi, lane);
            }
            n_pass += format_road(sm, D, g, cfg, best, out + (size_t)(c0 + jj) * 6, lane) ? 1u : 0u;
            __syncwarp();
        }
    }
    if (lane == 0 && n_pass)
        atomicAdd((unsigned long long *)(counts + 3), (unsigned long long)n_pass);
}

}  // namespace

size_t fit_smem_bytes(int warps_per_block) { return sizeof(WarpSmem) * (size_t)warps_per_block; }

int fit_persistent_blocks_per_sm(int warps_per_block) {
    int n = 0, n2 = 0;
    size_t smem = fit_smem_bytes(warps_per_block);
    cudaFuncSetAttribute(k_fit_persistent<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_fit_persistent<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fit_persistent<true>, warps_per_block * 32,
                                                      smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k_fit_persistent<false>,
                                                      warps_per_block * 32, smem) != cudaSuccess)
        return 0;
    return n < n2 ? n : n2;
}

cudaError_t launch_fit_persistent(const uint32_t *words, const uint64_t *event_off,
                                  const Dims *dims, const uint32_t *event_road,
                                  const RoadDesc *desc, uint64_t *counts, uint64_t road_cap,
                                  const int16_t *F, const int16_t *q, const svt_config cfg,
                                  const FusedRoads fr, uint32_t roads_per_chunk,
                                  uint32_t *out, unsigned long long *status,
                                  int warps_per_block, int grid, cudaStream_t st) {
    size_t smem = fit_smem_bytes(warps_per_block);
    if (cfg.chi2_cut < 32767u * 32767u)
        launch_after(k_fit_persistent<true>, grid, warps_per_block * 32, smem, st, words,
                     event_off, dims, event_road, desc, counts, road_cap, F, q, cfg, fr,
                     roads_per_chunk, out, status);
    else
        launch_after(k_fit_persistent<false>, grid, warps_per_block * 32, smem, st, words,
                     event_off, dims, event_road, desc, counts, road_cap, F, q, cfg, fr,
                     roads_per_chunk, out, status);
    return cudaGetLastError();
}

}  // namespace svt
