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
//     registers.  One combination then costs three 64-bit adds, a 16-bit
//     range test, three multiply-adds and one compare-select (the high word
//     of each sum is y_k + 32768; see eval_rows).  Only the three chi rows are
//     evaluated in the loop; the parameters are formed once for the winning
//     combination.
//   * Work: roads with more than small_max evaluated combinations are split
//     into items of `rows` rows and handled first (items taken from an atomic
//     counter; the road of an item is found by a 32-way warp search of the
//     short list of split roads).  Then warps take chunks of consecutive
//     roads (one coalesced load of their 32-byte descriptors) and fit every
//     remaining road whole, one warp per road; with the grouped instances two
//     consecutive SMALL roads of the same geometry go to the two halves of a
//     warp instead, or four TINY ones to its four quarters, or every TINY road
//     of the chunk to a lane of its own (see lane_fit).
//   * Each lane visits its combinations in increasing c within a column (or
//     within its block of rows of a column), so a strict '<' keeps the
//     smallest index among equal chi2; across columns, row blocks, lanes and
//     items the (chi2, c) pairs are merged as 64-bit keys (warp
//     shuffles; atomicMin on the road's key for split roads, which the warp
//     that retires the road's last item takes over).
//   * A warp lists the roads it has finished with their keys and, 31 or 32
//     at a time, writes their records one road per lane: recovering the hits
//     of the best combination and forming its three parameters is scalar
//     work that would otherwise hold all 32 lanes for every road.
#include "svt_kernels.cuh"

namespace svt {

namespace {

constexpr int ROWS_MAX = 64;

// A road's working set in shared memory, for roads with at most MH hits on
// every layer, NS suffix-table entries and NR rows per chunk.  All
// accumulator terms are kept multiplied by 2^(32 - oshift): the high word of a
// 64-bit sum of such terms is then exactly floor(sum / 2^oshift).
template <int MH, int NS, int NR>
struct RoadSmem {
    longlong2 T[N_LAYERS * MH][2];  // chi-row terms F[3+k][l] * x * 2^(32-oshift) of hit i of
                                    // layer l at [l*MH+i]: (k=3, k=4), (k=5, -); 32-byte entries
                                    // so a lookup is one 16-byte and one 8-byte load
    longlong2 S01[NS];              // suffix sums below the top suffix layer, rows 3, 4 [b']
    long long S5[NS];               // ... row 5
    longlong2 A01[NR];              // prefix sums incl. q, rows 3, 4, per row of the chunk
    long long A5[NR];               // ... row 5
    uint32_t x[N_LAYERS * MH];      // hit coordinates [l][i] (x = 0 for an empty layer)
    int32_t F[36];                  // F[s][m][k][l] at k*6+l (chi rows k = 3..5 only)
    int32_t q[6];                   // ... q[s][m][k] (k = 3..5 only)
    uint32_t n[N_LAYERS];           // n'_l = max(n_l, 1)
    uint32_t m[N_LAYERS];           // division magic of n'_l
    uint32_t off[N_LAYERS];         // index of the first hit of layer l in the road
    static constexpr uint32_t kMH = MH, kNR = NR;
};
// one road per warp; or two roads marked SMALL, one per half warp, each in
// half of the same space; or four roads marked TINY, one per quarter warp,
// each in a quarter of it
using WarpSmem = RoadSmem<MAX_HITS, 32, ROWS_MAX>;
using HalfSmem = RoadSmem<8, 16, 16>;
using QuarterSmem = RoadSmem<2, 16, 8>;
static_assert(2 * sizeof(HalfSmem) <= sizeof(WarpSmem), "two half slots fit in a warp slot");
static_assert(4 * sizeof(QuarterSmem) <= sizeof(WarpSmem), "four quarter slots fit in a warp slot");
static_assert(sizeof(HalfSmem) % 16 == 0, "half slots keep 16-byte alignment");
static_assert(sizeof(QuarterSmem) % 16 == 0, "quarter slots keep 16-byte alignment");
static_assert(sizeof(WarpSmem) % 16 == 0, "warp slots keep 16-byte alignment");
static_assert(sizeof(WarpSmem) >= 32 * 6 * sizeof(uint32_t), "a road slot holds 32 records");

// A warp's slot when each lane fits a TINY road alone (lane_fit): the lane's
// column sums B_k(b), at most 8 columns, in column j of the tables.
struct LaneTables {
    longlong2 B01[8][32];   // B_3(b), B_4(b) of lane j at [b][j]
    long long B5[8][32];    // B_5(b)
};
constexpr size_t SLOT_BYTES =
    sizeof(WarpSmem) > sizeof(LaneTables) ? sizeof(WarpSmem) : sizeof(LaneTables);
static_assert(SLOT_BYTES % 16 == 0, "slots keep 16-byte alignment");

// Roads a warp has finished but whose records it has not yet written: when 31
// or 32 are listed (and when the warp runs out of work) each lane writes one
// (write_record), so the per-road tail costs a lane rather than a warp.
struct RecordList {
    unsigned long long key[32];   // best key (UINT64_MAX: none passed)
    uint32_t road[32];
};
constexpr uint32_t GEO_SMALL = 1u << 28, GEO_TINY = 1u << 29;

// The W lanes (the warp, or one half of it) that fit one road.  Every
// warp-synchronous step of the per-road code names only these lanes, so the
// two halves of a warp may run their roads' loops with different trip counts.
template <int W>
struct Lanes {
    uint32_t gl;     // lane within the group
    uint32_t mask;   // the group's lanes
};
template <int W>
__device__ __forceinline__ Lanes<W> lanes_of(int lane) {
    Lanes<W> L;
    L.gl = (uint32_t)lane & (uint32_t)(W - 1);
    L.mask = W == 32 ? 0xffffffffu
                     : (((1u << W) - 1u) << ((uint32_t)lane & (uint32_t)(32 - W)));
    return L;
}

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

// Smallest 64-bit key over the group: the smallest high word, then the
// smallest low word among the lanes that hold it.
template <int W>
__device__ __forceinline__ unsigned long long group_min64(unsigned long long v,
                                                          const Lanes<W> &L) {
    const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
    uint32_t m_hi, m_lo;
    if constexpr (W == 32) {
        m_hi = __reduce_min_sync(0xffffffffu, hi);
        m_lo = __reduce_min_sync(0xffffffffu, hi == m_hi ? lo : 0xFFFFFFFFu);
    } else {
        m_hi = hi;
#pragma unroll
        for (int d = W / 2; d >= 1; d >>= 1) m_hi = min(m_hi, __shfl_xor_sync(L.mask, m_hi, d, W));
        m_lo = hi == m_hi ? lo : 0xFFFFFFFFu;
#pragma unroll
        for (int d = W / 2; d >= 1; d >>= 1) m_lo = min(m_lo, __shfl_xor_sync(L.mask, m_lo, d, W));
    }
    return ((unsigned long long)m_hi << 32) | m_lo;
}

__device__ __forceinline__ int32_t clamp_chi(int32_t y) { return max(min(y, 32767), -32767); }


// Road geometry unpacked from its descriptor (uniform over the road's lanes).
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
// in the group's slot.  Global loads are issued before any shared-memory work.
// A road has at most 96 hits (at most 48 in a half slot: 8 per layer), so
// three passes of W = 32 lanes, or of W = 16 lanes over a SMALL road, hold
// them all.
template <int W, typename SM>
__device__ __forceinline__ void road_setup(SM &sm, const uint32_t *__restrict__ words,
                                           const RoadDesc &D, const Geo &g,
                                           const int16_t *__restrict__ F,
                                           const int16_t *__restrict__ q, uint32_t sh,
                                           uint32_t xft, long long bias, const Lanes<W> &L) {
    constexpr uint32_t MH = SM::kMH;
    // the chi rows k = 3..5 only (18 + 3 constants): the record's parameter
    // rows are read from global memory by the lane that forms it
    constexpr int NFQ = (21 + W - 1) / W;
    const uint32_t rw = D.a.x, packed = D.a.y, gl = L.gl;
    const size_t cs = (size_t)rd_sector(D.a.z) * 64 + g.mask;
    int32_t fv[NFQ];
#pragma unroll
    for (int j = 0; j < NFQ; ++j) {
        const uint32_t e = gl + (uint32_t)W * j;
        fv[j] = e < 18 ? __ldg(F + cs * 36 + 18 + e) : (e < 21 ? __ldg(q + cs * 6 + e - 15) : 0);
    }
    uint32_t hv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const uint32_t h = gl + (uint32_t)W * j;
        hv[j] = h < g.total_hits ? __ldg(words + rw + 1 + h) : 0u;
    }
#pragma unroll
    for (int j = 0; j < NFQ; ++j) {
        const uint32_t e = gl + (uint32_t)W * j;
        if (e < 18) sm.F[18 + e] = fv[j];
        else if (e < 21) sm.q[e - 15] = fv[j];
    }
    const uint32_t nl = gl < N_LAYERS ? nhit_of(packed, gl) : 0u;
    uint32_t incl = nl;   // inclusive prefix of the layer counts
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        const uint32_t v = __shfl_up_sync(L.mask, incl, d, W);
        if (gl >= (uint32_t)d) incl += v;
    }
    if (gl < N_LAYERS) {
        // with track-trigger pairs layer 5 is no digit of its own (radix 1)
        const uint32_t np = (nl && !(xft && gl == N_LAYERS - 1)) ? nl : 1u;
        sm.n[gl] = np;
        sm.m[gl] = kDivMagic[np];
        sm.off[gl] = incl - nl;
        if (nl == 0) {   // a layer without hits contributes x = 0
            sm.x[gl * MH] = 0;
            sm.T[gl * MH][0] = make_longlong2(0, 0);
            sm.T[gl * MH][1].x = 0;
        }
    }
    __syncwarp(L.mask);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const uint32_t h = gl + (uint32_t)W * j;
        if (h < g.total_hits) {
            const uint32_t l = hit_layer(hv[j]);
            const uint32_t i = h - sm.off[l];   // hits are sorted by layer (validated)
            const uint32_t xc = hit_coord(hv[j]);
            sm.x[l * MH + i] = xc;
            longlong2 *t = sm.T[l * MH + i];
            t[0] = make_longlong2((long long)(sm.F[18 + l] * (int32_t)xc) << sh,
                                  (long long)(sm.F[24 + l] * (int32_t)xc) << sh);
            t[1].x = (long long)(sm.F[30 + l] * (int32_t)xc) << sh;
        }
    }
    __syncwarp(L.mask);
    if (xft) {
        // pair i: layer 4's entry i carries both coordinates of track-trigger
        // track i (equal counts are validated); layer 5 then adds nothing
        const uint32_t n4 = nhit_of(packed, 4);
        if (gl < n4) {
            longlong2 *t4 = sm.T[4 * MH + gl];
            const longlong2 *t5 = sm.T[5 * MH + gl];
            t4[0].x += t5[0].x;
            t4[0].y += t5[0].y;
            t4[1].x += t5[1].x;
        }
        __syncwarp(L.mask);
        if (gl == 0) {
            sm.T[5 * MH][0] = make_longlong2(0, 0);
            sm.T[5 * MH][1].x = 0;
        }
    }
    __syncwarp(L.mask);
    // S[b'] = bias + sum over the suffix layers below the top one, b' < NBp
    // (< 32; <= 16 for a SMALL road)
    // (NBp <= W for whole and half warps; a quarter warp takes two passes)
    for (uint32_t bp = gl; bp < g.NBp; bp += (uint32_t)W) {
        uint32_t rem = bp;
        long long S3 = bias, S4 = bias, S5 = bias;
#pragma unroll
        for (int l = N_LAYERS - 1; l >= 1; --l) {
            if ((uint32_t)l > g.split) {
                const uint32_t nl = sm.n[l];
                const uint32_t qd = div_by(rem, nl, sm.m[l]);
                const uint32_t i = rem - qd * nl;
                rem = qd;
                const longlong2 t01 = sm.T[l * MH + i][0];
                S3 += t01.x;
                S4 += t01.y;
                S5 += sm.T[l * MH + i][1].x;
            }
        }
        sm.S01[bp] = make_longlong2(S3, S4);
        sm.S5[bp] = S5;
    }
    __syncwarp(L.mask);
}

template <typename SM>
__device__ __forceinline__ void build_row(SM &sm, uint32_t split, uint32_t a, uint32_t slot,
                                          uint32_t qsh) {
    constexpr uint32_t MH = SM::kMH;
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
            const longlong2 t01 = sm.T[l * MH + i][0];
            A3 += t01.x;
            A4 += t01.y;
            A5 += sm.T[l * MH + i][1].x;
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

// Best key over rows [a_lo, a_hi) of the road, reduced over the group.  The
// key is (chi2 << 32) | (row << 9) | column; since columns < NB < 512 its low
// word orders exactly like the combination index c = row * NB + column.
// Each lane takes one column and runs down the rows of the chunk; in the last
// pass over the columns, when only w < W of them are left, the lanes form
// floor(W / w) groups of w and each group takes one block of the rows.
// GUARDED (valid when chi2_cut < 32767^2): a combination with a chi component
// of magnitude 32767 or more cannot pass, clamped or not.  One range test keeps
// only combinations with -32768 <= y_k <= 32767 for all three components; for
// those the sum of the squares is below 3 * 2^30 < 2^32 and is formed exactly
// in 32 bits, and the clamp changes no square that could still pass.
// Pass/fail, chi2 of passing combinations and the argmin are unchanged.
template <bool GUARDED, int W, typename SM>
__device__ __forceinline__ unsigned long long eval_rows(SM &sm, const Geo &g, uint32_t a_lo,
                                                        uint32_t a_hi, uint32_t qsh,
                                                        uint32_t init_chi, const Lanes<W> &L) {
    constexpr uint32_t MH = SM::kMH, NR = SM::kNR;
    unsigned long long best = ~0ull;
    const uint32_t NB = g.NB, NA = g.NA, C_eval = g.C_eval, NBp = g.NBp, top = g.split;
    const uint32_t mp = kDivMagic[NBp], gl = L.gl;
    for (uint32_t ac = a_lo; ac < a_hi; ac += NR) {
        const uint32_t ae = min(ac + NR, a_hi), rows = ae - ac;
#pragma unroll
        for (uint32_t r0 = 0; r0 < NR; r0 += (uint32_t)W)
            if (r0 + gl < rows) build_row(sm, top, ac + r0 + gl, r0 + gl, qsh);
        __syncwarp(L.mask);
        for (uint32_t b0 = 0; b0 < NB; b0 += (uint32_t)W) {
            uint32_t b = b0 + gl, lo = ac, hi = ae;
            if (NB - b0 < (uint32_t)W) {   // uniform over the group: the last, partial pass
                const uint32_t w = NB - b0, mw = kDivMagic[w];
                const uint32_t grp = div_by(gl, w, mw), n_grp = div_by((uint32_t)W, w, mw);
                const uint32_t len = div_by(rows + n_grp - 1u, n_grp, kDivMagic[n_grp]);
                b -= grp * w;
                lo = min(ac + grp * len, ae);   // groups past the last row get none
                hi = min(lo + len, ae);
            }
            // column b = is * NBp + bp: hit `is` of the top suffix layer and
            // entry bp of the suffix table
            const uint32_t is = div_by(b, NBp, mp), bp = b - is * NBp;
            const longlong2 t01 = sm.T[top * MH + is][0];
            const long long t5 = sm.T[top * MH + is][1].x;
            const longlong2 s01 = sm.S01[bp];
            const long long s5 = sm.S5[bp];
            const long long B3 = t01.x + s01.x, B4 = t01.y + s01.y, B5 = t5 + s5;
            if (hi == NA && lo < hi && (NA - 1) * NB + b >= C_eval) hi -= 1;
            uint32_t bchi = init_chi, ba = 0;
            // whole warps run longer columns: 8 rows per step there took 2-5 %
            // off the fit; half warps (small roads) keep 4
#pragma unroll(W == 32 ? 8 : 4)
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
        __syncwarp(L.mask);
    }
    return group_min64<W>(best, L);
}

// Best key of one road fitted whole by a group of W lanes (set-up and all its
// rows), on every lane of the group; UINT64_MAX when no combination passed or
// the road has none to evaluate.
template <bool GUARDED, int W, typename SM>
__device__ __forceinline__ unsigned long long fit_road(SM &sm, const uint32_t *__restrict__ words,
                                                       const RoadDesc &D,
                                                       const int16_t *__restrict__ F,
                                                       const int16_t *__restrict__ q,
                                                       const svt_config &cfg, uint32_t sh,
                                                       uint32_t qsh, uint32_t init_chi,
                                                       const Lanes<W> &L) {
    const Geo g = geo_of(D);
    if (g.C_eval == 0) return ~0ull;
    road_setup<W>(sm, words, D, g, F, q, sh, cfg.xft_pairs, kColBias<GUARDED>, L);
    return eval_rows<GUARDED, W>(sm, g, 0, g.NA, qsh, init_chi, L);
}

// The split of a TINY road for a quarter warp: the shortest suffix of at
// least 8 columns (every layer has one or two hits, so it has exactly 8 when
// the road has 8 or more combinations), one column per lane in a single pass.
// The combination index c = row * NB + column is the same whatever the split,
// so the key is re-expressed in the descriptor's split afterwards (see
// quarter_key).
__device__ __forceinline__ void quarter_geometry(Geo &g, uint32_t packed, uint32_t xft) {
    const RoadShape s = road_shape(packed, xft);
    uint32_t nb = 1, top = 0, NB = (uint32_t)s.C, ntop = s.n[0];
    bool found = false;
#pragma unroll
    for (int l = N_LAYERS - 1; l >= 0; --l) {
        nb *= s.n[l];
        if (!found && nb >= 8u) {
            top = (uint32_t)l;
            NB = nb;
            ntop = s.n[l];
            found = true;
        }
    }
    g.split = top;
    g.NBp = NB / ntop;
    g.NB = NB;
    g.NA = g.C_eval ? (g.C_eval + NB - 1) / NB : 0u;
}

// A key of the quarter split, (chi2, row, column), in the descriptor's split.
__device__ __forceinline__ unsigned long long quarter_key(unsigned long long best,
                                                          uint32_t NB_quarter,
                                                          uint32_t NB_desc) {
    if (best == ~0ull) return best;
    const uint32_t low = (uint32_t)best;
    const uint32_t c = (low >> 9) * NB_quarter + (low & 511u);
    const uint32_t row = c / NB_desc;
    return (best & 0xFFFFFFFF00000000ull) | (row << 9) | (c - row * NB_desc);
}

__device__ __forceinline__ RoadDesc shfl_desc(const uint4 &da, const uint4 &db, uint32_t src) {
    RoadDesc D;
    D.a.x = __shfl_sync(0xffffffffu, da.x, src);
    D.a.y = __shfl_sync(0xffffffffu, da.y, src);
    D.a.z = __shfl_sync(0xffffffffu, da.z, src);
    D.a.w = __shfl_sync(0xffffffffu, da.w, src);
    D.b.x = __shfl_sync(0xffffffffu, db.x, src);
    D.b.y = __shfl_sync(0xffffffffu, db.y, src);
    D.b.z = __shfl_sync(0xffffffffu, db.z, src);
    D.b.w = 0;
    return D;
}

// One TINY road (at most two hits on every layer, so at most 64
// combinations) fitted by one lane, and its record formed there.  The prefix
// layers 0..2 index the rows a and the suffix layers 3..5 the columns b,
// c = a * NB3 + b: the same combination index as in any other split, so the
// lane visits the combinations in increasing c and a strict '<' keeps the
// smallest c among equal chi2.  Every layer has radix 1 or 2, so the digits
// of a row or a column are single bits, and a sum over the layers is the sum
// of the first hits' terms plus, for every digit that is set, the layer's
// difference between its second and its first hit.  The column sums (at most
// 8) go to the lane's column of the slot's tables; each row's sums are formed
// once in registers.  With track-trigger pairs layer 5 has radix 1 and its
// hits' terms are added to those of their layer-4 partners, as in
// road_setup.  With L > 1 lanes to a road (lanes sub = 0..L-1 of a group of
// L consecutive lanes) each lane takes the rows a = sub (mod L) and the group
// merges its (chi2, c) keys; every lane of the group builds the same column
// sums in its own column.  The record is the one form_record writes: flags,
// the best c and its chi2, and the three parameter rows (Eq. 1) of the best
// combination formed in int64 from its hits' coordinates, which the lanes
// still hold.
struct LaneRecord {
    uint32_t w[6];
    bool pass;
};
template <bool GUARDED>
__device__ __forceinline__ LaneRecord lane_fit(LaneTables &tb, const uint32_t *__restrict__ words,
                                               const uint4 &da, const uint4 &db,
                                               const int16_t *__restrict__ F,
                                               const int16_t *__restrict__ q,
                                               const svt_config &cfg, uint32_t sh, uint32_t qsh,
                                               uint32_t init_chi, int lane, uint32_t L,
                                               uint32_t group_mask) {
    const uint32_t C_eval = da.w, packed = da.y, geo = db.x, xft = cfg.xft_pairs;
    const size_t cs = (size_t)rd_sector(da.z) * 64 + ((geo >> 13) & 63u);
    // The chi rows k = 3..5 of F as pairs of int16 (F[k][l], F[k][l+1]) for
    // even l (row k starts at element (cs * 36 + 6 k), an even index, so each
    // pair is 4-byte aligned), the pairs (q_2, q_3), (q_4, q_5); two hit words per
    // layer (the second repeats the first when the layer has one hit; a layer
    // without hits reads the road's header word and takes x = 0).  Every load
    // is issued before any is used.
    const uint32_t *F32 = reinterpret_cast<const uint32_t *>(F + cs * 36);
    const uint32_t *q32 = reinterpret_cast<const uint32_t *>(q + cs * 6);
    uint32_t fp[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) fp[j] = __ldg(F32 + 9 + j);
    const uint32_t q23 = __ldg(q32 + 1), q45 = __ldg(q32 + 2);
    uint32_t hw[N_LAYERS][2];
    {
        uint32_t off = da.x + 1;   // first hit word of layer l (hits are sorted by layer)
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l) {
            const uint32_t nl = nhit_of(packed, l);
            const uint32_t p0 = nl ? off : da.x;
            hw[l][0] = __ldg(words + p0);
            hw[l][1] = __ldg(words + (nl > 1u ? off + 1u : p0));
            off += nl;
        }
    }
    // the int16 at index j of a run of pairs (little-endian: the even element
    // in the low half)
    auto lo16 = [](uint32_t v) { return (int32_t)(int16_t)(v & 0xFFFFu); };
    auto hi16 = [](uint32_t v) { return (int32_t)v >> 16; };
    auto f_of = [&](int k, int l) -> int32_t {   // F[3 + k][l]
        const uint32_t v = fp[(k * 6 + l) >> 1];
        return (l & 1) ? hi16(v) : lo16(v);
    };
    // Every term is multiplied by P = 2^(32 - oshift) on its way into a 64-bit
    // sum (one wide multiply-add).  A0 and B0 hold the first hits' terms (with
    // q and the column bias); dA and dB the per-layer differences between a
    // layer's second and first hit, F (x1 - x0), which fit in 32 bits.
    const int32_t P = (int32_t)(1u << sh);
    long long A0[3], B0[3];
    int32_t dA[3][3], dB[3][3];
    uint32_t beta[N_LAYERS];   // 1 when the layer's radix is 2
    uint32_t xs[N_LAYERS];     // the layer's two coordinates, x0 | x1 << 16 (0: no hits)
    A0[0] = (long long)hi16(q23) << qsh;
    A0[1] = (long long)lo16(q45) << qsh;
    A0[2] = (long long)hi16(q45) << qsh;
#pragma unroll
    for (int k = 0; k < 3; ++k) B0[k] = kColBias<GUARDED>;
    const uint32_t n5 = nhit_of(packed, N_LAYERS - 1);
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) {
        const uint32_t nl = nhit_of(packed, l);
        const bool paired5 = xft && l == N_LAYERS - 1;
        beta[l] = (nl == 2u && !paired5) ? 1u : 0u;
        // with pairs, layer 4's entry i also carries layer 5's hit i
        const bool fold = xft && l == N_LAYERS - 2;
        const int32_t x0 = nl ? (int32_t)hit_coord(hw[l][0]) : 0;
        const int32_t x1 = nl ? (int32_t)hit_coord(hw[l][1]) : 0;
        xs[l] = (uint32_t)x0 | ((uint32_t)x1 << 16);
        const int32_t y0 = (fold && n5) ? (int32_t)hit_coord(hw[N_LAYERS - 1][0]) : 0;
        const int32_t y1 = (fold && n5) ? (int32_t)hit_coord(hw[N_LAYERS - 1][1]) : 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // |F x| < 2^30: one product, or a pair's two, and their
            // differences fit in 32 bits
            int32_t t0 = 0, d = 0;
            if (!paired5) {
                const int32_t fl = f_of(k, l);
                t0 = fl * x0;
                d = fl * (x1 - x0);
                if (fold) {
                    const int32_t f5 = f_of(k, N_LAYERS - 1);
                    t0 += f5 * y0;
                    d += f5 * (y1 - y0);
                }
            }
            if (l < 3) {
                A0[k] += (long long)t0 * P;
                dA[l][k] = d;
            } else {
                B0[k] += (long long)t0 * P;
                dB[l - 3][k] = d;
            }
        }
    }
    const uint32_t nbB = beta[3] + beta[4] + beta[5], NB3 = 1u << nbB;
    // column sums: column b's digits are bit b5 (layer 5), then layer 4, then layer 3
#pragma unroll
    for (uint32_t b = 0; b < 8u; ++b) {
        if (b < NB3) {
            const uint32_t d5 = b & beta[5], d4 = (b >> beta[5]) & beta[4],
                           d3 = (b >> (beta[5] + beta[4])) & beta[3];
            long long s[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                s[k] = B0[k];
                s[k] += (long long)(d3 ? dB[0][k] : 0) * P;
                s[k] += (long long)(d4 ? dB[1][k] : 0) * P;
                s[k] += (long long)(d5 ? dB[2][k] : 0) * P;
            }
            tb.B01[b][lane] = make_longlong2(s[0], s[1]);
            tb.B5[b][lane] = s[2];
        }
    }
    uint32_t bchi = init_chi, bc = 0;
    const uint32_t NA3 = 1u << (beta[0] + beta[1] + beta[2]), sub = (uint32_t)lane & (L - 1u);
    for (uint32_t a = sub, c0 = sub * NB3; a < NA3 && c0 < C_eval; a += L, c0 += L * NB3) {
        const uint32_t d2 = a & beta[2], d1 = (a >> beta[2]) & beta[1],
                       d0 = (a >> (beta[2] + beta[1])) & beta[0];
        long long A[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            A[k] = A0[k];
            A[k] += (long long)(d0 ? dA[0][k] : 0) * P;
            A[k] += (long long)(d1 ? dA[1][k] : 0) * P;
            A[k] += (long long)(d2 ? dA[2][k] : 0) * P;
        }
        const uint32_t nbr = min(NB3, C_eval - c0);   // columns of this row to evaluate
#pragma unroll
        for (uint32_t b = 0; b < 8u; ++b) {
            if (b < nbr) {
                const longlong2 v01 = tb.B01[b][lane];
                const long long v5 = tb.B5[b][lane];
                const int32_t y3 = hi_word(A[0] + v01.x);
                const int32_t y4 = hi_word(A[1] + v01.y);
                const int32_t y5 = hi_word(A[2] + v5);
                if (GUARDED) {   // as in eval_rows
                    const uint32_t g3 = (uint32_t)y3, g4 = (uint32_t)y4, g5 = (uint32_t)y5;
                    const uint32_t range = g3 | g4 | g5;
                    const uint32_t chi2 = g3 * g3 + g4 * g4 + g5 * g5 + (3u << 30) -
                                          ((g3 + g4 + g5) << 16);
                    if (range < 65536u && chi2 < bchi) {
                        bchi = chi2;
                        bc = c0 + b;
                    }
                } else {
                    const int32_t c3 = clamp_chi(y3), c4 = clamp_chi(y4), c5 = clamp_chi(y5);
                    const uint32_t chi2 =
                        (uint32_t)(c3 * c3) + (uint32_t)(c4 * c4) + (uint32_t)(c5 * c5);
                    if (chi2 < bchi) {
                        bchi = chi2;
                        bc = c0 + b;
                    }
                }
            }
        }
    }
    // the group's best: smallest chi2, then smallest c
    unsigned long long key = bchi != init_chi ? ((unsigned long long)bchi << 32) | bc : ~0ull;
    for (uint32_t d = 1; d < L; d <<= 1) {
        const unsigned long long o = __shfl_xor_sync(group_mask, key, d);
        key = o < key ? o : key;
    }
    bchi = (uint32_t)(key >> 32);
    bc = (uint32_t)key;
    // the record
    LaneRecord rec;
    rec.pass = C_eval > 0 && key != ~0ull;
    uint32_t flags = rec.pass ? SVT_FLAG_PASS : 0u;
    if (((geo >> 19) & 127u) == 0) flags |= SVT_FLAG_NO_HITS;
    if (geo & (1u << 27)) flags |= SVT_FLAG_BAD_PATTERN;
    if (geo & (1u << 26)) flags |= SVT_FLAG_OVERFLOW;
    rec.w[0] = rd_id(da.z) | (flags << 24);
    rec.w[1] = rec.pass ? bc : 0xFFFFFFFFu;
    rec.w[2] = rec.pass ? bchi : 0u;
    rec.w[3] = rec.w[4] = rec.w[5] = 0u;
    if (rec.pass) {
        // the parameter rows k = 0..2 of F and q
#pragma unroll
        for (int j = 0; j < 9; ++j) fp[j] = __ldg(F32 + j);
        const uint32_t q01 = __ldg(q32), q2x = __ldg(q32 + 1);
        // the best combination's digits (with pairs, layer 5 takes layer 4's)
        const uint32_t a = bc >> nbB, b = bc & (NB3 - 1u);
        uint32_t d[N_LAYERS];
        d[5] = b & beta[5];
        d[4] = (b >> beta[5]) & beta[4];
        d[3] = (b >> (beta[5] + beta[4])) & beta[3];
        d[2] = a & beta[2];
        d[1] = (a >> beta[2]) & beta[1];
        d[0] = (a >> (beta[2] + beta[1])) & beta[0];
        if (xft) d[5] = d[4];
        int32_t x[N_LAYERS];
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l) x[l] = (int32_t)((xs[l] >> (16u * d[l])) & 0xFFFFu);
        const int32_t qv[3] = {lo16(q01), hi16(q01), lo16(q2x)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            long long acc = (long long)qv[k] * (1ll << cfg.qshift);
#pragma unroll
            for (int l = 0; l < N_LAYERS; ++l) {
                const uint32_t v = fp[(k * 6 + l) >> 1];
                acc += (long long)((l & 1) ? hi16(v) : lo16(v)) * (long long)x[l];
            }
            rec.w[3 + k] = (uint32_t)(int32_t)(acc >> cfg.oshift);   // floor
        }
    }
    return rec;
}

// Record of road r from its best key (six words into w), formed by one lane
// (the warps of the fit kernel hand their finished roads out one per lane,
// see RecordList).
// For a road that passed, the hits of its best combination are the digits of
// c = row * NB + column in the radices n'_l (the column's digits for the
// suffix layers, the row's for the prefix layers), and the parameters
// p_k = floor((q_k 2^qshift + sum_l F_kl x_l) / 2^oshift), k = 0..2, are
// formed from them in int64 (Eq. 1 for the three parameter rows).  Every load
// is issued before any is used, with no branch between them (a layer without
// hits reads the road's header word and discards it).  Returns whether the
// road passed.
__device__ __forceinline__ bool form_record(const uint32_t *__restrict__ words,
                                            const RoadDesc *__restrict__ desc, uint32_t r,
                                            unsigned long long best,
                                            const int16_t *__restrict__ F,
                                            const int16_t *__restrict__ q,
                                            const svt_config &cfg, uint32_t *w) {
    const uint4 da = __ldg(&desc[r].a), db = __ldg(&desc[r].b);
    const uint32_t geo = db.x, packed = da.y, total_hits = (geo >> 19) & 127u;
    const bool pass = best != ~0ull;
    uint32_t flags = 0;
    if (total_hits == 0) flags |= SVT_FLAG_NO_HITS;
    if (geo & (1u << 27)) flags |= SVT_FLAG_BAD_PATTERN;
    if (geo & (1u << 26)) flags |= SVT_FLAG_OVERFLOW;
    uint32_t c = 0xFFFFFFFFu, chi2 = 0;
    int32_t p[3] = {0, 0, 0};
    if (pass) {
        flags |= SVT_FLAG_PASS;
        const uint32_t low = (uint32_t)best, row = low >> 9, col = low & 511u;
        const uint32_t split = geo & 7u;
        c = row * db.y + col;
        chi2 = (uint32_t)(best >> 32);
        uint32_t digit[N_LAYERS];
        uint32_t rem = col;
#pragma unroll
        for (int l = N_LAYERS - 1; l >= 0; --l) {
            if ((uint32_t)l + 1u == split) rem = row;   // the prefix layers take the row
            const uint32_t nl = nhit_of(packed, l);
            const uint32_t np = (nl && !(cfg.xft_pairs && l == N_LAYERS - 1)) ? nl : 1u;
            const uint32_t qd = div_by(rem, np, kDivMagic[np]);
            digit[l] = rem - qd * np;
            rem = qd;
        }
        if (cfg.xft_pairs) digit[N_LAYERS - 1] = digit[N_LAYERS - 2];   // the pair's own index
        const size_t cs = (size_t)rd_sector(da.z) * 64 + ((geo >> 13) & 63u);
        uint32_t hw[N_LAYERS];
        uint32_t off = da.x + 1;   // first hit word of layer l (hits are sorted by layer)
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l) {
            const uint32_t nl = nhit_of(packed, l);
            hw[l] = __ldg(words + (nl ? off + digit[l] : da.x));
            off += nl;
        }
        int32_t f[3][N_LAYERS], qk[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            qk[k] = __ldg(q + cs * 6 + k);
#pragma unroll
            for (int l = 0; l < N_LAYERS; ++l) f[k][l] = __ldg(F + cs * 36 + k * 6 + l);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            long long acc = (long long)qk[k] * (1ll << cfg.qshift);
#pragma unroll
            for (int l = 0; l < N_LAYERS; ++l) {
                const int32_t x = nhit_of(packed, l) ? (int32_t)hit_coord(hw[l]) : 0;
                acc += (long long)f[k][l] * (long long)x;
            }
            p[k] = (int32_t)(acc >> cfg.oshift);   // floor
        }
    }
    w[0] = rd_id(da.z) | (flags << 24);
    w[1] = c;
    w[2] = chi2;
    w[3] = (uint32_t)p[0];
    w[4] = (uint32_t)p[1];
    w[5] = (uint32_t)p[2];
    return pass;
}

// K4: persistent fit / cut / select / format.  GROUP 2: two consecutive SMALL
// roads of one chunk with the same geometry go to the two halves of the warp;
// GROUP 4: four consecutive TINY roads of the same geometry go to its four
// quarters (else two SMALL roads to its halves, as with GROUP 2); GROUP 32:
// every TINY road of the chunk goes to a lane of its own (lane k: the chunk's
// road k), then the warp fits the chunk's other roads one at a time.  Each is
// a separate instance, so that warps never switch between the code paths
// unless grouping was asked for.
// (GROUP 32 keeps every load of a lane's road in flight at once with up to 85
// registers a thread, blocks of at most 12 warps: 80 are used, three blocks of
// 8 warps per SM; with 64, loads were serialised or spilled and with 128 only
// 16 warps per SM were resident.  The others fit in 64, for two blocks of
// 512 threads.)
template <bool GUARDED, int GROUP>
__global__ void __launch_bounds__(GROUP == 32 ? 384 : 512, 2)
    k_fit_persistent(const uint32_t *__restrict__ words, const uint64_t *__restrict__ event_off,
                     const Dims *__restrict__ dims, const uint32_t *__restrict__ event_road,
                     const RoadDesc *__restrict__ desc, uint64_t *counts, uint64_t road_cap,
                     const int16_t *__restrict__ F, const int16_t *__restrict__ q,
                     const svt_config cfg, const FusedRoads fr, uint32_t roads_per_chunk,
                     uint32_t *out, unsigned long long *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem &sm = *reinterpret_cast<WarpSmem *>(smem_raw + SLOT_BYTES * (threadIdx.x >> 5));
    RecordList &rl = reinterpret_cast<RecordList *>(
        smem_raw + SLOT_BYTES * (blockDim.x >> 5))[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const Lanes<32> LW = lanes_of<32>(lane);
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
    // GROUP 32: lanes to a tiny road, so that chunks of 32, 16 or at most 8
    // roads fill the warp
    const uint32_t L = GROUP != 32 ? 1u : roads_per_chunk > 16 ? 1u : roads_per_chunk > 8 ? 2u : 4u;
    uint32_t n_rec = 0;    // entries of rl (uniform over the warp)
    uint32_t n_pass = 0;   // passing roads whose records this lane wrote, summed at exit
    // Each lane forms one listed record into the warp's road slot (free
    // between roads), then the warp stores the 6 * n_rec words with
    // consecutive lanes on consecutive words, so that the records of
    // consecutive roads go out as contiguous runs.
    auto flush = [&]() {
        __syncwarp();
        uint32_t *stage = reinterpret_cast<uint32_t *>(&sm);
        if ((uint32_t)lane < n_rec &&
            form_record(words, desc, rl.road[lane], rl.key[lane], F, q, cfg, stage + lane * 6))
            ++n_pass;
        __syncwarp();
        for (uint32_t e = (uint32_t)lane; e < n_rec * 6; e += 32) {
            const uint32_t i = e / 6;
            out[(size_t)rl.road[i] * 6 + (e - i * 6)] = stage[e];
        }
        n_rec = 0;
        __syncwarp();
    };

    // With four tiny roads per warp (GROUP 4) or one per lane (GROUP 32) a
    // batch without split roads skips phase 1 and hands every warp its first
    // chunk of phase 2 statically (warp w of block b takes chunk
    // w * gridDim.x + b, so that a batch of fewer chunks than warps spreads
    // over the SMs), the rest through the
    // counter counted from nw: the grid's warps then start without queueing
    // on one address, which for chunks this short is a large part of the
    // kernel (the paper's shape, 3000 events: 43 -> 37 us).  Otherwise every
    // claim goes through the counters (static first claims made the scaled
    // shape 6 % slower).
    const uint32_t nw = gridDim.x * (blockDim.x >> 5);
    const bool static_first = (GROUP == 4 || GROUP == 32) && n_items == 0;

    // phase 1: items of split roads
    while (!static_first) {
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
        road_setup<32>(sm, words, D, g, F, q, sh, cfg.xft_pairs, kColBias<GUARDED>, LW);
        const uint32_t a_lo = k * fr.rows;
        const uint32_t a_hi = min(a_lo + fr.rows, g.NA);
        const unsigned long long best = eval_rows<GUARDED, 32>(sm, g, a_lo, a_hi, qsh, init_chi, LW);
        uint32_t last = 0;
        if (lane == 0) {
            if (best != ~0ull) atomicMin(fr.key + r, best);
            __threadfence();
            last = (atomicSub(bl.pending + j, 1u) == 1u) ? 1u : 0u;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {   // every item of road r is done: list it with its final key
            if (n_rec == 32) flush();
            if (lane == 0) {
                __threadfence();
                rl.key[n_rec] = __ldcg(fr.key + r);
                rl.road[n_rec] = r;
            }
            n_rec += 1;
        }
        __syncwarp();
    }

    // phase 2: chunks of consecutive roads, each fitted whole by this warp,
    // or two SMALL roads side by side by its two halves
    for (bool first = true;; first = false) {
        uint32_t k = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;   // chunk index
        if (!(first && static_first)) {
            if (lane == 0) k = atomicAdd(bl.counters + 1, 1u) + (static_first ? nw : 0u);
            k = __shfl_sync(0xffffffffu, k, 0);
        }
        if ((uint64_t)k * roads_per_chunk >= R) break;
        const uint32_t c0 = k * roads_per_chunk;
        const uint32_t n = min(roads_per_chunk, R - c0);
        // this lane's road of the chunk (GROUP 32: L lanes to a road)
        const uint32_t jr = (uint32_t)lane / L;
        uint4 da = make_uint4(0, 0, 0, 0), db = make_uint4(0, 0, 0, 0);
        if (jr < n) {
            da = __ldg(&desc[c0 + jr].a);
            db = __ldg(&desc[c0 + jr].b);
        }
        if constexpr (GROUP == 32) {
            // the chunk's TINY roads, L lanes each, their records formed by
            // their first lanes and stored at once as runs of consecutive
            // words ...
            const bool mine = jr < n && (db.x & GEO_TINY) && da.w <= fr.small_max;
            const uint32_t lm = __ballot_sync(0xffffffffu, mine);
            const bool first_lane = ((uint32_t)lane & (L - 1u)) == 0;
            if (lm) {
                LaneRecord rec;
                if (mine)
                    rec = lane_fit<GUARDED>(*reinterpret_cast<LaneTables *>(&sm), words, da, db, F,
                                            q, cfg, sh, qsh, init_chi, lane, L, lm);
                __syncwarp();
                uint32_t *stage = reinterpret_cast<uint32_t *>(&sm);
                if (mine && first_lane) {
#pragma unroll
                    for (int j = 0; j < 6; ++j) stage[jr * 6 + j] = rec.w[j];
                    n_pass += rec.pass ? 1u : 0u;
                }
                __syncwarp();
                for (uint32_t e = (uint32_t)lane; e < n * 6; e += 32) {
                    const uint32_t i = e / 6;
                    if ((lm >> (i * L)) & 1u) out[(size_t)(c0 + i) * 6 + (e - i * 6)] = stage[e];
                }
                __syncwarp();
            }
            // ... then the others (not split) one per warp
            uint32_t rest = __ballot_sync(0xffffffffu,
                                          first_lane && jr < n && !mine && da.w <= fr.small_max);
            while (rest) {
                const uint32_t src = (uint32_t)__ffs(rest) - 1u, jj = src / L;
                rest &= rest - 1u;
                const RoadDesc D = shfl_desc(da, db, src);
                if (n_rec == 32) flush();
                const unsigned long long best =
                    fit_road<GUARDED, 32>(sm, words, D, F, q, cfg, sh, qsh, init_chi, LW);
                if (lane == 0) {
                    rl.key[n_rec] = best;
                    rl.road[n_rec] = c0 + jj;
                }
                n_rec += 1;
                __syncwarp();
            }
        } else {
            for (uint32_t jj = 0; jj < n;) {
                const RoadDesc D = shfl_desc(da, db, jj);
                if (D.a.w > fr.small_max) {   // split road: done in phase 1
                    ++jj;
                    continue;
                }
                if (n_rec > 32 - GROUP) flush();   // room for GROUP more
                if constexpr (GROUP == 4) {
                    // four TINY roads with the same hits per layer and the same
                    // number of combinations to evaluate, so that the quarters
                    // run their loops in step
                    if ((D.b.x & GEO_TINY) && jj + 3 < n) {
                        // lane k holds road c0 + k: one vote over the next four
                        const bool same = (db.x & GEO_TINY) && da.y == D.a.y && da.w == D.a.w;
                        const uint32_t votes = __ballot_sync(0xffffffffu, same);
                        if (((votes >> jj) & 15u) == 15u) {
                            // this lane's quarter and road
                            const uint32_t qt = (uint32_t)lane >> 3;
                            QuarterSmem &qs = reinterpret_cast<QuarterSmem *>(&sm)[qt];
                            const RoadDesc Dq = shfl_desc(da, db, jj + qt);
                            const Lanes<8> LQ = lanes_of<8>(lane);
                            Geo g = geo_of(Dq);
                            unsigned long long best = ~0ull;
                            if (g.C_eval) {
                                quarter_geometry(g, Dq.a.y, cfg.xft_pairs);
                                road_setup<8>(qs, words, Dq, g, F, q, sh, cfg.xft_pairs,
                                              kColBias<GUARDED>, LQ);
                                best = quarter_key(
                                    eval_rows<GUARDED, 8>(qs, g, 0, g.NA, qsh, init_chi, LQ), g.NB,
                                    Dq.b.y);
                            }
                            if ((lane & 7) == 0) {
                                rl.key[n_rec + qt] = best;
                                rl.road[n_rec + qt] = c0 + jj + qt;
                            }
                            n_rec += 4;
                            jj += 4;
                            __syncwarp();
                            continue;
                        }
                    }
                }
                if constexpr (GROUP >= 2) {
                    // two SMALL roads of the same geometry (split, NBp, ntop and NA),
                    // so that the two halves run their loops in step
                    if ((D.b.x & GEO_SMALL) && jj + 1 < n) {
                        const RoadDesc D2 = shfl_desc(da, db, jj + 1);
                        if ((D2.b.x & GEO_SMALL) && ((D.b.x ^ D2.b.x) & 0x1FFFu) == 0 &&
                            D.b.z == D2.b.z && D2.a.w <= fr.small_max) {
                            const uint32_t h = (uint32_t)lane >> 4;   // this lane's half and road
                            HalfSmem &hs = reinterpret_cast<HalfSmem *>(&sm)[h];
                            const unsigned long long best = fit_road<GUARDED, 16>(
                                hs, words, h ? D2 : D, F, q, cfg, sh, qsh, init_chi,
                                lanes_of<16>(lane));
                            if ((lane & 15) == 0) {
                                rl.key[n_rec + h] = best;
                                rl.road[n_rec + h] = c0 + jj + h;
                            }
                            n_rec += 2;
                            jj += 2;
                            __syncwarp();
                            continue;
                        }
                    }
                }
                const unsigned long long best =
                    fit_road<GUARDED, 32>(sm, words, D, F, q, cfg, sh, qsh, init_chi, LW);
                if (lane == 0) {
                    rl.key[n_rec] = best;
                    rl.road[n_rec] = c0 + jj;
                }
                n_rec += 1;
                jj += 1;
                __syncwarp();
            }
        }
    }
    flush();
    n_pass = __reduce_add_sync(0xffffffffu, n_pass);
    if (lane == 0 && n_pass)
        atomicAdd((unsigned long long *)(counts + 3), (unsigned long long)n_pass);
}

}  // namespace

size_t fit_smem_bytes(int warps_per_block) {
    return (SLOT_BYTES + sizeof(RecordList)) * (size_t)warps_per_block;
}

int fit_persistent_blocks_per_sm(int warps_per_block, uint32_t group) {
    const size_t smem = fit_smem_bytes(warps_per_block);
    int occ = 1 << 30;
    auto one = [&](auto kernel) {
        int n = 0;
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, warps_per_block * 32, smem) !=
            cudaSuccess)
            n = 0;
        occ = n < occ ? n : occ;
    };
    // both instances of the group (the chi2 cut picks one at launch)
    if (group == 32) {
        one(k_fit_persistent<true, 32>);
        one(k_fit_persistent<false, 32>);
    } else if (group == 4) {
        one(k_fit_persistent<true, 4>);
        one(k_fit_persistent<false, 4>);
    } else if (group == 2) {
        one(k_fit_persistent<true, 2>);
        one(k_fit_persistent<false, 2>);
    } else {
        one(k_fit_persistent<true, 1>);
        one(k_fit_persistent<false, 1>);
    }
    return occ;
}

cudaError_t launch_fit_persistent(const uint32_t *words, const uint64_t *event_off,
                                  const Dims *dims, const uint32_t *event_road,
                                  const RoadDesc *desc, uint64_t *counts, uint64_t road_cap,
                                  const int16_t *F, const int16_t *q, const svt_config cfg,
                                  const FusedRoads fr, uint32_t roads_per_chunk, uint32_t group,
                                  uint32_t *out, unsigned long long *status,
                                  int warps_per_block, int grid, cudaStream_t st) {
    const size_t smem = fit_smem_bytes(warps_per_block);
    const bool guarded = cfg.chi2_cut < 32767u * 32767u;
    auto launch = [&](auto kernel) {
        launch_after(kernel, grid, warps_per_block * 32, smem, st, words, event_off, dims,
                     event_road, desc, counts, road_cap, F, q, cfg, fr, roads_per_chunk, out,
                     status);
    };
    if (guarded) {
        if (group == 32) launch(k_fit_persistent<true, 32>);
        else if (group == 4) launch(k_fit_persistent<true, 4>);
        else if (group == 2) launch(k_fit_persistent<true, 2>);
        else launch(k_fit_persistent<true, 1>);
    } else {
        if (group == 32) launch(k_fit_persistent<false, 32>);
        else if (group == 4) launch(k_fit_persistent<false, 4>);
        else if (group == 2) launch(k_fit_persistent<false, 2>);
        else launch(k_fit_persistent<false, 1>);
    }
    return cudaGetLastError();
}

}  // namespace svt
