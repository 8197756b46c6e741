// svt_roads.cuh -- the fused path's per-road work description: the road
// descriptor that the road extraction builds and the persistent fit kernel
// reads, and the list of roads whose combinations are split into work items.
#pragma once

#include "svt_internal.cuh"

namespace svt {

// Per-road descriptor of the fused path (32 bytes), built once by the road
// extraction:
//   a = {header word index, hits per layer (5 bits each), header word,
//        evaluated combinations C_eval}
//   b = {geo, NB, NA, 0} with the split c = a_row * NB + b_col (see road_split),
//       NA = ceil(C_eval / NB) rows, and geo bits [2:0] split, [7:3] NBp (columns
//       below the top suffix layer, NB = ntop * NBp), [12:8] ntop, [18:13] layer
//       mask, [25:19] total hits, [26] OVERFLOW, [27] BAD_PATTERN, [28] SMALL:
//       at most 8 hits on every layer, NBp <= 16 and NA <= 16, so that half a
//       warp can fit the road (the fit kernel pairs such roads), [29] TINY: at
//       most 2 hits on every layer, NBp <= 16 and NA <= 8, so that a quarter
//       of a warp can fit it (the fit kernel can group four such roads).
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
    bool small = NBp <= 16u && NA <= 16u, tiny = NBp <= 16u && NA <= 8u;
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) {
        small = small && nhit_of(packed, l) <= 8u;
        tiny = tiny && nhit_of(packed, l) <= 2u;
    }
    const uint32_t geo = split | (NBp << 3) | (ntop << 8) | (s.mask << 13) | (s.total_hits << 19) |
                         ((!bad && C > cfg.max_comb) ? (1u << 26) : 0u) | (bad ? (1u << 27) : 0u) |
                         (small ? (1u << 28) : 0u) | (tiny ? (1u << 29) : 0u);
    RoadDesc d;
    d.a = make_uint4(rw, packed, hw, C_eval);
    d.b = make_uint4(geo, NB, NA, 0u);
    return d;
}

// Split roads of the fused path.  The road extraction appends each tile's
// split roads with one 64-bit atomic on `reserve` ((items << 32) | roads), so
// road slots and item ranges are reserved together and item_off increases
// with the slot; the fit kernel's work queues are counters[0] (items) and
// counters[1] (chunks of roads; past each warp's first chunk where the fit
// kernel hands those out statically).
struct BigList {
    uint32_t *road;                // split road of each slot
    uint32_t *item_off;            // its first work item
    uint32_t *pending;             // its items not yet finished
    unsigned long long *reserve;   // (items << 32) | roads appended so far
    uint32_t *counters;            // [0] items, [1] chunks taken from the queues
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

}  // namespace svt
