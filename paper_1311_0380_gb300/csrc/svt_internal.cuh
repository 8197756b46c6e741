// svt_internal.cuh -- device helpers shared by the CUDA kernels of the SVT
// track-fit library (word decoding, status reporting, block scans, exact small
// division, workspace carving).  Host-visible types come from include/svt.h.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/svt.h"

namespace svt {

// ---- word format (include/svt.h) -------------------------------------------
__host__ __device__ __forceinline__ uint32_t w_type(uint32_t w) { return w >> 30; }
__host__ __device__ __forceinline__ uint32_t ev_nroads(uint32_t w) { return w & 0xFFFu; }
__host__ __device__ __forceinline__ uint32_t rd_sector(uint32_t w) { return (w >> 21) & 0x1FFu; }
__host__ __device__ __forceinline__ uint32_t rd_id(uint32_t w) { return w & 0x1FFFFFu; }
__host__ __device__ __forceinline__ uint32_t hit_layer(uint32_t w) { return (w >> 27) & 7u; }
__host__ __device__ __forceinline__ uint32_t hit_reserved(uint32_t w) { return (w >> 15) & 0xFFFu; }
__host__ __device__ __forceinline__ uint32_t hit_coord(uint32_t w) { return w & 0x7FFFu; }

constexpr uint32_t TYPE_HIT = 0, TYPE_BAD = 1, TYPE_ROAD = 2, TYPE_EVENT = 3;
constexpr int N_LAYERS = 6;
constexpr int MAX_HITS = 16;

// packed hits per layer: 5 bits per layer
__host__ __device__ __forceinline__ uint32_t nhit_of(uint32_t packed, int l) {
    return (packed >> (5 * l)) & 31u;
}

// ---- status ---------------------------------------------------------------
__device__ __forceinline__ void report(unsigned long long *status, uint64_t word_index,
                                       uint32_t code) {
    atomicMin(status, (unsigned long long)((word_index << 8) | code));
}
__device__ __forceinline__ bool status_ok(const unsigned long long *status) {
    return *(volatile const unsigned long long *)status == ~0ull;
}

// ---- tiles of words ---------------------------------------------------------
constexpr int TILE_THREADS = 128;
constexpr int TILE_PER_THREAD = 8;
constexpr int TILE_WORDS = TILE_THREADS * TILE_PER_THREAD;  // 1024

__host__ __device__ __forceinline__ uint64_t n_tiles(uint64_t n_words) {
    return (n_words + TILE_WORDS - 1) / TILE_WORDS;
}

// ---- block-wide exclusive scan (blockDim.x == TILE_THREADS) ----------------
// Returns the exclusive prefix of `v` over the block and writes the block
// total to *total.  `smem` holds TILE_THREADS/32 + 1 entries.  With
// END_SYNC false the closing barrier is left out: the caller then reaches
// another barrier before `smem` is written again.
template <typename T, bool END_SYNC = true>
__device__ __forceinline__ T block_exclusive_scan(T v, T *smem, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_warps = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < n_warps) ? smem[lane] : T(0);
        T s = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < n_warps) smem[lane] = s - w;  // exclusive warp offsets
        if (lane == n_warps - 1) smem[n_warps] = s;
    }
    __syncthreads();
    T res = smem[warp] + x - v;
    *total = smem[n_warps];
    if (END_SYNC) __syncthreads();
    return res;
}

// ---- exact division by a small divisor ---------------------------------------
// For 1 <= d <= 16 and x < 2^24: q = x / d, using m = ceil(2^32 / d)
// (exact because x * (m*d - 2^32) < 2^32 in that range); d == 1 is special.
struct SmallDiv {
    uint32_t m;
    uint32_t d;
};
__host__ __device__ __forceinline__ SmallDiv make_div(uint32_t d) {
    SmallDiv r;
    r.d = d;
    r.m = (d <= 1) ? 0u : (uint32_t)((0xFFFFFFFFull / d) + 1ull);
    return r;
}
__device__ __forceinline__ uint32_t div_small(uint32_t x, SmallDiv v) {
    return v.d <= 1 ? x : __umulhi(x, v.m);
}
// m = ceil(2^32 / d) for d = 2..32 (0 for d < 2): x / d = umulhi(x, m) for
// x < 2^24 when d <= 16, and for x <= 64 when d <= 32.
static __device__ __constant__ uint32_t kDivMagic[33] = {
    0u, 0u, 2147483648u, 1431655766u, 1073741824u, 858993460u, 715827883u, 613566757u,
    536870912u, 477218589u, 429496730u, 390451573u, 357913942u, 330382100u, 306783379u,
    286331154u, 268435456u, 252645136u, 238609295u, 226050911u, 214748365u, 204522253u,
    195225787u, 186737709u, 178956971u, 171798692u, 165191050u, 159072863u, 153391690u,
    148102321u, 143165577u, 138547333u, 134217728u};
__device__ __forceinline__ uint32_t div_by(uint32_t x, uint32_t d, uint32_t m) {
    return d <= 1 ? x : __umulhi(x, m);
}

// ---- combination geometry of a road ----------------------------------------
// All quantities derived from the per-layer hit counts.
struct RoadShape {
    uint32_t n[N_LAYERS];   // n'_l = max(n_l, 1)
    uint32_t mask;          // layers with at least one hit
    uint32_t total_hits;
    uint32_t n_layers_hit;
    uint64_t C;             // prod n'_l
};
// With xft_pairs layer 5 is no digit of its own: its radix is 1 (it takes
// layer 4's hit index), while the mask and the hit count keep its hits.
__device__ __forceinline__ RoadShape road_shape(uint32_t packed, uint32_t xft_pairs = 0) {
    RoadShape s;
    s.mask = 0;
    s.total_hits = 0;
    s.n_layers_hit = 0;
    s.C = 1;
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) {
        uint32_t nl = nhit_of(packed, l);
        s.total_hits += nl;
        if (nl) {
            s.mask |= 1u << l;
            s.n_layers_hit += 1;
        }
        s.n[l] = (nl && !(xft_pairs && l == N_LAYERS - 1)) ? nl : 1u;
        s.C *= s.n[l];
    }
    return s;
}

// Split of the layers into a prefix {0..split-1} (index a, "rows") and a
// suffix {split..5} (index b, "columns"): c = a * NB + b.  The suffix is the
// shortest one with at least 32 combinations, so a warp's 32 lanes cover one
// row; roads with fewer than 32 combinations put everything in the suffix.
__device__ __forceinline__ void road_split(const RoadShape &s, uint32_t &split, uint32_t &NB) {
    uint32_t nb = 1;
    bool found = false;
    split = 0;
    NB = (uint32_t)s.C;
#pragma unroll
    for (int l = N_LAYERS - 1; l >= 0; --l) {
        nb *= s.n[l];
        if (!found && nb >= 32) {
            split = (uint32_t)l;
            NB = nb;
            found = true;
        }
    }
}

// ---- workspace carving -------------------------------------------------------
__host__ __device__ __forceinline__ size_t align_up(size_t v, size_t a) {
    return (v + a - 1) / a * a;
}

// A named NVTX range over the host-side enqueue of one stage (shown by the
// Nsight tools on the CPU timeline; a no-op when no tool is attached).
struct NvtxRange {
    __host__ explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    __host__ ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct Carver {
    char *base;
    size_t off;
    __host__ explicit Carver(void *b) : base((char *)b), off(0) {}
    template <typename T>
    __host__ T *take(size_t count) {
        off = align_up(off, 256);
        T *p = (T *)(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
    __host__ size_t size() const { return align_up(off, 256); }
};

}  // namespace svt
