// svt_plain.cu -- the plain per-stage path: combine writes every combination
// of one hit per layer, fit evaluates one combination per thread, select keeps
// the best passing combination per road, format packs the records.  This is
// the structure of the paper's Sec. 2.1 GPU port (one kernel per stage, the
// loops unrolled so that one thread handles one combination), kept here as
// the baseline of the fused path and as the per-stage C ABI.
#include "svt_kernels.cuh"

namespace svt {

namespace {

__device__ __forceinline__ uint64_t road_count(const uint64_t *n_roads, uint64_t road_cap) {
    uint64_t R = *n_roads;
    return R < road_cap ? R : road_cap;
}

__global__ void k_combine_count(const uint32_t *__restrict__ road_nhit,
                                const uint64_t *__restrict__ n_roads, uint64_t road_cap,
                                const svt_config cfg, uint32_t *road_flags, uint64_t *comb_cnt,
                                const unsigned long long *status) {
    if (!status_ok(status)) return;
    const uint64_t R = road_count(n_roads, road_cap);
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const RoadShape s = road_shape(road_nhit[r], cfg.xft_pairs);
        uint32_t flags = s.total_hits == 0 ? SVT_FLAG_NO_HITS : 0u;
        uint64_t n = 0;
        if (s.n_layers_hit < cfg.min_layers) {
            flags |= SVT_FLAG_BAD_PATTERN;
        } else {
            n = s.C;
            if (s.C > cfg.max_comb) {
                flags |= SVT_FLAG_OVERFLOW;
                n = cfg.max_comb;
            }
        }
        road_flags[r] = flags;
        comb_cnt[r] = n;
    }
}

// ---- exclusive scan of uint64 counts: per-tile sums, one-block scan, apply ----
constexpr int SCAN_THREADS = 256, SCAN_PER = 8, SCAN_TILE = SCAN_THREADS * SCAN_PER;

__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_u64_reduce(const uint64_t *__restrict__ a, const uint64_t *__restrict__ n_dev,
                      uint64_t cap, uint64_t *tile_sums, const unsigned long long *status) {
    __shared__ unsigned long long red[SCAN_THREADS / 32 + 1];
    if (!status_ok(status)) return;
    const uint64_t n = *n_dev < cap ? *n_dev : cap;
    const uint64_t T = (n + SCAN_TILE - 1) / SCAN_TILE;
    for (uint64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const uint64_t b = t * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_PER;
        unsigned long long s = 0;
#pragma unroll
        for (int j = 0; j < SCAN_PER; ++j) s += (b + j < n) ? a[b + j] : 0ull;
        unsigned long long tot;
        block_exclusive_scan<unsigned long long>(s, red, &tot);
        if (threadIdx.x == 0) tile_sums[t] = tot;
    }
}

__global__ void __launch_bounds__(1024)
    k_scan_u64_tiles(uint64_t *tile_sums, const uint64_t *__restrict__ n_dev, uint64_t cap,
                     const unsigned long long *status) {
    __shared__ unsigned long long sm[33];
    if (!status_ok(status)) return;
    const uint64_t n = *n_dev < cap ? *n_dev : cap;
    const uint64_t T = (n + SCAN_TILE - 1) / SCAN_TILE;
    unsigned long long carry = 0;
    for (uint64_t c0 = 0; c0 < T; c0 += 1024) {
        const uint64_t i = c0 + threadIdx.x;
        unsigned long long v = i < T ? tile_sums[i] : 0ull;
        unsigned long long tot;
        unsigned long long ex = block_exclusive_scan<unsigned long long>(v, sm, &tot);
        if (i < T) tile_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) tile_sums[T] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS)
    k_scan_u64_apply(uint64_t *a, const uint64_t *__restrict__ n_dev, uint64_t cap,
                     const uint64_t *__restrict__ tile_sums, uint64_t *total,
                     const unsigned long long *status) {
    __shared__ unsigned long long red[SCAN_THREADS / 32 + 1];
    if (!status_ok(status)) return;
    const uint64_t n = *n_dev < cap ? *n_dev : cap;
    const uint64_t T = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a[n] = tile_sums[T];
        if (total) *total = tile_sums[T];
    }
    for (uint64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const uint64_t b = t * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_PER;
        unsigned long long v[SCAN_PER], s = 0;
#pragma unroll
        for (int j = 0; j < SCAN_PER; ++j) {
            v[j] = (b + j < n) ? a[b + j] : 0ull;
            s += v[j];
        }
        unsigned long long tot;
        unsigned long long run = tile_sums[t] + block_exclusive_scan<unsigned long long>(s, red, &tot);
#pragma unroll
        for (int j = 0; j < SCAN_PER; ++j) {
            if (b + j < n) a[b + j] = run;
            run += v[j];
        }
    }
}

// Roads with more combinations than this are written (combine) and scanned
// (select) by a whole block in a second launch, so that one long road does
// not hold up a warp while the others have finished.
constexpr uint64_t PLAIN_BIG = 4096;

// Per-road metadata for the plain combine and select, read for a group of
// roads at once (one coalesced load per field) instead of road by road.
struct RoadMeta {
    uint64_t off, n;
    uint32_t word;   // road_nhit (combine) or road_flags (select)
};

// Metadata of road r (zeros past the last road).
__device__ __forceinline__ RoadMeta road_meta(const uint64_t *__restrict__ comb_off,
                                              const uint32_t *__restrict__ word, uint64_t R,
                                              uint64_t r) {
    RoadMeta m{0, 0, 0};
    if (r < R) {
        m.off = __ldg(comb_off + r);
        m.n = __ldg(comb_off + r + 1) - m.off;
        m.word = __ldg(word + r);
    }
    return m;
}

// Big roads of a block's group of blockDim.x roads, compacted into `list`
// (their metadata and index); returns how many (a block-wide call).
__device__ __forceinline__ uint32_t big_roads_of_group(const RoadMeta &mine, uint64_t r,
                                                       bool big, RoadMeta *list,
                                                       uint32_t *list_r, uint32_t *count) {
    if (threadIdx.x == 0) *count = 0;
    __syncthreads();
    if (big) {
        const uint32_t k = atomicAdd(count, 1u);
        list[k] = mine;
        list_r[k] = (uint32_t)r;
    }
    __syncthreads();
    return *count;
}

// Rows [a_begin, a_end) of one road's combinations in index order
// c = a * NB + b, with the layers split as in the fused path (road_split: a
// suffix of at least 32 combinations gives the column b, the prefix the row
// a).  A lane derives the suffix digits of its column once per pass over the
// columns; the prefix digits (the same for all lanes) are derived for the
// first row and then counted up row by row (layer split-1 fastest, a carry
// only when a digit wraps), so a combination costs a few instructions and
// two coalesced stores.
__device__ __forceinline__ void write_rows(uint32_t r, const RoadMeta &m, const RoadShape &s,
                                           uint32_t split, uint32_t NB, uint32_t a_begin,
                                           uint32_t a_end, uint32_t xft_pairs, int lane,
                                           uint32_t *comb_road, uint32_t *comb_hits) {
    uint32_t mg[N_LAYERS], top = 0;   // top: n'_l - 1 of every layer, 4 bits each
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) {
        mg[l] = kDivMagic[s.n[l]];
        top |= (s.n[l] - 1u) << (4 * l);
    }
    uint32_t ra = a_begin, pa0 = 0;   // prefix digits of the first row
#pragma unroll
    for (int l = N_LAYERS - 1; l >= 0; --l) {
        if ((uint32_t)l < split) {
            const uint32_t qd = div_by(ra, s.n[l], mg[l]);
            pa0 |= (ra - qd * s.n[l]) << (4 * l);
            ra = qd;
        }
    }
    for (uint32_t b0 = 0; b0 < NB; b0 += 32) {
        const uint32_t b = b0 + (uint32_t)lane;
        uint32_t rem = b, pb = 0;   // digits of the suffix layers split..5
#pragma unroll
        for (int l = N_LAYERS - 1; l >= 0; --l) {
            if ((uint32_t)l >= split) {
                const uint32_t qd = div_by(rem, s.n[l], mg[l]);
                pb |= (rem - qd * s.n[l]) << (4 * l);
                rem = qd;
            }
        }
        uint32_t pa = pa0;
        uint64_t c = (uint64_t)a_begin * NB + b;
        for (uint32_t a = a_begin; a < a_end; ++a, c += NB) {
            if (b < NB && c < m.n) {
                uint32_t packed = pa | pb;
                if (xft_pairs) packed |= ((packed >> 16) & 15u) << 20;   // layer 5 takes layer 4's hit
                comb_road[m.off + c] = r;
                comb_hits[m.off + c] = packed;
            }
            for (int l = (int)split - 1; l >= 0; --l) {   // next row
                const uint32_t sh = 4u * (uint32_t)l;
                if (((pa >> sh) & 15u) != ((top >> sh) & 15u)) {
                    pa += 1u << sh;
                    break;
                }
                pa &= ~(15u << sh);
            }
        }
    }
}

// A road per warp (roads of at most PLAIN_BIG combinations, each combination's
// digits by division; the next road's entries are read while this one is
// written), or a big road per block whose eight warps take one block of rows
// each (write_rows).
template <bool BIG>
__global__ void __launch_bounds__(256)
    k_combine_write(const uint32_t *__restrict__ road_nhit, const uint64_t *__restrict__ n_roads,
                    uint64_t road_cap, const uint64_t *__restrict__ comb_off, uint64_t comb_cap,
                    uint32_t xft_pairs, uint32_t *comb_road, uint32_t *comb_hits,
                    unsigned long long *status) {
    __shared__ RoadMeta list[256];
    __shared__ uint32_t list_r[256], list_n;
    if (!status_ok(status)) return;
    const uint64_t R = road_count(n_roads, road_cap);
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    if (!BIG && warp0 == 0 && lane == 0 && comb_off[R] > comb_cap) report(status, 0, SVT_ERR_OOM);
    if (!BIG) {
        RoadMeta m = road_meta(comb_off, road_nhit, R, warp0);
        for (uint64_t r = warp0; r < R; r += n_warps) {
            const RoadMeta next = road_meta(comb_off, road_nhit, R, r + n_warps);
            if (m.n && m.n <= PLAIN_BIG && m.off + m.n <= comb_cap) {
                const RoadShape s = road_shape(m.word, xft_pairs);
                uint32_t mg[N_LAYERS];
#pragma unroll
                for (int l = 0; l < N_LAYERS; ++l) mg[l] = kDivMagic[s.n[l]];
                for (uint64_t c = lane; c < m.n; c += 32) {
                    uint32_t rem = (uint32_t)c, packed = 0;
#pragma unroll
                    for (int l = N_LAYERS - 1; l >= 0; --l) {
                        const uint32_t qd = div_by(rem, s.n[l], mg[l]);
                        packed |= (rem - qd * s.n[l]) << (4 * l);
                        rem = qd;
                    }
                    if (xft_pairs) packed |= ((packed >> 16) & 15u) << 20;
                    comb_road[m.off + c] = (uint32_t)r;
                    comb_hits[m.off + c] = packed;
                }
            }
            m = next;
        }
    } else {
        const uint32_t warp = threadIdx.x >> 5, n_w = blockDim.x >> 5;
        for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x; g < R;
             g += (uint64_t)gridDim.x * blockDim.x) {
            const uint64_t r = g + threadIdx.x;
            const RoadMeta mine = road_meta(comb_off, road_nhit, R, r);
            const bool big = mine.n > PLAIN_BIG && mine.off + mine.n <= comb_cap;
            const uint32_t nb = big_roads_of_group(mine, r, big, list, list_r, &list_n);
            for (uint32_t k = 0; k < nb; ++k) {
                const RoadMeta m = list[k];
                const RoadShape s = road_shape(m.word, xft_pairs);
                uint32_t split, NB;
                road_split(s, split, NB);
                const uint32_t NA = (uint32_t)((m.n + NB - 1) / NB);
                const uint32_t per = (NA + n_w - 1) / n_w;
                const uint32_t a0 = min(warp * per, NA), a1 = min(a0 + per, NA);
                write_rows(list_r[k], m, s, split, NB, a0, a1, xft_pairs, lane, comb_road,
                           comb_hits);
            }
            __syncthreads();   // the list is rebuilt for the next group
        }
    }
}

// acc_k = q_k 2^qshift + sum_l F_kl x_l exactly, with 32-bit products:
// |F_kl x_l| <= 32768 * 32767 < 2^30, so every sum of two products is exact
// in int32; the three pair sums and q_k 2^qshift (|.| < 2^39) are added in
// int64.  With oshift >= 9, |y_k| < 2^31 and y_k = floor(acc_k / 2^oshift) is
// exact in int32.  Results: chi2 over the three clamped chi rows, p_0..p_2.
__device__ __forceinline__ uint32_t fit_rows(const int32_t (&Fk)[36], const long long (&qk)[6],
                                             const int32_t (&x)[N_LAYERS], uint32_t oshift,
                                             int32_t (&p)[3]) {
    int32_t y[N_LAYERS];
#pragma unroll
    for (int k = 0; k < N_LAYERS; ++k) {
        int32_t s2[3];
#pragma unroll
        for (int m = 0; m < 3; ++m)
            s2[m] = Fk[k * 6 + 2 * m] * x[2 * m] + Fk[k * 6 + 2 * m + 1] * x[2 * m + 1];
        const long long acc = qk[k] + (long long)s2[0] + (long long)s2[1] + (long long)s2[2];
        y[k] = (int32_t)(acc >> oshift);   // arithmetic shift: floor
    }
    uint32_t chi2 = 0;
#pragma unroll
    for (int k = 3; k < N_LAYERS; ++k) {
        const int32_t c = max(min(y[k], 32767), -32767);
        chi2 += (uint32_t)(c * c);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = y[k];
    return chi2;
}

// One combination with every input read from global memory (road data, hit
// words, the sector/pattern row of the constants).
__device__ __forceinline__ uint32_t fit_direct(const uint32_t *__restrict__ words,
                                               const uint32_t *__restrict__ road_word,
                                               const uint32_t *__restrict__ road_nhit,
                                               const int16_t *__restrict__ F,
                                               const int16_t *__restrict__ q,
                                               const svt_config &cfg, uint32_t r, uint32_t hits,
                                               int32_t (&p)[3]) {
    const uint32_t rw = __ldg(road_word + r);
    const uint32_t packed = __ldg(road_nhit + r);
    const uint32_t hw = __ldg(words + rw);
    uint32_t mask = 0, hoff = rw + 1;
    int32_t x[N_LAYERS];
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) {
        const uint32_t nl = nhit_of(packed, l);
        x[l] = nl ? (int32_t)hit_coord(__ldg(words + hoff + ((hits >> (4 * l)) & 15u))) : 0;
        mask |= nl ? (1u << l) : 0u;
        hoff += nl;
    }
    const size_t cs = (size_t)rd_sector(hw) * 64 + mask;
    int32_t Fk[36];
    long long qk[6];
#pragma unroll
    for (int i = 0; i < 36; ++i) Fk[i] = __ldg(F + cs * 36 + i);
#pragma unroll
    for (int k = 0; k < 6; ++k)
        qk[k] = (long long)((unsigned long long)(long long)__ldg(q + cs * 6 + k) << cfg.qshift);
    return fit_rows(Fk, qk, x, cfg.oshift, p);
}

// A road's row staged in shared memory by the plain fit: its constants as
// int32, q_k 2^qshift as int64 and, per layer, the index of its first hit in
// the road's coordinate list (0xFF for a layer without hits); the road's hit
// coordinates sit beside it (at most 96: 6 layers x 16).
constexpr int FIT_THREADS = 256;
constexpr int FIT_PER_THREAD = 8;
constexpr int FIT_TILE = FIT_THREADS * FIT_PER_THREAD;   // combinations per block tile
constexpr int FIT_STAGE_ROADS = 64;   // tiles over more roads read their inputs directly
struct alignas(16) StagedRow {
    int32_t F[36];
    long long q[6];
    uint8_t first[8];
    uint32_t pad[2];
};

__device__ __forceinline__ uint32_t fit_staged(const StagedRow &row,
                                               const uint16_t *__restrict__ coord,
                                               uint32_t oshift, uint32_t hits, int32_t (&p)[3]) {
    const uint2 fw = *reinterpret_cast<const uint2 *>(row.first);
    int32_t x[N_LAYERS];
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) {
        const uint32_t f0 = ((l < 4 ? fw.x : fw.y) >> (8 * (l & 3))) & 0xFFu;
        x[l] = f0 != 0xFFu ? (int32_t)coord[f0 + ((hits >> (4 * l)) & 15u)] : 0;
    }
    int32_t Fk[36];
    long long qk[6];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int4 v = reinterpret_cast<const int4 *>(row.F)[i];
        Fk[4 * i] = v.x;
        Fk[4 * i + 1] = v.y;
        Fk[4 * i + 2] = v.z;
        Fk[4 * i + 3] = v.w;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const longlong2 v = reinterpret_cast<const longlong2 *>(row.q)[i];
        qk[2 * i] = v.x;
        qk[2 * i + 1] = v.y;
    }
    return fit_rows(Fk, qk, x, oshift, p);
}

// One thread per combination, over block tiles of FIT_TILE consecutive
// combinations (thread t takes combinations t, t + 256, t + 512, ... of the
// tile and loads their entries first; 48 registers leave five blocks per SM).  Combinations are road-major, so a
// tile covers the roads comb_road[first] .. comb_road[last]; when there are
// at most FIT_STAGE_ROADS of them, their rows and hit coordinates are staged
// in shared memory once (coalesced loads) and the combinations of the tile
// need no other global load; otherwise each reads its inputs directly.
__global__ void __launch_bounds__(FIT_THREADS, 5)
    k_fit_plain(const uint32_t *__restrict__ words, const uint32_t *__restrict__ road_word,
                const uint32_t *__restrict__ road_nhit, const uint32_t *__restrict__ comb_road,
                const uint32_t *__restrict__ comb_hits, const uint64_t *__restrict__ n_combs,
                uint64_t comb_cap, const int16_t *__restrict__ F, const int16_t *__restrict__ q,
                const svt_config cfg, uint32_t *fit_chi2, int32_t *fit_par,
                const unsigned long long *status) {
    __shared__ StagedRow rows[FIT_STAGE_ROADS];
    __shared__ uint16_t coords[FIT_STAGE_ROADS][N_LAYERS * MAX_HITS];
    __shared__ uint32_t tile_r0, tile_nr;
    if (!status_ok(status)) return;
    const uint64_t n = *n_combs < comb_cap ? *n_combs : comb_cap;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint64_t j0 = (uint64_t)blockIdx.x * FIT_TILE; j0 < n; j0 += (uint64_t)gridDim.x * FIT_TILE) {
        const uint64_t j1 = min(j0 + (uint64_t)FIT_TILE, n);
        uint32_t rr[FIT_PER_THREAD], hh[FIT_PER_THREAD];
#pragma unroll
        for (int i = 0; i < FIT_PER_THREAD; ++i) {
            const uint64_t j = j0 + (uint64_t)(i * FIT_THREADS) + threadIdx.x;
            rr[i] = j < j1 ? __ldg(comb_road + j) : 0u;
            hh[i] = j < j1 ? __ldg(comb_hits + j) : 0u;
        }
        if (threadIdx.x == 0) {
            const uint32_t r0 = __ldg(comb_road + j0), r1 = __ldg(comb_road + j1 - 1);
            tile_r0 = r0;
            tile_nr = r1 - r0 + 1;   // roads are non-decreasing in j
        }
        __syncthreads();
        const uint32_t r0 = tile_r0, nr = tile_nr;
        const bool staged = nr <= (uint32_t)FIT_STAGE_ROADS;
        if (staged) {
            // warp w stages roads w, w + 8, ...: lane i of the F row (lanes
            // 0..3 twice), lanes 4..9 the q row, lanes 10..15 the layers, and
            // every lane some of the hit coordinates
            for (uint32_t rho = warp; rho < nr; rho += FIT_THREADS / 32) {
                const uint32_t r = r0 + rho;
                const uint32_t rw = __ldg(road_word + r), packed = __ldg(road_nhit + r);
                uint32_t mask = 0, total = 0;
#pragma unroll
                for (int l = 0; l < N_LAYERS; ++l) {
                    mask |= nhit_of(packed, l) ? (1u << l) : 0u;
                    total += nhit_of(packed, l);
                }
                total = min(total, (uint32_t)(N_LAYERS * MAX_HITS));
                const size_t cs = (size_t)rd_sector(__ldg(words + rw)) * 64 + mask;
                StagedRow &row = rows[rho];
                row.F[lane] = __ldg(F + cs * 36 + lane);
                if (lane < 4) {
                    row.F[32 + lane] = __ldg(F + cs * 36 + 32 + lane);
                } else if (lane < 10) {
                    const int k = lane - 4;
                    row.q[k] = (long long)((unsigned long long)(long long)__ldg(q + cs * 6 + k)
                                           << cfg.qshift);
                } else if (lane < 16) {
                    const int l = lane - 10;
                    uint32_t before = 0;   // hits on the layers below l
#pragma unroll
                    for (int m = 0; m < N_LAYERS - 1; ++m) before += m < l ? nhit_of(packed, m) : 0u;
                    row.first[l] = nhit_of(packed, l) ? (uint8_t)before : (uint8_t)0xFF;
                }
                for (uint32_t h = lane; h < total; h += 32)
                    coords[rho][h] = (uint16_t)hit_coord(__ldg(words + rw + 1 + h));
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < FIT_PER_THREAD; ++i) {
            const uint64_t j = j0 + (uint64_t)(i * FIT_THREADS) + threadIdx.x;
            if (j < j1) {
                int32_t p[3];
                const uint32_t chi2 =
                    staged ? fit_staged(rows[rr[i] - r0], coords[rr[i] - r0], cfg.oshift, hh[i], p)
                           : fit_direct(words, road_word, road_nhit, F, q, cfg, rr[i], hh[i], p);
                fit_chi2[j] = chi2;
#pragma unroll
                for (int k = 0; k < 3; ++k) fit_par[k * comb_cap + j] = p[k];
            }
        }
        __syncthreads();   // rows are reused by the next tile
    }
}

// Best passing combination of road r from its chi2 values, over the threads
// [idx, idx + step, ...) of the warp (step 32) or block (step 256): each
// visits its combinations in increasing c (a block keeps eight loads per
// thread in flight), so a strict '<' keeps the smallest index among equal chi2; the
// (chi2, c) keys are then merged (over the block through red, when BIG).
// Written by thread idx 0.
template <bool BIG>
__device__ __forceinline__ void select_road(uint32_t r, const RoadMeta &m,
                                            const uint32_t *__restrict__ fit_chi2,
                                            const int32_t *__restrict__ fit_par,
                                            uint64_t comb_cap, uint32_t init_chi, uint32_t idx,
                                            uint32_t step, int lane, unsigned long long *red,
                                            svt_best *best) {
    uint32_t bchi = init_chi, bc = 0;
    if (!BIG && m.off + m.n <= comb_cap) {
        for (uint64_t c = idx; c < m.n; c += step) {
            const uint32_t v = __ldg(fit_chi2 + m.off + c);
            if (v < bchi) {
                bchi = v;
                bc = (uint32_t)c;
            }
        }
    } else if (m.off + m.n <= comb_cap) {
        for (uint64_t c0 = idx; c0 < m.n; c0 += 8ull * step) {
            uint32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint64_t c = c0 + (uint64_t)u * step;
                v[u] = c < m.n ? __ldg(fit_chi2 + m.off + c) : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (v[u] < bchi) {
                    bchi = v[u];
                    bc = (uint32_t)(c0 + (uint64_t)u * step);
                }
        }
    }
    unsigned long long key = bchi != init_chi ? (((unsigned long long)bchi << 32) | bc) : ~0ull;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, key, d);
        key = o < key ? o : key;
    }
    if (BIG) {
        if (lane == 0) red[threadIdx.x >> 5] = key;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) key = red[w] < key ? red[w] : key;
        __syncthreads();   // red is reused by the next road
    }
    if (idx == 0) {
        svt_best b;
        b.flags = m.word;
        if (key != ~0ull) {
            const uint32_t c = (uint32_t)key;
            b.flags |= SVT_FLAG_PASS;
            b.comb = c;
            b.chi2 = (uint32_t)(key >> 32);
            b.p[0] = fit_par[m.off + c];
            b.p[1] = fit_par[comb_cap + m.off + c];
            b.p[2] = fit_par[2 * comb_cap + m.off + c];
        } else {
            b.comb = 0xFFFFFFFFu;
            b.chi2 = 0;
            b.p[0] = b.p[1] = b.p[2] = 0;
        }
        best[r] = b;
    }
}

// Chi-square cut and best combination of each road: a road per warp (roads of
// at most PLAIN_BIG combinations), or a big road per block.
template <bool BIG>
__global__ void __launch_bounds__(256)
    k_select(const uint32_t *__restrict__ fit_chi2, const int32_t *__restrict__ fit_par,
             uint64_t comb_cap, const uint64_t *__restrict__ comb_off,
             const uint32_t *__restrict__ road_flags, const uint64_t *__restrict__ n_roads,
             uint64_t road_cap, const svt_config cfg, svt_best *best,
             const unsigned long long *status) {
    __shared__ unsigned long long red[8];
    __shared__ RoadMeta list[256];
    __shared__ uint32_t list_r[256], list_n;
    if (!status_ok(status)) return;
    const uint64_t R = road_count(n_roads, road_cap);
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t init_chi = cfg.chi2_cut == 0xFFFFFFFFu ? 0xFFFFFFFFu : cfg.chi2_cut + 1u;
    if (!BIG) {
        RoadMeta m = road_meta(comb_off, road_flags, R, warp0);
        for (uint64_t r = warp0; r < R; r += n_warps) {
            const RoadMeta next = road_meta(comb_off, road_flags, R, r + n_warps);
            if (m.n <= PLAIN_BIG)
                select_road<false>((uint32_t)r, m, fit_chi2, fit_par, comb_cap, init_chi,
                                   (uint32_t)lane, 32u, lane, red, best);
            m = next;
        }
    } else {
        for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x; g < R;
             g += (uint64_t)gridDim.x * blockDim.x) {
            const uint64_t r = g + threadIdx.x;
            const RoadMeta mine = road_meta(comb_off, road_flags, R, r);
            const uint32_t nb = big_roads_of_group(mine, r, mine.n > PLAIN_BIG, list, list_r,
                                                   &list_n);
            for (uint32_t k = 0; k < nb; ++k)
                select_road<true>(list_r[k], list[k], fit_chi2, fit_par, comb_cap, init_chi,
                                  threadIdx.x, blockDim.x, lane, red, best);
            __syncthreads();   // the list is rebuilt for the next group
        }
    }
}

__global__ void k_format(const svt_best *__restrict__ best, const uint32_t *__restrict__ words,
                         const uint32_t *__restrict__ road_word,
                         const uint64_t *__restrict__ n_roads, uint64_t road_cap, uint32_t *out,
                         const unsigned long long *status) {
    if (!status_ok(status)) return;
    const uint64_t R = road_count(n_roads, road_cap);
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const svt_best b = best[r];
        const uint32_t hw = __ldg(words + road_word[r]);
        uint32_t *o = out + r * 6;
        o[0] = rd_id(hw) | (b.flags << 24);
        o[1] = b.comb;
        o[2] = b.chi2;
        o[3] = (uint32_t)b.p[0];
        o[4] = (uint32_t)b.p[1];
        o[5] = (uint32_t)b.p[2];
    }
}

int grid_for(uint64_t n, int threads, int max_grid) {
    uint64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b < (uint64_t)max_grid ? b : (uint64_t)max_grid);
}

}  // namespace

void launch_combine_count(const uint32_t *road_nhit, const uint64_t *n_roads, uint64_t road_cap,
                          const svt_config cfg, uint32_t *road_flags, uint64_t *comb_cnt,
                          const unsigned long long *status, int grid, cudaStream_t st) {
    k_combine_count<<<grid_for(road_cap, 256, grid), 256, 0, st>>>(road_nhit, n_roads, road_cap,
                                                                   cfg, road_flags, comb_cnt,
                                                                   status);
}

void launch_scan_u64(uint64_t *a, const uint64_t *n_dev, uint64_t cap, uint64_t *tile_sums,
                     uint64_t *total, const unsigned long long *status, int grid, cudaStream_t st) {
    int g = grid_for(cap, SCAN_TILE, grid);
    k_scan_u64_reduce<<<g, SCAN_THREADS, 0, st>>>(a, n_dev, cap, tile_sums, status);
    k_scan_u64_tiles<<<1, 1024, 0, st>>>(tile_sums, n_dev, cap, status);
    k_scan_u64_apply<<<g, SCAN_THREADS, 0, st>>>(a, n_dev, cap, tile_sums, total, status);
}

size_t scan_u64_tile_count(uint64_t cap) { return (cap + SCAN_TILE - 1) / SCAN_TILE + 1; }

void launch_combine_write(const uint32_t *road_nhit, const uint64_t *n_roads, uint64_t road_cap,
                          const uint64_t *comb_off, uint64_t comb_cap, uint32_t xft_pairs,
                          uint32_t *comb_road, uint32_t *comb_hits, unsigned long long *status,
                          int grid, cudaStream_t st) {
    k_combine_write<false><<<grid_for(road_cap * 32, 256, grid), 256, 0, st>>>(
        road_nhit, n_roads, road_cap, comb_off, comb_cap, xft_pairs, comb_road, comb_hits, status);
    k_combine_write<true><<<grid_for(road_cap, 256, grid), 256, 0, st>>>(
        road_nhit, n_roads, road_cap, comb_off, comb_cap, xft_pairs, comb_road, comb_hits, status);
}

void launch_fit_plain(const uint32_t *words, const uint32_t *road_word, const uint32_t *road_nhit,
                      const uint32_t *comb_road, const uint32_t *comb_hits,
                      const uint64_t *n_combs, uint64_t comb_cap, const int16_t *F,
                      const int16_t *q, const svt_config cfg, uint32_t *fit_chi2,
                      int32_t *fit_par, const unsigned long long *status, int grid,
                      cudaStream_t st) {
    k_fit_plain<<<grid_for((comb_cap + FIT_TILE - 1) / FIT_TILE * FIT_THREADS, FIT_THREADS, grid),
                  FIT_THREADS, 0, st>>>(
        words, road_word, road_nhit, comb_road, comb_hits, n_combs, comb_cap, F, q, cfg, fit_chi2,
        fit_par, status);
}

void launch_select(const uint32_t *fit_chi2, const int32_t *fit_par, uint64_t comb_cap,
                   const uint64_t *comb_off, const uint32_t *road_flags, const uint64_t *n_roads,
                   uint64_t road_cap, const svt_config cfg, svt_best *best,
                   const unsigned long long *status, int grid, cudaStream_t st) {
    k_select<false><<<grid_for(road_cap * 32, 256, grid), 256, 0, st>>>(
        fit_chi2, fit_par, comb_cap, comb_off, road_flags, n_roads, road_cap, cfg, best, status);
    k_select<true><<<grid_for(road_cap, 256, grid), 256, 0, st>>>(
        fit_chi2, fit_par, comb_cap, comb_off, road_flags, n_roads, road_cap, cfg, best, status);
}

void launch_format(const svt_best *best, const uint32_t *words, const uint32_t *road_word,
                   const uint64_t *n_roads, uint64_t road_cap, uint32_t *out,
                   const unsigned long long *status, int grid, cudaStream_t st) {
    k_format<<<grid_for(road_cap, 256, grid), 256, 0, st>>>(best, words, road_word, n_roads,
                                                           road_cap, out, status);
}

}  // namespace svt
