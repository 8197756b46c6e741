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

__global__ void k_combine_write(const uint32_t *__restrict__ road_nhit,
                                const uint64_t *__restrict__ n_roads, uint64_t road_cap,
                                const uint64_t *__restrict__ comb_off, uint64_t comb_cap,
                                uint32_t xft_pairs, uint32_t *comb_road, uint32_t *comb_hits,
                                unsigned long long *status) {
    if (!status_ok(status)) return;
    const uint64_t R = road_count(n_roads, road_cap);
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    if (warp0 == 0 && lane == 0 && comb_off[R] > comb_cap) report(status, 0, SVT_ERR_OOM);
    for (uint64_t r = warp0; r < R; r += n_warps) {
        const uint64_t off = comb_off[r], n = comb_off[r + 1] - off;
        if (off + n > comb_cap) continue;
        const RoadShape s = road_shape(road_nhit[r], xft_pairs);
        uint32_t m[N_LAYERS];
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l) m[l] = kDivMagic[s.n[l]];
        for (uint64_t c = lane; c < n; c += 32) {
            uint32_t rem = (uint32_t)c, packed = 0;   // c < max_comb < 2^32
#pragma unroll
            for (int l = N_LAYERS - 1; l >= 0; --l) {
                const uint32_t qd = div_by(rem, s.n[l], m[l]);
                packed |= (rem - qd * s.n[l]) << (4 * l);
                rem = qd;
            }
            if (xft_pairs) packed |= ((packed >> 16) & 15u) << 20;   // layer 5 takes layer 4's hit
            comb_road[off + c] = (uint32_t)r;
            comb_hits[off + c] = packed;
        }
    }
}

__global__ void k_fit_plain(const uint32_t *__restrict__ words,
                            const uint32_t *__restrict__ road_word,
                            const uint32_t *__restrict__ road_nhit,
                            const uint32_t *__restrict__ comb_road,
                            const uint32_t *__restrict__ comb_hits,
                            const uint64_t *__restrict__ n_combs, uint64_t comb_cap,
                            const int16_t *__restrict__ F, const int16_t *__restrict__ q,
                            const svt_config cfg, uint32_t *fit_chi2, int32_t *fit_par,
                            const unsigned long long *status) {
    if (!status_ok(status)) return;
    const uint64_t n = *n_combs < comb_cap ? *n_combs : comb_cap;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = __ldg(comb_road + j);
        const uint32_t hits = __ldg(comb_hits + j);
        const uint32_t rw = __ldg(road_word + r);
        const uint32_t packed = __ldg(road_nhit + r);
        const uint32_t hw = __ldg(words + rw);
        uint32_t mask = 0, hoff = rw + 1;
        uint32_t x[N_LAYERS];
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l) {
            const uint32_t nl = nhit_of(packed, l);
            x[l] = nl ? hit_coord(__ldg(words + hoff + ((hits >> (4 * l)) & 15u))) : 0u;
            mask |= nl ? (1u << l) : 0u;
            hoff += nl;
        }
        const size_t cs = (size_t)rd_sector(hw) * 64 + mask;
        const int16_t *Fs = F + cs * 36;
        const int16_t *qs = q + cs * 6;
        // acc_k exactly, with 32-bit products: |F_kl x_l| <= 32768 * 32767 < 2^30,
        // so every sum of two products is exact in int32; the three pair sums
        // and q_k 2^qshift (|.| < 2^39) are added in int64.  With oshift >= 9,
        // |y_k| < 2^31 and y_k is exact in int32.
        int32_t y[N_LAYERS];
#pragma unroll
        for (int k = 0; k < N_LAYERS; ++k) {
            int32_t s2[3];
#pragma unroll
            for (int m = 0; m < 3; ++m)
                s2[m] = (int32_t)__ldg(Fs + k * 6 + 2 * m) * (int32_t)x[2 * m] +
                        (int32_t)__ldg(Fs + k * 6 + 2 * m + 1) * (int32_t)x[2 * m + 1];
            const long long acc =
                (long long)((unsigned long long)(long long)__ldg(qs + k) << cfg.qshift) +
                (long long)s2[0] + (long long)s2[1] + (long long)s2[2];
            y[k] = (int32_t)(acc >> cfg.oshift);   // arithmetic shift: floor
        }
        uint32_t chi2 = 0;
#pragma unroll
        for (int k = 3; k < N_LAYERS; ++k) {
            const int32_t c = max(min(y[k], 32767), -32767);
            chi2 += (uint32_t)(c * c);
        }
        fit_chi2[j] = chi2;
        fit_par[j] = y[0];
        fit_par[comb_cap + j] = y[1];
        fit_par[2 * comb_cap + j] = y[2];
    }
}

__global__ void k_select(const uint32_t *__restrict__ fit_chi2,
                         const int32_t *__restrict__ fit_par, uint64_t comb_cap,
                         const uint64_t *__restrict__ comb_off,
                         const uint32_t *__restrict__ road_flags,
                         const uint64_t *__restrict__ n_roads, uint64_t road_cap,
                         const svt_config cfg, svt_best *best,
                         const unsigned long long *status) {
    if (!status_ok(status)) return;
    const uint64_t R = road_count(n_roads, road_cap);
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t init_chi = cfg.chi2_cut == 0xFFFFFFFFu ? 0xFFFFFFFFu : cfg.chi2_cut + 1u;
    for (uint64_t r = warp0; r < R; r += n_warps) {
        const uint64_t off = comb_off[r], n = comb_off[r + 1] - off;
        uint32_t bchi = init_chi, bc = 0;
        if (off + n <= comb_cap) {
            for (uint64_t c = lane; c < n; c += 32) {
                const uint32_t chi2 = __ldg(fit_chi2 + off + c);
                if (chi2 < bchi) {   // c increases per lane: keeps the smallest index
                    bchi = chi2;
                    bc = (uint32_t)c;
                }
            }
        }
        unsigned long long key = bchi != init_chi ? (((unsigned long long)bchi << 32) | bc) : ~0ull;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            unsigned long long o = __shfl_xor_sync(0xffffffffu, key, d);
            key = o < key ? o : key;
        }
        if (lane == 0) {
            svt_best b;
            b.flags = road_flags[r];
            if (key != ~0ull) {
                const uint32_t c = (uint32_t)key;
                b.flags |= SVT_FLAG_PASS;
                b.comb = c;
                b.chi2 = (uint32_t)(key >> 32);
                b.p[0] = fit_par[off + c];
                b.p[1] = fit_par[comb_cap + off + c];
                b.p[2] = fit_par[2 * comb_cap + off + c];
            } else {
                b.comb = 0xFFFFFFFFu;
                b.chi2 = 0;
                b.p[0] = b.p[1] = b.p[2] = 0;
            }
            best[r] = b;
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
    k_combine_write<<<grid_for(road_cap * 32, 256, grid), 256, 0, st>>>(
        road_nhit, n_roads, road_cap, comb_off, comb_cap, xft_pairs, comb_road, comb_hits, status);
}

void launch_fit_plain(const uint32_t *words, const uint32_t *road_word, const uint32_t *road_nhit,
                      const uint32_t *comb_road, const uint32_t *comb_hits,
                      const uint64_t *n_combs, uint64_t comb_cap, const int16_t *F,
                      const int16_t *q, const svt_config cfg, uint32_t *fit_chi2,
                      int32_t *fit_par, const unsigned long long *status, int grid,
                      cudaStream_t st) {
    k_fit_plain<<<grid_for(comb_cap, 256, grid), 256, 0, st>>>(
        words, road_word, road_nhit, comb_road, comb_hits, n_combs, comb_cap, F, q, cfg, fit_chi2,
        fit_par, status);
}

void launch_select(const uint32_t *fit_chi2, const int32_t *fit_par, uint64_t comb_cap,
                   const uint64_t *comb_off, const uint32_t *road_flags, const uint64_t *n_roads,
                   uint64_t road_cap, const svt_config cfg, svt_best *best,
                   const unsigned long long *status, int grid, cudaStream_t st) {
    k_select<<<grid_for(road_cap * 32, 256, grid), 256, 0, st>>>(
        fit_chi2, fit_par, comb_cap, comb_off, road_flags, n_roads, road_cap, cfg, best, status);
}

void launch_format(const svt_best *best, const uint32_t *words, const uint32_t *road_word,
                   const uint64_t *n_roads, uint64_t road_cap, uint32_t *out,
                   const unsigned long long *status, int grid, cudaStream_t st) {
    k_format<<<grid_for(road_cap, 256, grid), 256, 0, st>>>(best, words, road_word, n_roads,
                                                           road_cap, out, status);
}

}  // namespace svt
