// svt_fused.cu -- combine + fit + chi-square cut + best-per-road + format of
// the paper's Sec. 2 / Sec. 2.1 in one persistent kernel.
//
// Design (GB300 first; the paper's Kepler port used one thread per
// combination and a separate kernel per stage):
//   * The fit is linear, so with the layers split into a prefix (rows, index
//     a) and a suffix (columns, index b) every accumulator is
//         acc_k(a, b) = A_k(a) + B_k(b),
//     A_k(a) = q_k 2^qshift + sum_{prefix l} F_kl x_l,  B_k(b) = sum_{suffix l} F_kl x_l,
//     exactly in int64.  A warp owns one work item -- up to rows_per_item rows
//     of one road -- builds the per-hit terms F_kl x_l and the item's A rows in
//     shared memory, and each lane holds the B of one column in registers.
//     One combination then costs three 64-bit adds, three funnel shifts,
//     the clamp, three multiply-adds and one compare.  Only the three chi rows
//     are evaluated in the loop; the parameters are recomputed once for the
//     winning combination.
//   * Work items come from a global atomic counter (dynamic load balance over
//     uneven roads); the road of an item is found by a 32-way warp search of
//     the per-road item offsets.
//   * Each lane visits its combinations in increasing c within a column, so a
//     strict '<' keeps the smallest index among equal chi2; across columns,
//     lanes and items the (chi2, c) pairs are merged as 64-bit keys with
//     atomicMin on the road's slot.  The warp that retires a road's last item
//     formats its record.
#include "svt_kernels.cuh"

namespace svt {

namespace {

constexpr int ROWS_MAX = 64;

struct WarpSmem {
    int32_t T[N_LAYERS * MAX_HITS * 3];   // chi-row terms F[3+k][l] * x, [l][i][k]
    int32_t cF[18];                       // F[3+k][l] at k*6+l
    int32_t cq[3];
    int32_t pad[3];
    longlong2 A[ROWS_MAX][2];             // (A3, A4), (A5, -)
};

// K3: item offsets per road, road slots, records of roads that are not fitted
__global__ void __launch_bounds__(TILE_THREADS)
    k_items(const uint32_t *__restrict__ words, const uint32_t *__restrict__ road_word,
            const uint32_t *__restrict__ road_nhit, uint64_t road_cap,
            const Dims *__restrict__ dims, const uint32_t *__restrict__ tile_roads,
            const uint32_t *__restrict__ tile_items, const uint32_t *__restrict__ road_items,
            uint32_t *road_item_off, unsigned long long *road_best, uint32_t *road_pending,
            uint32_t *out, uint32_t *item_counter, unsigned long long *status) {
    __shared__ uint32_t red[TILE_THREADS / 32 + 1];
    if (!status_ok(status)) return;
    const uint64_t T = n_tiles(dims->n_words);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *item_counter = 0;
        uint64_t R = tile_roads[T];
        if (R <= road_cap) road_item_off[R] = tile_items[T];
    }
    for (uint64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const uint64_t r0 = tile_roads[t], r1 = tile_roads[t + 1];
        const uint64_t rb = r0 + (uint64_t)threadIdx.x * TILE_PER_THREAD;
        uint32_t w[TILE_PER_THREAD], s = 0;
#pragma unroll
        for (int j = 0; j < TILE_PER_THREAD; ++j) {
            w[j] = (rb + j < r1 && rb + j < road_cap) ? road_items[rb + j] : 0u;
            s += w[j];
        }
        uint32_t total;
        uint32_t run = tile_items[t] + block_exclusive_scan<uint32_t>(s, red, &total);
#pragma unroll
        for (int j = 0; j < TILE_PER_THREAD; ++j) {
            const uint64_t r = rb + j;
            if (r >= r1 || r >= road_cap) break;
            road_item_off[r] = run;
            run += w[j];
            road_pending[r] = w[j];
            road_best[r] = ~0ull;
            if (w[j] == 0) {   // fewer layers than min_layers: not fitted
                const uint32_t hw = __ldg(words + road_word[r]);
                const uint32_t flags = SVT_FLAG_BAD_PATTERN |
                                       (road_nhit[r] == 0 ? SVT_FLAG_NO_HITS : 0u);
                uint32_t *o = out + r * 6;
                o[0] = rd_id(hw) | (flags << 24);
                o[1] = 0xFFFFFFFFu;
                o[2] = 0; o[3] = 0; o[4] = 0; o[5] = 0;
            }
        }
    }
}

// largest r in [0, R) with off[r] <= it (off non-decreasing, off[0] = 0)
__device__ __forceinline__ uint32_t find_road(const uint32_t *__restrict__ off, uint32_t R,
                                              uint32_t it, int lane) {
    uint32_t lo = 0, hi = R;
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

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
        v = o < v ? o : v;
    }
    return v;
}

__device__ __forceinline__ int32_t clamp_chi(int32_t y) { return max(min(y, 32767), -32767); }

// Record of road r from its best key (called by the warp that retires the road).
__device__ void format_road(const uint32_t *__restrict__ words, uint32_t rw, uint32_t packed,
                            const int16_t *__restrict__ F, const int16_t *__restrict__ q,
                            const svt_config &cfg, unsigned long long best, uint32_t *o,
                            uint64_t *counts, int lane) {
    const RoadShape s = road_shape(packed);
    const uint32_t hw = __ldg(words + rw);
    const uint32_t sector = rd_sector(hw);
    const bool pass = best != ~0ull;
    uint32_t flags = 0;
    if (s.total_hits == 0) flags |= SVT_FLAG_NO_HITS;
    if (s.C > cfg.max_comb) flags |= SVT_FLAG_OVERFLOW;
    if (pass) flags |= SVT_FLAG_PASS;
    int32_t p = 0;
    const uint32_t c = (uint32_t)best;
    if (pass && lane < 3) {
        uint32_t rem = c, idx[N_LAYERS];
#pragma unroll
        for (int l = N_LAYERS - 1; l >= 0; --l) {
            idx[l] = rem % s.n[l];
            rem /= s.n[l];
        }
        const size_t cs = (size_t)sector * 64 + s.mask;
        long long acc = (long long)__ldg(q + cs * 6 + lane) * (1ll << cfg.qshift);
        uint32_t hoff = rw + 1;
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l) {
            const uint32_t nl = nhit_of(packed, l);
            const uint32_t x = nl ? hit_coord(__ldg(words + hoff + idx[l])) : 0u;
            acc += (long long)__ldg(F + cs * 36 + lane * 6 + l) * (long long)x;
            hoff += nl;
        }
        p = (int32_t)(acc >> cfg.oshift);   // arithmetic shift: floor
    }
    const int32_t p0 = __shfl_sync(0xffffffffu, p, 0);
    const int32_t p1 = __shfl_sync(0xffffffffu, p, 1);
    const int32_t p2 = __shfl_sync(0xffffffffu, p, 2);
    if (lane == 0) {
        o[0] = rd_id(hw) | (flags << 24);
        o[1] = pass ? c : 0xFFFFFFFFu;
        o[2] = pass ? (uint32_t)(best >> 32) : 0u;
        o[3] = (uint32_t)p0;
        o[4] = (uint32_t)p1;
        o[5] = (uint32_t)p2;
        if (pass && counts) atomicAdd((unsigned long long *)(counts + 3), 1ull);
    }
}

// K4: persistent fit / cut / select / format
__global__ void k_fit_persistent(const uint32_t *__restrict__ words,
                                 const uint32_t *__restrict__ road_word,
                                 const uint32_t *__restrict__ road_nhit,
                                 const uint32_t *__restrict__ road_item_off,
                                 const uint64_t *__restrict__ n_roads_p, uint64_t road_cap,
                                 const uint64_t *__restrict__ total_items_p,
                                 const int16_t *__restrict__ F, const int16_t *__restrict__ q,
                                 const svt_config cfg, uint32_t rows_per_item,
                                 unsigned long long *road_best, uint32_t *road_pending,
                                 uint32_t *out, uint32_t *item_counter, uint64_t *counts,
                                 unsigned long long *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem &sm = reinterpret_cast<WarpSmem *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    if (!status_ok(status)) return;
    const uint64_t R64 = *n_roads_p;
    if (R64 > road_cap || R64 == 0) return;
    const uint32_t R = (uint32_t)R64;
    const uint64_t total_items64 = *total_items_p;
    if (total_items64 > 0xFFFFFFFFull) return;
    const uint32_t total_items = (uint32_t)total_items64;
    const uint32_t os = cfg.oshift;
    const uint32_t init_chi = cfg.chi2_cut == 0xFFFFFFFFu ? 0xFFFFFFFFu : cfg.chi2_cut + 1u;

    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(item_counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= total_items) break;
        const uint32_t r = find_road(road_item_off, R, it, lane);
        const uint32_t k_item = it - __ldg(road_item_off + r);
        const uint32_t rw = __ldg(road_word + r);
        const uint32_t packed = __ldg(road_nhit + r);
        const uint32_t hw = __ldg(words + rw);
        const RoadShape s = road_shape(packed);
        const uint32_t C = (uint32_t)s.C;
        const uint32_t C_eval = C > cfg.max_comb ? cfg.max_comb : C;
        uint32_t split, NB;
        road_split(s, split, NB);
        const uint32_t NA = (C_eval + NB - 1) / NB;
        const uint32_t a_lo = k_item * rows_per_item;
        const uint32_t a_hi = min(a_lo + rows_per_item, NA);

        // constants of the chi rows for (sector, mask)
        const size_t cs = (size_t)rd_sector(hw) * 64 + s.mask;
        if (lane < 18) sm.cF[lane] = __ldg(F + cs * 36 + 18 + lane);
        else if (lane < 21) sm.cq[lane - 18] = __ldg(q + cs * 6 + 3 + (lane - 18));
        // layers without hits contribute x = 0
        if (lane < N_LAYERS && nhit_of(packed, lane) == 0) {
            sm.T[(lane * MAX_HITS) * 3 + 0] = 0;
            sm.T[(lane * MAX_HITS) * 3 + 1] = 0;
            sm.T[(lane * MAX_HITS) * 3 + 2] = 0;
        }
        __syncwarp();
        // per-hit terms
        for (uint32_t h = lane; h < s.total_hits; h += 32) {
            const uint32_t x = __ldg(words + rw + 1 + h);
            const uint32_t l = hit_layer(x);
            uint32_t i = h;
#pragma unroll
            for (int ll = 0; ll < N_LAYERS; ++ll)
                if ((uint32_t)ll < l) i -= nhit_of(packed, ll);
            const int32_t xc = (int32_t)hit_coord(x);
            int32_t *t = sm.T + (l * MAX_HITS + i) * 3;
            t[0] = sm.cF[0 * 6 + l] * xc;
            t[1] = sm.cF[1 * 6 + l] * xc;
            t[2] = sm.cF[2 * 6 + l] * xc;
        }
        SmallDiv dv[N_LAYERS];
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l) dv[l] = make_div(s.n[l]);
        __syncwarp();
        // A rows of this item
        if ((uint32_t)lane < a_hi - a_lo) {
            uint32_t rem = a_lo + lane;
            long long A3 = (long long)sm.cq[0] * (1ll << cfg.qshift);
            long long A4 = (long long)sm.cq[1] * (1ll << cfg.qshift);
            long long A5 = (long long)sm.cq[2] * (1ll << cfg.qshift);
#pragma unroll
            for (int l = N_LAYERS - 1; l >= 0; --l) {
                if ((uint32_t)l < split) {
                    const uint32_t qd = div_small(rem, dv[l]);
                    const uint32_t i = rem - qd * s.n[l];
                    rem = qd;
                    const int32_t *t = sm.T + (l * MAX_HITS + i) * 3;
                    A3 += t[0];
                    A4 += t[1];
                    A5 += t[2];
                }
            }
            sm.A[lane][0] = make_longlong2(A3, A4);
            sm.A[lane][1] = make_longlong2(A5, 0);
        }
        if (lane + 32 < (int)(a_hi - a_lo)) {
            uint32_t rem = a_lo + lane + 32;
            long long A3 = (long long)sm.cq[0] * (1ll << cfg.qshift);
            long long A4 = (long long)sm.cq[1] * (1ll << cfg.qshift);
            long long A5 = (long long)sm.cq[2] * (1ll << cfg.qshift);
#pragma unroll
            for (int l = N_LAYERS - 1; l >= 0; --l) {
                if ((uint32_t)l < split) {
                    const uint32_t qd = div_small(rem, dv[l]);
                    const uint32_t i = rem - qd * s.n[l];
                    rem = qd;
                    const int32_t *t = sm.T + (l * MAX_HITS + i) * 3;
                    A3 += t[0];
                    A4 += t[1];
                    A5 += t[2];
                }
            }
            sm.A[lane + 32][0] = make_longlong2(A3, A4);
            sm.A[lane + 32][1] = make_longlong2(A5, 0);
        }
        __syncwarp();

        unsigned long long best = ~0ull;
        for (uint32_t b0 = 0; b0 < NB; b0 += 32) {
            const uint32_t b = b0 + lane;
            long long B3 = 0, B4 = 0, B5 = 0;
            {
                uint32_t rem = b;
#pragma unroll
                for (int l = N_LAYERS - 1; l >= 0; --l) {
                    if ((uint32_t)l >= split) {
                        const uint32_t qd = div_small(rem, dv[l]);
                        const uint32_t i = min(rem - qd * s.n[l], (uint32_t)MAX_HITS - 1);
                        rem = qd;
                        const int32_t *t = sm.T + (l * MAX_HITS + i) * 3;
                        B3 += t[0];
                        B4 += t[1];
                        B5 += t[2];
                    }
                }
            }
            uint32_t a_end = a_hi;
            if (b >= NB)
                a_end = a_lo;
            else if (a_hi == NA && (NA - 1) * NB + b >= C_eval)
                a_end = a_hi - 1;
            uint32_t bchi = init_chi, bc = 0;
            uint32_t c = a_lo * NB + b;
            const longlong2 *Ap = &sm.A[0][0];
            for (uint32_t a = a_lo; a < a_end; ++a, c += NB, Ap += 2) {
                const longlong2 v01 = Ap[0];
                const longlong2 v2 = Ap[1];
                const long long s3 = v01.x + B3, s4 = v01.y + B4, s5 = v2.x + B5;
                const int32_t y3 = clamp_chi((int32_t)__funnelshift_r((uint32_t)s3, (uint32_t)(s3 >> 32), os));
                const int32_t y4 = clamp_chi((int32_t)__funnelshift_r((uint32_t)s4, (uint32_t)(s4 >> 32), os));
                const int32_t y5 = clamp_chi((int32_t)__funnelshift_r((uint32_t)s5, (uint32_t)(s5 >> 32), os));
                const uint32_t chi2 = (uint32_t)(y3 * y3) + (uint32_t)(y4 * y4) + (uint32_t)(y5 * y5);
                if (chi2 < bchi) {
                    bchi = chi2;
                    bc = c;
                }
            }
            if (bchi != init_chi) {
                const unsigned long long key = ((unsigned long long)bchi << 32) | bc;
                best = key < best ? key : best;
            }
        }
        best = warp_min64(best);
        uint32_t last = 0;
        if (lane == 0) {
            if (best != ~0ull) atomicMin(road_best + r, best);
            __threadfence();
            last = (atomicSub(road_pending + r, 1u) == 1u) ? 1u : 0u;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            const unsigned long long fb = __ldcg(road_best + r);
            format_road(words, rw, packed, F, q, cfg, fb, out + (size_t)r * 6, counts, lane);
        }
        __syncwarp();
    }
}

}  // namespace

void launch_items(const uint32_t *words, const uint32_t *road_word, const uint32_t *road_nhit,
                  uint64_t road_cap, const Dims *dims,
                  uint64_t max_words, const uint32_t *tile_roads, const uint32_t *tile_items,
                  const uint32_t *road_items, uint32_t *road_item_off,
                  unsigned long long *road_best, uint32_t *road_pending, uint32_t *out,
                  uint32_t *item_counter, unsigned long long *status, int grid,
                  cudaStream_t st) {
    uint64_t T = n_tiles(max_words);
    int g = (int)(T < (uint64_t)grid ? T : (uint64_t)grid);
    if (g < 1) g = 1;
    k_items<<<g, TILE_THREADS, 0, st>>>(words, road_word, road_nhit, road_cap, dims, tile_roads,
                                       tile_items, road_items, road_item_off, road_best,
                                       road_pending, out, item_counter, status);
}

size_t fit_smem_bytes(int warps_per_block) { return sizeof(WarpSmem) * (size_t)warps_per_block; }

int fit_persistent_blocks_per_sm(int warps_per_block, uint32_t rows_per_item) {
    (void)rows_per_item;
    int n = 0;
    size_t smem = fit_smem_bytes(warps_per_block);
    cudaFuncSetAttribute(k_fit_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fit_persistent, warps_per_block * 32,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_fit_persistent(const uint32_t *words, const uint32_t *road_word,
                                  const uint32_t *road_nhit, const uint32_t *road_item_off,
                                  const uint64_t *n_roads, uint64_t road_cap,
                                  const uint64_t *total_items, const int16_t *F,
                                  const int16_t *q, const svt_config cfg, uint32_t rows_per_item,
                                  unsigned long long *road_best, uint32_t *road_pending,
                                  uint32_t *out, uint32_t *item_counter, uint64_t *counts,
                                  unsigned long long *status, int warps_per_block, int grid,
                                  cudaStream_t st) {
    size_t smem = fit_smem_bytes(warps_per_block);
    k_fit_persistent<<<grid, warps_per_block * 32, smem, st>>>(
        words, road_word, road_nhit, road_item_off, n_roads, road_cap, total_items, F, q, cfg,
        rows_per_item, road_best, road_pending, out, item_counter, counts, status);
    return cudaGetLastError();
}

}  // namespace svt
