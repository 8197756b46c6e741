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
//   * Each lane visits its combinations in increasing c within a column, so a
//     strict '<' keeps the smallest index among equal chi2; across columns,
//     lanes and items the (chi2, c) pairs are merged as 64-bit keys (warp
//     shuffles; atomicMin on the road's slot for split roads, whose record is
//     written by the warp that retires the road's last item).
#include "svt_kernels.cuh"

namespace svt {

namespace {

constexpr int ROWS_MAX = 64;

// All accumulator terms are kept multiplied by 2^(32 - oshift): the high word
// of a 64-bit sum of such terms is then exactly floor(sum / 2^oshift).
struct WarpSmem {
    long long T[N_LAYERS * MAX_HITS * 3]; // chi-row terms F[3+k][l] * x * 2^(32-oshift), [l][i][k]
    longlong2 S[32][2];                   // suffix sums below the top suffix layer, [b'](3 rows)
    longlong2 A[ROWS_MAX][2];             // prefix sums incl. q, per row: (A3, A4), (A5, -)
    int32_t cF[18];                       // F[3+k][l] at k*6+l
    int32_t cq[3];
    int32_t pad[3];
    SmallDiv dv[N_LAYERS];                // exact division by n'_l
    uint32_t n[N_LAYERS];                 // n'_l = max(n_l, 1)
    // road geometry (warp-uniform): c = a * NB + b, b = i_top * NBp + b'
    uint32_t split, NB, NA, C_eval, NBp, d_hi, d_lo, total_hits;
};

// K3: the list of split roads
__global__ void __launch_bounds__(TILE_THREADS)
    k_big_list(const uint4 *__restrict__ desc, uint64_t road_cap, const Dims *__restrict__ dims,
               const uint32_t *__restrict__ tile_roads, const uint32_t *__restrict__ tile_big,
               const uint32_t *__restrict__ tile_bigitems, const FusedRoads fr, BigList bl,
               unsigned long long *status) {
    __shared__ uint32_t red[TILE_THREADS / 32 + 1];
    if (!status_ok(status)) return;
    const uint64_t T = n_tiles(dims->n_words);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bl.counters[0] = 0;
        bl.counters[1] = 0;
        bl.item_off[tile_big[T]] = tile_bigitems[T];
    }
    for (uint64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const uint64_t r0 = tile_roads[t], r1 = min((uint64_t)tile_roads[t + 1], road_cap);
        const uint64_t rb = r0 + (uint64_t)threadIdx.x * TILE_PER_THREAD;
        uint32_t it[TILE_PER_THREAD], n_it = 0, n_big = 0;
#pragma unroll
        for (int j = 0; j < TILE_PER_THREAD; ++j) {
            it[j] = 0;
            if (rb + j < r1) {
                const uint4 d = desc[rb + j];
                it[j] = road_big_items(d.y, d.w, fr);
            }
            n_it += it[j];
            n_big += it[j] ? 1u : 0u;
        }
        uint32_t tot;
        uint32_t item_run = tile_bigitems[t] + block_exclusive_scan<uint32_t>(n_it, red, &tot);
        uint32_t big_run = tile_big[t] + block_exclusive_scan<uint32_t>(n_big, red, &tot);
#pragma unroll
        for (int j = 0; j < TILE_PER_THREAD; ++j) {
            if (!it[j]) continue;
            bl.road[big_run] = (uint32_t)(rb + j);
            bl.item_off[big_run] = item_run;
            bl.best[big_run] = ~0ull;
            bl.pending[big_run] = it[j];
            big_run += 1;
            item_run += it[j];
        }
    }
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

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
        v = o < v ? o : v;
    }
    return v;
}

__device__ __forceinline__ int32_t clamp_chi(int32_t y) { return max(min(y, 32767), -32767); }

// Constants of the chi rows, per-hit terms and suffix table of road D in the
// warp's slot.
__device__ __forceinline__ void road_setup(WarpSmem &sm, const uint32_t *__restrict__ words,
                                           const uint4 D, const int16_t *__restrict__ F,
                                           const int16_t *__restrict__ q, uint32_t sh, int lane) {
    const uint32_t packed = D.y;
    if (lane == 0) {
        const RoadShape rs = road_shape(packed);
        uint32_t split, NB;
        road_split(rs, split, NB);
        uint32_t ntop = 1;
#pragma unroll
        for (int l = 0; l < N_LAYERS; ++l)
            if ((uint32_t)l == split) ntop = rs.n[l];
        const uint32_t NBp = NB / ntop;
        sm.split = split;
        sm.NB = NB;
        sm.C_eval = D.w;
        sm.NA = (D.w + NB - 1) / NB;
        sm.NBp = NBp;
        sm.d_hi = 32u / NBp;
        sm.d_lo = 32u - (32u / NBp) * NBp;
        sm.total_hits = rs.total_hits;
    }
    if (lane < N_LAYERS) {
        const uint32_t nl = nhit_of(packed, lane);
        sm.n[lane] = nl ? nl : 1u;
        sm.dv[lane] = make_div(nl ? nl : 1u);
    }
    uint32_t mask = 0;
#pragma unroll
    for (int l = 0; l < N_LAYERS; ++l) mask |= nhit_of(packed, l) ? (1u << l) : 0u;
    const size_t cs = (size_t)rd_sector(D.z) * 64 + mask;
    if (lane < 18) sm.cF[lane] = __ldg(F + cs * 36 + 18 + lane);
    else if (lane < 21) sm.cq[lane - 18] = __ldg(q + cs * 6 + 3 + (lane - 18));
    // layers without hits contribute x = 0
    if (lane < N_LAYERS && nhit_of(packed, lane) == 0) {
        sm.T[(lane * MAX_HITS) * 3 + 0] = 0;
        sm.T[(lane * MAX_HITS) * 3 + 1] = 0;
        sm.T[(lane * MAX_HITS) * 3 + 2] = 0;
    }
    __syncwarp();
    const uint32_t total_hits = sm.total_hits;
    for (uint32_t h = lane; h < total_hits; h += 32) {
        const uint32_t x = __ldg(words + D.x + 1 + h);
        const uint32_t l = hit_layer(x);
        uint32_t i = h;
#pragma unroll
        for (int ll = 0; ll < N_LAYERS; ++ll)
            if ((uint32_t)ll < l) i -= nhit_of(packed, ll);
        const int32_t xc = (int32_t)hit_coord(x);
        long long *t = sm.T + (l * MAX_HITS + i) * 3;
        t[0] = (long long)(sm.cF[0 * 6 + l] * xc) << sh;
        t[1] = (long long)(sm.cF[1 * 6 + l] * xc) << sh;
        t[2] = (long long)(sm.cF[2 * 6 + l] * xc) << sh;
    }
    __syncwarp();
    // S[b'] = sum over the suffix layers below the top one, b' < NBp (< 32)
    const uint32_t split = sm.split;
    if ((uint32_t)lane < sm.NBp) {
        uint32_t rem = lane;
        long long S3 = 0, S4 = 0, S5 = 0;
#pragma unroll
        for (int l = N_LAYERS - 1; l >= 1; --l) {
            if ((uint32_t)l > split) {
                const uint32_t qd = div_small(rem, sm.dv[l]);
                const uint32_t i = rem - qd * sm.n[l];
                rem = qd;
                const long long *t = sm.T + (l * MAX_HITS + i) * 3;
                S3 += t[0];
                S4 += t[1];
                S5 += t[2];
            }
        }
        sm.S[lane][0] = make_longlong2(S3, S4);
        sm.S[lane][1] = make_longlong2(S5, 0);
    }
    __syncwarp();
}

__device__ __forceinline__ void build_row(WarpSmem &sm, uint32_t split, uint32_t a,
                                          uint32_t slot, uint32_t qsh) {
    uint32_t rem = a;
    long long A3 = (long long)sm.cq[0] << qsh;
    long long A4 = (long long)sm.cq[1] << qsh;
    long long A5 = (long long)sm.cq[2] << qsh;
#pragma unroll
    for (int l = N_LAYERS - 1; l >= 0; --l) {
        if ((uint32_t)l < split) {
            const uint32_t qd = div_small(rem, sm.dv[l]);
            const uint32_t i = rem - qd * sm.n[l];
            rem = qd;
            const long long *t = sm.T + (l * MAX_HITS + i) * 3;
            A3 += t[0];
            A4 += t[1];
            A5 += t[2];
        }
    }
    sm.A[slot][0] = make_longlong2(A3, A4);
    sm.A[slot][1] = make_longlong2(A5, 0);
}

__device__ __forceinline__ int32_t hi_word(long long v) {
    return (int32_t)((unsigned long long)v >> 32);
}

// Best (chi2 << 32 | c) over rows [a_lo, a_hi) of the road, reduced over the
// warp.  NOCLAMP (valid when chi2_cut < 32767^2): the squares are summed
// unclamped in 64 bits; any combination with a chi component of magnitude
// 32767 or more then exceeds the cut under both readings, and below that the
// clamp is the identity, so pass/fail, chi2 of passing combinations and the
// argmin are unchanged.
template <bool NOCLAMP>
__device__ __forceinline__ unsigned long long eval_rows(WarpSmem &sm, uint32_t a_lo,
                                                        uint32_t a_hi, uint32_t qsh,
                                                        uint32_t init_chi, int lane) {
    unsigned long long best = ~0ull;
    const uint32_t NB = sm.NB, NA = sm.NA, C_eval = sm.C_eval, NBp = sm.NBp;
    const uint32_t top = sm.split, d_lo = sm.d_lo, d_hi = sm.d_hi;
    const uint32_t is0 = (uint32_t)lane / NBp, bp0 = (uint32_t)lane - is0 * NBp;
    for (uint32_t ac = a_lo; ac < a_hi; ac += ROWS_MAX) {
        const uint32_t ae = min(ac + (uint32_t)ROWS_MAX, a_hi);
        if (ac + lane < ae) build_row(sm, top, ac + lane, lane, qsh);
        if (ac + lane + 32 < ae) build_row(sm, top, ac + lane + 32, lane + 32, qsh);
        __syncwarp();
        uint32_t is = is0, bp = bp0;   // column b = is * NBp + bp
        for (uint32_t b0 = 0; b0 < NB; b0 += 32) {
            const uint32_t b = b0 + (uint32_t)lane;
            if (b < NB) {
                const long long *t = sm.T + (top * MAX_HITS + is) * 3;
                const longlong2 s01 = sm.S[bp][0], s2 = sm.S[bp][1];
                const long long B3 = t[0] + s01.x, B4 = t[1] + s01.y, B5 = t[2] + s2.x;
                uint32_t a_end = ae;
                if (ae == NA && (NA - 1) * NB + b >= C_eval) a_end = ae - 1;
                uint32_t bchi = init_chi, ba = 0;
                const longlong2 *Ap = &sm.A[0][0];
#pragma unroll 4
                for (uint32_t a = ac; a < a_end; ++a, Ap += 2) {
                    const longlong2 v01 = Ap[0];
                    const longlong2 v2 = Ap[1];
                    const int32_t y3 = hi_word(v01.x + B3);
                    const int32_t y4 = hi_word(v01.y + B4);
                    const int32_t y5 = hi_word(v2.x + B5);
                    if (NOCLAMP) {
                        unsigned long long v = (unsigned long long)((long long)y3 * y3);
                        v += (unsigned long long)((long long)y4 * y4);
                        v += (unsigned long long)((long long)y5 * y5);
                        if (v < (unsigned long long)bchi) {
                            bchi = (uint32_t)v;
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
                    const unsigned long long key = ((unsigned long long)bchi << 32) | (ba * NB + b);
                    best = key < best ? key : best;
                }
            }
            bp += d_lo;
            is += d_hi;
            if (bp >= NBp) {
                bp -= NBp;
                is += 1;
            }
        }
        __syncwarp();
    }
    return warp_min64(best);
}

// Record of a road from its best key (all lanes call; lanes 0..2 recompute p).
__device__ __forceinline__ void format_road(const uint32_t *__restrict__ words, const uint4 D,
                            const int16_t *__restrict__ F, const int16_t *__restrict__ q,
                            const svt_config &cfg, unsigned long long best, uint32_t *o,
                            uint64_t *counts, int lane) {
    const uint32_t packed = D.y;
    const RoadShape s = road_shape(packed);
    const bool pass = best != ~0ull;
    uint32_t flags = 0;
    if (s.total_hits == 0) flags |= SVT_FLAG_NO_HITS;
    if (s.n_layers_hit < cfg.min_layers)
        flags |= SVT_FLAG_BAD_PATTERN;
    else if (s.C > cfg.max_comb)
        flags |= SVT_FLAG_OVERFLOW;
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
        const size_t cs = (size_t)rd_sector(D.z) * 64 + s.mask;
        long long acc = (long long)__ldg(q + cs * 6 + lane) * (1ll << cfg.qshift);
        uint32_t hoff = D.x + 1;
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
        o[0] = rd_id(D.z) | (flags << 24);
        o[1] = pass ? c : 0xFFFFFFFFu;
        o[2] = pass ? (uint32_t)(best >> 32) : 0u;
        o[3] = (uint32_t)p0;
        o[4] = (uint32_t)p1;
        o[5] = (uint32_t)p2;
        if (pass && counts) atomicAdd((unsigned long long *)(counts + 3), 1ull);
    }
}

// K4: persistent fit / cut / select / format
template <bool NOCLAMP>
__global__ void __launch_bounds__(512, 2) k_fit_persistent(const uint32_t *__restrict__ words,
                                 const uint4 *__restrict__ desc,
                                 const uint64_t *__restrict__ counts_in, uint64_t road_cap,
                                 const uint64_t *__restrict__ n_big_p,
                                 const int16_t *__restrict__ F, const int16_t *__restrict__ q,
                                 const svt_config cfg, const FusedRoads fr,
                                 uint32_t roads_per_chunk, BigList bl, uint32_t *out,
                                 uint64_t *counts, unsigned long long *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem &sm = reinterpret_cast<WarpSmem *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    if (!status_ok(status)) return;
    const uint64_t R64 = counts_in[0];
    if (R64 > road_cap || R64 == 0) return;
    const uint32_t R = (uint32_t)R64;
    const uint64_t n_items64 = counts_in[1];
    if (n_items64 > 0xFFFFFFFFull) return;
    const uint32_t n_items = (uint32_t)n_items64;
    const uint32_t n_big = (uint32_t)*n_big_p;
    const uint32_t sh = 32u - cfg.oshift, qsh = cfg.qshift + sh;
    const uint32_t init_chi = cfg.chi2_cut == 0xFFFFFFFFu ? 0xFFFFFFFFu : cfg.chi2_cut + 1u;

    // phase 1: items of split roads
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(bl.counters + 0, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const uint32_t j = find_slot(bl.item_off, n_big, it, lane);
        const uint32_t r = __ldg(bl.road + j);
        const uint32_t k = it - __ldg(bl.item_off + j);
        const uint4 D = __ldg(desc + r);
        road_setup(sm, words, D, F, q, sh, lane);
        const uint32_t a_lo = k * fr.rows;
        const uint32_t a_hi = min(a_lo + fr.rows, sm.NA);
        const unsigned long long best = eval_rows<NOCLAMP>(sm, a_lo, a_hi, qsh, init_chi, lane);
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
            format_road(words, D, F, q, cfg, fb, out + (size_t)r * 6, counts, lane);
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
        uint4 d = make_uint4(0, 0, 0, 0);
        if ((uint32_t)lane < n) d = __ldg(desc + c0 + lane);
        for (uint32_t jj = 0; jj < n; ++jj) {
            uint4 D;
            D.x = __shfl_sync(0xffffffffu, d.x, jj);
            D.y = __shfl_sync(0xffffffffu, d.y, jj);
            D.z = __shfl_sync(0xffffffffu, d.z, jj);
            D.w = __shfl_sync(0xffffffffu, d.w, jj);
            if (D.w > fr.small_max) continue;   // split road: done in phase 1
            unsigned long long best = ~0ull;
            if (D.w > 0) {
                road_setup(sm, words, D, F, q, sh, lane);
                best = eval_rows<NOCLAMP>(sm, 0, sm.NA, qsh, init_chi, lane);
            }
            format_road(words, D, F, q, cfg, best, out + (size_t)(c0 + jj) * 6, counts, lane);
            __syncwarp();
        }
    }
}

}  // namespace

void launch_big_list(const uint4 *desc, uint64_t road_cap, const Dims *dims, uint64_t max_words,
                     const uint32_t *tile_roads, const uint32_t *tile_big,
                     const uint32_t *tile_bigitems, const FusedRoads fr, BigList bl,
                     unsigned long long *status, int grid, cudaStream_t st) {
    uint64_t T = n_tiles(max_words);
    int g = (int)(T < (uint64_t)grid ? T : (uint64_t)grid);
    if (g < 1) g = 1;
    k_big_list<<<g, TILE_THREADS, 0, st>>>(desc, road_cap, dims, tile_roads, tile_big,
                                          tile_bigitems, fr, bl, status);
}

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

cudaError_t launch_fit_persistent(const uint32_t *words, const uint4 *desc, const uint64_t *counts,
                                  uint64_t road_cap, const uint64_t *n_big, const int16_t *F,
                                  const int16_t *q, const svt_config cfg, const FusedRoads fr,
                                  uint32_t roads_per_chunk, BigList bl, uint32_t *out,
                                  uint64_t *counts_out, unsigned long long *status,
                                  int warps_per_block, int grid, cudaStream_t st) {
    size_t smem = fit_smem_bytes(warps_per_block);
    if (cfg.chi2_cut < 32767u * 32767u)
        k_fit_persistent<true><<<grid, warps_per_block * 32, smem, st>>>(
            words, desc, counts, road_cap, n_big, F, q, cfg, fr, roads_per_chunk, bl, out,
            counts_out, status);
    else
        k_fit_persistent<false><<<grid, warps_per_block * 32, smem, st>>>(
            words, desc, counts, road_cap, n_big, F, q, cfg, fr, roads_per_chunk, bl, out,
            counts_out, status);
    return cudaGetLastError();
}

}  // namespace svt
