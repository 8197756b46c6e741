// svt_calib.cu -- FP32 relaxation of the linearised fit for calibrating its
// constants (the paper's Sec. 2 form p = f.x + q without the integer shift
// and clamp):
//     y_t = F[s_t] x_t + q[s_t]                       (6 rows per track)
//     L   = (1/N) sum_t [ sum_{k<3} w_k (y_tk - theta_tk)^2 + sum_{k>=3} y_tk^2 ]
// with hand-written forward and backward kernels.
//
// Tracks are first sorted by sector (stable counting sort on the device);
// every kernel then works on "items" of at most CALIB_CHUNK consecutive tracks
// of one sector: the forward, the loss alone and the general backward take
// one warp per item, the fused loss-and-gradient pass a contiguous run of
// items per warp with its final sums made by the warps that complete each
// sector (atomic tickets, no waiting).  Every reduction runs in a fixed order
// (lanes, then items or segments in index order), so results are bitwise
// reproducible run to run.
#include <mutex>

#include "svt_kernels.cuh"

namespace svt {

namespace {

constexpr int CALIB_CHUNK = 256;          // tracks per item (8 per lane)
constexpr int SORT_TILE = 1024;           // tracks per histogram tile
constexpr int NPAR = 42;                  // 36 entries of F[s] + 6 of q[s]


__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// ---- stable counting sort by sector ------------------------------------------
__global__ void k_hist(const int32_t *__restrict__ sector, uint64_t n, uint32_t S, uint32_t T,
                       uint32_t *counts, unsigned long long *status) {
    __shared__ uint32_t h[512];
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) h[s] = 0;
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < SORT_TILE; j += blockDim.x) {
            const uint64_t i = (uint64_t)t * SORT_TILE + j;
            if (i < n) {
                const int32_t s = sector[i];
                if (s < 0 || (uint32_t)s >= S) {
                    report(status, i, SVT_ERR_BAD_SECTOR);
                } else {
                    atomicAdd(&h[s], 1u);
                }
            }
        }
        __syncthreads();
        for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) counts[(uint64_t)s * T + t] = h[s];
        __syncthreads();
    }
}

// exclusive scan of counts[0..n) in one block; n = S * T
__global__ void __launch_bounds__(1024) k_scan_counts(uint32_t *counts, uint64_t n) {
    __shared__ uint32_t sm[33];
    uint32_t carry = 0;
    for (uint64_t c0 = 0; c0 < n; c0 += 4096) {
        const uint64_t i0 = c0 + (uint64_t)threadIdx.x * 4;
        uint32_t v[4], s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (i0 + k < n) ? counts[i0 + k] : 0u;
            s += v[k];
        }
        uint32_t tot;
        uint32_t run = carry + block_exclusive_scan<uint32_t>(s, sm, &tot);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < n) counts[i0 + k] = run;
            run += v[k];
        }
        carry += tot;
    }
}

// one warp per tile: stable ranks inside the tile by rounds of 32 tracks
__global__ void k_scatter(const int32_t *__restrict__ sector, uint64_t n, uint32_t S, uint32_t T,
                          const uint32_t *__restrict__ base, int32_t *perm) {
    __shared__ uint32_t cnt[512];
    const int lane = threadIdx.x;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        for (uint32_t s = lane; s < S; s += 32) cnt[s] = 0;
        __syncwarp();
        for (int r = 0; r < SORT_TILE / 32; ++r) {
            const uint64_t i = (uint64_t)t * SORT_TILE + r * 32 + lane;
            const bool valid = i < n;
            const int32_t s = valid ? sector[i] : -1;
            const bool ok = valid && s >= 0 && (uint32_t)s < S;
            const uint32_t key = ok ? (uint32_t)s : 0xFFFFFFFFu;
            const uint32_t match = __match_any_sync(0xffffffffu, key);
            const uint32_t rank = __popc(match & ((1u << lane) - 1u));
            uint32_t before = 0;
            if (ok) before = cnt[s];
            __syncwarp();
            if (ok) {
                perm[base[(uint64_t)s * T + t] + before + rank] = (int32_t)i;
                if (rank == 0) cnt[s] = before + __popc(match);
            }
            __syncwarp();
        }
    }
}

// sector_off and the item table, one block
__global__ void __launch_bounds__(1024)
    k_items(const uint32_t *__restrict__ base, uint32_t S, uint32_t T, uint64_t n,
            int32_t *sector_off, int32_t *sector_item, int32_t *item_sector, int32_t *item_start,
            int32_t *n_items, uint32_t max_items) {
    __shared__ uint32_t sm[33];
    __shared__ uint32_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < S; c0 += 1024) {
        const uint32_t s = c0 + threadIdx.x;
        uint32_t off = 0, len = 0;
        if (s < S) {
            off = base[(uint64_t)s * T];
            const uint32_t end = (s + 1 < S) ? base[(uint64_t)(s + 1) * T] : (uint32_t)n;
            len = end - off;
            sector_off[s] = (int32_t)off;
        }
        const uint32_t items = (len + CALIB_CHUNK - 1) / CALIB_CHUNK;
        uint32_t tot;
        const uint32_t first = carry_s + block_exclusive_scan<uint32_t>(items, sm, &tot);
        if (s < S) sector_item[s] = (int32_t)first;
        for (uint32_t k = 0; k < items; ++k) {
            if (first + k < max_items) {
                item_sector[first + k] = (int32_t)s;
                item_start[first + k] = (int32_t)(off + k * CALIB_CHUNK);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sector_off[S] = (int32_t)n;
        sector_item[S] = (int32_t)carry_s;
        *n_items = (int32_t)carry_s;
    }
}

__global__ void k_gather(const float *__restrict__ src, uint32_t width,
                         const int32_t *__restrict__ perm, uint64_t n, float *dst) {
    const uint64_t total = n * width;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = k / width, c = k % width;
        dst[k] = src[(uint64_t)perm[i] * width + c];
    }
}

// ---- forward / loss / backward -------------------------------------------------
struct Item {
    uint32_t s, start, end;
};

__device__ __forceinline__ Item item_of(const int32_t *item_sector, const int32_t *item_start,
                                        const int32_t *sector_off, uint32_t i) {
    Item it;
    it.s = (uint32_t)item_sector[i];
    it.start = (uint32_t)item_start[i];
    const uint32_t send = (uint32_t)sector_off[it.s + 1];
    it.end = min(it.start + (uint32_t)CALIB_CHUNK, send);
    return it;
}

// F[s] and q[s] of the item's sector in the warp's shared slot (q may be null
// where only F is needed: the offsets then read as 0)
__device__ __forceinline__ void load_consts(float *c, const float *__restrict__ F,
                                            const float *__restrict__ q, uint32_t s, int lane) {
    for (int j = lane; j < NPAR; j += 32) {
        if (j < 36)
            c[j] = F[(size_t)s * 36 + j];
        else
            c[j] = q ? q[(size_t)s * 6 + (j - 36)] : 0.f;
    }
    __syncwarp();
}

__device__ __forceinline__ void eval_track(const float *c, const float *__restrict__ x, uint32_t t,
                                           float xv[6], float y[6]) {
    const float2 *xp = reinterpret_cast<const float2 *>(x + (size_t)t * 6);
    float2 a = xp[0], b = xp[1], d = xp[2];
    xv[0] = a.x; xv[1] = a.y; xv[2] = b.x; xv[3] = b.y; xv[4] = d.x; xv[5] = d.y;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float acc = c[36 + k];
#pragma unroll
        for (int l = 0; l < 6; ++l) acc = fmaf(c[k * 6 + l], xv[l], acc);
        y[k] = acc;
    }
}

__global__ void __launch_bounds__(256, 6)
    k_forward(const float *__restrict__ x, const int32_t *__restrict__ item_sector,
              const int32_t *__restrict__ item_start,
              const int32_t *__restrict__ sector_off, const int32_t *__restrict__ n_items,
              const float *__restrict__ F, const float *__restrict__ q, float *y) {
    __shared__ float cs[8][48];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t NI = (uint32_t)*n_items;
    for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + wib; i < NI; i += gridDim.x * (blockDim.x >> 5)) {
        const Item it = item_of(item_sector, item_start, sector_off, i);
        load_consts(cs[wib], F, q, it.s, lane);
        // the item's tracks in CALIB_CHUNK / 32 unrolled steps, so their loads
        // are in flight together (same order as a plain loop)
#pragma unroll
        for (int k = 0; k < CALIB_CHUNK / 32; ++k) {
            const uint32_t t = it.start + (uint32_t)lane + 32u * k;
            if (t >= it.end) continue;
            float xv[6], yv[6];
            eval_track(cs[wib], x, t, xv, yv);
            float2 *yp = reinterpret_cast<float2 *>(y + (size_t)t * 6);
            yp[0] = make_float2(yv[0], yv[1]);
            yp[1] = make_float2(yv[2], yv[3]);
            yp[2] = make_float2(yv[4], yv[5]);
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256, 8)
    k_loss_items(const float *__restrict__ x, const float *__restrict__ theta,
                 const int32_t *__restrict__ item_sector,
                 const int32_t *__restrict__ item_start,
                 const int32_t *__restrict__ sector_off,
                 const int32_t *__restrict__ n_items, const float *__restrict__ F,
                 const float *__restrict__ q, const float *__restrict__ w,
                 float *item_loss) {
    __shared__ float cs[8][48];
    allow_next_grid();   // the final reduction may be scheduled; it waits for this grid
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t NI = (uint32_t)*n_items;
    const float w0 = w[0], w1 = w[1], w2 = w[2];
    for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + wib; i < NI; i += gridDim.x * (blockDim.x >> 5)) {
        const Item it = item_of(item_sector, item_start, sector_off, i);
        load_consts(cs[wib], F, q, it.s, lane);
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < CALIB_CHUNK / 32; ++k) {
            const uint32_t t = it.start + (uint32_t)lane + 32u * k;
            if (t >= it.end) continue;
            float xv[6], yv[6];
            eval_track(cs[wib], x, t, xv, yv);
            const float r0 = yv[0] - theta[(size_t)t * 3 + 0];
            const float r1 = yv[1] - theta[(size_t)t * 3 + 1];
            const float r2 = yv[2] - theta[(size_t)t * 3 + 2];
            acc += w0 * r0 * r0 + w1 * r1 * r1 + w2 * r2 * r2 + yv[3] * yv[3] + yv[4] * yv[4] +
                   yv[5] * yv[5];
        }
        acc = warp_sum(acc);
        if (lane == 0) item_loss[i] = acc;
        __syncwarp();
    }
}

// one block: loss = (sum of the item partials) / n in a fixed order: thread
// t sums items t, t + 1024, t + 2048, ... in that order (eight loads in
// flight at a time), then the block sums the 1024 partials by a fixed tree
__global__ void __launch_bounds__(1024)
    k_loss_final(const float *__restrict__ item_loss, const int32_t *__restrict__ n_items,
                 uint64_t n, float *loss) {
    constexpr uint32_t B = 1024, U = 8;
    __shared__ float sm[32];
    wait_prior_grid();   // the item partials are complete (see launch_after)
    const uint32_t NI = (uint32_t)*n_items;
    float total = 0.f;
    uint32_t i = threadIdx.x;
    for (; i + (U - 1) * B < NI; i += U * B) {
        float v[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) v[u] = item_loss[i + u * B];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) total += v[u];
    }
    for (; i < NI; i += B) total += item_loss[i];
    total = warp_sum(total);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = total;
    __syncthreads();
    if (threadIdx.x < 32) {
        const float u = warp_sum(sm[threadIdx.x]);
        if (threadIdx.x == 0) *loss = n ? u / (float)n : 0.f;
    }
}

// per item of the general backward: sum_t g_t x_t^T and sum_t g_t with g
// from grad_y, and dx_t = F[s]^T g_t when dx is given
__global__ void k_grad_items(const float *__restrict__ x, const float *__restrict__ grad_y,
                             const int32_t *__restrict__ item_sector,
                             const int32_t *__restrict__ item_start,
                             const int32_t *__restrict__ sector_off,
                             const int32_t *__restrict__ n_items, const float *__restrict__ F,
                             float *item_grad, float *dx) {
    __shared__ float cs[8][48];
    // per warp: the 32 lanes' partials, row stride NPAR + 1 (odd, so that both
    // the row writes and the column reads are free of bank conflicts)
    __shared__ float red_s[8][32 * (NPAR + 1)];
    allow_next_grid();   // the final reduction may be scheduled; it waits for this grid
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t NI = (uint32_t)*n_items;
    for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + wib; i < NI; i += gridDim.x * (blockDim.x >> 5)) {
        const Item it = item_of(item_sector, item_start, sector_off, i);
        load_consts(cs[wib], F, nullptr, it.s, lane);
        float acc[NPAR];
#pragma unroll
        for (int j = 0; j < NPAR; ++j) acc[j] = 0.f;
        // two tracks per step keep two tracks' loads in flight (the 42
        // accumulators leave room for only 16 warps per SM); each lane still
        // adds its tracks in increasing order
#pragma unroll 2
        for (uint32_t t = it.start + lane; t < it.end; t += 32) {
            float xv[6], g[6];
            {
                const float2 *xp = reinterpret_cast<const float2 *>(x + (size_t)t * 6);
                const float2 *gp = reinterpret_cast<const float2 *>(grad_y + (size_t)t * 6);
                float2 a = xp[0], b = xp[1], d = xp[2];
                xv[0] = a.x; xv[1] = a.y; xv[2] = b.x; xv[3] = b.y; xv[4] = d.x; xv[5] = d.y;
                a = gp[0]; b = gp[1]; d = gp[2];
                g[0] = a.x; g[1] = a.y; g[2] = b.x; g[3] = b.y; g[4] = d.x; g[5] = d.y;
                if (dx) {
                    float dv[6];
#pragma unroll
                    for (int l = 0; l < 6; ++l) {
                        float s = 0.f;
#pragma unroll
                        for (int k = 0; k < 6; ++k) s = fmaf(cs[wib][k * 6 + l], g[k], s);
                        dv[l] = s;
                    }
                    float2 *dp = reinterpret_cast<float2 *>(dx + (size_t)t * 6);
                    dp[0] = make_float2(dv[0], dv[1]);
                    dp[1] = make_float2(dv[2], dv[3]);
                    dp[2] = make_float2(dv[4], dv[5]);
                }
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {
#pragma unroll
                for (int l = 0; l < 6; ++l) acc[k * 6 + l] = fmaf(g[k], xv[l], acc[k * 6 + l]);
                acc[36 + k] += g[k];
            }
        }
        // the item's sums over the lanes: every lane writes its partials, then
        // lane j adds column j (and j + 32) over the lanes in lane order
        float *red = red_s[wib];
#pragma unroll
        for (int j = 0; j < NPAR; ++j) red[lane * (NPAR + 1) + j] = acc[j];
        __syncwarp();
        for (int j = lane; j < NPAR; j += 32) {
            float total = 0.f;
#pragma unroll 8
            for (int m = 0; m < 32; ++m) total += red[m * (NPAR + 1) + j];
            item_grad[(size_t)i * NPAR + j] = total;
        }
        __syncwarp();
    }
}

// per (sector, entry): sum of the sector's item partials in index order, scaled
__global__ void k_grad_final(const float *__restrict__ item_grad,
                             const int32_t *__restrict__ sector_item, uint32_t S,
                             const float *__restrict__ scale_dev, float scale, float *dF,
                             float *dq) {
    wait_prior_grid();   // the item partials are complete (see launch_after)
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S * NPAR) return;
    const uint32_t s = k / NPAR, j = k % NPAR;
    const uint32_t first = (uint32_t)sector_item[s], last = (uint32_t)sector_item[s + 1];
    float total = 0.f;
    uint32_t m = first;
    for (; m + 8 <= last; m += 8) {   // eight loads in flight, added in index order
        float v[8];
#pragma unroll
        for (uint32_t u = 0; u < 8; ++u) v[u] = item_grad[(size_t)(m + u) * NPAR + j];
#pragma unroll
        for (uint32_t u = 0; u < 8; ++u) total += v[u];
    }
    for (; m < last; ++m) total += item_grad[(size_t)m * NPAR + j];
    const float sc = scale * (scale_dev ? *scale_dev : 1.f);
    if (j < 36)
        dF[(size_t)s * 36 + j] = total * sc;
    else
        dq[(size_t)s * 6 + (j - 36)] = total * sc;
}

// ---- the loss and its gradient in one pass --------------------------------------
constexpr int LG_BT = 4;   // tracks per lane whose loads are in flight together

// The loss and its gradient in one pass over the tracks.  Warp w of the grid
// takes the contiguous items [w per, (w + 1) per) (per = ceil(items /
// warps)); their sectors and first tracks are looked up together, one item
// per lane, before any of them is used.  Every lane loads LG_BT of its tracks
// (x and theta; the index is clamped to the last track, so the loads need
// only the item's first track) before using any of them, while the item's
// end and, for a new sector, its constants are fetched, then adds its tracks'
// loss terms and the 42 products g x^T, g (g = dL/dy up to the factor 2/N)
// in track order for as long as consecutive items belong to one sector; with
// WY it also writes each track's y = F x + q.  When the sector changes, or
// the warp's items end, the lanes' partials are summed through shared memory
// (four runs of eight lanes in lane order, then the runs in a fixed tree)
// into the slot of the segment's first item.  The final sums need no second
// launch: after writing a segment the warp adds the segment's item count to
// its sector's ticket (atomicAdd after a fence); the warp that completes the
// sector's count sums the sector's segments in warp order -- their slots
// follow from `per` alone --, writes dF[s], dq[s] and the sector's loss,
// then adds the sector's item count to the batch's ticket; the warp that
// completes that count sums the sector losses in sector order.  Nothing waits
// on another warp, and for a given grid every sum runs in a fixed order, so
// repeated calls give identical bits.  Sectors without tracks get zero
// gradients.  The tickets (tickets[0..S]) must be zero at entry; every warp
// that completes one sets it back to zero, so a call leaves them ready for
// the next.
template <bool WY>
__global__ void __launch_bounds__(256, 2)
    k_loss_grad(const float *__restrict__ x, const float *__restrict__ theta,
                const int32_t *__restrict__ item_sector, const int32_t *__restrict__ item_start,
                const int32_t *__restrict__ sector_off, const int32_t *__restrict__ sector_item,
                const int32_t *__restrict__ n_items, uint32_t S, uint64_t n,
                const float *__restrict__ F, const float *__restrict__ q,
                const float *__restrict__ w, const float *__restrict__ scale_dev,
                float *item_loss, float *item_grad, float *sector_loss, unsigned int *tickets,
                float *loss, float *dF, float *dq, float *y) {
    constexpr int TPL = CALIB_CHUNK / 32;   // tracks per lane and item
    // per warp: F[s] and q[s] as six rows of eight floats (F[r][0..5], q[r], 0)
    __shared__ __align__(16) float cs[8][48];
    __shared__ float red_s[8][32 * (NPAR + 1)];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + wib, nw = gridDim.x * (blockDim.x >> 5);
    const uint32_t NI = (uint32_t)*n_items;
    const float scale = (n ? 2.0f / (float)n : 0.f) * (scale_dev ? *scale_dev : 1.f);
    for (uint32_t s = gw; s < S; s += nw) {
        if (sector_item[s + 1] != sector_item[s]) continue;
        for (int j = lane; j < NPAR; j += 32) {
            if (j < 36)
                dF[(size_t)s * 36 + j] = 0.f;
            else
                dq[(size_t)s * 6 + (j - 36)] = 0.f;
        }
    }
    if (NI == 0) {
        if (gw == 0 && lane == 0) *loss = 0.f;
        return;
    }
    const uint32_t per = (NI + nw - 1) / nw;
    const uint32_t i0 = gw * per, i1 = min(i0 + per, NI);
    if (i0 >= i1) return;
    const float w0 = w[0], w1 = w[1], w2 = w[2];
    const uint32_t last_track = (uint32_t)n - 1;
    float acc[NPAR];
    float lacc = 0.f;
#pragma unroll
    for (int j = 0; j < NPAR; ++j) acc[j] = 0.f;
    uint32_t seg = i0;   // first item of the current segment
    float *c = cs[wib];
    for (uint32_t base = i0; base < i1; base += 32) {
        // the next 32 items' sector, first track and end, one item per lane
        const uint32_t cnt = min(32u, i1 - base);
        uint32_t m_s = 0, m_start = 0, m_end = 0;
        if ((uint32_t)lane < cnt) {
            m_s = (uint32_t)__ldg(item_sector + base + lane);
            m_start = (uint32_t)__ldg(item_start + base + lane);
            m_end = min(m_start + (uint32_t)CALIB_CHUNK, (uint32_t)__ldg(sector_off + m_s + 1));
        }
        const uint32_t after = base + cnt < i1 ? (uint32_t)__ldg(item_sector + base + cnt) : ~0u;
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t i = base + k;
            const uint32_t is = __shfl_sync(0xffffffffu, m_s, (int)k);
            const uint32_t start = __shfl_sync(0xffffffffu, m_start, (int)k);
#pragma unroll 1
            for (int h = 0; h < TPL; h += LG_BT) {
                float xv[LG_BT][6], th[LG_BT][3];
#pragma unroll
                for (int kk = 0; kk < LG_BT; ++kk) {
                    const uint32_t t = min(start + (uint32_t)lane + 32u * (h + kk), last_track);
                    const float2 *xp = reinterpret_cast<const float2 *>(x + (size_t)t * 6);
                    const float2 a = __ldg(xp), b = __ldg(xp + 1), d = __ldg(xp + 2);
                    xv[kk][0] = a.x; xv[kk][1] = a.y; xv[kk][2] = b.x;
                    xv[kk][3] = b.y; xv[kk][4] = d.x; xv[kk][5] = d.y;
                    th[kk][0] = __ldg(theta + (size_t)t * 3 + 0);
                    th[kk][1] = __ldg(theta + (size_t)t * 3 + 1);
                    th[kk][2] = __ldg(theta + (size_t)t * 3 + 2);
                }
                const uint32_t iend = __shfl_sync(0xffffffffu, m_end, (int)k);
                if (h == 0 && i == seg) {
                    // a new segment's constants, fetched while the tracks are in flight
                    for (int j = lane; j < 48; j += 32) {
                        const int r = j >> 3, l = j & 7;
                        c[j] = l < 6 ? __ldg(F + (size_t)is * 36 + r * 6 + l)
                                     : (l == 6 ? __ldg(q + (size_t)is * 6 + r) : 0.f);
                    }
                    __syncwarp();
                }
#pragma unroll
                for (int kk = 0; kk < LG_BT; ++kk) {
                    const uint32_t t = start + (uint32_t)lane + 32u * (h + kk);
                    if (t >= iend) continue;
                    float g[6];
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
                        const float4 u = *reinterpret_cast<const float4 *>(c + r * 8);
                        const float4 v = *reinterpret_cast<const float4 *>(c + r * 8 + 4);
                        float e = v.z;
                        e = fmaf(u.x, xv[kk][0], e);
                        e = fmaf(u.y, xv[kk][1], e);
                        e = fmaf(u.z, xv[kk][2], e);
                        e = fmaf(u.w, xv[kk][3], e);
                        e = fmaf(v.x, xv[kk][4], e);
                        e = fmaf(v.y, xv[kk][5], e);
                        g[r] = e;
                    }
                    if (WY) {
                        float2 *yp = reinterpret_cast<float2 *>(y + (size_t)t * 6);
                        yp[0] = make_float2(g[0], g[1]);
                        yp[1] = make_float2(g[2], g[3]);
                        yp[2] = make_float2(g[4], g[5]);
                    }
                    const float r0 = g[0] - th[kk][0], r1 = g[1] - th[kk][1], r2 = g[2] - th[kk][2];
                    lacc += w0 * r0 * r0 + w1 * r1 * r1 + w2 * r2 * r2 + g[3] * g[3] +
                            g[4] * g[4] + g[5] * g[5];
                    g[0] = w0 * r0;
                    g[1] = w1 * r1;
                    g[2] = w2 * r2;
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
#pragma unroll
                        for (int l = 0; l < 6; ++l) acc[r * 6 + l] = fmaf(g[r], xv[kk][l], acc[r * 6 + l]);
                        acc[36 + r] += g[r];
                    }
                }
            }
            // does the segment end with this item?
            const uint32_t next_s = __shfl_sync(0xffffffffu, m_s, (int)min(k + 1, 31u));
            if (i + 1 != i1 && (k + 1 < cnt ? next_s : after) == is) continue;
            // the segment's sums over the lanes into its first item's slot: four
            // runs of eight lanes in lane order, then the runs in a fixed tree
            {
                float *red = red_s[wib];
#pragma unroll
                for (int j = 0; j < NPAR; ++j) red[lane * (NPAR + 1) + j] = acc[j];
                __syncwarp();
                for (int j = lane; j < NPAR; j += 32) {
                    float part[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float v = red[(8 * u) * (NPAR + 1) + j];
#pragma unroll
                        for (int m = 1; m < 8; ++m) v += red[(8 * u + m) * (NPAR + 1) + j];
                        part[u] = v;
                    }
                    item_grad[(size_t)seg * NPAR + j] = (part[0] + part[1]) + (part[2] + part[3]);
                }
                const float lt = warp_sum(lacc);
                if (lane == 0) item_loss[seg] = lt;
                __syncwarp();
            }
            const uint32_t seg_items = i + 1 - seg;
            seg = i + 1;
            lacc = 0.f;
#pragma unroll
            for (int j = 0; j < NPAR; ++j) acc[j] = 0.f;
            // the sector's ticket
            const uint32_t a = (uint32_t)sector_item[is], b = (uint32_t)sector_item[is + 1];
            __threadfence();
            unsigned int last = 0;
            if (lane == 0) last = atomicAdd(&tickets[is], seg_items) + seg_items == b - a;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (!last) continue;
            __threadfence();
            if (lane == 0) tickets[is] = 0u;   // ready for the next call
            // the sector's segments: one per warp whose items meet [a, b), in warp order
            const uint32_t wa = a / per, wz = (b - 1) / per;
            for (int j = lane; j < NPAR; j += 32) {
                float total = 0.f;
                uint32_t v = wa;
                for (; v + 8 <= wz + 1; v += 8) {   // eight loads in flight, added in order
                    float u8[8];
#pragma unroll
                    for (uint32_t u = 0; u < 8; ++u)
                        u8[u] = __ldcg(item_grad + (size_t)max(a, (v + u) * per) * NPAR + j);
#pragma unroll
                    for (uint32_t u = 0; u < 8; ++u) total += u8[u];
                }
                for (; v <= wz; ++v) total += __ldcg(item_grad + (size_t)max(a, v * per) * NPAR + j);
                if (j < 36)
                    dF[(size_t)is * 36 + j] = total * scale;
                else
                    dq[(size_t)is * 6 + (j - 36)] = total * scale;
            }
            float sl = 0.f;
            for (uint32_t v = wa + (uint32_t)lane; v <= wz; v += 32)
                sl += __ldcg(item_loss + max(a, v * per));
            sl = warp_sum(sl);
            if (lane == 0) sector_loss[is] = sl;
            __syncwarp();
            // the batch's ticket counts the items of summed sectors
            __threadfence();
            unsigned int fin = 0;
            if (lane == 0) fin = atomicAdd(&tickets[S], b - a) + (b - a) == NI;
            fin = __shfl_sync(0xffffffffu, fin, 0);
            if (fin) {
                __threadfence();
                if (lane == 0) tickets[S] = 0u;   // ready for the next call
                float tl[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {   // S <= 512: every sector loss in flight at once
                    const uint32_t s2 = (uint32_t)lane + 32u * u;
                    tl[u] = (s2 < S && sector_item[s2 + 1] != sector_item[s2])
                                ? __ldcg(sector_loss + s2)
                                : 0.f;
                }
                float t = 0.f;
#pragma unroll
                for (int u = 0; u < 16; ++u) t += tl[u];
                t = warp_sum(t);
                if (lane == 0) *loss = t / (float)n;
            }
        }
    }
}

// ---- the fused pass with its tracks staged by the bulk-copy unit ------------------
// The loss and its gradient as k_loss_grad computes them, in two kernels
// chained by programmatic dependent launch, for x and theta that start on a
// 16-byte boundary (the launcher takes k_loss_grad otherwise).
//
// k_loss_grad_bulk takes the track loads off the lanes: the x and theta rows
// of each item are copied to the warp's shared-memory buffers by one
// cp.async.bulk per array (completion counted on an mbarrier per buffer),
// NBUF - 1 items ahead of the item the warp adds up, so that every warp
// always has an item's bytes in flight while it computes.  A bulk copy moves
// 16-byte aligned spans of a multiple of 16 bytes, hence the copied range
// [lo, hi) is the item's track range widened to multiples of four tracks
// (4 x 24 bytes of x, 4 x 12 of theta) and cut at the last multiple of four
// at or below n, so no byte past either array is read; the at most three
// tracks past that cut are read from global memory by their lanes.  The end
// of item i is the first track of item i + 1 (the items tile the sorted
// tracks), n for the last item.  The I items are cut into runs for the first
// W warps (W the smaller of I and the grid's warps) that differ by one item
// at most (CalibRuns), so that every SM gets work.  Each warp writes one
// partial per segment (a run of its items in one sector) into the slot of
// the segment's first item, as k_loss_grad does, and takes no ticket.
//
// k_lg_final, once the first kernel has completed, sums each sector's
// segment partials in warp order (one thread per sector and entry, every
// sector including those without tracks) and, in its last block, the
// sectors' losses in a fixed tree.  Every sum runs in a fixed order for a
// given grid, so repeated calls give identical bits.  (Taking the final sums
// in the first kernel by tickets, as k_loss_grad does, put a chain of
// fences, atomics and loads after the last warp's compute that took longer
// than the dependent launch.)
//
// Every wait on a copy is bounded; a copy that does not land within the
// bound sets the flag word the launcher passes (the workspace's tickets[S +
// 1]), and k_lg_final then writes a NaN loss and clears it.
constexpr int ST_TRACKS = CALIB_CHUNK + 4;                 // an item with its widening
constexpr uint32_t ST_XBYTES = ST_TRACKS * 24u;            // x rows of a buffer
constexpr uint32_t ST_BUF = ST_TRACKS * 36u;               // x rows, then theta rows
constexpr uint32_t BULK_WAIT_SPINS = 1u << 20;
static_assert(ST_XBYTES % 16 == 0 && ST_BUF % 16 == 0, "bulk copy spans");
static_assert(32 * (NPAR + 1) * 4 <= (int)ST_XBYTES, "the lane sums reuse an x buffer");

// the cut of I items into runs for the first W = min(warps, I) warps: the
// first I mod W warps take one item more than the others (no division in
// first(); warp_of() divides by a 32-bit value)
struct CalibRuns {
    uint32_t nwe, qi, rq;
    __device__ __forceinline__ CalibRuns(uint32_t warps, uint32_t items) {
        nwe = max(1u, min(warps, items));
        qi = items / nwe;
        rq = items % nwe;
    }
    __device__ __forceinline__ uint32_t first(uint32_t v) const { return v * qi + min(v, rq); }
    __device__ __forceinline__ uint32_t warp_of(uint32_t i) const {   // the run holding item i
        const uint32_t big = rq * (qi + 1);
        return i < big ? i / (qi + 1) : rq + (i - big) / qi;
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(m)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// generic-proxy accesses of shared memory before this point are ordered
// before later bulk-copy (async-proxy) writes
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(m)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(m))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// false when the phase did not complete within the bound
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *m, uint32_t parity) {
    for (uint32_t k = 0; k < BULK_WAIT_SPINS; ++k)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}

// F[s] (rows of six) and q[s] as six rows of eight floats, entries lane and
// lane + 32 of the 48
__device__ __forceinline__ void fetch_consts(const float *__restrict__ F,
                                             const float *__restrict__ q, uint32_t s, int lane,
                                             float &k0, float &k1) {
    auto one = [&](int j) {
        const int r = j >> 3, l = j & 7;
        return l < 6 ? __ldg(F + (size_t)s * 36 + r * 6 + l)
                     : (l == 6 ? __ldg(q + (size_t)s * 6 + r) : 0.f);
    };
    k0 = one(lane);
    k1 = lane < 16 ? one(lane + 32) : 0.f;
}

template <bool WY, bool GRAD, int WARPS, int NBUF>
__global__ void __launch_bounds__(WARPS * 32, 1)
    k_loss_grad_bulk(const float *__restrict__ x, const float *__restrict__ theta,
                     const int32_t *__restrict__ item_sector,
                     const int32_t *__restrict__ item_start, const int32_t *__restrict__ n_items,
                     uint64_t n, const float *__restrict__ F, const float *__restrict__ q,
                     const float *__restrict__ w, float *item_loss, float *item_grad,
                     unsigned int *flag, float *y) {
    constexpr int TPL = CALIB_CHUNK / 32;   // tracks per lane and item
    extern __shared__ __align__(128) unsigned char st_buf[];
    __shared__ __align__(16) float cs[WARPS][48];
    __shared__ __align__(8) uint64_t bars[WARPS][NBUF];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t gw = blockIdx.x * WARPS + wib, nw = gridDim.x * WARPS;
    allow_next_grid();   // k_lg_final's blocks may take SMs as this grid's blocks leave
    const uint32_t NI = (uint32_t)*n_items;
    if (NI == 0) return;
    const CalibRuns runs(nw, NI);
    if (gw >= runs.nwe) return;
    const uint32_t i0 = runs.first(gw), i1 = runs.first(gw + 1);
    unsigned char *wbuf = st_buf + (size_t)wib * NBUF * ST_BUF;
    uint64_t *mb = bars[wib];
    if (lane == 0) {
#pragma unroll
        for (int b = 0; b < NBUF; ++b) mbar_init(&mb[b], 1);
        mbar_init_fence();
    }
    __syncwarp();
    const float w0 = w[0], w1 = w[1], w2 = w[2];
    const uint32_t n32 = (uint32_t)n, n4 = n32 & ~3u;
    // sector, first track and end of 32 items, one per lane: the current
    // batch [base, base + 32) and the next
    uint32_t base = i0;
    uint32_t c_s = 0, c_st = 0, c_en = 0, x_s = 0, x_st = 0, x_en = 0;
    auto fetch = [&](uint32_t b0, uint32_t &ms, uint32_t &mst, uint32_t &men) {
        const uint32_t i = b0 + (uint32_t)lane;
        ms = mst = men = 0;
        if (i < i1) {
            ms = (uint32_t)__ldg(item_sector + i);
            mst = (uint32_t)__ldg(item_start + i);
            men = i + 1 < NI ? (uint32_t)__ldg(item_start + i + 1) : n32;
        }
    };
    auto info = [&](uint32_t j, uint32_t &s, uint32_t &st, uint32_t &en) {
        const uint32_t d = j - base;   // below 64
        const int src = (int)(d & 31u);
        const uint32_t a0 = __shfl_sync(0xffffffffu, c_s, src), b0 = __shfl_sync(0xffffffffu, x_s, src);
        const uint32_t a1 = __shfl_sync(0xffffffffu, c_st, src), b1 = __shfl_sync(0xffffffffu, x_st, src);
        const uint32_t a2 = __shfl_sync(0xffffffffu, c_en, src), b2 = __shfl_sync(0xffffffffu, x_en, src);
        s = d < 32 ? a0 : b0;
        st = d < 32 ? a1 : b1;
        en = d < 32 ? a2 : b2;
    };
    auto span = [&](uint32_t st, uint32_t en, uint32_t &lo, uint32_t &hi) {
        lo = st & ~3u;
        hi = max(lo, min((en + 3u) & ~3u, n4));
    };
    // copy item j's rows into buffer b (every lane's reads of b are done)
    auto issue = [&](uint32_t j, int b) {
        uint32_t s, st, en, lo, hi;
        info(j, s, st, en);
        span(st, en, lo, hi);
        __syncwarp();
        if (lane == 0) {
            unsigned char *d = wbuf + (size_t)b * ST_BUF;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&mb[b], (hi - lo) * 36u);
            if (hi > lo) {
                bulk_copy_g2s(d, x + (size_t)lo * 6, (hi - lo) * 24u, &mb[b]);
                bulk_copy_g2s(d + ST_XBYTES, theta + (size_t)lo * 3, (hi - lo) * 12u, &mb[b]);
            }
        }
    };
    fetch(base, c_s, c_st, c_en);
    fetch(base + 32, x_s, x_st, x_en);
#pragma unroll
    for (int b = 0; b < NBUF - 1; ++b)
        if (i0 + (uint32_t)b < i1) issue(i0 + (uint32_t)b, b);
    float k0, k1;   // the constants of the next segment, fetched one item ahead
    {
        uint32_t s, st, en;
        info(i0, s, st, en);
        fetch_consts(F, q, s, lane, k0, k1);
    }
    // per lane: acc[6k + l] = sum r_k x_l, acc[36 + k] = sum r_k with
    // r = y - theta in rows 0..2 and r = y in rows 3..5 (the weights w_k of
    // rows 0..2 are applied once, at the segment's end), l3[k] = sum r_k^2
    // for k < 3 and l3[3] = sum over rows 3..5
    float acc[NPAR], l3[4];
#pragma unroll
    for (int j = 0; j < NPAR; ++j) acc[j] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) l3[k] = 0.f;
    uint32_t seg = i0, phase = 0u, bad = 0u, ever_bad = 0u;
    float *c = cs[wib];
    int b = 0;   // buffer of item i
    for (uint32_t i = i0; i < i1; ++i) {
        if (i - base >= 32u) {   // the next batch of lookups
            base += 32;
            c_s = x_s; c_st = x_st; c_en = x_en;
            fetch(base + 32, x_s, x_st, x_en);
        }
        uint32_t is, start, iend;
        info(i, is, start, iend);
        if (i + NBUF - 1 < i1) issue(i + NBUF - 1, (b + NBUF - 1) % NBUF);
        if (i == seg) {   // a new segment's constants
            __syncwarp();
            c[lane] = k0;
            if (lane < 16) c[lane + 32] = k1;
            __syncwarp();
        }
        uint32_t nxt_s = ~0u;
        if (i + 1 < i1) {
            uint32_t st2, en2;
            info(i + 1, nxt_s, st2, en2);
            if (nxt_s != is) fetch_consts(F, q, nxt_s, lane, k0, k1);
        }
        uint32_t lo, hi;
        span(start, iend, lo, hi);
        if (!mbar_wait_bounded(&mb[b], (phase >> b) & 1u)) bad = 1u;
        phase ^= 1u << b;
        const float *xs = reinterpret_cast<const float *>(wbuf + (size_t)b * ST_BUF);
        const float *ts = reinterpret_cast<const float *>(wbuf + (size_t)b * ST_BUF + ST_XBYTES);
        float cr[6][8];   // the segment's constants, in registers for the item
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const float4 p = *reinterpret_cast<const float4 *>(c + r * 8);
            const float4 v = *reinterpret_cast<const float4 *>(c + r * 8 + 4);
            cr[r][0] = p.x; cr[r][1] = p.y; cr[r][2] = p.z; cr[r][3] = p.w;
            cr[r][4] = v.x; cr[r][5] = v.y; cr[r][6] = v.z; cr[r][7] = 0.f;
        }
#pragma unroll 2
        for (int u = 0; u < TPL; ++u) {
            const uint32_t t = start + (uint32_t)lane + 32u * (uint32_t)u;
            if (t >= iend) break;
            float xv[6], th[3];
            if (t < hi) {
                const float2 *xp = reinterpret_cast<const float2 *>(xs + (size_t)(t - lo) * 6);
                const float2 a = xp[0], bb = xp[1], d = xp[2];
                xv[0] = a.x; xv[1] = a.y; xv[2] = bb.x; xv[3] = bb.y; xv[4] = d.x; xv[5] = d.y;
                const float *tp = ts + (size_t)(t - lo) * 3;
                th[0] = tp[0]; th[1] = tp[1]; th[2] = tp[2];
            } else {   // past the last multiple of four tracks
#pragma unroll
                for (int l = 0; l < 6; ++l) xv[l] = __ldg(x + (size_t)t * 6 + l);
#pragma unroll
                for (int l = 0; l < 3; ++l) th[l] = __ldg(theta + (size_t)t * 3 + l);
            }
            float g[6];
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                float e = cr[r][6];
                e = fmaf(cr[r][0], xv[0], e);
                e = fmaf(cr[r][1], xv[1], e);
                e = fmaf(cr[r][2], xv[2], e);
                e = fmaf(cr[r][3], xv[3], e);
                e = fmaf(cr[r][4], xv[4], e);
                e = fmaf(cr[r][5], xv[5], e);
                g[r] = e;
            }
            if (WY) {
                float2 *yp = reinterpret_cast<float2 *>(y + (size_t)t * 6);
                yp[0] = make_float2(g[0], g[1]);
                yp[1] = make_float2(g[2], g[3]);
                yp[2] = make_float2(g[4], g[5]);
            }
            g[0] -= th[0];
            g[1] -= th[1];
            g[2] -= th[2];
            l3[0] = fmaf(g[0], g[0], l3[0]);
            l3[1] = fmaf(g[1], g[1], l3[1]);
            l3[2] = fmaf(g[2], g[2], l3[2]);
            l3[3] = fmaf(g[3], g[3], l3[3]);
            l3[3] = fmaf(g[4], g[4], l3[3]);
            l3[3] = fmaf(g[5], g[5], l3[3]);
            if (GRAD) {
#pragma unroll
                for (int r = 0; r < 6; ++r) {
#pragma unroll
                    for (int l = 0; l < 6; ++l) acc[r * 6 + l] = fmaf(g[r], xv[l], acc[r * 6 + l]);
                    acc[36 + r] += g[r];
                }
            }
        }
        const int bi = b;
        b = b + 1 == NBUF ? 0 : b + 1;
        // does the segment end with this item?
        if (i + 1 != i1 && nxt_s == is) continue;
        {   // the segment's sums over the lanes, through item i's x buffer
#pragma unroll
            for (int l = 0; l < 6; ++l) {
                acc[l] *= w0;
                acc[6 + l] *= w1;
                acc[12 + l] *= w2;
            }
            acc[36] *= w0;
            acc[37] *= w1;
            acc[38] *= w2;
            const float lacc = fmaf(w0, l3[0], fmaf(w1, l3[1], fmaf(w2, l3[2], l3[3])));
            if (GRAD) {
                float *red = reinterpret_cast<float *>(wbuf + (size_t)bi * ST_BUF);
                __syncwarp();
#pragma unroll
                for (int j = 0; j < NPAR; ++j) red[lane * (NPAR + 1) + j] = acc[j];
                __syncwarp();
                for (int j = lane; j < NPAR; j += 32) {
                    float part[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float v = red[(8 * u) * (NPAR + 1) + j];
#pragma unroll
                        for (int m = 1; m < 8; ++m) v += red[(8 * u + m) * (NPAR + 1) + j];
                        part[u] = v;
                    }
                    item_grad[(size_t)seg * NPAR + j] = (part[0] + part[1]) + (part[2] + part[3]);
                }
            }
            const float lt = warp_sum(lacc);
            if (lane == 0) item_loss[seg] = lt;
            __syncwarp();
        }
        seg = i + 1;
#pragma unroll
        for (int j = 0; j < NPAR; ++j) acc[j] = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) l3[k] = 0.f;
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1u);
        ever_bad |= bad;
        bad = 0u;
    }
    // after a wait that gave up, wait (bounded again) for the last copy into
    // each buffer before the block's shared memory is released
    if (ever_bad) {
#pragma unroll
        for (int bb = 0; bb < NBUF; ++bb) mbar_wait_bounded(&mb[bb], ((phase >> bb) & 1u) ^ 1u);
    }
}


// the final sums of the staged pass (see above): blocks [0, ncol) one thread
// per (sector, entry) (ncol = 0: the loss alone), block ncol the loss; nw =
// the first kernel's warps
constexpr int LGF_THREADS = 512;
__global__ void __launch_bounds__(LGF_THREADS)
    k_lg_final(const float *__restrict__ item_grad, const float *__restrict__ item_loss,
               const int32_t *__restrict__ sector_item, const int32_t *__restrict__ n_items,
               uint32_t S, uint64_t n, uint32_t nw, uint32_t ncol,
               const float *__restrict__ scale_dev, unsigned int *flag, float *loss, float *dF,
               float *dq) {
    wait_prior_grid();
    const uint32_t NI = (uint32_t)*n_items;
    const float scale = (n ? 2.0f / (float)n : 0.f) * (scale_dev ? *scale_dev : 1.f);
    const CalibRuns runs(nw, NI);
    auto first = [&](uint32_t v) { return runs.first(v); };
    auto warp_of = [&](uint32_t i) { return runs.warp_of(i); };
    if (blockIdx.x < ncol) {
        const uint32_t k = blockIdx.x * LGF_THREADS + threadIdx.x;
        if (k >= S * NPAR) return;
        const uint32_t s = k / NPAR, j = k % NPAR;
        const uint32_t a = (uint32_t)sector_item[s], e = (uint32_t)sector_item[s + 1];
        float total = 0.f;
        if (e > a) {
            const uint32_t wa = warp_of(a), wz = warp_of(e - 1);
#pragma unroll 4
            for (uint32_t v = wa; v <= wz; ++v) total += item_grad[(size_t)max(a, first(v)) * NPAR + j];
        }
        if (j < 36)
            dF[(size_t)s * 36 + j] = total * scale;
        else
            dq[(size_t)s * 6 + (j - 36)] = total * scale;
        return;
    }
    // the loss: each thread its sectors' segment losses in order, then the
    // threads' sums by a fixed shuffle tree per warp and over the warps
    __shared__ float wsum[LGF_THREADS / 32];
    float sl = 0.f;
    for (uint32_t s = threadIdx.x; s < S; s += LGF_THREADS) {
        const uint32_t a = (uint32_t)sector_item[s], e = (uint32_t)sector_item[s + 1];
        if (e > a) {
            const uint32_t wa = warp_of(a), wz = warp_of(e - 1);
#pragma unroll 4
            for (uint32_t v = wa; v <= wz; ++v) sl += item_loss[max(a, first(v))];
        }
    }
    sl = warp_sum(sl);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = sl;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < LGF_THREADS / 32 ? wsum[threadIdx.x] : 0.f;
        t = warp_sum(t);
        if (threadIdx.x == 0) {
            const unsigned int f = *flag;
            if (f) *flag = 0u;
            *loss = n == 0 ? 0.f : (f ? __int_as_float(0x7fc00000) : t / (float)n);
        }
    }
}

// out_F = g dF, out_q = g dq over S sectors, one launch
__global__ void k_grad_scale(const float *__restrict__ g, const float *__restrict__ dF,
                             const float *__restrict__ dq, uint32_t S, float *out_F,
                             float *out_q) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    const float v = *g;
    if (k < S * 36)
        out_F[k] = dF[k] * v;
    else if (k < S * NPAR)
        out_q[k - S * 36] = dq[k - S * 36] * v;
}

}  // namespace

// ---- launchers used by svt_abi.cu -------------------------------------------------
// the staged pass's blocks: 12 warps without y (more warps to hide the
// per-warp latency), 8 with y (whose stores favour fewer warps), two
// buffers per warp each
constexpr int LGB_NBUF = 2, LGB_WARPS_NOY = 12, LGB_WARPS_Y = 8;

size_t calib_bulk_smem(int warps) { return (size_t)warps * LGB_NBUF * ST_BUF; }

// the staged pass's three instances: loss and gradient, the same with y,
// the loss alone
enum { LGB_GRAD = 0, LGB_GRAD_Y = 1, LGB_LOSS = 2 };
constexpr int lgb_warps(int kind) { return kind == LGB_GRAD_Y ? LGB_WARPS_Y : LGB_WARPS_NOY; }

// resident blocks per SM of each instance on the current device (0: it
// cannot be launched, the register-staged kernels are taken); the first call
// on a device raises the kernels' dynamic shared-memory limit
const int *calib_bulk_blocks_per_sm() {
    constexpr int MAXD = 64;
    static std::once_flag once[MAXD];
    static int per_sm[MAXD][3];
    static const int none[3] = {0, 0, 0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXD) return none;
    std::call_once(once[dev], [dev] {
        auto one = [&](auto kernel, int warps) {
            const int smem = (int)calib_bulk_smem(warps);
            int k = 0;
            if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                    cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, kernel, warps * 32, smem) !=
                    cudaSuccess)
                k = 0;
            return k;
        };
        per_sm[dev][LGB_GRAD] =
            one(k_loss_grad_bulk<false, true, LGB_WARPS_NOY, LGB_NBUF>, LGB_WARPS_NOY);
        per_sm[dev][LGB_GRAD_Y] =
            one(k_loss_grad_bulk<true, true, LGB_WARPS_Y, LGB_NBUF>, LGB_WARPS_Y);
        per_sm[dev][LGB_LOSS] =
            one(k_loss_grad_bulk<false, false, LGB_WARPS_NOY, LGB_NBUF>, LGB_WARPS_NOY);
        (void)cudaGetLastError();
    });
    return per_sm[dev];
}

// the staged pass when x and theta are 16-byte aligned and it can be
// launched; false: the caller takes the register-staged kernels
bool launch_loss_grad_bulk(int kind, const float *x, const float *theta,
                           const int32_t *item_sector, const int32_t *item_start,
                           const int32_t *sector_item, const int32_t *n_items, uint32_t S,
                           uint64_t n, const float *F, const float *q, const float *w,
                           const float *scale_dev, float *item_loss, float *item_grad,
                           unsigned int *flag, float *loss, float *dF, float *dq, float *y,
                           int sms, cudaStream_t st) {
    if ((((uintptr_t)x | (uintptr_t)theta) & 15u) != 0) return false;
    const int per_sm = calib_bulk_blocks_per_sm()[kind];
    if (per_sm <= 0) return false;
    const int g = max(sms, 1) * per_sm, warps = lgb_warps(kind);
    const size_t smem = calib_bulk_smem(warps);
    if (kind == LGB_GRAD_Y)
        k_loss_grad_bulk<true, true, LGB_WARPS_Y, LGB_NBUF><<<g, warps * 32, smem, st>>>(
            x, theta, item_sector, item_start, n_items, n, F, q, w, item_loss, item_grad, flag, y);
    else if (kind == LGB_GRAD)
        k_loss_grad_bulk<false, true, LGB_WARPS_NOY, LGB_NBUF><<<g, warps * 32, smem, st>>>(
            x, theta, item_sector, item_start, n_items, n, F, q, w, item_loss, item_grad, flag,
            nullptr);
    else
        k_loss_grad_bulk<false, false, LGB_WARPS_NOY, LGB_NBUF><<<g, warps * 32, smem, st>>>(
            x, theta, item_sector, item_start, n_items, n, F, q, w, item_loss, item_grad, flag,
            nullptr);
    const uint32_t ncol = kind == LGB_LOSS ? 0u : (S * NPAR + LGF_THREADS - 1) / LGF_THREADS;
    launch_after(k_lg_final, ncol + 1, LGF_THREADS, 0, st, (const float *)item_grad,
                 (const float *)item_loss, sector_item, n_items, S, n, (uint32_t)(g * warps), ncol,
                 scale_dev, flag, loss, dF, dq);
    return true;
}

uint32_t calib_max_items(uint64_t n, uint32_t S) {
    return (uint32_t)((n + CALIB_CHUNK - 1) / CALIB_CHUNK + S);
}
uint32_t calib_tiles(uint64_t n) { return (uint32_t)((n + SORT_TILE - 1) / SORT_TILE); }

void launch_calib_sort(const int32_t *sector, uint64_t n, uint32_t S, uint32_t *counts,
                       int32_t *perm, int32_t *sector_off, int32_t *sector_item,
                       int32_t *item_sector, int32_t *item_start, int32_t *n_items,
                       unsigned long long *status, int grid, cudaStream_t st) {
    const uint32_t T = calib_tiles(n);
    const int g = (int)min((uint32_t)grid, max(T, 1u));
    if (T > 0) k_hist<<<g, 256, 0, st>>>(sector, n, S, T, counts, status);
    k_scan_counts<<<1, 1024, 0, st>>>(counts, (uint64_t)S * T);
    if (T > 0) k_scatter<<<g, 32, 0, st>>>(sector, n, S, T, counts, perm);
    if (T > 0)
        k_items<<<1, 1024, 0, st>>>(counts, S, T, n, sector_off, sector_item, item_sector,
                                    item_start, n_items, calib_max_items(n, S));
}

void launch_calib_gather(const float *src, uint32_t width, const int32_t *perm, uint64_t n,
                         float *dst, int grid, cudaStream_t st) {
    k_gather<<<grid, 256, 0, st>>>(src, width, perm, n, dst);
}

void launch_calib_forward(const float *x, const int32_t *item_sector, const int32_t *item_start,
                          const int32_t *sector_off, const int32_t *n_items, uint32_t max_items,
                          const float *F, const float *q, float *y, int grid, cudaStream_t st) {
    // one warp per item (8 per block); the block scheduler keeps the SMs full
    const int g = (int)((max_items + 7) / 8 + 1);
    (void)grid;
    k_forward<<<g, 256, 0, st>>>(x, item_sector, item_start, sector_off, n_items, F, q, y);
}

void launch_calib_loss(const float *x, const float *theta, const int32_t *item_sector,
                       const int32_t *item_start, const int32_t *sector_off,
                       const int32_t *sector_item, const int32_t *n_items, uint32_t max_items,
                       uint32_t S, uint64_t n, const float *F, const float *q, const float *w,
                       float *item_loss, unsigned int *flag, float *loss, int sms, int grid,
                       cudaStream_t st) {
    if (launch_loss_grad_bulk(LGB_LOSS, x, theta, item_sector, item_start, sector_item, n_items,
                              S, n, F, q, w, nullptr, item_loss, nullptr, flag, loss, nullptr,
                              nullptr, nullptr, sms, st))
        return;
    // one warp per item (8 per block); the block scheduler keeps the SMs full
    const int g = (int)((max_items + 7) / 8 + 1);
    (void)grid;
    k_loss_items<<<g, 256, 0, st>>>(x, theta, item_sector, item_start, sector_off, n_items, F, q, w,
                                   item_loss);
    launch_after(k_loss_final, 1, 1024, 0, st, item_loss, n_items, n, loss);
}

void launch_calib_loss_grad(const float *x, const float *theta, const int32_t *item_sector,
                            const int32_t *item_start, const int32_t *sector_off,
                            const int32_t *sector_item, const int32_t *n_items, uint32_t S,
                            uint64_t n, const float *F, const float *q, const float *w,
                            const float *scale_dev, float *item_loss, float *item_grad,
                            float *sector_loss, unsigned int *tickets, float *loss, float *dF,
                            float *dq, float *y, int sms, cudaStream_t st) {
    if (launch_loss_grad_bulk(y ? LGB_GRAD_Y : LGB_GRAD, x, theta, item_sector, item_start,
                              sector_item, n_items, S, n, F, q, w, scale_dev, item_loss,
                              item_grad, tickets + S + 1, loss, dF, dq, y, sms, st))
        return;
    // two resident blocks of 8 warps per SM, each warp a contiguous run of items
    const int g = max(sms, 1) * 2;
    if (y)
        k_loss_grad<true><<<g, 256, 0, st>>>(x, theta, item_sector, item_start, sector_off,
                                             sector_item, n_items, S, n, F, q, w, scale_dev,
                                             item_loss, item_grad, sector_loss, tickets, loss, dF,
                                             dq, y);
    else
        k_loss_grad<false><<<g, 256, 0, st>>>(x, theta, item_sector, item_start, sector_off,
                                              sector_item, n_items, S, n, F, q, w, scale_dev,
                                              item_loss, item_grad, sector_loss, tickets, loss,
                                              dF, dq, y);
}

void launch_calib_grad_scale(const float *g, const float *dF, const float *dq, uint32_t S,
                             float *out_F, float *out_q, cudaStream_t st) {
    k_grad_scale<<<(S * NPAR + 255) / 256, 256, 0, st>>>(g, dF, dq, S, out_F, out_q);
}

void launch_calib_grad(const float *x, const float *grad_y, const int32_t *item_sector,
                       const int32_t *item_start, const int32_t *sector_off,
                       const int32_t *sector_item, const int32_t *n_items, uint32_t max_items,
                       uint32_t S, const float *F, float *item_grad, float *dF, float *dq,
                       float *dx, int grid, cudaStream_t st) {
    const int g = (int)min((uint32_t)grid, (max_items + 7) / 8 + 1);
    k_grad_items<<<g, 256, 0, st>>>(x, grad_y, item_sector, item_start, sector_off, n_items, F,
                                    item_grad, dx);
    launch_after(k_grad_final, (S * NPAR + 255) / 256, 256, 0, st, item_grad, sector_item, S,
                 (const float *)nullptr, 1.0f, dF, dq);
}

}  // namespace svt
