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
                       const int32_t *n_items, uint32_t max_items, uint64_t n, const float *F,
                       const float *q, const float *w, float *item_loss, float *loss, int grid,
                       cudaStream_t st) {
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
