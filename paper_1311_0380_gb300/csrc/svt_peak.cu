// svt_peak.cu -- arithmetic throughput of this GPU, measured: context for the
// fit kernel's integer-ALU and issue rooflines.
//
// Every thread runs rings of eight chains.  Each new value reads its
// neighbour chain's previous value, so no chain has a closed form the compiler
// could fold, while the eight chains give enough independent work per thread
// to keep the pipes full at full occupancy.
//   mode 0: int32 3-input adds (a + b + c)
//   mode 1: int32 multiply-adds (a * b + c)
//   mode 2: both, as two independent rings interleaved
//   mode 3: fp32 multiply and fused multiply-add (the fastest instruction
//           stream: a measure of the schedulers' issue rate)
#include "svt_kernels.cuh"

namespace svt {

namespace {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;

// operations per chain and step of each mode
__host__ __device__ constexpr int peak_ops(int mode) { return mode == 0 || mode == 1 ? 1 : 2; }

template <int MODE>
__global__ void __launch_bounds__(PEAK_THREADS)
    k_pipe_peak(uint32_t iters, uint32_t seed, uint32_t *sink) {
    uint32_t a[PEAK_CHAINS], m[PEAK_CHAINS];
    float f[PEAK_CHAINS];
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) {
        a[i] = (threadIdx.x + 1u) * (uint32_t)(2 * i + 3) + seed;
        m[i] = a[i] ^ 0x55u;
        f[i] = (float)a[i] * 1e-9f;
    }
    const uint32_t c = seed ^ 0x9E3779B9u;
    const float fc = 1.0000001f, fd = 1e-7f;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int i = 0; i < PEAK_CHAINS; ++i) {
                const int j = (i + 1) % PEAK_CHAINS;
                if (MODE == 0 || MODE == 2) a[i] = a[i] + a[j] + c;
                if (MODE == 1 || MODE == 2) m[i] = m[i] * m[j] + c;
                if (MODE == 3) f[i] = fmaf(f[i], fc, f[j] * fd);
            }
        }
    }
    uint32_t r = 0;
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) {
        r ^= a[i] ^ m[i];
        sum += f[i];
    }
    // keeps the work alive; almost never taken
    if (r == seed || sum == 1234.5f) sink[blockIdx.x & 255u] = r;
}

}  // namespace

}  // namespace svt

extern "C" int svt_pipe_peak(uint32_t mode, uint32_t iters, double *ops_per_s, double *seconds,
                             void *stream) {
    using namespace svt;
    if (mode > 3 || iters < 1 || !ops_per_s) return SVT_ERR_BAD_ARG;
    int device = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return SVT_ERR_CUDA;
    void (*kernel)(uint32_t, uint32_t, uint32_t *) =
        mode == 0 ? k_pipe_peak<0>
                  : (mode == 1 ? k_pipe_peak<1> : (mode == 2 ? k_pipe_peak<2> : k_pipe_peak<3>));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, PEAK_THREADS, 0) !=
            cudaSuccess ||
        per_sm < 1)
        return SVT_ERR_CUDA;
    const int grid = sms * per_sm;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SVT_OK;
    float ms = 0.f;
    if (cudaMalloc(&sink, 256 * sizeof(uint32_t)) != cudaSuccess) return SVT_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = SVT_ERR_CUDA;
        goto out;
    }
    kernel<<<grid, PEAK_THREADS, 0, st>>>(iters < 64 ? iters : 64, 12345u, sink);   // warm-up
    if (cudaEventRecord(e0, st) != cudaSuccess) { rc = SVT_ERR_CUDA; goto out; }
    kernel<<<grid, PEAK_THREADS, 0, st>>>(iters, 12345u, sink);
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        ms <= 0.f) {
        rc = SVT_ERR_CUDA;
        goto out;
    }
    *ops_per_s = (double)grid * PEAK_THREADS * (double)iters * 4.0 * PEAK_CHAINS *
                 peak_ops((int)mode) / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3;
out:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}
