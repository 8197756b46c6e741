// svt_noalloc.cu -- svt_run without a caller-provided workspace.
//
// Some callers cannot allocate device memory at all: a trigger front-end
// process that only receives device pointers from the framework that owns
// the GPU, a real-time loop whose rules forbid allocation (with its latency
// and failure modes) once data taking has started, or a host program that
// links this library without a device allocator of its own.  For them this
// entry point takes its scratch from one fixed array that lives in the
// library itself.  The array is reserved on a device when this code is
// loaded there -- under CUDA's default lazy module loading, at the first
// svt_run_noalloc call on that device -- and held until the process exits;
// every call on that device shares it.
#include <mutex>

#include "svt_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;   // 32 MiB per device

// The shared scratch.  In host code this name is only a stand-in for the
// device array; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices];   // null until a lookup on that device succeeds
std::mutex g_scratch_mu;

// Device address of the scratch on the current device.  Only a successful
// lookup is kept: a failed one (for example a first call made while the
// stream is being captured, when the module cannot be loaded) leaves the
// slot empty, clears the error and is tried again on the next call.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SVT_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SVT_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SVT_OK;
}

}  // namespace

extern "C" {

size_t svt_run_noalloc_scratch_bytes(void) { return kScratchBytes; }

int svt_run_noalloc(const uint32_t *d_words, uint64_t n_words, const uint64_t *d_event_off,
                    uint64_t n_events, const int16_t *d_F, const int16_t *d_q,
                    const svt_config *cfg, uint64_t road_cap, uint32_t *d_out,
                    uint32_t *d_event_road, uint64_t *d_counts, uint64_t *d_status,
                    const svt_schedule *sched, void *stream) {
    const size_t need = svt_run_workspace_size(n_words, n_events, road_cap, sched);
    if (need > kScratchBytes) return SVT_ERR_OOM;
    void *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != SVT_OK) return rc;
    // svt_run initialises every part of the workspace it reads (status,
    // counters, scans, per-road slots) at the start of each call, so the
    // previous call's contents in the shared array do not leak into this one.
    return svt_run(d_words, n_words, d_event_off, n_events, d_F, d_q, cfg, road_cap, d_out,
                   d_event_road, d_counts, d_status, scratch, kScratchBytes, sched, nullptr,
                   stream);
}

}  // extern "C"
