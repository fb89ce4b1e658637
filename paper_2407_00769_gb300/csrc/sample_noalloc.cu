// Post-selection for callers that cannot allocate device memory.
//
// tn_sample() allocates two small device buffers on every call (the k chosen
// indices and probabilities, before they are copied to the host).  Some
// callers cannot allow that: a plug-in running inside a host application
// that owns all device memory through its own pool and forbids other
// allocations, or a latency-critical thread that must never enter the CUDA
// allocator (cudaMalloc and cudaFree can synchronize the whole device).
// tn_sample_noalloc() runs the same top-k kernel with that scratch held in a
// fixed array in device global memory, so it allocates nothing.
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>
#include <string>

#include "kernels.cuh"

namespace {

constexpr int kMaxK = TN_SAMPLE_NOALLOC_MAX_K;

// The k results, then the multi-block selection's scratch for k <= kMaxK
// (its header, per-block counts and the k kept entries).
constexpr size_t kSelectBytes = 4096 + 1024 * 8 + (size_t)kMaxK * 16;
struct SampleScratch {
    int64_t idx[kMaxK];
    double prob[kMaxK];
    __align__(256) uint8_t select[kSelectBytes];
};

// 44 KiB in every device that loads this library, kept until the process
// exits.  Host code must not pass this name to a kernel: on the host it is
// only a stand-in for the symbol, not a device address.
static __device__ __align__(256) SampleScratch g_sample_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char *g_scratch_addr[kMaxDevices] = {};

// Device address of g_sample_scratch on the current device, looked up once
// per device (with that device current) and cached.
int scratch_for_current_device(char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return tn::record_error(TN_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return tn::record_error(TN_EUNSUPPORTED, "device index beyond the scratch table");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sample_scratch);
        if (e != cudaSuccess || !p)
            return tn::record_error(TN_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                                  cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<char *>(p);
    }
    *out = g_scratch_addr[dev];
    return TN_OK;
}

}  // namespace

extern "C" int tn_sample_noalloc(const double *d_amps, int32_t n_open, int32_t k, int64_t *out_idx,
                                 double *out_prob, void *stream) {
    if (!d_amps || !out_idx || !out_prob) return tn::record_error(TN_EINVAL, "NULL argument");
    if (n_open < 0 || n_open > 30) return tn::record_error(TN_EINVAL, "n_open must be in 0..30");
    const int64_t n = (int64_t)1 << n_open;
    if (k < 1 || k > n) return tn::record_error(TN_EINVAL, "k must be in 1..2^n_open");
    if (k > kMaxK)
        return tn::record_error(TN_EINVAL, "tn_sample_noalloc: k = " + std::to_string(k) +
                                               " exceeds its fixed scratch of " +
                                               std::to_string(kMaxK) +
                                               " results (use tn_sample for larger k)");
    char *base = nullptr;
    const int rc = scratch_for_current_device(&base);
    if (rc != TN_OK) return rc;
    int64_t *d_idx = reinterpret_cast<int64_t *>(base + offsetof(SampleScratch, idx));
    double *d_prob = reinterpret_cast<double *>(base + offsetof(SampleScratch, prob));
    cudaStream_t s = (cudaStream_t)stream;
    // the kernels write entries 0..k-1 of both arrays and initialise the
    // selection's header themselves; nothing is read before it is written,
    // so no clearing is needed
    if (tn::topk_scratch_bytes(n, k) > kSelectBytes)
        return tn::record_error(TN_EUNSUPPORTED, "tn_sample_noalloc: selection scratch exceeds its fixed size");
    cudaError_t e = tn::launch_topk_select((const double2 *)d_amps, n, k, base + offsetof(SampleScratch, select),
                                           d_idx, d_prob, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_idx, d_idx, (size_t)k * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_prob, d_prob, (size_t)k * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return tn::record_error(TN_ECUDA, std::string("tn_sample_noalloc: ") + cudaGetErrorString(e));
    return TN_OK;
}
