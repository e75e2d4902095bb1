// noalloc.cu -- k-clique counting for callers that cannot allocate device memory.
//
// citron_count needs a caller-provided workspace.  Some callers have no way to provide one:
// host applications and plugin frameworks that own the device heap and forbid allocation after
// start-up, real-time loops that cannot afford the implicit synchronisation of cudaMalloc and
// cudaFree, and plain C callers that have no allocator of their own.  For them this file keeps
// the counting scratch in one fixed, file-scope device array.
//
// The array is a static __device__ object: every GPU that loads the library holds its
// kNoAllocBytes until the process exits.  In host code the symbol is only a host-side stand-in,
// so its device address is looked up once per device with cudaGetSymbolAddress (on the first
// call made with that device current) and that address is what the kernels receive.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "citron.h"
#include "common.cuh"

namespace citron_host {
cudaError_t run_count(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_cols, uint32_t k,
                      CountRun &run, uint32_t *err, Carver &c, cudaStream_t s, int num_sms,
                      unsigned long long *h_result);
}  // namespace citron_host

namespace {

// Stated limits of the fixed scratch: at most kNoAllocMaxN vertices.  The first 256 bytes hold
// the device error word; the rest holds the root lists, queue counters and the sum.
constexpr uint32_t kNoAllocMaxN = 1u << 16;
constexpr size_t kNoAllocBytes = (size_t)1 << 20;  // 1 MiB per device
constexpr size_t kHeaderBytes = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mutex;
void *g_device_ptr[64] = {};
int g_num_sms[64] = {};

// Device address of the scratch array for the current device (looked up on first use).
cudaError_t scratch_for_current_device(void **ptr, int *sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_device_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_num_sms[dev] = v;
        g_device_ptr[dev] = p;
    }
    *ptr = g_device_ptr[dev];
    *sms = g_num_sms[dev];
    return cudaSuccess;
}

citron_status status_of(cudaError_t e)
{
    if (e == cudaSuccess) return CITRON_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? CITRON_E_WORKSPACE : CITRON_E_CUDA;
}

}  // namespace

extern "C" citron_status citron_count_noalloc(uint32_t n, const uint64_t *d_dag_off,
                                              const uint32_t *d_dag_cols, uint32_t k,
                                              uint64_t *h_count, void *stream)
{
    using namespace citron_host;
    if (!h_count || !d_dag_off || k == 0) return CITRON_E_INVALID;
    if (k > CITRON_MAX_K || n > kNoAllocMaxN) return CITRON_E_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    void *base = nullptr;
    int sms = 0;
    cudaError_t e = scratch_for_current_device(&base, &sms);
    if (e != cudaSuccess) return status_of(e);
    uint32_t *err = (uint32_t *)base;
    // the array keeps the previous call's contents: clear the error word before any kernel
    if ((e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s))) return status_of(e);
    if (k == 1) {
        *h_count = n;
        return status_of(cudaStreamSynchronize(s));
    }
    if (k == 2) {
        uint64_t m = 0;
        e = cudaMemcpyAsync(&m, d_dag_off + n, sizeof(m), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return status_of(e);
        *h_count = m;
        return CITRON_OK;
    }
    if (n && !d_dag_cols) return CITRON_E_INVALID;
    Carver c((char *)base + kHeaderBytes, kNoAllocBytes - kHeaderBytes);
    CountRun run;  // defaults: every region the count reads is cleared inside run_count
    unsigned long long result = 0;
    e = run_count(n, d_dag_off, d_dag_cols, k, run, err, c, s, sms, &result);
    if (e) return status_of(e);
    uint32_t code = 0;
    e = cudaMemcpyAsync(&code, err, sizeof(code), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return status_of(e);
    switch (code) {
        case citron::kDevOk: *h_count = result; return CITRON_OK;
        case citron::kDevTimeout: return CITRON_E_TIMEOUT;
        case citron::kDevOverflow: return CITRON_E_OVERFLOW;
        case citron::kDevTooLong: return CITRON_E_UNSUPPORTED;
        case citron::kDevBadInput: return CITRON_E_INVALID;
        case citron::kDevScratch: return CITRON_E_WORKSPACE;
        case citron::kDevBudget: return CITRON_E_BUDGET;
        default: return CITRON_E_CUDA;
    }
}
