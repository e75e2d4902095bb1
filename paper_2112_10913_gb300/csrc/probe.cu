// probe.cu -- peak rate of the counting phase's unit of work on this device: the 32-bit word
// operation (AND of two candidate words, POPC, add), on register operands, so that no memory
// level limits it.  Every thread keeps 8 independent chains; the operands change every
// iteration (a ^= s) so that nothing is loop-invariant.  Per word: AND, POPC, IADD, XOR.
#include <cuda_runtime.h>
#include <stdint.h>

#include "citron.h"
#include "common.cuh"

namespace citron {

constexpr int kProbeChains = 8;

// Receives a count only when a thread's sum hits one chosen value, so that the compiler must
// keep every chain; device code names it directly.
static __device__ unsigned long long g_probe_sink;

__global__ __launch_bounds__(1024) void k_probe_word_ops(uint32_t iters, uint32_t seed)
{
    uint32_t a[kProbeChains], b[kProbeChains], s[kProbeChains];
    const uint32_t x = seed ^ (blockIdx.x * 1024u + threadIdx.x) * 2654435761u;
#pragma unroll
    for (int j = 0; j < kProbeChains; j++) {
        a[j] = x * (2 * j + 1) + 0x9e3779b9u * j;
        b[j] = ~x ^ (0x85ebca6bu * (j + 1));
        s[j] = 0;
    }
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < kProbeChains; j++) {
            s[j] += __popc(a[j] & b[j]);
            a[j] ^= s[j];
        }
    }
    uint32_t t = 0;
#pragma unroll
    for (int j = 0; j < kProbeChains; j++) t += s[j];
    if (t == 0x7fffffffu) atomicAdd(&g_probe_sink, 1ull);
}

}  // namespace citron

extern "C" citron_status citron_probe_word_ops(uint32_t blocks_per_sm, uint32_t iters,
                                               double *h_ops_per_s, float *h_ms, void *stream)
{
    using namespace citron;
    if (!h_ops_per_s || blocks_per_sm == 0 || blocks_per_sm > 8 || iters == 0) return CITRON_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return CITRON_E_CUDA;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) || cudaEventCreate(&b)) {
        if (a) cudaEventDestroy(a);
        return CITRON_E_CUDA;
    }
    const uint32_t grid = (uint32_t)sms * blocks_per_sm;
    k_probe_word_ops<<<grid, 1024, 0, st>>>(8, 1u);  // warm-up (module load)
    cudaEventRecord(a, st);
    k_probe_word_ops<<<grid, 1024, 0, st>>>(iters, 12345u);
    cudaEventRecord(b, st);
    citron_host::note_launches(2);
    e = cudaGetLastError();
    if (!e) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (!e) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e) return CITRON_E_CUDA;
    const double ops = (double)grid * 1024.0 * (double)iters * kProbeChains;
    *h_ops_per_s = ms > 0 ? ops / (ms * 1e-3) : 0.0;
    if (h_ms) *h_ms = ms;
    return CITRON_OK;
}
