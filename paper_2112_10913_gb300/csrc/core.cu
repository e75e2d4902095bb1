// core.cu -- core ordering (Algorithm OrdCore, Sec. III) computed in synchronous peeling rounds.
//
// Each round first raises the level to the smallest remaining degree (the level never falls),
// then removes every remaining vertex whose remaining degree is at most the level, all together,
// and only then lowers the remaining degrees of their neighbours.  rank orders the vertices by
// (removal round, id).  A vertex's later neighbours were all present when its round began, so its
// out-degree is at most that round's level and the maximum out-degree is the degeneracy -- the
// property the paper wants from the core ordering (Sec. III, Table II) -- while the rounds run in
// parallel instead of one vertex per step.
//
// One cooperative persistent kernel runs every round.  Per round, one warp per frontier vertex
// walks its adjacency row and decrements the degrees of the neighbours still present with
// atomics; a neighbour whose degree falls from level + 1 to level joins the next frontier (only one
// decrement can make that step, so it is pushed exactly once).  A round that leaves no frontier
// raises the level to the grid minimum of the remaining degrees and rebuilds the frontier with a
// scan.  Rounds are separated by a grid barrier whose wait is bounded in time.  The ranks then
// come from the stable radix sort of the ids by round (order.cu).
#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace citron {

constexpr uint32_t kPresent = 0xffffffffu;  // round_of[] of a vertex not removed yet
constexpr int kCoreThreads = 1024;
constexpr unsigned long long kGridWaitNs = 4000000000ull;  // 4 s per barrier at most

struct CoreState {
    unsigned int bar_count;
    unsigned int bar_gen;
    unsigned int cnt[3];  // frontier sizes, ring over rounds (round t's frontier in cnt[t % 3])
    unsigned int gmin;    // smallest remaining degree (level raise)
    unsigned int rounds;
    unsigned int level;
};

__device__ __forceinline__ uint32_t load_relaxed(unsigned int *p)
{
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> r(*p);
    return r.load(cuda::memory_order_relaxed);
}

// Barrier over all blocks of a cooperative launch (all of them resident).  Returns false on every
// thread of the block when the wait (at most wait_ns) gave up or some block has reported an
// error, so that the kernel can return; the other blocks then give up at their next barrier.
__device__ bool grid_barrier(CoreState *s, uint32_t *err, unsigned long long wait_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(s->bar_gen), cnt(s->bar_count);
        const unsigned int g = gen.load(cuda::memory_order_acquire);
        __threadfence();
        int ok = 1;
        if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1) {
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.store(g + 1, cuda::memory_order_release);
        } else {
            const unsigned long long t0 = global_ns();
            uint32_t spins = 0;
            while (gen.load(cuda::memory_order_acquire) == g) {
                if ((++spins & 63u) == 0 && global_ns() - t0 > wait_ns) {
                    set_error(err, kDevTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (load_relaxed(err)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ __launch_bounds__(kCoreThreads) void k_core_peel(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ cols,
    uint32_t *cur, uint32_t *round_of, uint32_t *fa, uint32_t *fb, CoreState *s, uint32_t *err,
    unsigned long long wait_ns, uint32_t absent_block)
{
    // injected fault (tests only): this block never arrives at the first barrier, so that the
    // other blocks' bounded wait there must run out
    if (blockIdx.x == absent_block) return;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31, gwarp = tid >> 5, nwarps = nthreads >> 5;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;

    for (uint32_t v = tid; v < n; v += nthreads) {
        const uint64_t a = off[v], b = off[v + 1];
        if (b < a || b > arcs) set_error(err, kDevBadInput);
        cur[v] = b >= a ? (uint32_t)(b - a) : 0u;
        round_of[v] = kPresent;
    }
    if (leader) s->gmin = kPresent;
    if (!grid_barrier(s, err, wait_ns)) return;

    uint32_t t = 0, level = 0, removed = 0, f = 0;
    uint32_t *F = fa, *N = fb;
    while (removed < n) {
        if (f == 0) {
            // Raise the level to the smallest remaining degree ...
            uint32_t m = kPresent;
            for (uint32_t v = tid; v < n; v += nthreads)
                if (__ldcg(round_of + v) == kPresent) m = min(m, __ldcg(cur + v));
            m = __reduce_min_sync(kFull, m);
            if (lane == 0 && m != kPresent) atomicMin(&s->gmin, m);
            if (!grid_barrier(s, err, wait_ns)) return;
            const uint32_t least = load_relaxed(&s->gmin);
            if (least == kPresent) {  // nothing left although removed < n: inconsistent input
                set_error(err, kDevBadInput);
                return;
            }
            level = max(level, least);
            // ... and take every present vertex of degree <= level as this round's frontier.
            for (uint32_t v0 = tid - lane; v0 < n; v0 += nthreads) {
                const uint32_t v = v0 + lane;
                const bool take = v < n && __ldcg(round_of + v) == kPresent && __ldcg(cur + v) <= level;
                const uint32_t mask = __ballot_sync(kFull, take);
                uint32_t base = 0;
                if (lane == 0 && mask) base = atomicAdd(&s->cnt[t % 3], (unsigned)__popc(mask));
                base = __shfl_sync(kFull, base, 0);
                if (take) {
                    __stcg(F + base + __popc(mask & lanemask_lt()), v);
                    __stcg(round_of + v, t);
                }
            }
            if (!grid_barrier(s, err, wait_ns)) return;
            f = load_relaxed(&s->cnt[t % 3]);
            if (leader) s->gmin = kPresent;  // every block read it before the barrier above
            if (f == 0 || f > n - removed) {
                set_error(err, kDevBadInput);
                return;
            }
        }
        // Remove the frontier: lower the degrees of the neighbours still present.
        if (leader) s->cnt[(t + 2) % 3] = 0;  // last read at the start of round t - 1
        const uint32_t nxt = (t + 1) % 3;
        for (uint32_t i = gwarp; i < f; i += nwarps) {
            const uint32_t v = __ldcg(F + i);
            const uint64_t a = off[v], b = min(off[v + 1], arcs);
            for (uint64_t e0 = a; e0 < b; e0 += 32) {
                const uint64_t e = e0 + lane;
                bool push = false;
                uint32_t w = 0;
                if (e < b) {
                    w = cols[e];
                    if (w >= n)
                        set_error(err, kDevBadInput);
                    else if (__ldcg(round_of + w) == kPresent)
                        push = atomicSub(cur + w, 1u) == level + 1;
                }
                const uint32_t mask = __ballot_sync(kFull, push);
                if (mask) {
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(&s->cnt[nxt], (unsigned)__popc(mask));
                    base = __shfl_sync(kFull, base, 0);
                    if (push) {
                        __stcg(N + base + __popc(mask & lanemask_lt()), w);
                        __stcg(round_of + w, t + 1);
                    }
                }
            }
        }
        if (!grid_barrier(s, err, wait_ns)) return;
        removed += f;
        t++;
        f = load_relaxed(&s->cnt[t % 3]);
        if (f > n - removed) {
            set_error(err, kDevBadInput);
            return;
        }
        uint32_t *tmp = F;
        F = N;
        N = tmp;
    }
    if (leader) {
        s->rounds = t;
        s->level = level;
    }
}

}  // namespace citron

namespace citron_host {

using namespace citron;

cudaError_t launch_rank_by_key(uint32_t n, const uint32_t *keys, uint32_t key_bound, uint32_t *rank,
                               uint32_t *perm, uint32_t *err, Carver &c, cudaStream_t st);
size_t order_ws_bytes(uint32_t n);

size_t core_ws_bytes(uint32_t n)
{
    Sizer s;
    s.take<CoreState>(1);
    for (int i = 0; i < 4; i++) s.take<uint32_t>((size_t)n + 1);  // cur, round_of, two frontiers
    return s.used + order_ws_bytes(n);
}

// Synchronous: the round count sizes the radix sort.  Device errors land in err.
cudaError_t launch_core_order(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                              uint32_t *rank, uint32_t *perm, uint32_t *h_level,
                              uint32_t *h_rounds, uint32_t *err, Carver &c, cudaStream_t st,
                              int num_sms)
{
    CoreState *state = c.take<CoreState>(1);
    uint32_t *cur = c.take<uint32_t>((size_t)n + 1);
    uint32_t *round_of = c.take<uint32_t>((size_t)n + 1);
    uint32_t *fa = c.take<uint32_t>((size_t)n + 1);
    uint32_t *fb = c.take<uint32_t>((size_t)n + 1);
    if (!c.ok) return cudaErrorMemoryAllocation;
    if (h_level) *h_level = 0;
    if (h_rounds) *h_rounds = 0;
    if (n == 0) return cudaSuccess;
    int dev = 0, coop = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!e && !coop) return cudaErrorNotSupported;
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_core_peel, kCoreThreads, 0);
    if (!e && per_sm < 1) return cudaErrorLaunchOutOfResources;
    if (!e) e = cudaMemsetAsync(state, 0, sizeof(CoreState), st);
    if (e) return e;
    // One thread per vertex at most (fewer blocks make cheaper barriers), all blocks resident.
    uint32_t grid = (n + kCoreThreads - 1) / kCoreThreads;
    if (grid > (uint32_t)(num_sms * per_sm)) grid = (uint32_t)(num_sms * per_sm);
    const citron_faults f = injected_faults();
    unsigned long long wait_ns = f.barrier_wait_ns ? f.barrier_wait_ns : kGridWaitNs;
    uint32_t absent = f.barrier_absent_block ? f.barrier_absent_block - 1 : 0xffffffffu;
    void *args[] = {&n, &arcs, &off, &cols, &cur, &round_of, &fa, &fb, &state, &err, &wait_ns, &absent};
    e = cudaLaunchCooperativeKernel((const void *)k_core_peel, dim3(grid), dim3(kCoreThreads), args,
                                    0, st);
    note_launches(1);
    if (e) return e;
    CoreState hs = {};
    uint32_t code = 0;
    e = cudaMemcpyAsync(&hs, state, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(&code, err, sizeof(code), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return e;
    if (code) return cudaSuccess;  // reported from the error word by the caller
    if (h_level) *h_level = hs.level;
    if (h_rounds) *h_rounds = hs.rounds;
    return launch_rank_by_key(n, round_of, hs.rounds, rank, perm, err, c, st);
}

}  // namespace citron_host
