// common.cuh -- internal helpers of the CUDA path (not part of the C ABI).
//
// Device-side error reporting, the workspace carver, warp/block scans and the decoupled
// look-back tile prefix used by the single-pass compaction and scan kernels.
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "citron.h"

namespace citron {

constexpr uint32_t kFull = 0xffffffffu;

// Device error word layout (first 64 bytes of every workspace): word 0 = first error code.
enum DevErr : uint32_t {
    kDevOk = 0,
    kDevTimeout = 1,      // a bounded spin gave up
    kDevOverflow = 2,     // a uint64 sum wrapped
    kDevTooLong = 3,      // a row exceeded a compiled capacity
    kDevBadInput = 4,     // input violated the CSR contract where the kernel checks it
    kDevScratch = 5,      // workspace sized for a smaller max out-degree than the input has
    kDevBudget = 6,       // the count's time budget ran out
};

__device__ __forceinline__ void set_error(uint32_t *err, uint32_t code)
{
    atomicCAS(err, 0u, code);
}

// Spin limit for every device wait (decoupled look-back).  Each probe is an L2 round trip
// (~1 us under load), so the limit bounds a wait to a few seconds at most.
constexpr uint32_t kSpinLimit = 1u << 22;

// Bounds of the decoupled look-back waits, passed to every kernel that waits on another tile:
// the spin limit and, for fault-injection tests only, a tile that never publishes its prefix
// (~0u: none), so that its successor's bounded wait must run out.
struct WaitCfg {
    uint32_t spin_limit = kSpinLimit;
    uint32_t stall_tile = 0xffffffffu;
};

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Time budget of one count shared by all of its launches: clock0 holds the global time of the
// first check (0 before it); a block asks before it takes more work.
struct Budget {
    unsigned long long *clock0 = nullptr;
    unsigned long long ns = 0;  // 0: no limit

    __device__ __forceinline__ bool over(uint32_t *err) const
    {
        if (!ns) return false;
        const unsigned long long now = global_ns();
        unsigned long long t0 = *(volatile unsigned long long *)clock0;
        if (t0 == 0) {
            t0 = atomicCAS(clock0, 0ull, now);
            if (t0 == 0) t0 = now;
        }
        // another block may have started the clock a moment after this one read the timer
        if (now <= t0 || now - t0 <= ns) return false;
        set_error(err, kDevBudget);
        return true;
    }
};

// Exact uint64 accumulation into a global counter; flags a wrap past 2^64 - 1.
__device__ __forceinline__ void add_checked(unsigned long long *dst, unsigned long long v,
                                            uint32_t *err)
{
    if (v == 0) return;
    unsigned long long old = atomicAdd(dst, v);
    if (old + v < old) set_error(err, kDevOverflow);
}

// Warp sum of uint64 lane values with wrap detection.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v, uint32_t *err)
{
    bool wrapped = false;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(kFull, v, o);
        unsigned long long s = v + w;
        wrapped |= s < v;
        v = s;
    }
    if (__any_sync(kFull, wrapped) && (threadIdx.x & 31) == 0) set_error(err, kDevOverflow);
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Inclusive warp scan (uint32).
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive block scan of one uint32 per thread; returns the exclusive prefix and the total.
// `scratch` needs blockDim.x / 32 + 1 words.  Contains __syncthreads.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *scratch, uint32_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t incl = warp_incl_scan(v);
    if (lane == 31) scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? scratch[lane] : 0;
        uint32_t si = warp_incl_scan(s);
        if (lane < nw) scratch[lane] = si - s;
        if (lane == nw - 1) scratch[nw] = si;
    }
    __syncthreads();
    uint32_t r = scratch[warp] + incl - v;
    total = scratch[nw];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------------------------
// Decoupled look-back (single-pass prefix over tiles).  status[t] packs a 2-bit flag and a 62-bit
// value: flag 1 = the tile's own aggregate is published, flag 2 = its inclusive prefix is.
// Tiles take ids from an atomic ticket in launch order, so a tile only ever waits on tiles that
// are already running; every wait is bounded by kSpinLimit and reports kDevTimeout.

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void publish(unsigned long long *status, uint32_t t,
                                        unsigned long long v)
{
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> ref(status[t]);
    ref.store(v, cuda::memory_order_release);
}

__device__ __forceinline__ unsigned long long peek(unsigned long long *status, long long t)
{
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> ref(status[t]);
    return ref.load(cuda::memory_order_acquire);
}

// Called by ONE full warp of the tile's block.  Returns the exclusive prefix of tile t and
// publishes its inclusive prefix.  `agg` must be the same on all lanes.
__device__ __forceinline__ unsigned long long lookback_warp(unsigned long long *status, uint32_t t,
                                                            unsigned long long agg, uint32_t *err,
                                                            const WaitCfg &wc)
{
    const int lane = threadIdx.x & 31;
    if (t == wc.stall_tile) return 0;  // injected fault: this tile never publishes
    if (t == 0) {
        if (lane == 0) publish(status, 0, kFlagPre | agg);
        return 0;
    }
    if (lane == 0) publish(status, t, kFlagAgg | agg);
    unsigned long long excl = 0;
    long long j = (long long)t - 1;
    uint32_t spins = 0;
    while (true) {
        long long idx = j - lane;
        unsigned long long s = idx >= 0 ? peek(status, idx) : kFlagPre;
        unsigned long long flag = s & ~kValMask;
        uint32_t pre = __ballot_sync(kFull, flag == kFlagPre);
        uint32_t zero = __ballot_sync(kFull, flag == 0);
        uint32_t upto = pre ? ((__ffs(pre) == 32) ? kFull : ((1u << __ffs(pre)) - 1)) : kFull;
        if (zero & upto) {
            if (++spins > wc.spin_limit) {
                if (lane == 0) set_error(err, kDevTimeout);
                break;
            }
            continue;
        }
        unsigned long long v = (upto >> lane) & 1 ? (s & kValMask) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        excl += v;
        if (pre) break;
        j -= 32;
    }
    if (lane == 0) publish(status, t, kFlagPre | ((excl + agg) & kValMask));
    return excl;
}

// Where a finished root's count goes, besides the grand total: the per-root array and/or the
// total of the root's group (the graph it belongs to, in a batch of graphs).
struct RootSink {
    unsigned long long *per_root;        // per root (optional)
    const uint32_t *group_of_row;        // group of each root (optional, with group_counts)
    unsigned long long *group_counts;    // per-group totals
    uint32_t ngroups;
    // per DAG arc e = (u, v) (optional, k >= 3): the k-cliques whose first two vertices are u, v,
    // i.e. the count of the edge task of e (zeroed by the classification pass, then added to)
    unsigned long long *per_arc;

    __device__ __forceinline__ void put(uint32_t u, unsigned long long r, uint32_t *err) const
    {
        if (per_root) per_root[u] = r;
        if (group_counts) {
            const uint32_t g = group_of_row[u];
            if (g < ngroups) add_checked(&group_counts[g], r, err);
            else set_error(err, kDevBadInput);
        }
    }
    // A root counted by several blocks (a split heavy root): each adds its part.
    __device__ __forceinline__ void add(uint32_t u, unsigned long long r, uint32_t *err) const
    {
        if (per_root) add_checked(&per_root[u], r, err);
        if (group_counts) {
            const uint32_t g = group_of_row[u];
            if (g < ngroups) add_checked(&group_counts[g], r, err);
            else set_error(err, kDevBadInput);
        }
    }
    __device__ __forceinline__ bool wants_root_total() const { return per_root || group_counts; }
};

// A heavy root whose units (edge tasks, or edge sub-tasks (u, a_t, b)) any block may take: the
// block that took the root from the queue publishes it here; blocks that find the root queue
// empty rebuild its local subgraph and take units from the same cursor.
struct HeavySlot {
    uint32_t u;       // the root
    uint32_t units;   // size of its unit space
    uint32_t cursor;  // next unit to take (may run past `units`)
    uint32_t ready;   // 1 once u and units are published
};

struct HelpTable {
    HeavySlot *slots = nullptr;
    uint32_t cap = 0;
    uint32_t *nslots = nullptr;  // slots taken so far (may run past cap: those roots get no help)
};

// Which roots a counting pass takes, besides the out-degree prune: with group_of_row set, only
// the roots whose group asks for this pass's k (group_k[group] == k).
struct RootFilter {
    const uint32_t *group_of_row = nullptr;
    const uint32_t *group_k = nullptr;
    uint32_t ngroups = 0;
    uint32_t k = 0;

    __device__ __forceinline__ bool takes(uint32_t u) const
    {
        if (!group_of_row) return true;
        const uint32_t g = group_of_row[u];
        return g < ngroups && group_k[g] == k;
    }
};

}  // namespace citron

// ---------------------------------------------------------------------------------------------
// Host side: workspace carving (every region 256-byte aligned).

namespace citron_host {

// Path thresholds of the counting phase (see count.cu).
// The instrumented bitmap kernel (word-op counting, per-arc output) is compiled for k <= 8 only:
// the deep recursion of k = 9..12 takes most of the build's time, and debug modes there are rare.
constexpr uint32_t kInstrumentedMaxK = 8;

struct CountPlan {
    uint32_t small_max = 32;       // roots with out-degree <= this use the warp-register path
    uint32_t bitmap_max = 1024;    // ... <= this use the shared-memory bitmap path
    uint32_t warps_per_cta = 32;   // warps per block of the bitmap path (fewer if shared memory is short)
    uint32_t compact_max = 128;    // candidate sets up to this size are re-encoded compactly (0: never)
    uint32_t max_blocks = 0;       // cap on the blocks of each counting launch (0: no cap)
    uint32_t split_min = 384;      // bitmap-path roots of at least this out-degree share their units
                                   // with idle blocks (0xffffffff: never)
};

// Options and outputs of one counting call.
struct CountRun {
    CountPlan plan;
    citron::RootSink sink = {nullptr, nullptr, nullptr, 0, nullptr};  // per-root / group / arc outputs
    citron::RootFilter filter;                               // roots of this pass
    bool count_work = false;                 // instrumented launch: count word operations
    bool time_kernels = false;               // record device time of the counting kernels
    bool balance = false;                    // record when each bitmap-path block starts and ends
    unsigned long long budget_ns = 0;        // device time the count may take (0: no limit)
    unsigned long long work = 0;             // out: word operations (AND + POPC of 32-bit words)
    float kernel_ms[3] = {0, 0, 0};          // out: warp-register, bitmap, sorted-list kernels
    float busy_ms[2] = {0, 0};               // out: bitmap kernel's span (first start to last end)
                                             // and tail (first block end to last block end)
};

// Number of kernels this library has launched (all devices, all threads).
void note_launches(unsigned n);
unsigned long long launches();

// Faults injected by citron_set_faults (all zero in normal operation).
citron_faults injected_faults();
// Look-back bounds under the injected faults.
inline citron::WaitCfg wait_cfg()
{
    const citron_faults f = injected_faults();
    citron::WaitCfg w;
    if (f.lookback_spin_limit) w.spin_limit = f.lookback_spin_limit;
    if (f.lookback_stall_tile) w.stall_tile = f.lookback_stall_tile - 1;
    return w;
}

struct Carver {
    char *base;
    size_t cap;
    size_t used = 0;
    bool ok = true;
    Carver(void *p, size_t bytes) : base((char *)p), cap(bytes) {}
    template <class T>
    T *take(size_t count)
    {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (used + bytes > cap || !base) {
            ok = false;
            used += bytes;
            return nullptr;
        }
        T *p = (T *)(base + used);
        used += bytes;
        return p;
    }
};

// Size-only twin of Carver used by the *_bytes queries.
struct Sizer {
    size_t used = 0;
    template <class T>
    void take(size_t count) { used += (count * sizeof(T) + 255) & ~size_t(255); }
};

}  // namespace citron_host
