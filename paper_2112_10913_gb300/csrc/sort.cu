// sort.cu -- stable ranking of the vertex ids by a key: the degree ordering of Sec. II / Sec. IV
// (key = d(u), ties by id), the degree ordering of many graphs at once (key = (graph, d(u)), ties
// by id) and the removal rounds of the core ordering.
//
// A least-significant-digit radix sort with 8-bit digits in the single-sweep form: one launch
// computes the digit histograms of every pass at once (k_os_hist), then each pass is ONE launch
// (k_os_scatter) in which every tile of 4096 ids ranks its ids stably by the pass's digit (warp
// __match_any_sync peers, per-warp digit counts, a running per-digit base over 16 rounds),
// publishes its 256 digit counts and learns the counts of the tiles before it by a decoupled
// look-back per digit (one thread per digit, eight predecessors read per probe), then scatters.
// The key of an id is read again in every pass (the degree from the offsets, or the key arrays):
// only the ids move.  The ids enter in ascending order, so stability gives the id tie-break; the
// passes of a second, more significant key (the graph of each vertex) come after those of the
// first.  A pass whose digit is the same for every id keeps the order and skips the look-back.
// The last pass writes rank[id] = position and, optionally, perm[position] = id.
#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace citron {

constexpr int kOsThreads = 256;
constexpr int kOsItems = 16;
constexpr uint32_t kOsTile = kOsThreads * kOsItems;  // keys per tile
constexpr int kOsMaxPasses = 8;
constexpr int kOsWindow = 8;  // predecessors read per look-back probe

// The sort keys of an id: the first key (keys[id], or the degree off[id+1] - off[id] when keys
// is NULL) for passes 0 .. lo_passes-1, then the second key hi[id] (optional).
struct SortKeys {
    const uint64_t *off;
    const uint32_t *keys;
    const uint32_t *hi;
    int lo_passes;

    __device__ __forceinline__ uint32_t digit(uint32_t id, int pass) const
    {
        if (pass < lo_passes) {
            const uint32_t key = keys ? keys[id] : (uint32_t)min(off[id + 1] - off[id], (uint64_t)0xffffffffull);
            return (key >> (8 * pass)) & 255u;
        }
        return (hi[id] >> (8 * (pass - lo_passes))) & 255u;
    }
};

// hist[p * 256 + d] = number of keys whose digit p is d, for every pass p at once.
__global__ __launch_bounds__(kOsThreads) void k_os_hist(SortKeys sk, uint32_t n, int passes,
                                                        uint32_t *hist)
{
    __shared__ uint32_t cnt[kOsMaxPasses * 256];
    for (int i = threadIdx.x; i < passes * 256; i += kOsThreads) cnt[i] = 0;
    __syncthreads();
    // the loop bound is uniform over the block, so every lane reaches each __match_any_sync
    for (uint32_t i0 = blockIdx.x * kOsThreads; i0 < n; i0 += gridDim.x * kOsThreads) {
        const uint32_t i = i0 + threadIdx.x;
        const bool valid = i < n;
        for (int p = 0; p < passes; p++) {
            const uint32_t d = valid ? sk.digit(i, p) : 256u;
            // keys of a warp often share a digit (small degrees): one atomic per distinct digit
            const uint32_t peers = __match_any_sync(kFull, d);
            if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[p * 256 + d], __popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += kOsThreads)
        if (cnt[i]) atomicAdd(&hist[i], cnt[i]);
}

// One pass of the sort over tiles taken in launch order (ticket).  status[t * 256 + d] holds the
// look-back word of tile t and digit d (flag in the top two bits: the tile's own count, or the
// inclusive prefix over tiles 0..t).
__global__ __launch_bounds__(kOsThreads) void k_os_scatter(
    SortKeys sk, const uint32_t *__restrict__ vals_in, uint32_t n, int pass,
    const uint32_t *__restrict__ hist, unsigned long long *status, uint32_t *ticket,
    uint32_t *vals_out, uint32_t *rank_out, uint32_t *perm_out, uint32_t *err, WaitCfg wc)
{
    __shared__ uint32_t s_gstart[256];      // first position of each digit in the output
    __shared__ uint32_t s_base[256];        // running count of each digit in this tile
    __shared__ uint32_t s_wcnt[kOsThreads / 32][256];
    __shared__ uint32_t s_scan[kOsThreads / 32 + 1];
    __shared__ uint32_t s_tile;
    __shared__ int s_trivial;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        s_tile = atomicAdd(ticket, 1u);
        s_trivial = 0;
    }
    const uint32_t hd = hist[pass * 256 + tid];
    __syncthreads();
    if (hd == n) s_trivial = 1;  // every key has this digit: the pass keeps the order
    uint32_t total;
    s_gstart[tid] = block_excl_scan(hd, s_scan, total);
    s_base[tid] = 0;
    const uint32_t t = s_tile;
    const uint32_t tile0 = t * kOsTile;
    __syncthreads();
    const bool trivial = s_trivial != 0;

    uint32_t dig[kOsItems], val[kOsItems], pos[kOsItems];
#pragma unroll
    for (int r = 0; r < kOsItems; r++) {
        const uint32_t idx = tile0 + r * kOsThreads + tid;
        const bool valid = idx < n;
        val[r] = valid ? (vals_in ? vals_in[idx] : idx) : 0u;
        dig[r] = valid && val[r] < n ? sk.digit(val[r], pass) : 0u;
    }
    if (!trivial) {
        // stable local ranks: keys are visited in index order (round-major, thread-minor)
#pragma unroll
        for (int r = 0; r < kOsItems; r++) {
#pragma unroll
            for (int w = 0; w < kOsThreads / 32; w++) s_wcnt[w][tid] = 0;
            __syncthreads();
            const uint32_t idx = tile0 + r * kOsThreads + tid;
            const uint32_t d = idx < n ? dig[r] : 256u;
            const uint32_t peers = __match_any_sync(kFull, d);
            const uint32_t lrank = __popc(peers & lanemask_lt());
            if (d < 256 && lrank == 0) s_wcnt[warp][d] = __popc(peers);
            __syncthreads();
            {  // thread tid owns digit tid: exclusive prefix over warps plus the running base
                uint32_t run = s_base[tid];
#pragma unroll
                for (int w = 0; w < kOsThreads / 32; w++) {
                    const uint32_t c = s_wcnt[w][tid];
                    s_wcnt[w][tid] = run;
                    run += c;
                }
                s_base[tid] = run;
            }
            __syncthreads();
            pos[r] = d < 256 ? s_wcnt[warp][d] + lrank : 0u;
            __syncthreads();
        }
        // decoupled look-back for digit tid
        const uint32_t agg = s_base[tid];
        unsigned long long excl = 0;
        if (t != wc.stall_tile) {  // an injected fault withholds this tile's words
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> mine(status[(size_t)t * 256 + tid]);
            if (t == 0) {
                mine.store(kFlagPre | agg, cuda::memory_order_release);
            } else {
                mine.store(kFlagAgg | agg, cuda::memory_order_release);
                long long j = (long long)t - 1;
                uint32_t spins = 0;
                bool done = false;
                while (!done) {
                    unsigned long long w[kOsWindow];
#pragma unroll
                    for (int q = 0; q < kOsWindow; q++) {
                        const long long jj = j - q;
                        w[q] = jj >= 0 ? peek(status, jj * 256 + tid) : kFlagPre;
                    }
                    // walk from the nearest predecessor: stop at a prefix, wait on a gap
                    unsigned long long add = 0;
                    int gap = -1;
                    bool pre = false;
#pragma unroll
                    for (int q = 0; q < kOsWindow; q++) {
                        if (gap < 0 && !pre) {
                            const unsigned long long f = w[q] & ~kValMask;
                            if (f == 0) {
                                gap = q;
                            } else {
                                add += w[q] & kValMask;
                                pre = f == kFlagPre;
                            }
                        }
                    }
                    excl += add;  // the words before the gap (or up to the prefix) are counted
                    if (pre) {
                        done = true;
                    } else if (gap >= 0) {
                        j -= gap;
                        if (++spins > wc.spin_limit) {
                            set_error(err, kDevTimeout);
                            break;
                        }
                    } else {
                        j -= kOsWindow;
                    }
                }
                mine.store(kFlagPre | ((excl + agg) & kValMask), cuda::memory_order_release);
            }
        }
        s_wcnt[0][tid] = (uint32_t)excl;  // s_wcnt is free now: tile's start of each digit
        __syncthreads();
    }
    const bool last = rank_out != nullptr;
#pragma unroll
    for (int r = 0; r < kOsItems; r++) {
        const uint32_t idx = tile0 + r * kOsThreads + tid;
        if (idx >= n) continue;
        uint32_t gpos;
        if (trivial) {
            gpos = idx;
        } else {
            const uint32_t d = dig[r];
            gpos = s_gstart[d] + s_wcnt[0][d] + pos[r];
        }
        if (gpos >= n) {  // only after a look-back gave up
            set_error(err, kDevTimeout);
            continue;
        }
        if (vals_out) vals_out[gpos] = val[r];
        if (last) {
            if (val[r] < n) rank_out[val[r]] = gpos;
            if (perm_out) perm_out[gpos] = val[r];
        }
    }
}

}  // namespace citron

namespace citron_host {

using namespace citron;

static int sort_passes(uint64_t key_bound)
{
    int bits = 0;
    while (bits < 32 && ((key_bound ? key_bound - 1 : 0) >> bits) != 0) bits++;
    return bits <= 8 ? 1 : (bits + 7) / 8;
}

size_t order_ws_bytes(uint32_t n)
{
    Sizer s;
    const size_t ntiles = ((size_t)n + kOsTile - 1) / kOsTile + 1;
    s.take<uint32_t>((size_t)n);                                // ids ping
    s.take<uint32_t>((size_t)n);                                // ids pong
    s.take<uint32_t>(kOsMaxPasses * 256 + kOsMaxPasses);        // histograms, tickets
    s.take<unsigned long long>(ntiles * 256 * kOsMaxPasses);   // look-back words
    return s.used;
}

// Stable ranks of the ids 0..n-1 by (hi[id], key(id)), key = the degree (keys0 == NULL) or
// keys0[id] below key_bound, hi (optional) below hi_bound.  rank[id] = position; perm[position]
// = id when perm != NULL.
static cudaError_t sort_ids(uint32_t n, const uint64_t *off, const uint32_t *keys0, uint64_t key_bound,
                            const uint32_t *hi, uint64_t hi_bound, uint32_t *rank, uint32_t *perm,
                            uint32_t *err, Carver &c, cudaStream_t st)
{
    const int lo_passes = sort_passes(key_bound);
    const int passes = lo_passes + (hi ? sort_passes(hi_bound) : 0);
    if (passes > kOsMaxPasses) return cudaErrorInvalidValue;
    const uint32_t ntiles = (uint32_t)(((uint64_t)n + kOsTile - 1) / kOsTile);
    uint32_t *vals[2] = {c.take<uint32_t>(n), c.take<uint32_t>(n)};
    uint32_t *hist = c.take<uint32_t>(kOsMaxPasses * 256 + kOsMaxPasses);
    unsigned long long *status = c.take<unsigned long long>(((size_t)ntiles + 1) * 256 * kOsMaxPasses);
    if (!c.ok) return cudaErrorMemoryAllocation;
    if (n == 0) return cudaSuccess;
    uint32_t *tickets = hist + kOsMaxPasses * 256;
    cudaError_t e = cudaMemsetAsync(hist, 0, (kOsMaxPasses * 256 + kOsMaxPasses) * sizeof(uint32_t), st);
    if (!e) e = cudaMemsetAsync(status, 0, (size_t)ntiles * 256 * passes * sizeof(unsigned long long), st);
    if (e) return e;
    SortKeys sk;
    sk.off = off;
    sk.keys = keys0;
    sk.hi = hi;
    sk.lo_passes = lo_passes;
    uint32_t hgrid = (n + kOsThreads * 8 - 1) / (kOsThreads * 8);
    if (hgrid > 1024) hgrid = 1024;
    k_os_hist<<<hgrid, kOsThreads, 0, st>>>(sk, n, passes, hist);
    const WaitCfg wc = wait_cfg();
    const uint32_t *vin = nullptr;
    for (int p = 0; p < passes; p++) {
        const bool last = p == passes - 1;
        uint32_t *vout = last ? nullptr : vals[p & 1];
        k_os_scatter<<<ntiles, kOsThreads, 0, st>>>(sk, vin, n, p, hist, status + (size_t)ntiles * 256 * p,
                                                    tickets + p, vout, last ? rank : nullptr,
                                                    last ? perm : nullptr, err, wc);
        vin = vout;
    }
    note_launches(1 + passes);
    return cudaGetLastError();
}

cudaError_t launch_order(uint32_t n, const uint64_t *off, uint32_t *rank, uint32_t *perm,
                         uint32_t *err, Carver &c, cudaStream_t st)
{
    return sort_ids(n, off, nullptr, n, nullptr, 0, rank, perm, err, c, st);
}

// Degree ordering of a disjoint union of graphs, graph by graph: (group, degree, id).
cudaError_t launch_order_grouped(uint32_t n, const uint64_t *off, const uint32_t *group,
                                 uint32_t ngroups, uint32_t *rank, uint32_t *perm, uint32_t *err,
                                 Carver &c, cudaStream_t st)
{
    return sort_ids(n, off, nullptr, n, group, ngroups ? ngroups : 1, rank, perm, err, c, st);
}

// Ranks by (key, id) for keys below key_bound (the core ordering's removal rounds).
cudaError_t launch_rank_by_key(uint32_t n, const uint32_t *keys, uint32_t key_bound, uint32_t *rank,
                               uint32_t *perm, uint32_t *err, Carver &c, cudaStream_t st)
{
    return sort_ids(n, nullptr, keys, key_bound ? key_bound : 1, nullptr, 0, rank, perm, err, c, st);
}

}  // namespace citron_host
