// count.cu -- counting phase on sm_103a (Algorithm Counting, Sec. III, with CITRON's subgraphs,
// Sec. V-B).
//
// Every k-clique is counted once, at its first vertex u in the DAG order ("root"), as a
// (k-1)-clique of the subgraph induced by N+(u) (Sec. II: g_u with V(g_u) = N+(u)).  Roots with
// fewer than k-1 out-neighbours are skipped (the prune of Sec. V-B).  Roots are split by their
// out-degree D:
//   D <= small_max (<= 32)  k_count_small: one warp per root.  Row i of the local subgraph
//       (V(g_u) ∩ N+(a_i), Algorithm GenSubgraph of CITRON) is a 32-bit mask held by lane i.  The
//       recursion runs warp-uniform on candidate masks; the penultimate level adds subgraph
//       degrees for all candidates in one step (Counting's l = 2 branch, Sec. V-B last paragraph).
//   D <= bitmap_max (<= 1024) k_count_mid: one block per root, roots taken largest-D first from
//       a device queue.  The local subgraph is a D x D bitmap in shared memory built by
//       intersecting the sorted list N+(u) with every N+(a_i) (binary search of each element of
//       N+(a_i) in N+(u), lists kept sorted as in the paper).  Its edges (u, a_i) are the tasks
//       of the block's warps (edge-parallel counting); a warp recurses with the candidate set
//       spread over its lanes, one 32-bit word per lane, using ballot / popc / shuffles.
//   D > bitmap_max  k_count_list: one warp per root, candidate sets kept as sorted lists in
//       global scratch, intersections by binary search (the sorted-list form of Sec. V-B).
// Counts are exact uint64; every addition into a shared total checks for wrap-around.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

#include "count_impl.cuh"

namespace citron {

// ------------------------------------------------------------------------------------------
// Root classification.

__global__ void k_classify(uint32_t n, const uint64_t *__restrict__ dag_off, uint32_t need,
                           uint32_t small_max, uint32_t bitmap_max, uint32_t *small_list,
                           uint32_t *big_list, uint32_t *mid_hist, CountStats *st,
                           unsigned long long *per_root, unsigned long long *per_arc,
                           RootFilter filter)
{
    __shared__ uint32_t s_cnt[2], s_base[2], s_max[3];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x < 3) s_max[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t D = 0;
    int cls = -1;  // 0 small, 1 big, 2 mid
    if (u < n) {
        const uint64_t d64 = dag_off[u + 1] - dag_off[u];
        D = (uint32_t)min(d64, (uint64_t)0xffffffffull);
        if (per_root) per_root[u] = 0;
        if (per_arc)  // debug output: every arc of the row starts at zero
            for (uint64_t e = dag_off[u]; e < dag_off[u + 1]; e++) per_arc[e] = 0;
        if (D >= need && filter.takes(u)) cls = D <= small_max ? 0 : (D <= bitmap_max ? 2 : 1);
    }
    uint32_t off_in_warp[2] = {0, 0}, warp_base[2] = {0, 0};
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const uint32_t bal = __ballot_sync(kFull, cls == c);
        off_in_warp[c] = __popc(bal & lanemask_lt());
        if (bal && lane == 0) warp_base[c] = atomicAdd(&s_cnt[c], __popc(bal));
        warp_base[c] = __shfl_sync(kFull, warp_base[c], 0);
    }
    if (cls == 2) atomicAdd(&mid_hist[D], 1u);
    uint32_t m = D;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
    if (lane == 0 && m) atomicMax(&s_max[2], m);
    if (cls == 2) atomicMax(&s_max[0], D);
    if (cls == 1) atomicMax(&s_max[1], D);
    __syncthreads();
    if (threadIdx.x == 0) {
        s_base[0] = s_cnt[0] ? atomicAdd(&st->n_small, s_cnt[0]) : 0;
        s_base[1] = s_cnt[1] ? atomicAdd(&st->n_big, s_cnt[1]) : 0;
        if (s_max[0]) atomicMax(&st->max_mid, s_max[0]);
        if (s_max[1]) atomicMax(&st->max_big, s_max[1]);
        if (s_max[2]) atomicMax(&st->max_all, s_max[2]);
    }
    __syncthreads();
    if (cls == 0) small_list[s_base[0] + warp_base[0] + off_in_warp[0]] = u;
    if (cls == 1) big_list[s_base[1] + warp_base[1] + off_in_warp[1]] = u;
}

// Bin starts for the mid roots in DESCENDING out-degree: cursor[d] = #roots with degree > d.
__global__ __launch_bounds__(1024) void k_mid_bins(const uint32_t *hist, uint32_t bins,
                                                    uint32_t *cursor, CountStats *st)
{
    __shared__ uint32_t scratch[33];
    // reversed index: position i holds degree bins-1-i
    const uint32_t per = (bins + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(bins, threadIdx.x * per), hi = min(bins, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; i++) s += hist[bins - 1 - i];
    uint32_t total;
    uint32_t run = block_excl_scan(s, scratch, total);
    for (uint32_t i = lo; i < hi; i++) {
        const uint32_t d = bins - 1 - i;
        cursor[d] = run;
        run += hist[d];
    }
    if (threadIdx.x == 0) st->n_mid = total;
}

__global__ void k_mid_scatter(uint32_t n, const uint64_t *__restrict__ dag_off, uint32_t need,
                              uint32_t small_max, uint32_t bitmap_max, uint32_t *cursor,
                              uint32_t *mid_list, RootFilter filter)
{
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t D = 0xffffffffu;
    if (u < n) {
        const uint64_t d64 = dag_off[u + 1] - dag_off[u];
        if (d64 >= need && d64 > small_max && d64 <= bitmap_max && filter.takes(u)) D = (uint32_t)d64;
    }
    const uint32_t peers = __match_any_sync(kFull, D);
    if (D == 0xffffffffu) return;
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if ((threadIdx.x & 31) == leader) base = atomicAdd(&cursor[D], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    mid_list[base + __popc(peers & lanemask_lt())] = u;
}

// Group of each DAG row: row rank[v] belongs to the group of vertex v (relabelled DAG).
__global__ void k_batch_rows(uint32_t n, const uint32_t *__restrict__ rank,
                             const uint32_t *__restrict__ group_of_vertex, uint32_t *group_of_row,
                             uint32_t *err)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint32_t r = rank[v];
    if (r < n) group_of_row[r] = group_of_vertex[v];
    else set_error(err, kDevBadInput);
}

// Groups with k = 1 count their vertices, groups with k = 2 their arcs.
__global__ void k_batch_trivial(uint32_t n, const uint64_t *__restrict__ dag_off,
                                const uint32_t *__restrict__ group_of_row,
                                const uint32_t *__restrict__ group_k, uint32_t ngroups,
                                unsigned long long *group_counts, uint32_t *err)
{
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const uint32_t g = group_of_row[u];
    if (g >= ngroups) {
        set_error(err, kDevBadInput);
        return;
    }
    const uint32_t k = group_k[g];
    if (k == 1) add_checked(&group_counts[g], 1ull, err);
    else if (k == 2) add_checked(&group_counts[g], dag_off[u + 1] - dag_off[u], err);
}

__global__ void k_per_root_trivial(uint32_t n, const uint64_t *dag_off, uint32_t k,
                                   unsigned long long *per_root)
{
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) per_root[u] = k == 1 ? 1ull : (unsigned long long)(dag_off[u + 1] - dag_off[u]);
}

// Copy of a DAG slice to a new place: offsets re-based, column ids shifted (citron_dag_append).
// Grid-stride over the n + 1 offsets, then over the arcs.
__global__ void k_dag_append(uint32_t n, const uint64_t *__restrict__ src_off,
                             const uint32_t *__restrict__ src_cols, uint32_t src_row,
                             uint64_t *__restrict__ dst_off, uint32_t *__restrict__ dst_cols,
                             uint32_t dst_row, uint64_t dst_arc)
{
    const uint64_t base = src_off[0];
    const uint64_t arcs = src_off[n] - base;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = i0; i <= n; i += stride) dst_off[i] = src_off[i] - base + dst_arc;
    for (uint64_t e = i0; e < arcs; e += stride) dst_cols[dst_arc + e] = src_cols[base + e] - src_row + dst_row;
}

// Sets count uint64 values (the injected seed of the device totals, tests only).
__global__ void k_fill_u64(unsigned long long *p, uint32_t count, unsigned long long v)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[i] = v;
}

}  // namespace citron

namespace citron_host {

using namespace citron;

cudaError_t launch_dag_append(uint32_t n, const uint64_t *src_off, const uint32_t *src_cols,
                              uint32_t src_row, uint64_t *dst_off, uint32_t *dst_cols,
                              uint32_t dst_row, uint64_t dst_arc, cudaStream_t s)
{
    k_dag_append<<<304, 256, 0, s>>>(n, src_off, src_cols, src_row, dst_off, dst_cols, dst_row, dst_arc);
    note_launches(1);
    return cudaGetLastError();
}

// Seeds `count` device totals with the injected count_seed (no-op in normal operation).
cudaError_t seed_totals(unsigned long long *p, uint32_t count, cudaStream_t s)
{
    const unsigned long long seed = injected_faults().count_seed;
    if (!seed || !count) return cudaSuccess;
    k_fill_u64<<<(count + 255) / 256, 256, 0, s>>>(p, count, seed);
    note_launches(1);
    return cudaGetLastError();
}

size_t count_ws_bytes(uint32_t n, uint32_t max_outdeg, int num_sms)
{
    Sizer s;
    s.take<CountStats>(1);
    s.take<unsigned long long>(4);
    s.take<uint32_t>(8);                      // queue counters
    s.take<uint32_t>((size_t)n + 1);          // small list
    s.take<uint32_t>((size_t)n + 1);          // mid list
    s.take<uint32_t>((size_t)n + 1);          // big list
    s.take<uint32_t>(kBitmapCap + 2);         // mid histogram
    s.take<uint32_t>(kBitmapCap + 2);         // mid cursors
    s.take<HeavySlot>(kHelpSlots);            // help table of heavy roots
    s.take<unsigned long long>(2 * (size_t)num_sms * kMidBlocksPerSmCap);  // block start/end
    // sorted-list scratch: one (k-3)-level stack per warp, sized for the largest root, so that
    // every root can take the list path (tuned thresholds send any root there)
    const uint32_t list_warps = (uint32_t)num_sms * kListWarps;
    s.take<uint32_t>((size_t)max_outdeg * list_warps * (kMaxK - 3) + 1);
    return s.used;
}

// Runs the count for k >= 3.  Returns a CUDA error, or cudaErrorMemoryAllocation when the
// workspace is too small.  The host value lands in *h_result.
cudaError_t run_count(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_cols, uint32_t k,
                      CountRun &run, uint32_t *err, Carver &c, cudaStream_t s, int num_sms,
                      unsigned long long *h_result)
{
    CountStats *st = c.take<CountStats>(1);
    unsigned long long *result = c.take<unsigned long long>(4);  // total, work, budget clock
    uint32_t *next = c.take<uint32_t>(8);
    uint32_t *small_list = c.take<uint32_t>((size_t)n + 1);
    uint32_t *mid_list = c.take<uint32_t>((size_t)n + 1);
    uint32_t *big_list = c.take<uint32_t>((size_t)n + 1);
    uint32_t *hist = c.take<uint32_t>(kBitmapCap + 2);
    uint32_t *cursor = c.take<uint32_t>(kBitmapCap + 2);
    MidAux aux;
    aux.help.slots = c.take<HeavySlot>(kHelpSlots);
    aux.help.cap = kHelpSlots;
    aux.help.nslots = next + 2;
    aux.block_ns = c.take<unsigned long long>(2 * (size_t)num_sms * kMidBlocksPerSmCap);
    aux.budget.clock0 = result + 2;
    aux.budget.ns = run.budget_ns;
    if (!c.ok) return cudaErrorMemoryAllocation;
    // the rest of the workspace is list-path scratch
    uint32_t *list_scratch = (uint32_t *)(c.base + c.used);
    const size_t list_words = c.cap > c.used ? (c.cap - c.used) / sizeof(uint32_t) : 0;
    unsigned long long *work = result + 1;
    const CountPlan &plan = run.plan;

    cudaError_t e;
    if ((e = cudaMemsetAsync(st, 0, sizeof(CountStats), s))) return e;
    if ((e = cudaMemsetAsync(result, 0, 4 * sizeof(unsigned long long), s))) return e;
    if ((e = seed_totals(result, 1, s))) return e;
    if ((e = cudaMemsetAsync(next, 0, 8 * sizeof(uint32_t), s))) return e;
    if ((e = cudaMemsetAsync(hist, 0, (kBitmapCap + 2) * sizeof(uint32_t), s))) return e;
    if ((e = cudaMemsetAsync(aux.help.slots, 0, kHelpSlots * sizeof(HeavySlot), s))) return e;
    const uint32_t need = k - 1;
    const uint32_t blocks = (n + 255) / 256;
    if (n) {
        k_classify<<<blocks, 256, 0, s>>>(n, dag_off, need, plan.small_max, plan.bitmap_max,
                                          small_list, big_list, hist, st, run.sink.per_root,
                                          run.sink.per_arc, run.filter);
        k_mid_bins<<<1, 1024, 0, s>>>(hist, plan.bitmap_max + 1, cursor, st);
        k_mid_scatter<<<blocks, 256, 0, s>>>(n, dag_off, need, plan.small_max, plan.bitmap_max,
                                             cursor, mid_list, run.filter);
        note_launches(3);
    }
    CountStats hs;
    if ((e = cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
#define CITRON_CASE(KK)                                                                           \
    case KK:                                                                                      \
        e = launch_count_##KK(run, dag_off, dag_cols, hs, st, small_list, mid_list, big_list,     \
                               next, list_scratch, list_words, result, work, aux, err, s,         \
                               num_sms);                                                          \
        break;
    switch (k) {
        CITRON_CASE(3)
        CITRON_CASE(4)
        CITRON_CASE(5)
        CITRON_CASE(6)
        CITRON_CASE(7)
        CITRON_CASE(8)
        CITRON_CASE(9)
        CITRON_CASE(10)
        CITRON_CASE(11)
        CITRON_CASE(12)
        default: return cudaErrorInvalidValue;
    }
#undef CITRON_CASE
    if (e) return e;
    unsigned long long out[2] = {0, 0};
    if ((e = cudaMemcpyAsync(out, result, sizeof(out), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    *h_result = out[0];
    run.work = out[1];
    return cudaSuccess;
}

// Capture-safe variant of run_count: no host synchronisation.  Launch configurations come from
// upper bounds (every row a root, the largest row max_outdeg) instead of the classification's
// statistics; the kernels read the real list sizes on the device and exit when they are done.
cudaError_t run_count_async(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_cols, uint32_t k,
                            uint32_t max_outdeg, CountRun &run, uint32_t *err, Carver &c,
                            cudaStream_t s, int num_sms)
{
    CountStats *st = c.take<CountStats>(1);
    unsigned long long *result = c.take<unsigned long long>(4);  // total, work, budget clock
    uint32_t *next = c.take<uint32_t>(8);
    uint32_t *small_list = c.take<uint32_t>((size_t)n + 1);
    uint32_t *mid_list = c.take<uint32_t>((size_t)n + 1);
    uint32_t *big_list = c.take<uint32_t>((size_t)n + 1);
    uint32_t *hist = c.take<uint32_t>(kBitmapCap + 2);
    uint32_t *cursor = c.take<uint32_t>(kBitmapCap + 2);
    MidAux aux;
    aux.help.slots = c.take<HeavySlot>(kHelpSlots);
    aux.help.cap = kHelpSlots;
    aux.help.nslots = next + 2;
    aux.block_ns = c.take<unsigned long long>(2 * (size_t)num_sms * kMidBlocksPerSmCap);
    aux.budget.clock0 = result + 2;
    aux.budget.ns = run.budget_ns;
    if (!c.ok) return cudaErrorMemoryAllocation;
    uint32_t *list_scratch = (uint32_t *)(c.base + c.used);
    const size_t list_words = c.cap > c.used ? (c.cap - c.used) / sizeof(uint32_t) : 0;
    unsigned long long *work = result + 1;
    const CountPlan &plan = run.plan;
    cudaError_t e;
    if ((e = cudaMemsetAsync(st, 0, sizeof(CountStats), s))) return e;
    if ((e = cudaMemsetAsync(result, 0, 4 * sizeof(unsigned long long), s))) return e;
    if ((e = cudaMemsetAsync(next, 0, 8 * sizeof(uint32_t), s))) return e;
    if ((e = cudaMemsetAsync(hist, 0, (kBitmapCap + 2) * sizeof(uint32_t), s))) return e;
    if ((e = cudaMemsetAsync(aux.help.slots, 0, kHelpSlots * sizeof(HeavySlot), s))) return e;
    if (n == 0 || max_outdeg < k - 1) return cudaSuccess;
    const uint32_t need = k - 1;
    const uint32_t blocks = (n + 255) / 256;
    k_classify<<<blocks, 256, 0, s>>>(n, dag_off, need, plan.small_max, plan.bitmap_max, small_list,
                                      big_list, hist, st, nullptr, nullptr, run.filter);
    k_mid_bins<<<1, 1024, 0, s>>>(hist, plan.bitmap_max + 1, cursor, st);
    k_mid_scatter<<<blocks, 256, 0, s>>>(n, dag_off, need, plan.small_max, plan.bitmap_max, cursor,
                                         mid_list, run.filter);
    note_launches(3);
    CountStats hs = {};
    hs.n_small = max_outdeg >= need ? n : 0;
    hs.max_mid = max_outdeg < plan.bitmap_max ? max_outdeg : plan.bitmap_max;
    hs.n_mid = hs.max_mid > plan.small_max ? n : 0;
    hs.max_big = max_outdeg;
    hs.n_big = max_outdeg > plan.bitmap_max ? n : 0;
    run.time_kernels = false;
#define CITRON_CASE(KK)                                                                           \
    case KK:                                                                                      \
        e = launch_count_##KK(run, dag_off, dag_cols, hs, st, small_list, mid_list, big_list,     \
                              next, list_scratch, list_words, result, work, aux, err, s,         \
                              num_sms);                                                          \
        break;
    switch (k) {
        CITRON_CASE(3)
        CITRON_CASE(4)
        CITRON_CASE(5)
        CITRON_CASE(6)
        CITRON_CASE(7)
        CITRON_CASE(8)
        CITRON_CASE(9)
        CITRON_CASE(10)
        CITRON_CASE(11)
        CITRON_CASE(12)
        default: return cudaErrorInvalidValue;
    }
#undef CITRON_CASE
    return e;
}

cudaError_t launch_batch_rows(uint32_t n, const uint32_t *rank, const uint32_t *group_of_vertex,
                              uint32_t *group_of_row, uint32_t *err, cudaStream_t s)
{
    if (n) {
        k_batch_rows<<<(n + 255) / 256, 256, 0, s>>>(n, rank, group_of_vertex, group_of_row, err);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_trivial(uint32_t n, const uint64_t *dag_off, const uint32_t *group_of_row,
                                 const uint32_t *group_k, uint32_t ngroups,
                                 unsigned long long *counts, uint32_t *err, cudaStream_t s)
{
    if (n) {
        k_batch_trivial<<<(n + 255) / 256, 256, 0, s>>>(n, dag_off, group_of_row, group_k, ngroups,
                                                       counts, err);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_per_root_trivial(uint32_t n, const uint64_t *dag_off, uint32_t k,
                                    unsigned long long *per_root, cudaStream_t s)
{
    if (n) {
        k_per_root_trivial<<<(n + 255) / 256, 256, 0, s>>>(n, dag_off, k, per_root);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace citron_host
