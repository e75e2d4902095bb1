// order.cu -- ordering phase on sm_103a: degree ordering, DAG construction, input validation.
//
//   Degree ordering (Sec. II, Sec. IV): rank = position of u when sorted by (d(u), u), by the
//     single-sweep radix sort of sort.cu.
//   Algorithm GenOrdering (Sec. IV), fused into ONE pass over the arcs:
//     k_tile_rows       : for every tile of 4096 arcs, the first vertex whose row starts in it;
//     k_dag_compact     : keep-test of every arc, block scan, decoupled look-back prefix over
//                         tiles, coalesced store of the kept arcs (the DAG columns, already sorted
//                         per row) and of the DAG row offsets.  The count pass, PrefixSum and the
//                         fill pass of the listing become one read of cols and one write of the DAG.
//   The DAG of any rank, relabelled to ranks, is built in relabel.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace citron {

// ------------------------------------------------------------------------------------------
// Algorithm GenOrdering, fused.

constexpr int kGoThreads = 256;
constexpr int kGoItems = 16;
constexpr uint32_t kGoTile = kGoThreads * kGoItems;  // 4096 arcs
constexpr uint32_t kGoRowCap = 2048;                 // row starts cached in shared memory

// first_row[b] = min{u : off[u] >= p_b}, p_b = b*tile for b < ntiles, p_ntiles = arcs.
// Thread per vertex u in [0, n]: it owns the positions p with off[u-1] < p <= off[u].
__global__ void k_tile_rows(uint32_t n, uint64_t arcs, const uint64_t *off, uint32_t tile,
                            uint32_t ntiles, uint32_t *first_row)
{
    const uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > n) return;
    const uint64_t hi = off[u];
    // tiles b < ntiles with lo < b*tile <= hi
    uint64_t b0 = (u == 0) ? 0 : off[u - 1] / tile + 1;
    uint64_t b1 = hi / tile;  // inclusive
    if (b1 > ntiles - 1) b1 = ntiles - 1;
    for (uint64_t b = b0; b <= b1 && b < ntiles; b++) first_row[b] = (uint32_t)u;
    const bool owns_end = (u == 0) ? (arcs <= hi) : (off[u - 1] < arcs && arcs <= hi);
    if (owns_end) first_row[ntiles] = (uint32_t)u;
}

// deg[u] = off[u+1] - off[u] (clamped to 32 bits): the key of the degree ordering.
__global__ void k_degrees(uint32_t n, const uint64_t *__restrict__ off, uint32_t *__restrict__ deg)
{
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) deg[u] = (uint32_t)min(off[u + 1] - off[u], (uint64_t)0xffffffffull);
}

// Algorithm GenOrdering (Sec. IV) in one pass over the arcs in tiles of 4096: keep-test of every
// arc (u -> v kept iff (d(u), u) < (d(v), v), key = degree), block scan, decoupled look-back
// prefix over tiles, coalesced store of the kept ids (rows keep the input's order, so they stay
// sorted) and of the row offsets.  Every thread issues the key gathers of its 16 arcs before it
// uses any of them.
__global__ __launch_bounds__(kGoThreads) void k_dag_compact(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ cols,
    const uint32_t *__restrict__ key, const uint32_t *__restrict__ first_row, uint32_t ntiles,
    uint64_t *__restrict__ out_off, uint32_t *__restrict__ out_vals, uint64_t out_cap,
    unsigned long long *status, uint32_t *ticket, uint32_t *err, int vec4, WaitCfg wc)
{
    __shared__ uint64_t s_row[kGoRowCap + 1];
    __shared__ uint32_t s_key[kGoRowCap + 1];
    __shared__ uint32_t s_out[kGoTile];
    __shared__ uint32_t s_pref[kGoThreads];
    __shared__ uint16_t s_mask[kGoThreads];
    __shared__ uint32_t s_scan[kGoThreads / 32 + 1];
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_excl;

    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) return;
    const uint64_t t0 = (uint64_t)t * kGoTile;
    const uint64_t t1 = min(t0 + kGoTile, arcs);
    const uint32_t u_first = first_row[t];
    const uint32_t u_next = first_row[t + 1];
    // Offsets that break the CSR contract (validate first) make the tile publish an empty
    // aggregate and flag the error instead of reading out of range.
    const bool bad = u_first > n || u_next > n || u_next < u_first || (t > 0 && u_first == 0);
    // vertex owning arc t0: the last u with off[u] <= t0
    const uint32_t r0 = bad ? 0 : ((off[u_first] == t0) ? u_first : u_first - 1);
    const uint32_t nrows = bad ? 0 : u_next - r0;  // rows r0 .. u_next-1 may hold arcs of this tile
    const bool cached = nrows + 1 <= kGoRowCap + 1;
    if (bad && tid == 0) set_error(err, kDevBadInput);
    if (cached) {
        for (uint32_t i = tid; i <= nrows; i += kGoThreads) {
            s_row[i] = off[r0 + i];
            s_key[i] = (r0 + i < n) ? key[r0 + i] : 0u;
        }
    }
    __syncthreads();
    auto row_start = [&](uint32_t r) -> uint64_t {  // off[r] for r in [r0, u_next]
        return cached ? s_row[r - r0] : off[r];
    };
    auto row_key = [&](uint32_t r) -> uint32_t { return cached ? s_key[r - r0] : key[r]; };

    const uint64_t a0 = bad ? t1 : t0 + (uint64_t)tid * kGoItems;
    uint32_t v[kGoItems], kv[kGoItems];
    if (vec4 && a0 + kGoItems <= t1) {
        const uint4 *p = reinterpret_cast<const uint4 *>(cols + a0);
#pragma unroll
        for (int q = 0; q < kGoItems / 4; q++) {
            uint4 x = __ldg(p + q);
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kGoItems; j++) v[j] = (a0 + j < t1) ? cols[a0 + j] : 0;
    }
    // all key gathers in flight before any is used
#pragma unroll
    for (int j = 0; j < kGoItems; j++) kv[j] = (a0 + j < t1 && v[j] < n) ? __ldg(key + v[j]) : 0u;
    // row of this thread's first arc: last r in [r0, u_next] with off[r] <= a0
    uint32_t r = r0;
    if (a0 < t1) {
        uint32_t lo = r0, hi = u_next;  // invariant off[lo] <= a0
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo + 1) / 2;
            if (row_start(mid) <= a0) lo = mid;
            else hi = mid - 1;
        }
        r = lo;
    }
    uint32_t mask = 0;
    if (a0 < t1) {
        uint64_t re = row_start(r + 1);
        uint32_t ku = row_key(r);
#pragma unroll
        for (int j = 0; j < kGoItems; j++) {
            const uint64_t a = a0 + j;
            if (a < t1) {
                while (re <= a) {
                    r++;
                    re = row_start(r + 1);
                    ku = row_key(r);
                }
                const uint32_t w = v[j];
                if (w >= n) {
                    set_error(err, kDevBadInput);
                    continue;
                }
                const bool keep = ku < kv[j] || (ku == kv[j] && r < w);
                if (keep) mask |= 1u << j;
            }
        }
    }
    s_mask[tid] = (uint16_t)mask;
    uint32_t total;
    const uint32_t pref = block_excl_scan(__popc(mask), s_scan, total);
    s_pref[tid] = pref;
    {
        uint32_t p = pref;
#pragma unroll
        for (int j = 0; j < kGoItems; j++)
            if (mask >> j & 1) s_out[p++] = v[j];
    }
    if (tid < 32) {
        unsigned long long e = lookback_warp(status, t, total, err, wc);
        if (tid == 0) s_excl = e;
    }
    __syncthreads();
    const unsigned long long excl = s_excl;
    if (excl + total > out_cap) {  // more kept arcs than half the input: asymmetric input
        if (tid == 0) set_error(err, kDevBadInput);
        return;
    }
    for (uint32_t i = tid; i < total; i += kGoThreads) out_vals[excl + i] = s_out[i];
    if (bad) return;
    // row offsets of the vertices whose rows start inside this tile
    for (uint32_t u = u_first + tid; u < u_next; u += kGoThreads) {
        const uint32_t pos = (uint32_t)(row_start(u) - t0);
        const uint32_t q = pos / kGoItems, j = pos % kGoItems;
        out_off[u] = excl + s_pref[q] + __popc((uint32_t)s_mask[q] & ((1u << j) - 1));
    }
    if (t == ntiles - 1) {  // trailing vertices whose rows start at the end of the arcs
        for (uint32_t u = first_row[ntiles] + tid; u <= n; u += kGoThreads) out_off[u] = excl + total;
    }
}

// ------------------------------------------------------------------------------------------
// Validation of the CSR contract (offsets, range, order, loops, symmetry).

__global__ void k_validate(uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off,
                           const uint32_t *__restrict__ cols, uint32_t *bad)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[n] != arcs)) atomicMin(bad, 1u);
    for (uint32_t u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
        const uint64_t b = off[u], e = off[u + 1];
        if (e < b || e > arcs) {
            if (lane == 0) atomicMin(bad, 1u);
            continue;
        }
        for (uint64_t i = b + lane; i < e; i += 32) {
            const uint32_t v = cols[i];
            uint32_t code = 0;
            if (v >= n) code = 2;
            else if (i > b && cols[i - 1] >= v) code = 3;
            else if (v == u) code = 4;
            else {  // reverse arc v -> u by binary search in row v
                uint64_t lo = off[v], hi = off[v + 1];
                if (hi < lo || hi > arcs) code = 1;
                else {
                    while (lo < hi) {
                        const uint64_t mid = lo + (hi - lo) / 2;
                        if (cols[mid] < u) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo >= off[v + 1] || cols[lo] != u) code = 5;
                }
            }
            if (code) atomicMin(bad, code);
        }
    }
}

// Largest row length of a CSR given its offsets.
__global__ void k_max_rowlen(uint32_t n, const uint64_t *off, uint32_t *out)
{
    uint32_t best = 0;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        best = max(best, (uint32_t)min(off[u + 1] - off[u], (uint64_t)0xffffffffull));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}
}  // namespace citron

// ------------------------------------------------------------------------------------------
// Host launchers (called from api.cu).

namespace citron_host {

using namespace citron;

size_t relabel_ws_bytes(uint32_t n, uint64_t arcs);
cudaError_t launch_relabel_dag(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                               const uint32_t *rank, uint64_t *dag_off, uint32_t *dag_cols,
                               uint32_t *d_max_outdeg, uint32_t *err, Carver &c, cudaStream_t st,
                               int num_sms);

size_t dag_ws_bytes(uint32_t n, uint64_t arcs)
{
    Sizer s;
    const uint64_t ntiles = (arcs + kGoTile - 1) / kGoTile;
    s.take<uint32_t>(ntiles + 2);             // first_row
    s.take<unsigned long long>(ntiles + 1);   // look-back status (compaction)
    s.take<uint32_t>(8);                      // tickets, counters
    s.take<uint32_t>((size_t)n + 1);          // degrees
    const size_t r = relabel_ws_bytes(n, arcs);
    return r > s.used ? r : s.used;
}

cudaError_t launch_tile_rows(uint32_t n, uint64_t arcs, const uint64_t *off, uint32_t tile,
                             uint32_t ntiles, uint32_t *first_row, cudaStream_t st)
{
    k_tile_rows<<<(n + 1 + 255) / 256, 256, 0, st>>>(n, arcs, off, tile, ntiles, first_row);
    note_launches(1);
    return cudaGetLastError();
}

// Returns cudaErrorMemoryAllocation if the workspace is short; device errors land in err.
cudaError_t launch_build_dag(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                             const uint32_t *rank, uint64_t *dag_off, uint32_t *dag_cols,
                             uint32_t *d_max_outdeg, uint32_t *err, Carver &c, cudaStream_t st,
                             int num_sms)
{
    if (rank)
        return launch_relabel_dag(n, arcs, off, cols, rank, dag_off, dag_cols, d_max_outdeg, err, c,
                                  st, num_sms);
    const uint64_t ntiles64 = (arcs + kGoTile - 1) / kGoTile;
    uint32_t *first_row = c.take<uint32_t>(ntiles64 + 2);
    unsigned long long *status = c.take<unsigned long long>(ntiles64 + 1);
    uint32_t *ctr = c.take<uint32_t>(8);
    uint32_t *keys = c.take<uint32_t>((size_t)n + 1);
    if (!c.ok) return cudaErrorMemoryAllocation;
    if (ntiles64 >= 0xffffffffull) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctr, 0, 8 * sizeof(uint32_t), st))) return e;
    if (arcs == 0 || n == 0) {
        return cudaMemsetAsync(dag_off, 0, ((size_t)n + 1) * sizeof(uint64_t), st);
    }
    const uint32_t ntiles = (uint32_t)ntiles64;
    const int vec4 = ((uintptr_t)cols % 16) == 0;
    if ((e = cudaMemsetAsync(status, 0, ntiles64 * sizeof(unsigned long long), st))) return e;
    if ((e = launch_tile_rows(n, arcs, off, kGoTile, ntiles, first_row, st))) return e;
    k_degrees<<<(n + 255) / 256, 256, 0, st>>>(n, off, keys);
    k_dag_compact<<<ntiles, kGoThreads, 0, st>>>(n, arcs, off, cols, keys, first_row, ntiles, dag_off,
                                                 dag_cols, arcs / 2, status, ctr, err, vec4, wait_cfg());
    note_launches(2);
    if (d_max_outdeg) {
        k_max_rowlen<<<num_sms * 4, 256, 0, st>>>(n, dag_off, d_max_outdeg);
        note_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_validate(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                            uint32_t *bad, cudaStream_t st, int num_sms)
{
    k_validate<<<num_sms * 8, 256, 0, st>>>(n, arcs, off, cols, bad);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace citron_host

