// order.cu -- ordering phase on sm_103a: degree ordering, DAG construction, input validation.
//
//   Degree ordering (Sec. II, Sec. IV): rank = position of u when sorted by (d(u), u).
//     k_radix_hist / k_radix_scatter: stable LSD radix sort of the ids by degree, 8-bit digits;
//     ids enter in ascending order, so stability supplies the id tie-break.
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
// Radix sort of vertex ids by degree.

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // 4096 keys per block

__device__ __forceinline__ uint32_t degree_of(const uint64_t *off, uint32_t u)
{
    return (uint32_t)(off[u + 1] - off[u]);
}

// Per-block histogram of one 8-bit digit.  hist is digit-major: hist[d * nblocks + b].
__global__ __launch_bounds__(kRsThreads) void k_radix_hist(const uint64_t *off, const uint32_t *keys,
                                                           uint32_t n, int shift, uint32_t *hist,
                                                           uint32_t nblocks)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kRsTile;
#pragma unroll 4
    for (int i = 0; i < kRsItems; i++) {
        uint32_t idx = base + i * kRsThreads + threadIdx.x;
        if (idx < n) {
            uint32_t key = keys ? keys[idx] : degree_of(off, idx);
            atomicAdd(&cnt[(key >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of one uint32 array by a single block of 1024 threads (sizes here are
// 256 x blocks).  Each warp owns one contiguous segment and walks it 32 entries at a time, so
// every load and store is coalesced.
__global__ __launch_bounds__(1024) void k_scan_small(uint32_t *data, uint32_t count)
{
    __shared__ uint32_t s_warp[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t seg = ((count + 31) / 32 + 31) & ~31u;
    const uint32_t lo = min(count, (uint32_t)w * seg), hi = min(count, lo + seg);
    constexpr int kBatch = 8;  // loads of one lane in flight together
    uint32_t sum = 0;
    for (uint32_t b = lo; b < hi; b += 32 * kBatch) {
        uint32_t v[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; t++) {
            const uint32_t i = b + t * 32 + lane;
            v[t] = i < hi ? data[i] : 0u;
        }
#pragma unroll
        for (int t = 0; t < kBatch; t++) sum += v[t];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    if (lane == 0) s_warp[w] = sum;
    __syncthreads();
    if (w == 0) {
        const uint32_t v = s_warp[lane];
        const uint32_t incl = warp_incl_scan(v);
        s_warp[lane] = incl - v;
    }
    __syncthreads();
    uint32_t carry = s_warp[w];
    for (uint32_t b = lo; b < hi; b += 32 * kBatch) {
        uint32_t v[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; t++) {
            const uint32_t i = b + t * 32 + lane;
            v[t] = i < hi ? data[i] : 0u;
        }
#pragma unroll
        for (int t = 0; t < kBatch; t++) {
            const uint32_t i = b + t * 32 + lane;
            const uint32_t incl = warp_incl_scan(v[t]);
            if (i < hi) data[i] = carry + incl - v[t];
            carry += __shfl_sync(kFull, incl, 31);
        }
    }
}

// Stable scatter of one digit.  Keys of a tile are visited in index order (round-major,
// thread-minor); ranks inside a round come from __match_any_sync peers and a per-digit prefix
// over the warps.  On the last pass the permutation and the rank array are written.
__global__ __launch_bounds__(kRsThreads) void k_radix_scatter(
    const uint64_t *off, const uint32_t *keys_in, const uint32_t *vals_in, uint32_t n, int shift,
    const uint32_t *hist, uint32_t nblocks, uint32_t *keys_out, uint32_t *vals_out,
    uint32_t *rank_out)
{
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[kRsThreads / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5;
    base[tid] = hist[tid * nblocks + blockIdx.x];
    const uint32_t tile = blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; r++) {
#pragma unroll
        for (int w = 0; w < kRsThreads / 32; w++) wcnt[w][tid] = 0;
        __syncthreads();
        const uint32_t idx = tile + r * kRsThreads + tid;
        const bool valid = idx < n;
        uint32_t key = 0, val = 0, d = 256;
        if (valid) {
            key = keys_in ? keys_in[idx] : degree_of(off, idx);
            val = vals_in ? vals_in[idx] : idx;
            d = (key >> shift) & 255u;
        }
        const uint32_t peers = __match_any_sync(kFull, d);
        const uint32_t lrank = __popc(peers & lanemask_lt());
        if (valid && lrank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {  // thread tid owns digit tid: exclusive prefix over warps, plus the running base
            uint32_t run = base[tid];
#pragma unroll
            for (int w = 0; w < kRsThreads / 32; w++) {
                uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wcnt[warp][d] + lrank;
            if (keys_out) keys_out[pos] = key;
            vals_out[pos] = val;
            if (rank_out) rank_out[val] = pos;
        }
        __syncthreads();
    }
}

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

size_t order_ws_bytes(uint32_t n)
{
    Sizer s;
    const uint32_t nb = (n + kRsTile - 1) / kRsTile + 1;
    s.take<uint32_t>((size_t)n);        // keys ping
    s.take<uint32_t>((size_t)n);        // keys pong
    s.take<uint32_t>((size_t)n);        // vals ping
    s.take<uint32_t>((size_t)n);        // vals pong
    s.take<uint32_t>((size_t)256 * nb);  // histogram
    return s.used;
}

static int radix_passes(uint32_t n)
{
    int bits = 0;
    while (bits < 32 && ((uint64_t)(n ? n - 1 : 0) >> bits) != 0) bits++;
    return bits <= 8 ? 1 : (bits + 7) / 8;
}

// Stable LSD sort of the ids 0..n-1 by a key: the degree (keys0 == NULL) or keys0[id].  Writes
// rank[id] = position and, when perm != NULL, perm[position] = id.  `passes` 8-bit digits.
static cudaError_t sort_ids(uint32_t n, const uint64_t *off, const uint32_t *keys0, int passes,
                            uint32_t *rank, uint32_t *perm, Carver &c, cudaStream_t st)
{
    const uint32_t nb = (n + kRsTile - 1) / kRsTile;
    uint32_t *keys[2] = {c.take<uint32_t>(n), c.take<uint32_t>(n)};
    uint32_t *vals[2] = {c.take<uint32_t>(n), c.take<uint32_t>(n)};
    uint32_t *hist = c.take<uint32_t>((size_t)256 * (nb + 1));
    if (!c.ok) return cudaErrorMemoryAllocation;
    if (n == 0) return cudaSuccess;
    const uint32_t *kin = keys0, *vin = nullptr;
    for (int p = 0; p < passes; p++) {
        const bool last = p == passes - 1;
        k_radix_hist<<<nb, kRsThreads, 0, st>>>(off, kin, n, 8 * p, hist, nb);
        k_scan_small<<<1, 1024, 0, st>>>(hist, 256 * nb);
        uint32_t *kout = last ? nullptr : keys[p & 1];
        uint32_t *vout = last ? (perm ? perm : vals[p & 1]) : vals[p & 1];
        k_radix_scatter<<<nb, kRsThreads, 0, st>>>(off, kin, vin, n, 8 * p, hist, nb, kout, vout,
                                                   last ? rank : nullptr);
        note_launches(3);
        kin = kout;
        vin = vout;
    }
    return cudaGetLastError();
}

cudaError_t launch_order(uint32_t n, const uint64_t *off, uint32_t *rank, uint32_t *perm,
                         Carver &c, cudaStream_t st)
{
    return sort_ids(n, off, nullptr, radix_passes(n), rank, perm, c, st);
}

// Ranks by (key, id) for keys below key_bound (the core ordering's removal rounds).
cudaError_t launch_rank_by_key(uint32_t n, const uint32_t *keys, uint32_t key_bound, uint32_t *rank,
                               uint32_t *perm, Carver &c, cudaStream_t st)
{
    return sort_ids(n, nullptr, keys, radix_passes(key_bound ? key_bound : 1), rank, perm, c, st);
}

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

