// order.cu -- ordering phase on sm_103a: degree ordering, DAG construction, input validation.
//
//   Degree ordering (Sec. II, Sec. IV): rank = position of u when sorted by (d(u), u).
//     k_radix_hist / k_radix_scatter: stable LSD radix sort of the ids by degree, 8-bit digits;
//     ids enter in ascending order, so stability supplies the id tie-break.
//   Algorithm GenOrdering (Sec. IV), fused into ONE pass over the arcs:
//     k_tile_rows       : for every tile of 4096 arcs, the first vertex whose row starts in it;
//     k_dag_compact<0>  : keep-test of every arc, block scan, decoupled look-back prefix over
//                         tiles, coalesced store of the kept arcs (the DAG columns, already sorted
//                         per row) and of the DAG row offsets.  The count pass, PrefixSum and the
//                         fill pass of the listing become one read of cols and one write of the DAG.
//   Relabelled DAG from any rank (Sec. II directionalizing, rows renamed to ranks):
//     k_dag_compact<1> (kept ranks, input row order) -> k_rl_rowlen -> k_scan_rowlen (look-back)
//     -> k_rl_sort (per-row sort into rank order; k_rl_sort_long for rows above 512).
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

// One pass over the arcs in tiles of 4096: keep-test of every arc, block scan, decoupled look-back
// prefix over tiles, coalesced store of the kept values and of the row offsets.
//   ORDER = 0 (Algorithm GenOrdering, Sec. IV): key = degree; u -> v kept iff
//             (d(u), u) < (d(v), v); the kept value is v.  Rows keep the input's order.
//   ORDER = 1 (any rank): key = rank; kept iff rank[v] > rank[u]; the kept value is rank[v]
//             (rows stay in input order, unsorted: the relabel pass sorts them).
// Every thread issues the key gathers of its 16 arcs before it uses any of them.
template <int ORDER>
__global__ __launch_bounds__(kGoThreads) void k_dag_compact(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ cols,
    const uint32_t *__restrict__ key, const uint32_t *__restrict__ first_row, uint32_t ntiles,
    uint64_t *__restrict__ out_off, uint32_t *__restrict__ out_vals, uint64_t out_cap,
    unsigned long long *status, uint32_t *ticket, uint32_t *err, int vec4)
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
                const bool keep = ORDER == 0 ? (ku < kv[j] || (ku == kv[j] && r < w)) : (kv[j] > ku);
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
            if (mask >> j & 1) s_out[p++] = ORDER == 0 ? v[j] : kv[j];
    }
    if (tid < 32) {
        unsigned long long e = lookback_warp(status, t, total, err);
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
// Relabelled DAG from a rank permutation.

// rowlen[rank[u]] = length of u's kept row (G[u+1] - G[u]); the largest goes to max_len.
__global__ void k_rl_rowlen(uint32_t n, const uint64_t *__restrict__ G,
                            const uint32_t *__restrict__ rank, uint32_t *__restrict__ rowlen,
                            uint32_t *max_len, uint32_t *err)
{
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t len = 0;
    if (u < n) {
        const uint32_t ru = rank[u];
        len = (uint32_t)min(G[u + 1] - G[u], (uint64_t)0xffffffffull);
        if (ru < n) rowlen[ru] = len;
        else set_error(err, kDevBadInput);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(kFull, len, o));
    if ((threadIdx.x & 31) == 0 && len) atomicMax(max_len, len);
}

constexpr int kScThreads = 256;
constexpr int kScItems = 16;
constexpr uint32_t kScTile = kScThreads * kScItems;

// dag_off[i] = sum of rowlen[0..i), dag_off[n] = total; single pass with look-back.
__global__ __launch_bounds__(kScThreads) void k_scan_rowlen(uint32_t n, const uint32_t *rowlen,
                                                            uint64_t *dag_off, uint32_t ntiles,
                                                            unsigned long long *status,
                                                            uint32_t *ticket, uint32_t *err)
{
    __shared__ uint32_t s_scan[kScThreads / 32 + 1];
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) return;
    const uint64_t i0 = (uint64_t)t * kScTile + (uint64_t)tid * kScItems;
    uint32_t v[kScItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScItems; j++) {
        v[j] = (i0 + j < n) ? rowlen[i0 + j] : 0;
        s += v[j];
    }
    uint32_t total;
    const uint32_t pref = block_excl_scan(s, s_scan, total);
    if (tid < 32) {
        unsigned long long e = lookback_warp(status, t, total, err);
        if (tid == 0) s_excl = e;
    }
    __syncthreads();
    unsigned long long run = s_excl + pref;
#pragma unroll
    for (int j = 0; j < kScItems; j++) {
        if (i0 + j < n) dag_off[i0 + j] = run;
        run += v[j];
    }
    if (t == ntiles - 1 && tid == kScThreads - 1) dag_off[n] = run;
}

// Bitonic sort of a power-of-two buffer in shared memory by one warp (or one block when
// `block` is set).
__device__ __forceinline__ void bitonic_smem(uint32_t *s, uint32_t p, int lane, int width,
                                             bool block)
{
    for (uint32_t k = 2; k <= p; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = lane; i < p; i += width) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const uint32_t a = s[i], b = s[ixj];
                    const bool asc = (i & k) == 0;
                    if ((a > b) == asc) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            if (block) __syncthreads();
            else __syncwarp();
        }
    }
}

// Ascending bitonic sort of 32*E values held by one warp in registers, striped: value e of
// lane l has index e*32 + l.  Partners closer than 32 are on other lanes (shuffles), farther
// ones are in the same lane's registers.
template <int E>
__device__ __forceinline__ void warp_sort_striped(uint32_t (&v)[E], int lane)
{
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int je = j >> 5;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    if ((e & je) == 0) {
                        const int e2 = e | je;
                        const bool asc = (((uint32_t)(e * 32 + lane)) & k) == 0;
                        const uint32_t a = v[e], b = v[e2];
                        const bool sw = (a > b) == asc;
                        v[e] = sw ? b : a;
                        v[e2] = sw ? a : b;
                    }
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const bool asc = (((uint32_t)(e * 32 + lane)) & k) == 0;
                    const uint32_t q = __shfl_xor_sync(kFull, v[e], j);
                    v[e] = (lower == asc) ? min(v[e], q) : max(v[e], q);
                }
            }
        }
    }
}

// Loads a row of len <= 32*E values (striped, padded with the maximum), sorts it in registers
// and stores it to dst.
template <int E>
__device__ __forceinline__ void warp_sort_row(const uint32_t *src, uint32_t len, uint32_t *dst, int lane)
{
    uint32_t v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t i = e * 32 + lane;
        v[e] = i < len ? src[i] : 0xffffffffu;
    }
    warp_sort_striped<E>(v, lane);
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t i = e * 32 + lane;
        if (i < len) dst[i] = v[e];
    }
}

constexpr int kRlWarps = 8;
constexpr uint32_t kRlRows = 256;     // rows per block step
constexpr uint32_t kRlStage = 8192;   // kept entries staged in shared memory per step
constexpr uint32_t kRlWarpCap = 512;  // rows up to this length are sorted by one warp
constexpr uint32_t kLongCap = 32768;  // longest relabelled row this build sorts (power of 2)

// Relabel: the kept row of input vertex u (values = ranks, input order) becomes row rank[u] of
// the DAG, sorted.  A block takes 256 consecutive input rows at a time.  Their offsets, ranks and
// destinations are staged in shared memory (coalesced, independent loads) and, when the rows'
// entries fit, the entries too (one coalesced copy: the rows are contiguous).  Rows of at most
// 32 entries are then sorted with one thread per entry: its place is the number of smaller
// entries in its row (ranks are distinct).  Rows up to 512 entries are sorted by one warp in
// registers (bitonic, up to 16 values per lane); longer rows are listed for k_rl_sort_long.
__global__ __launch_bounds__(kRlWarps * 32) void k_rl_sort(
    uint32_t n, const uint64_t *__restrict__ G, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ rank, const uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, uint64_t dag_cap, uint32_t *long_rows, uint32_t *n_long,
    uint32_t *err)
{
    __shared__ uint64_t s_g[kRlRows + 1];
    __shared__ uint64_t s_dst[kRlRows];
    __shared__ uint32_t s_vals[kRlStage];
    __shared__ uint8_t s_rowid[kRlStage];  // row (within the step) of each staged entry of a short row
    static_assert(kRlRows <= 256, "row ids are 8-bit");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (uint32_t r0 = blockIdx.x * kRlRows; r0 < n; r0 += gridDim.x * kRlRows) {
        const uint32_t cnt = min(kRlRows, n - r0);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i <= cnt; i += blockDim.x) s_g[i] = G[r0 + i];
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t ru = rank[r0 + i];
            s_dst[i] = ru < n ? dag_off[ru] : ~0ull;
        }
        __syncthreads();
        const uint64_t base = s_g[0];
        const uint64_t total = s_g[cnt] - base;
        const bool staged = total <= kRlStage;
        if (staged) {
            for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) s_vals[i] = vals[base + i];
            for (uint32_t i = w; i < cnt; i += kRlWarps) {  // row ids of the short rows' entries
                const uint32_t rb = (uint32_t)(s_g[i] - base), re = (uint32_t)(s_g[i + 1] - base);
                if (re - rb <= 32 && rb + lane < re) s_rowid[rb + lane] = (uint8_t)i;
            }
        }
        __syncthreads();
        // short rows: one thread per staged entry
        if (staged) {
            for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
                // entries of long rows hold a stale id: the range check sends them to the warps
                const uint32_t lo = s_rowid[e];
                if (lo >= cnt) continue;
                const uint32_t rb = (uint32_t)(s_g[lo] - base), len = (uint32_t)(s_g[lo + 1] - s_g[lo]);
                if (e < rb || e >= rb + len || len > 32) continue;
                const uint64_t dst = s_dst[lo];
                if (dst == ~0ull || dst + len > dag_cap) {
                    set_error(err, kDevBadInput);
                    continue;
                }
                const uint32_t x = s_vals[e];
                uint32_t pos = 0;
                for (uint32_t j = 0; j < len; j++) pos += s_vals[rb + j] < x;
                dag_cols[dst + pos] = x;
            }
        }
        // longer rows (and every row of a step whose entries were not staged): one warp each
        for (uint32_t i = w; i < cnt; i += kRlWarps) {
            const uint64_t b = s_g[i];
            const uint32_t len = (uint32_t)(s_g[i + 1] - b);
            if (len == 0 || (staged && len <= 32)) continue;
            const uint64_t dst = s_dst[i];
            if (dst == ~0ull || dst + len > dag_cap) {
                if (lane == 0) set_error(err, kDevBadInput);
                continue;
            }
            const uint32_t *src = staged ? s_vals + (b - base) : vals + b;
            uint32_t *out = dag_cols + dst;
            if (len <= 32) warp_sort_row<1>(src, len, out, lane);
            else if (len <= 64) warp_sort_row<2>(src, len, out, lane);
            else if (len <= 128) warp_sort_row<4>(src, len, out, lane);
            else if (len <= 256) warp_sort_row<8>(src, len, out, lane);
            else if (len <= kRlWarpCap) warp_sort_row<16>(src, len, out, lane);
            else if (lane == 0) long_rows[atomicAdd(n_long, 1u)] = r0 + i;
        }
    }
}

// One block per long row; dynamic shared memory holds the padded row.
__global__ __launch_bounds__(1024) void k_rl_sort_long(
    uint32_t n, const uint64_t *__restrict__ G, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ rank, const uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, uint64_t dag_cap, const uint32_t *long_rows,
    const uint32_t *n_long, uint32_t cap, uint32_t *err)
{
    extern __shared__ uint32_t s_row[];
    for (uint32_t it = blockIdx.x; it < *n_long; it += gridDim.x) {
        const uint32_t u = long_rows[it];
        const uint32_t ru = rank[u];
        const uint64_t b = G[u];
        const uint32_t len = (uint32_t)(G[u + 1] - b);
        if (len > cap || ru >= n) {
            if (threadIdx.x == 0) set_error(err, len > cap ? kDevTooLong : kDevBadInput);
            continue;
        }
        uint32_t p = 64;
        while (p < len) p <<= 1;
        for (uint32_t j = threadIdx.x; j < p; j += blockDim.x) s_row[j] = j < len ? vals[b + j] : 0xffffffffu;
        __syncthreads();
        bitonic_smem(s_row, p, threadIdx.x, blockDim.x, true);
        const uint64_t dst = dag_off[ru];
        if (dst + len <= dag_cap)
            for (uint32_t j = threadIdx.x; j < len; j += blockDim.x) dag_cols[dst + j] = s_row[j];
        else if (threadIdx.x == 0)
            set_error(err, kDevBadInput);
        __syncthreads();
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

size_t dag_ws_bytes(uint32_t n, uint64_t arcs)
{
    Sizer s;
    const uint64_t ntiles = (arcs + kGoTile - 1) / kGoTile;
    s.take<uint32_t>(ntiles + 2);             // first_row
    s.take<unsigned long long>(ntiles + 1);   // look-back status (compaction)
    s.take<uint32_t>(8);                      // tickets, counters
    s.take<uint32_t>((size_t)n + 1);          // degrees / rowlen
    s.take<unsigned long long>((size_t)n / kScTile + 2);  // look-back status (scan)
    s.take<uint32_t>((size_t)n + 1);          // long rows
    s.take<uint64_t>((size_t)n + 1);          // kept-row offsets in input order
    s.take<uint32_t>(arcs / 2 + 1);           // kept ranks in input order
    return s.used;
}

// Returns cudaErrorMemoryAllocation if the workspace is short; device errors land in err.
cudaError_t launch_build_dag(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                             const uint32_t *rank, uint64_t *dag_off, uint32_t *dag_cols,
                             uint32_t *d_max_outdeg, uint32_t *err, Carver &c, cudaStream_t st,
                             int num_sms)
{
    const uint64_t ntiles64 = (arcs + kGoTile - 1) / kGoTile;
    uint32_t *first_row = c.take<uint32_t>(ntiles64 + 2);
    unsigned long long *status = c.take<unsigned long long>(ntiles64 + 1);
    uint32_t *ctr = c.take<uint32_t>(8);
    uint32_t *keys = c.take<uint32_t>((size_t)n + 1);
    const uint32_t sc_tiles = (n + kScTile - 1) / kScTile;
    unsigned long long *sc_status = c.take<unsigned long long>((size_t)n / kScTile + 2);
    uint32_t *long_rows = c.take<uint32_t>((size_t)n + 1);
    uint64_t *G = c.take<uint64_t>((size_t)n + 1);
    uint32_t *kept = c.take<uint32_t>(arcs / 2 + 1);
    if (!c.ok) return cudaErrorMemoryAllocation;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctr, 0, 8 * sizeof(uint32_t), st))) return e;
    if (arcs == 0 || n == 0) {
        return cudaMemsetAsync(dag_off, 0, ((size_t)n + 1) * sizeof(uint64_t), st);
    }
    const uint32_t ntiles = (uint32_t)ntiles64;
    const int vec4 = ((uintptr_t)cols % 16) == 0;
    if ((e = cudaMemsetAsync(status, 0, ntiles64 * sizeof(unsigned long long), st))) return e;
    k_tile_rows<<<(n + 1 + 255) / 256, 256, 0, st>>>(n, arcs, off, kGoTile, ntiles, first_row);
    note_launches(1);
    if (!rank) {
        k_degrees<<<(n + 255) / 256, 256, 0, st>>>(n, off, keys);
        k_dag_compact<0><<<ntiles, kGoThreads, 0, st>>>(n, arcs, off, cols, keys, first_row, ntiles,
                                                       dag_off, dag_cols, arcs / 2, status, ctr,
                                                       err, vec4);
        note_launches(2);
        if (d_max_outdeg) {
            k_max_rowlen<<<num_sms * 4, 256, 0, st>>>(n, dag_off, d_max_outdeg);
            note_launches(1);
        }
        return cudaGetLastError();
    }
    if ((e = cudaMemsetAsync(sc_status, 0, ((size_t)sc_tiles + 1) * sizeof(unsigned long long), st)))
        return e;
    if ((e = cudaMemsetAsync(keys, 0, ((size_t)n + 1) * sizeof(uint32_t), st))) return e;
    uint32_t *max_len = ctr + 2;
    uint32_t *n_long = ctr + 3;
    k_dag_compact<1><<<ntiles, kGoThreads, 0, st>>>(n, arcs, off, cols, rank, first_row, ntiles, G,
                                                   kept, arcs / 2, status, ctr, err, vec4);
    k_rl_rowlen<<<(n + 255) / 256, 256, 0, st>>>(n, G, rank, keys, max_len, err);
    k_scan_rowlen<<<sc_tiles, kScThreads, 0, st>>>(n, keys, dag_off, sc_tiles, sc_status, ctr + 1,
                                                   err);
    uint32_t rl_grid = (n + kRlRows - 1) / kRlRows;
    if (rl_grid > (uint32_t)num_sms * 6) rl_grid = (uint32_t)num_sms * 6;
    k_rl_sort<<<rl_grid, kRlWarps * 32, 0, st>>>(n, G, kept, rank, dag_off, dag_cols, arcs / 2,
                                                 long_rows, n_long, err);
    const uint32_t cap_bytes = kLongCap * sizeof(uint32_t);
    if ((e = cudaFuncSetAttribute(k_rl_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  cap_bytes)))
        return e;
    k_rl_sort_long<<<num_sms, 1024, cap_bytes, st>>>(n, G, kept, rank, dag_off, dag_cols, arcs / 2,
                                                     long_rows, n_long, kLongCap, err);
    note_launches(5);
    if (d_max_outdeg)
        if ((e = cudaMemcpyAsync(d_max_outdeg, max_len, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)))
            return e;
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

