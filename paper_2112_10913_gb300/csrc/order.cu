// order.cu -- ordering phase on sm_103a: degree ordering, DAG construction, input validation.
//
//   Degree ordering (Sec. II, Sec. IV): rank = position of u when sorted by (d(u), u).
//     k_radix_hist / k_radix_scatter: stable LSD radix sort of the ids by degree, 8-bit digits;
//     ids enter in ascending order, so stability supplies the id tie-break.
//   Algorithm GenOrdering (Sec. IV), fused into ONE pass over the arcs:
//     k_tile_rows     : for every tile of 4096 arcs, the first vertex whose row starts in it;
//     k_gen_ordering  : keep-test of every arc, block scan, decoupled look-back prefix over tiles,
//                       coalesced store of the kept arcs (the DAG columns, already sorted per
//                       row) and of the DAG row offsets.  The count pass, PrefixSum and the fill
//                       pass of the listing become one read of cols and one write of the DAG.
//   Relabelled DAG from any rank (Sec. II directionalizing, rows renamed to ranks):
//     k_outdeg_rank -> k_scan_rowlen (look-back) -> k_fill_rank (+ k_fill_rank_long).
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

// Exclusive scan of one uint32 array by a single block (sizes here are 256 x blocks).
__global__ __launch_bounds__(1024) void k_scan_small(uint32_t *data, uint32_t count)
{
    __shared__ uint32_t scratch[33];
    const uint32_t per = (count + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(count, threadIdx.x * per), hi = min(count, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; i++) s += data[i];
    uint32_t total;
    uint32_t run = block_excl_scan(s, scratch, total);
    for (uint32_t i = lo; i < hi; i++) {
        uint32_t v = data[i];
        data[i] = run;
        run += v;
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

__device__ __forceinline__ bool degree_before(uint64_t du, uint32_t u, uint64_t dv, uint32_t v)
{
    return du < dv || (du == dv && u < v);
}

__global__ __launch_bounds__(kGoThreads) void k_gen_ordering(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ cols,
    const uint32_t *__restrict__ first_row, uint32_t ntiles, uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, uint64_t dag_cap, unsigned long long *status,
    uint32_t *ticket, uint32_t *err, int vec4)
{
    __shared__ uint64_t s_row[kGoRowCap + 1];
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
    if (cached)
        for (uint32_t i = tid; i <= nrows; i += kGoThreads) s_row[i] = off[r0 + i];
    __syncthreads();
    auto row_start = [&](uint32_t r) -> uint64_t {  // off[r] for r in [r0, u_next]
        return cached ? s_row[r - r0] : off[r];
    };

    // Rows of this thread's first arc: last r in [r0, u_next] with off[r] <= a.
    const uint64_t a0 = bad ? t1 : t0 + (uint64_t)tid * kGoItems;
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
    uint32_t v[kGoItems];
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
    uint32_t mask = 0;
    if (a0 < t1) {
        uint64_t rs = row_start(r), re = row_start(r + 1);
#pragma unroll
        for (int j = 0; j < kGoItems; j++) {
            const uint64_t a = a0 + j;
            if (a < t1) {
                while (re <= a) {
                    r++;
                    rs = re;
                    re = row_start(r + 1);
                }
                const uint32_t w = v[j];
                if (w >= n) {
                    set_error(err, kDevBadInput);
                    continue;
                }
                const uint64_t du = re - rs;
                const uint64_t dw = __ldg(off + w + 1) - __ldg(off + w);
                if (degree_before(du, r, dw, w)) mask |= 1u << j;
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
        unsigned long long e = lookback_warp(status, t, total, err);
        if (tid == 0) s_excl = e;
    }
    __syncthreads();
    const unsigned long long excl = s_excl;
    if (excl + total > dag_cap) {  // more kept arcs than half the input: asymmetric input
        if (tid == 0) set_error(err, kDevBadInput);
        return;
    }
    for (uint32_t i = tid; i < total; i += kGoThreads) dag_cols[excl + i] = s_out[i];
    if (bad) return;
    // DAG row offsets of the vertices whose rows start inside this tile.
    for (uint32_t u = u_first + tid; u < u_next; u += kGoThreads) {
        const uint32_t pos = (uint32_t)(row_start(u) - t0);
        const uint32_t q = pos / kGoItems, j = pos % kGoItems;
        dag_off[u] = excl + s_pref[q] + __popc((uint32_t)s_mask[q] & ((1u << j) - 1));
    }
    if (t == ntiles - 1) {  // trailing vertices whose rows start at the end of the arcs
        for (uint32_t u = first_row[ntiles] + tid; u <= n; u += kGoThreads) dag_off[u] = excl + total;
    }
}

// ------------------------------------------------------------------------------------------
// Relabelled DAG from a rank permutation.

// rowlen[rank[u]] = #{v in N(u) : rank[v] > rank[u]}; warp per vertex.
__global__ void k_outdeg_rank(uint32_t n, const uint64_t *__restrict__ off,
                              const uint32_t *__restrict__ cols, const uint32_t *__restrict__ rank,
                              uint32_t *__restrict__ rowlen, uint32_t *max_len, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    uint32_t best = 0;
    for (uint32_t u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
        const uint64_t b = off[u], e = off[u + 1];
        const uint32_t ru = rank[u];
        if (ru >= n) {
            if (lane == 0) set_error(err, kDevBadInput);
            continue;
        }
        uint32_t c = 0;
        for (uint64_t i = b + lane; i < e; i += 32) {
            const uint32_t v = cols[i];
            if (v < n) c += rank[v] > ru;
            else set_error(err, kDevBadInput);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) rowlen[ru] = c;
        best = max(best, c);
    }
    if (lane == 0 && best) atomicMax(max_len, best);
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

constexpr int kFrWarps = 8;
constexpr uint32_t kFrCap = 1024;  // rows up to this length are sorted by one warp

// Fill row rank[u] with the ranks of u's later neighbours, sorted.  Warp per vertex; longer
// rows are listed for k_fill_rank_long.
__global__ __launch_bounds__(kFrWarps * 32) void k_fill_rank(
    uint32_t n, const uint64_t *__restrict__ off, const uint32_t *__restrict__ cols,
    const uint32_t *__restrict__ rank, const uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, uint32_t *long_rows, uint32_t *n_long)
{
    __shared__ uint32_t s_buf[kFrWarps][kFrCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *buf = s_buf[w];
    const uint32_t warps = gridDim.x * kFrWarps;
    for (uint32_t u = blockIdx.x * kFrWarps + w; u < n; u += warps) {
        const uint32_t ru = rank[u];
        if (ru >= n) continue;
        const uint64_t ob = dag_off[ru];
        const uint32_t len = (uint32_t)(dag_off[ru + 1] - ob);
        if (len == 0) continue;
        if (len > kFrCap) {
            if (lane == 0) long_rows[atomicAdd(n_long, 1u)] = u;
            continue;
        }
        const uint64_t b = off[u], e = off[u + 1];
        uint32_t fill = 0;
        for (uint64_t i = b; i < e; i += 32) {
            uint32_t x = 0;
            bool keep = false;
            if (i + lane < e && cols[i + lane] < n) {
                x = rank[cols[i + lane]];
                keep = x > ru;
            }
            const uint32_t bal = __ballot_sync(kFull, keep);
            const uint32_t pos = fill + __popc(bal & lanemask_lt());
            if (keep && pos < len) buf[pos] = x;
            fill += __popc(bal);
        }
        if (len <= 32) {
            // one element per lane; bitonic network over shuffles
            uint32_t x = lane < len ? buf[lane] : 0xffffffffu;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const uint32_t y = __shfl_xor_sync(kFull, x, j);
                    const bool up = (lane & k) == 0;
                    const bool lower = (lane & j) == 0;
                    x = (lower == up) ? min(x, y) : max(x, y);
                }
            }
            if (lane < len) dag_cols[ob + lane] = x;
        } else {
            uint32_t p = 64;
            while (p < len) p <<= 1;
            for (uint32_t i = len + lane; i < p; i += 32) buf[i] = 0xffffffffu;
            __syncwarp();
            bitonic_smem(buf, p, lane, 32, false);
            for (uint32_t i = lane; i < len; i += 32) dag_cols[ob + i] = buf[i];
        }
        __syncwarp();
    }
}

constexpr uint32_t kLongCap = 32768;  // longest relabelled row this build sorts (power of 2)

// One block per long row; dynamic shared memory holds the padded row.
__global__ __launch_bounds__(1024) void k_fill_rank_long(
    uint32_t n, const uint64_t *__restrict__ off, const uint32_t *__restrict__ cols,
    const uint32_t *__restrict__ rank, const uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, const uint32_t *long_rows, const uint32_t *n_long,
    uint32_t cap, uint32_t *err)
{
    extern __shared__ uint32_t s_row[];
    __shared__ uint32_t s_fill;
    __shared__ uint32_t s_scan[33];
    for (uint32_t it = blockIdx.x; it < *n_long; it += gridDim.x) {
        const uint32_t u = long_rows[it];
        const uint32_t ru = rank[u];
        const uint64_t ob = dag_off[ru];
        const uint32_t len = (uint32_t)(dag_off[ru + 1] - ob);
        if (len > cap) {
            if (threadIdx.x == 0) set_error(err, kDevTooLong);
            continue;
        }
        if (threadIdx.x == 0) s_fill = 0;
        __syncthreads();
        const uint64_t b = off[u], e = off[u + 1];
        for (uint64_t i0 = b; i0 < e; i0 += blockDim.x) {
            const uint64_t i = i0 + threadIdx.x;
            uint32_t x = 0, keep = 0;
            if (i < e && cols[i] < n) {
                x = rank[cols[i]];
                keep = x > ru;
            }
            uint32_t tot;
            const uint32_t pos = block_excl_scan(keep, s_scan, tot);
            if (keep && s_fill + pos < len) s_row[s_fill + pos] = x;
            __syncthreads();
            if (threadIdx.x == 0) s_fill += tot;
            __syncthreads();
        }
        uint32_t p = 64;
        while (p < len) p <<= 1;
        for (uint32_t i = len + threadIdx.x; i < p; i += blockDim.x) s_row[i] = 0xffffffffu;
        __syncthreads();
        bitonic_smem(s_row, p, threadIdx.x, blockDim.x, true);
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) dag_cols[ob + i] = s_row[i];
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

cudaError_t launch_order(uint32_t n, const uint64_t *off, uint32_t *rank, uint32_t *perm,
                         Carver &c, cudaStream_t st)
{
    const uint32_t nb = (n + kRsTile - 1) / kRsTile;
    uint32_t *keys[2] = {c.take<uint32_t>(n), c.take<uint32_t>(n)};
    uint32_t *vals[2] = {c.take<uint32_t>(n), c.take<uint32_t>(n)};
    uint32_t *hist = c.take<uint32_t>((size_t)256 * (nb + 1));
    if (!c.ok) return cudaErrorMemoryAllocation;
    if (n == 0) return cudaSuccess;
    const int passes = radix_passes(n);
    const uint32_t *kin = nullptr, *vin = nullptr;
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

size_t dag_ws_bytes(uint32_t n, uint64_t arcs)
{
    Sizer s;
    const uint64_t ntiles = (arcs + kGoTile - 1) / kGoTile;
    s.take<uint32_t>(ntiles + 2);             // first_row
    s.take<unsigned long long>(ntiles + 1);   // look-back status (GenOrdering)
    s.take<uint32_t>(8);                      // tickets, counters
    s.take<uint32_t>((size_t)n + 1);          // rowlen (relabel)
    s.take<unsigned long long>((size_t)n / kScTile + 2);  // look-back status (scan)
    s.take<uint32_t>((size_t)n + 1);          // long rows
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
    uint32_t *rowlen = c.take<uint32_t>((size_t)n + 1);
    const uint32_t sc_tiles = (n + kScTile - 1) / kScTile;
    unsigned long long *sc_status = c.take<unsigned long long>((size_t)n / kScTile + 2);
    uint32_t *long_rows = c.take<uint32_t>((size_t)n + 1);
    if (!c.ok) return cudaErrorMemoryAllocation;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctr, 0, 8 * sizeof(uint32_t), st))) return e;
    if (arcs == 0 || n == 0) {
        return cudaMemsetAsync(dag_off, 0, ((size_t)n + 1) * sizeof(uint64_t), st);
    }
    if (!rank) {
        const uint32_t ntiles = (uint32_t)ntiles64;
        if ((e = cudaMemsetAsync(status, 0, ntiles64 * sizeof(unsigned long long), st))) return e;
        k_tile_rows<<<(n + 1 + 255) / 256, 256, 0, st>>>(n, arcs, off, kGoTile, ntiles, first_row);
        const int vec4 = ((uintptr_t)cols % 16) == 0;
        k_gen_ordering<<<ntiles, kGoThreads, 0, st>>>(n, arcs, off, cols, first_row, ntiles, dag_off,
                                                     dag_cols, arcs / 2, status, ctr, err, vec4);
        note_launches(2);
        if (d_max_outdeg) {
            k_max_rowlen<<<num_sms * 4, 256, 0, st>>>(n, dag_off, d_max_outdeg);
            note_launches(1);
        }
        return cudaGetLastError();
    }
    if ((e = cudaMemsetAsync(sc_status, 0, ((size_t)sc_tiles + 1) * sizeof(unsigned long long), st)))
        return e;
    uint32_t *max_len = ctr + 2;
    uint32_t *n_long = ctr + 3;
    k_outdeg_rank<<<num_sms * 8, 256, 0, st>>>(n, off, cols, rank, rowlen, max_len, err);
    k_scan_rowlen<<<sc_tiles, kScThreads, 0, st>>>(n, rowlen, dag_off, sc_tiles, sc_status, ctr + 1,
                                                   err);
    k_fill_rank<<<num_sms * 8, kFrWarps * 32, 0, st>>>(n, off, cols, rank, dag_off, dag_cols,
                                                       long_rows, n_long);
    const uint32_t cap_bytes = kLongCap * sizeof(uint32_t);
    if ((e = cudaFuncSetAttribute(k_fill_rank_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  cap_bytes)))
        return e;
    k_fill_rank_long<<<num_sms, 1024, cap_bytes, st>>>(n, off, cols, rank, dag_off, dag_cols,
                                                       long_rows, n_long, kLongCap, err);
    note_launches(4);
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

