// relabel.cu -- the DAG of any total order, relabelled to ranks (Sec. II directionalisation with
// the rows renamed by position in the order).
//
// Row r of the output belongs to the vertex u of rank r and holds the ranks of u's neighbours of
// higher rank, ascending.  With the degree rank of citron_order this is the degree-ordered DAG
// (Sec. II, Sec. IV) in rank space, where every local subgraph of the counting phase is
// upper-triangular.
//
// Four launches, none of which waits on another block:
//   k_rl_prologue : rowlen[r] = 0 and perm[rank[u]] = u (the vertex of each rank);
//   k_rl_keep     : one pass over the arcs in tiles of 4096.  Per arc u->v the keep-test
//                   rank[v] > rank[u] (the rank gathers of a tile are all in flight before any
//                   is used); the kept ranks of each row are compacted IN the row's own input
//                   range (kept[off[u] ..]), so no global prefix is needed.  Every (row, tile)
//                   piece takes its place in the row with one atomicAdd on rowlen[rank[u]],
//                   which ends up holding the row's out-degree in rank order;
//   k_scan_rowlen : dag_off = exclusive prefix of rowlen (single pass, decoupled look-back) and
//                   the largest row;
//   k_rl_fill     : rows in RANK order, 256 per step: each row's kept ranks are gathered from its
//                   input range into shared memory at their output position, sorted there
//                   (rows of <= 32 by counting the smaller entries, <= 512 by one warp's
//                   register bitonic sort) and the step's output range dag_cols[dag_off[r0] ..
//                   dag_off[r0 + 256]) is written out contiguously; rows above 512 are listed
//                   for k_rl_fill_long (one block per row).
// The kernels after k_rl_keep return at once when the error word is set: offsets computed
// after an error are not trusted.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace citron {

constexpr int kKeThreads = 256;
constexpr int kKeItems = 16;
constexpr uint32_t kKeTile = kKeThreads * kKeItems;  // arcs per tile of k_rl_keep
constexpr uint32_t kKeRowCap = 2048;                 // row offsets cached in shared memory
constexpr int32_t kNoSlot = INT32_MIN;               // a row piece that may not be written

// rowlen[r] = 0 for every rank, perm[rank[u]] = u.
__global__ void k_rl_prologue(uint32_t n, const uint32_t *__restrict__ rank, uint32_t *rowlen,
                              uint32_t *perm, uint32_t *err)
{
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    rowlen[u] = 0;
    const uint32_t r = rank[u];
    if (r < n) perm[r] = u;
    else set_error(err, kDevBadInput);
}

// Number of kept arcs before tile position x (0 <= x <= 4096) from the per-thread prefix and
// keep masks of the tile.
__device__ __forceinline__ uint32_t tile_prefix(const uint32_t *s_pref, const uint16_t *s_mask,
                                                uint32_t x)
{
    const uint32_t q = x / kKeItems, b = x % kKeItems;
    if (q >= (uint32_t)kKeThreads) return s_pref[kKeThreads];
    return s_pref[q] + __popc((uint32_t)s_mask[q] & ((1u << b) - 1u));
}

// Rows of a tile with more than kKeRowCap rows (long runs of empty rows): every kept arc takes
// its place in its row with its own atomic.  Offsets are read from global memory.
__device__ __noinline__ void rl_keep_uncached(uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off,
                                              const uint32_t *__restrict__ cols,
                                              const uint32_t *__restrict__ rank, uint32_t r0,
                                              uint32_t u_next, uint64_t t0, uint64_t t1,
                                              uint32_t *kept, uint32_t *rowlen, uint32_t *err)
{
    const uint64_t a0 = t0 + (uint64_t)threadIdx.x * kKeItems;
    if (a0 >= t1) return;
    uint32_t lo = r0, hi = u_next;  // last r with off[r] <= a0
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo + 1) / 2;
        if (off[mid] <= a0) lo = mid;
        else hi = mid - 1;
    }
    uint32_t r = lo;
    uint64_t rs = off[r], re = off[r + 1];
    for (int j = 0; j < kKeItems; j++) {
        const uint64_t a = a0 + j;
        if (a >= t1) break;
        while (re <= a && r + 1 < u_next) {
            r++;
            rs = re;
            re = off[r + 1];
        }
        const uint32_t v = cols[a];
        const uint32_t ku = rank[r];
        if (v >= n || ku >= n || rs > re || re > arcs) {
            set_error(err, kDevBadInput);
            continue;
        }
        const uint32_t kv = rank[v];
        if (kv > ku) {
            const uint32_t pos = atomicAdd(&rowlen[ku], 1u);
            if (pos < re - rs) kept[rs + pos] = kv;
            else set_error(err, kDevBadInput);
        }
    }
}

// first_row[b] = min{u : off[u] >= b * 4096} (k_tile_rows, order.cu).  Positions inside a tile
// are 32-bit offsets from its first arc t0; the tile's rows are cached with their starts
// clamped to the tile.
__global__ __launch_bounds__(kKeThreads) void k_rl_keep(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ cols,
    const uint32_t *__restrict__ rank, const uint32_t *__restrict__ first_row, uint32_t *kept,
    uint32_t *rowlen, uint32_t *err, int vec4)
{
    __shared__ uint32_t s_rel[kKeRowCap + 1];  // row starts - t0, clamped to [0, len]
    __shared__ uint32_t s_key[kKeRowCap];      // rank of each row
    __shared__ int32_t s_delta[kKeRowCap];     // place of the row's piece minus P(piece start)
    __shared__ uint32_t s_out[kKeTile];        // kept ranks in tile order
    __shared__ uint16_t s_krow[kKeTile];       // tile row of each kept rank
    __shared__ uint32_t s_pref[kKeThreads + 1];
    __shared__ uint16_t s_mask[kKeThreads];
    __shared__ uint32_t s_scan[kKeThreads / 32 + 1];

    const int tid = threadIdx.x;
    const uint32_t t = blockIdx.x;
    const uint64_t t0 = (uint64_t)t * kKeTile;
    const uint64_t t1 = min(t0 + kKeTile, arcs);
    const uint32_t len = (uint32_t)(t1 - t0);
    const uint32_t u_first = first_row[t];
    const uint32_t u_next = first_row[t + 1];
    const bool bad = u_first > n || u_next > n || u_next < u_first || (t > 0 && u_first == 0);
    if (bad) {
        if (tid == 0) set_error(err, kDevBadInput);
        return;
    }
    // rows r0 .. u_next-1 can hold arcs of this tile (r0 = last row starting at or before t0)
    const uint64_t o_first = off[u_first];
    const uint32_t r0 = (o_first == t0) ? u_first : u_first - 1;
    const uint32_t nrows = u_next - r0;
    if (nrows > kKeRowCap || nrows == 0) {
        rl_keep_uncached(n, arcs, off, cols, rank, r0, u_next, t0, t1, kept, rowlen, err);
        return;
    }
    const uint64_t row0_start = off[r0];
    for (uint32_t i = tid; i <= nrows; i += kKeThreads) {
        const uint64_t o = off[r0 + i];
        s_rel[i] = o <= t0 ? 0u : (o - t0 >= len ? len : (uint32_t)(o - t0));
        if (i < nrows) s_key[i] = rank[r0 + i];
    }
    __syncthreads();

    const uint32_t p0 = (uint32_t)tid * kKeItems;
    uint32_t v[kKeItems], kv[kKeItems];
    if (vec4 && p0 + kKeItems <= len) {
        const uint4 *p = reinterpret_cast<const uint4 *>(cols + t0 + p0);
#pragma unroll
        for (int q = 0; q < kKeItems / 4; q++) {
            const uint4 x = __ldg(p + q);
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kKeItems; j++) v[j] = (p0 + j < len) ? cols[t0 + p0 + j] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kKeItems; j++) kv[j] = (p0 + j < len && v[j] < n) ? __ldg(rank + v[j]) : 0u;

    // tile row of this thread's first arc: last i with s_rel[i] <= p0 (s_rel[0] = 0)
    uint32_t ri0 = 0;
    if (p0 < len) {
        uint32_t lo = 0, hi = nrows - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (s_rel[mid] <= p0) lo = mid;
            else hi = mid - 1;
        }
        ri0 = lo;
    }

    uint32_t mask = 0;
    if (p0 < len) {
        uint32_t ri = ri0, re = s_rel[ri + 1], ku = s_key[ri];
#pragma unroll
        for (int j = 0; j < kKeItems; j++) {
            const uint32_t p = p0 + j;
            if (p < len) {
                while (re <= p && ri + 1 < nrows) {
                    ri++;
                    re = s_rel[ri + 1];
                    ku = s_key[ri];
                }
                if (v[j] >= n) set_error(err, kDevBadInput);
                else if (kv[j] > ku) mask |= 1u << j;
            }
        }
    }
    s_mask[tid] = (uint16_t)mask;
    uint32_t total;
    s_pref[tid] = block_excl_scan(__popc(mask), s_scan, total);
    if (tid == 0) s_pref[kKeThreads] = total;
    __syncthreads();

    // each row piece reserves its place in its row with one atomic (thread per row)
    for (uint32_t i = tid; i < nrows; i += kKeThreads) {
        const uint32_t f = s_rel[i], e = s_rel[i + 1];
        int32_t delta = kNoSlot;
        if (e > f) {
            const uint32_t pf = tile_prefix(s_pref, s_mask, f);
            const uint32_t cnt = tile_prefix(s_pref, s_mask, e) - pf;
            if (cnt) {
                // the first and the last row may extend beyond the tile
                uint64_t rowlen_true = e - f;
                if (i == 0 || i == nrows - 1) {
                    const uint64_t b = off[r0 + i], c = off[r0 + i + 1];
                    rowlen_true = (b <= c && c <= arcs) ? c - b : 0;
                }
                const uint32_t key = s_key[i];
                if (key < n) {
                    const uint32_t base = atomicAdd(&rowlen[key], cnt);
                    // a row cannot keep more arcs than it has (else the rank is not a
                    // permutation); places stay far below 2^31
                    if ((uint64_t)base + cnt <= rowlen_true && base < 0x40000000u)
                        delta = (int32_t)base - (int32_t)pf;
                    else
                        set_error(err, kDevBadInput);
                } else {
                    set_error(err, kDevBadInput);
                }
            }
        }
        s_delta[i] = delta;
    }
    // kept ranks to shared memory in tile order, with their rows
    if (mask) {
        uint32_t ri = ri0, re = s_rel[ri + 1], q = s_pref[tid];
#pragma unroll
        for (int j = 0; j < kKeItems; j++) {
            const uint32_t p = p0 + j;
            if (p < len) {
                while (re <= p && ri + 1 < nrows) {
                    ri++;
                    re = s_rel[ri + 1];
                }
                if (mask >> j & 1) {
                    s_out[q] = kv[j];
                    s_krow[q] = (uint16_t)ri;
                    q++;
                }
            }
        }
    }
    __syncthreads();
    // consecutive kept ranks of a row piece go to consecutive places of the row
    for (uint32_t q = tid; q < total; q += kKeThreads) {
        const uint32_t ri = s_krow[q];
        const int32_t delta = s_delta[ri];
        if (delta == kNoSlot) continue;
        const uint64_t rs = ri == 0 ? row0_start : t0 + s_rel[ri];
        kept[rs + (uint64_t)(int64_t)((int64_t)delta + q)] = s_out[q];
    }
}

constexpr int kScThreads = 256;
constexpr int kScItems = 16;
constexpr uint32_t kScTile = kScThreads * kScItems;

// dag_off[i] = sum of rowlen[0..i), dag_off[n] = total (single pass with look-back); the largest
// row goes to max_len.
__global__ __launch_bounds__(kScThreads) void k_scan_rowlen(uint32_t n, const uint32_t *rowlen,
                                                            uint64_t *dag_off, uint32_t ntiles,
                                                            unsigned long long *status,
                                                            uint32_t *ticket, uint32_t *max_len,
                                                            uint32_t *err, WaitCfg wc)
{
    __shared__ uint32_t s_scan[kScThreads / 32 + 1];
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = *(volatile uint32_t *)err ? 0xffffffffu : atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= ntiles) return;
    const uint64_t i0 = (uint64_t)t * kScTile + (uint64_t)tid * kScItems;
    uint32_t v[kScItems];
    uint32_t s = 0, mx = 0;
#pragma unroll
    for (int j = 0; j < kScItems; j++) {
        v[j] = (i0 + j < n) ? rowlen[i0 + j] : 0;
        s += v[j];
        mx = max(mx, v[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    if ((tid & 31) == 0 && mx) atomicMax(max_len, mx);
    uint32_t total;
    const uint32_t pref = block_excl_scan(s, s_scan, total);
    if (tid < 32) {
        unsigned long long e = lookback_warp(status, t, total, err, wc);
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
// and stores it to dst (dst may alias src).
template <int E>
__device__ __forceinline__ void warp_sort_row(const uint32_t *src, uint32_t len, uint32_t *dst, int lane)
{
    uint32_t v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t i = e * 32 + lane;
        v[e] = i < len ? src[i] : 0xffffffffu;
    }
    __syncwarp();
    warp_sort_striped<E>(v, lane);
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t i = e * 32 + lane;
        if (i < len) dst[i] = v[e];
    }
}

// Sorts a row of 33..512 values with one warp; false when it is longer (left to the long path).
__device__ __forceinline__ bool warp_sort_any(const uint32_t *src, uint32_t len, uint32_t *dst, int lane)
{
    if (len <= 32) warp_sort_row<1>(src, len, dst, lane);
    else if (len <= 64) warp_sort_row<2>(src, len, dst, lane);
    else if (len <= 128) warp_sort_row<4>(src, len, dst, lane);
    else if (len <= 256) warp_sort_row<8>(src, len, dst, lane);
    else if (len <= 512) warp_sort_row<16>(src, len, dst, lane);
    else return false;
    return true;
}

constexpr int kFiWarps = 8;
constexpr uint32_t kFiRows = 256;     // ranks per block step
constexpr uint32_t kFiStage = 8192;   // values staged in shared memory per step
constexpr uint32_t kLongCap = 32768;  // longest relabelled row this build sorts (power of 2)

__global__ __launch_bounds__(kFiWarps * 32) void k_rl_fill(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ perm,
    const uint32_t *__restrict__ kept, const uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, uint64_t dag_cap, uint32_t *long_rows, uint32_t *n_long,
    uint32_t *err)
{
    __shared__ uint64_t s_dst[kFiRows + 1];
    __shared__ uint64_t s_src[kFiRows];
    __shared__ uint32_t s_vals[kFiStage];
    __shared__ uint8_t s_rowid[kFiStage];
    __shared__ int s_stop;
    static_assert(kFiRows <= 256, "row ids are 8-bit");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_stop = *(volatile uint32_t *)err != 0;
    __syncthreads();
    if (s_stop) return;
    for (uint32_t r0 = blockIdx.x * kFiRows; r0 < n; r0 += gridDim.x * kFiRows) {
        const uint32_t cnt = min(kFiRows, n - r0);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i <= cnt; i += blockDim.x) s_dst[i] = dag_off[r0 + i];
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint32_t u = perm[r0 + i];
            uint64_t src = ~0ull;
            if (u < n) {
                // the kept entries of u live in u's own input range
                const uint64_t b = off[u], e = off[u + 1];
                const uint64_t len = dag_off[r0 + i + 1] - dag_off[r0 + i];
                if (b <= e && e <= arcs && len <= e - b) src = b;
            }
            if (src == ~0ull) set_error(err, kDevBadInput);
            s_src[i] = src;
        }
        if (threadIdx.x == 0) s_stop = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x)
            if (s_dst[i + 1] < s_dst[i]) s_stop = 1;
        __syncthreads();
        const uint64_t base = s_dst[0];
        const uint64_t total = s_dst[cnt] - base;
        if (s_stop || s_dst[cnt] > dag_cap) {  // offsets not monotone, or more kept arcs than m
            if (threadIdx.x == 0) set_error(err, kDevBadInput);
            continue;
        }
        const bool staged = total <= kFiStage;
        if (staged) {
            // gather every row's kept entries to their output position (warp per row)
            for (uint32_t i = w; i < cnt; i += kFiWarps) {
                const uint32_t rb = (uint32_t)(s_dst[i] - base), len = (uint32_t)(s_dst[i + 1] - s_dst[i]);
                const uint64_t src = s_src[i];
                if (src == ~0ull) continue;
                for (uint32_t j = lane; j < len; j += 32) {
                    s_vals[rb + j] = kept[src + j];
                    s_rowid[rb + j] = (uint8_t)i;
                }
            }
            __syncthreads();
            // rows of <= 32: one thread per entry, place = number of smaller entries (ranks are
            // distinct); the result lands in global memory directly (each row is one segment)
            for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
                const uint32_t i = s_rowid[e];
                if (i >= cnt || s_src[i] == ~0ull) continue;  // entry of a row that was not gathered
                const uint32_t rb = (uint32_t)(s_dst[i] - base), len = (uint32_t)(s_dst[i + 1] - s_dst[i]);
                if (len > 32) continue;
                const uint32_t x = s_vals[e];
                uint32_t pos = 0;
                for (uint32_t j = 0; j < len; j++) pos += s_vals[rb + j] < x;
                dag_cols[base + rb + pos] = x;
            }
            // longer rows: one warp each, sorted in registers
            for (uint32_t i = w; i < cnt; i += kFiWarps) {
                const uint32_t rb = (uint32_t)(s_dst[i] - base), len = (uint32_t)(s_dst[i + 1] - s_dst[i]);
                if (len <= 32 || s_src[i] == ~0ull) continue;
                if (!warp_sort_any(s_vals + rb, len, dag_cols + base + rb, lane) && lane == 0)
                    long_rows[atomicAdd(n_long, 1u)] = r0 + i;
            }
        } else {
            for (uint32_t i = w; i < cnt; i += kFiWarps) {
                const uint32_t len = (uint32_t)(s_dst[i + 1] - s_dst[i]);
                const uint64_t src = s_src[i];
                if (len == 0 || src == ~0ull) continue;
                if (!warp_sort_any(kept + src, len, dag_cols + s_dst[i], lane) && lane == 0)
                    long_rows[atomicAdd(n_long, 1u)] = r0 + i;
            }
        }
    }
}

// One block per listed long row; dynamic shared memory holds the padded row.
__global__ __launch_bounds__(1024) void k_rl_fill_long(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ perm,
    const uint32_t *__restrict__ kept, const uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, uint64_t dag_cap, const uint32_t *long_rows,
    const uint32_t *n_long, uint32_t cap, uint32_t *err)
{
    extern __shared__ uint32_t s_row[];
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = *(volatile uint32_t *)err != 0;
    __syncthreads();
    if (s_stop) return;
    for (uint32_t it = blockIdx.x; it < *n_long; it += gridDim.x) {
        const uint32_t r = long_rows[it];
        if (r >= n) continue;
        const uint32_t u = perm[r];
        const uint64_t dst = dag_off[r];
        const uint64_t len64 = dag_off[r + 1] - dst;
        if (u >= n || len64 > cap || dst + len64 > dag_cap || off[u] + len64 > min(off[u + 1], arcs)) {
            if (threadIdx.x == 0) set_error(err, len64 > cap ? kDevTooLong : kDevBadInput);
            continue;
        }
        const uint32_t len = (uint32_t)len64;
        const uint64_t b = off[u];
        uint32_t p = 64;
        while (p < len) p <<= 1;
        for (uint32_t j = threadIdx.x; j < p; j += blockDim.x) s_row[j] = j < len ? kept[b + j] : 0xffffffffu;
        __syncthreads();
        for (uint32_t k = 2; k <= p; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = threadIdx.x; i < p; i += blockDim.x) {
                    const uint32_t ixj = i ^ j;
                    if (ixj > i) {
                        const uint32_t x = s_row[i], y = s_row[ixj];
                        if ((x > y) == ((i & k) == 0)) {
                            s_row[i] = y;
                            s_row[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t j = threadIdx.x; j < len; j += blockDim.x) dag_cols[dst + j] = s_row[j];
        __syncthreads();
    }
}

}  // namespace citron

namespace citron_host {

using namespace citron;

size_t relabel_ws_bytes(uint32_t n, uint64_t arcs)
{
    Sizer s;
    s.take<uint32_t>((arcs + kKeTile - 1) / kKeTile + 2);  // first_row
    s.take<uint32_t>(8);                                    // tickets, counters
    s.take<uint32_t>((size_t)n + 1);                        // rowlen (rank order)
    s.take<uint32_t>((size_t)n + 1);                        // perm
    s.take<unsigned long long>((size_t)n / kScTile + 2);    // look-back status (scan)
    s.take<uint32_t>((size_t)n + 1);                        // long rows
    s.take<uint32_t>(arcs + 1);                             // kept ranks, in-row layout
    return s.used;
}

cudaError_t launch_tile_rows(uint32_t n, uint64_t arcs, const uint64_t *off, uint32_t tile,
                             uint32_t ntiles, uint32_t *first_row, cudaStream_t st);

// Relabelled DAG of the order `rank`.  Device errors land in err.
cudaError_t launch_relabel_dag(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                               const uint32_t *rank, uint64_t *dag_off, uint32_t *dag_cols,
                               uint32_t *d_max_outdeg, uint32_t *err, Carver &c, cudaStream_t st,
                               int num_sms)
{
    const uint64_t ntiles64 = (arcs + kKeTile - 1) / kKeTile;
    uint32_t *first_row = c.take<uint32_t>(ntiles64 + 2);
    uint32_t *ctr = c.take<uint32_t>(8);
    uint32_t *rowlen = c.take<uint32_t>((size_t)n + 1);
    uint32_t *perm = c.take<uint32_t>((size_t)n + 1);
    const uint32_t sc_tiles = (n + kScTile - 1) / kScTile;
    unsigned long long *sc_status = c.take<unsigned long long>((size_t)n / kScTile + 2);
    uint32_t *long_rows = c.take<uint32_t>((size_t)n + 1);
    uint32_t *kept = c.take<uint32_t>(arcs + 1);
    if (!c.ok) return cudaErrorMemoryAllocation;
    if (ntiles64 >= 0xffffffffull) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctr, 0, 8 * sizeof(uint32_t), st))) return e;
    if (arcs == 0 || n == 0) return cudaMemsetAsync(dag_off, 0, ((size_t)n + 1) * sizeof(uint64_t), st);
    if ((e = cudaMemsetAsync(sc_status, 0, ((size_t)sc_tiles + 1) * sizeof(unsigned long long), st)))
        return e;
    const uint32_t ntiles = (uint32_t)ntiles64;
    const int vec4 = ((uintptr_t)cols % 16) == 0;
    uint32_t *ticket = ctr, *max_len = ctr + 2, *n_long = ctr + 3;
    if ((e = launch_tile_rows(n, arcs, off, kKeTile, ntiles, first_row, st))) return e;
    k_rl_prologue<<<(n + 255) / 256, 256, 0, st>>>(n, rank, rowlen, perm, err);
    k_rl_keep<<<ntiles, kKeThreads, 0, st>>>(n, arcs, off, cols, rank, first_row, kept, rowlen, err, vec4);
    k_scan_rowlen<<<sc_tiles, kScThreads, 0, st>>>(n, rowlen, dag_off, sc_tiles, sc_status, ticket,
                                                   max_len, err, wait_cfg());
    uint32_t grid = (n + kFiRows - 1) / kFiRows;
    if (grid > (uint32_t)num_sms * 8) grid = (uint32_t)num_sms * 8;
    k_rl_fill<<<grid, kFiWarps * 32, 0, st>>>(n, arcs, off, perm, kept, dag_off, dag_cols, arcs / 2,
                                              long_rows, n_long, err);
    const uint32_t cap_bytes = kLongCap * sizeof(uint32_t);
    if ((e = cudaFuncSetAttribute(k_rl_fill_long, cudaFuncAttributeMaxDynamicSharedMemorySize, cap_bytes)))
        return e;
    k_rl_fill_long<<<num_sms, 1024, cap_bytes, st>>>(n, arcs, off, perm, kept, dag_off, dag_cols,
                                                     arcs / 2, long_rows, n_long, kLongCap, err);
    note_launches(5);
    if (d_max_outdeg)
        if ((e = cudaMemcpyAsync(d_max_outdeg, max_len, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)))
            return e;
    return cudaGetLastError();
}

}  // namespace citron_host
