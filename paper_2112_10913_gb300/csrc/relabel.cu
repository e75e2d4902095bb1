// relabel.cu -- the DAG of any total order, relabelled to ranks (Sec. II directionalisation with
// the rows renamed by position in the order).
//
// Row r of the output belongs to the vertex u of rank r and holds the ranks of u's neighbours of
// higher rank, ascending.  With the degree rank of citron_order this is the degree-ordered DAG
// (Sec. II, Sec. IV) in rank space, where every local subgraph of the counting phase is
// upper-triangular.
//
// Six launches; no block waits on another, and only the scan waits on earlier tiles:
//   k_rl_prologue : rowlen[r] = 0 and perm[rank[u]] = u (the vertex of each rank);
//   k_rl_keep     : one pass over the arcs, one chunk of 512 arcs per warp and no block-wide
//                   barrier.  Per arc u->v the keep-test rank[v] > rank[u] (the 16 rank gathers
//                   of a lane are all in flight before any is used); the kept ranks of each row
//                   are placed IN the row's own input range (kept[off[u] ..]), so no global
//                   prefix is needed: a warp-aggregated shared counter per row gives each kept
//                   arc its place in its row piece, and every (row, chunk) piece takes its place
//                   in the row with one atomicAdd on rowlen[rank[u]], which ends up holding the
//                   row's out-degree in rank order;
//   k_scan_rowlen : dag_off = exclusive prefix of rowlen (single pass, decoupled look-back) and
//                   the largest row;
//   k_rl_fill     : rows in RANK order, one row per lane: a row of <= 32 entries is sorted by its
//                   lane in registers (a bitonic network of 4..32 values); longer rows are listed;
//   k_rl_fill_mid : one listed row per warp, claimed dynamically, sorted by the whole warp in
//                   registers (bitonic over the lanes): rows of 33..256 entries, then (second
//                   launch, more registers per lane) 257..1024; longer rows are listed again for
//                   k_rl_fill_long (one block per row).
// The kernels after k_rl_keep return at once when the error word is set: offsets computed
// after an error are not trusted.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace citron {


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

// A chunk of 512 arcs per warp; no block-wide barrier anywhere, so every warp runs at its own
// pace and the per-arc rank gathers of many warps overlap.
constexpr uint32_t kWkArcs = 512;    // arcs per warp chunk (4 quads of 4 arcs per lane)
constexpr uint32_t kWkRowCap = 64;   // rows of a chunk handled in shared memory
constexpr int kWkWarps = 8;          // warps per block

// A chunk overlapping more than kWkRowCap rows (long runs of empty rows): every kept arc takes
// its place in its row with its own atomic; offsets come from global memory.
__device__ __noinline__ void rl_keep_uncached(uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off,
                                              const uint32_t *__restrict__ cols,
                                              const uint32_t *__restrict__ rank, uint32_t r0,
                                              uint32_t u_next, uint64_t c0, uint64_t c1,
                                              uint32_t *kept, uint32_t *rowlen, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    for (uint64_t a = c0 + lane; a < c1; a += 32) {
        uint32_t lo = r0, hi = u_next;  // the last r with off[r] <= a
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo + 1) / 2;
            if (off[mid] <= a) lo = mid;
            else hi = mid - 1;
        }
        if (lo >= n) {  // offsets that are not monotone
            set_error(err, kDevBadInput);
            continue;
        }
        const uint64_t rs = off[lo], re = off[lo + 1];
        const uint32_t v = cols[a], ku = rank[lo];
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

// first_row[c] = min{u : off[u] >= c * 512} (k_tile_rows, order.cu).  Lane l holds the 16
// consecutive arcs 16l .. 16l+15 of its chunk.  The place of a kept arc inside its row piece is
// the number of kept arcs before it in the chunk (a warp prefix over the keep flags) minus that
// number at the piece's start; every (row, chunk) piece reserves its place in the row with one
// global atomic.
__global__ __launch_bounds__(kWkWarps * 32) void k_rl_keep(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ cols,
    const uint32_t *__restrict__ rank, const uint32_t *__restrict__ first_row, uint32_t nchunks,
    uint32_t *kept, uint32_t *rowlen, uint32_t *err, int vec4)
{
    __shared__ uint32_t s_rel[kWkWarps][kWkRowCap + 1];  // row starts - c0, clamped to [0, len]
    __shared__ uint32_t s_key[kWkWarps][kWkRowCap];      // rank of each row
    __shared__ int32_t s_place[kWkWarps][kWkRowCap];     // place of the row's piece minus P(start)
    __shared__ uint32_t s_excl[kWkWarps][33];            // kept arcs before each lane's arcs
    __shared__ uint16_t s_keep[kWkWarps][32];            // each lane's keep flags
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t c = blockIdx.x * kWkWarps + w;
    if (c >= nchunks) return;
    const uint64_t c0 = (uint64_t)c * kWkArcs;
    const uint64_t c1 = min(c0 + kWkArcs, arcs);
    const uint32_t len = (uint32_t)(c1 - c0);
    const uint32_t u_first = first_row[c], u_next = first_row[c + 1];
    if (u_first > n || u_next > n || u_next < u_first || (c > 0 && u_first == 0)) {
        if (lane == 0) set_error(err, kDevBadInput);
        return;
    }
    const uint32_t r0 = (off[u_first] == c0) ? u_first : u_first - 1;
    const uint32_t nrows = u_next - r0;
    if (nrows > kWkRowCap || nrows == 0) {
        rl_keep_uncached(n, arcs, off, cols, rank, r0, u_next, c0, c1, kept, rowlen, err);
        return;
    }
    for (uint32_t i = lane; i <= nrows; i += 32) {
        const uint64_t o = off[r0 + i];
        s_rel[w][i] = o <= c0 ? 0u : (o - c0 >= len ? len : (uint32_t)(o - c0));
        if (i < nrows) s_key[w][i] = rank[r0 + i];
    }
    const uint64_t row0_start = off[r0];
    const uint32_t p0 = 16u * lane;
    uint32_t v[16], kv[16];
    if (vec4 && p0 + 16 <= len) {
        const uint4 *src = reinterpret_cast<const uint4 *>(cols + c0 + p0);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint4 x = __ldg(src + q);
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = p0 + j < len ? cols[c0 + p0 + j] : 0u;
    }
#pragma unroll
    for (int j = 0; j < 16; j++) kv[j] = (p0 + j < len && v[j] < n) ? __ldg(rank + v[j]) : 0u;
    __syncwarp();
    // the row of this lane's first arc: the last i with s_rel[i] <= p0
    uint32_t ri0 = 0;
    if (p0 < len) {
        uint32_t lo = 0, hi = nrows - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (s_rel[w][mid] <= p0) lo = mid;
            else hi = mid - 1;
        }
        ri0 = lo;
    }
    uint32_t keep = 0;
    if (p0 < len) {
        uint32_t ri = ri0, re = s_rel[w][ri + 1], ku = s_key[w][ri];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const uint32_t p = p0 + j;
            if (p < len) {
                while (re <= p && ri + 1 < nrows) {
                    re = s_rel[w][++ri + 1];
                    ku = s_key[w][ri];
                }
                if (v[j] >= n) set_error(err, kDevBadInput);
                else if (kv[j] > ku) keep |= 1u << j;
            }
        }
    }
    const uint32_t cnt = __popc(keep);
    const uint32_t incl = warp_incl_scan(cnt);
    s_excl[w][lane] = incl - cnt;
    if (lane == 31) s_excl[w][32] = incl;
    s_keep[w][lane] = (uint16_t)keep;
    __syncwarp();
    // P(x): kept arcs of the chunk before position x
    auto P = [&](uint32_t x) -> uint32_t {
        const uint32_t q = x >> 4, b = x & 15;
        return q >= 32 ? s_excl[w][32] : s_excl[w][q] + __popc((uint32_t)s_keep[w][q] & ((1u << b) - 1u));
    };
    for (uint32_t i = lane; i < nrows; i += 32) {
        const uint32_t f = s_rel[w][i], e = s_rel[w][i + 1];
        int32_t place = INT32_MIN;
        const uint32_t pf = P(f), k = e > f ? P(e) - pf : 0u;
        if (k) {
            const uint32_t key = s_key[w][i];
            uint64_t rowlen_true = e - f;
            if (i == 0 || i == nrows - 1) {  // the first and the last row may extend beyond the chunk
                const uint64_t b = off[r0 + i], t = off[r0 + i + 1];
                rowlen_true = (b <= t && t <= arcs) ? t - b : 0;
            }
            if (key < n) {
                const uint32_t base = atomicAdd(&rowlen[key], k);
                // a row cannot keep more arcs than it has (else the rank is not a permutation)
                if ((uint64_t)base + k <= rowlen_true && base < 0x40000000u) place = (int32_t)base - (int32_t)pf;
                else set_error(err, kDevBadInput);
            } else {
                set_error(err, kDevBadInput);
            }
        }
        s_place[w][i] = place;
    }
    __syncwarp();
    if (keep) {
        uint32_t ri = ri0, re = s_rel[w][ri + 1];
        uint32_t q = s_excl[w][lane];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const uint32_t p = p0 + j;
            if (p < len) {
                while (re <= p && ri + 1 < nrows) re = s_rel[w][++ri + 1];
                if ((keep >> j) & 1) {
                    const int32_t place = s_place[w][ri];
                    if (place != INT32_MIN) {
                        const uint64_t rs = ri == 0 ? row0_start : c0 + s_rel[w][ri];
                        kept[rs + (uint64_t)(int64_t)((int64_t)place + q)] = kv[j];
                    }
                    q++;
                }
            }
        }
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

// Sorts a row of up to MAXLEN (256 or 1024) values with one warp; false when it is longer (left
// to the next path).
template <uint32_t MAXLEN>
__device__ __forceinline__ bool warp_sort_upto(const uint32_t *src, uint32_t len, uint32_t *dst, int lane)
{
    if (len <= 32) { warp_sort_row<1>(src, len, dst, lane); return true; }
    if (len <= 64) { warp_sort_row<2>(src, len, dst, lane); return true; }
    if (len <= 128) { warp_sort_row<4>(src, len, dst, lane); return true; }
    if (len <= 256) { warp_sort_row<8>(src, len, dst, lane); return true; }
    if constexpr (MAXLEN >= 512) {
        if (len <= 512) { warp_sort_row<16>(src, len, dst, lane); return true; }
    }
    if constexpr (MAXLEN >= 1024) {
        if (len <= 1024) { warp_sort_row<32>(src, len, dst, lane); return true; }
    }
    return false;
}

constexpr int kFiWarps = 8;
constexpr int kFmWarps = 4;
constexpr int kFmMidBlocks = 8;  // blocks of kFmWarps warps per SM for rows of 33..256 entries
constexpr uint32_t kLongCap = 32768;  // longest relabelled row this build sorts (power of 2)

// Ascending bitonic sorting network over N registers (N a power of two): every index is known at
// compile time, so the values never leave the registers.
template <int N>
__device__ __forceinline__ void net_sort(uint32_t (&v)[N])
{
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; i++) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t a = v[i], b = v[l];
                    const bool up = (i & k) == 0;
                    v[i] = up ? min(a, b) : max(a, b);
                    v[l] = up ? max(a, b) : min(a, b);
                }
            }
        }
    }
}

// Loads a row of len <= N values (padded with the maximum), sorts it in the thread's registers and
// stores it.
template <int N>
__device__ __forceinline__ void thread_sort_row(const uint32_t *__restrict__ src, uint32_t len,
                                                uint32_t *__restrict__ dst)
{
    uint32_t v[N];
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = (uint32_t)i < len ? src[i] : 0xffffffffu;
    net_sort<N>(v);
#pragma unroll
    for (int i = 0; i < N; i++)
        if ((uint32_t)i < len) dst[i] = v[i];
}

// Rows in rank order, one row per lane: the 32 lanes of a warp take 32 consecutive ranks, whose
// out-degrees are alike (ranks follow the degree), so the lanes' work is alike.  A row of at most
// 32 entries is sorted by its lane alone, in registers (a sorting network of 4, 8, 16 or 32
// values).  Longer rows are listed (rows[0 .. *n_mid)) for k_rl_fill_mid: in a degree order they
// sit at the top ranks, and sorting them here would leave those few warps with most of the work.
__global__ __launch_bounds__(kFiWarps * 32) void k_rl_fill(
    uint32_t n, uint64_t arcs, const uint64_t *__restrict__ off, const uint32_t *__restrict__ perm,
    const uint32_t *__restrict__ kept, const uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, uint64_t dag_cap, uint32_t *mid_rows, uint32_t *n_mid,
    uint32_t *err)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (*(volatile uint32_t *)err) return;  // an earlier pass failed: its offsets are not trusted
    const uint64_t stride = (uint64_t)gridDim.x * kFiWarps * 32;
    for (uint64_t r0 = ((uint64_t)blockIdx.x * kFiWarps + w) * 32; r0 < n; r0 += stride) {
        const uint64_t r = r0 + lane;
        uint32_t len = 0;
        uint64_t src = 0, dst = 0;
        if (r < n) {
            const uint32_t u = perm[r];
            dst = dag_off[r];
            const uint64_t l64 = dag_off[r + 1] - dst;
            bool ok = u < n;
            if (ok) {
                src = off[u];
                const uint64_t e = off[u + 1];
                ok = src <= e && e <= arcs && l64 <= e - src && dst + l64 <= dag_cap && dst <= dst + l64;
            }
            if (ok) len = (uint32_t)l64;
            else set_error(err, kDevBadInput);
        }
        const uint32_t *in = kept + src;
        uint32_t *out = dag_cols + dst;
        if (len == 1) out[0] = in[0];
        else if (len >= 2 && len <= 4) thread_sort_row<4>(in, len, out);
        else if (len >= 5 && len <= 8) thread_sort_row<8>(in, len, out);
        else if (len >= 9 && len <= 16) thread_sort_row<16>(in, len, out);
        else if (len >= 17 && len <= 32) thread_sort_row<32>(in, len, out);
        const uint32_t longer = __ballot_sync(kFull, len > 32);
        if (longer) {
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(n_mid, (uint32_t)__popc(longer));
            at = __shfl_sync(kFull, at, 0);
            if (len > 32) mid_rows[at + __popc(longer & lanemask_lt())] = (uint32_t)r;
        }
    }
}

// Listed rows, one per warp, in the order the warps claim them (one atomic per row; a row's sort
// costs far more).  Two instances: rows of 33..256 entries (8 registers of values per lane, so
// that 32 warps fit an SM), then rows of 257..1024 (32 per lane, 128 registers); each lists the
// rows it cannot take for the next (k_rl_fill_long above 1024).
template <uint32_t MAXLEN, int MINB>
__global__ __launch_bounds__(kFmWarps * 32, MINB) void k_rl_fill_mid(
    const uint32_t *__restrict__ perm, const uint32_t *__restrict__ kept,
    const uint64_t *__restrict__ off, const uint64_t *__restrict__ dag_off,
    uint32_t *__restrict__ dag_cols, const uint32_t *in_rows, const uint32_t *n_in, uint32_t *cursor,
    uint32_t *out_rows, uint32_t *n_out, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    if (*(volatile uint32_t *)err) return;
    const uint32_t total = *n_in;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(cursor, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= total) break;
        const uint32_t r = in_rows[it];
        // listed by k_rl_fill after its bounds checks: r < n, perm[r] < n, the row fits
        const uint64_t src = off[perm[r]], dst = dag_off[r];
        const uint32_t len = (uint32_t)(dag_off[r + 1] - dst);
        if (!warp_sort_upto<MAXLEN>(kept + src, len, dag_cols + dst, lane) && lane == 0)
            out_rows[atomicAdd(n_out, 1u)] = r;
    }
}

// One block per listed row above 1024 entries; dynamic shared memory holds the padded row.
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
    s.take<uint32_t>((arcs + kWkArcs - 1) / kWkArcs + 2);  // first_row
    s.take<uint32_t>(8);                                    // tickets, counters
    s.take<uint32_t>((size_t)n + 1);                        // rowlen (rank order)
    s.take<uint32_t>((size_t)n + 1);                        // perm
    s.take<unsigned long long>((size_t)n / kScTile + 2);    // look-back status (scan)
    s.take<uint32_t>((size_t)n + 1);                        // rows above 32 entries
    s.take<uint32_t>((size_t)n + 1);                        // rows above 256 entries
    s.take<uint32_t>((size_t)n + 1);                        // rows above 1024 entries
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
    const uint64_t ntiles64 = (arcs + kWkArcs - 1) / kWkArcs;
    uint32_t *first_row = c.take<uint32_t>(ntiles64 + 2);
    uint32_t *ctr = c.take<uint32_t>(8);
    uint32_t *rowlen = c.take<uint32_t>((size_t)n + 1);
    uint32_t *perm = c.take<uint32_t>((size_t)n + 1);
    const uint32_t sc_tiles = (n + kScTile - 1) / kScTile;
    unsigned long long *sc_status = c.take<unsigned long long>((size_t)n / kScTile + 2);
    uint32_t *mid_rows = c.take<uint32_t>((size_t)n + 1);
    uint32_t *big_rows = c.take<uint32_t>((size_t)n + 1);
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
    uint32_t *ticket = ctr, *max_len = ctr + 2, *n_long = ctr + 3, *n_mid = ctr + 4, *cursor = ctr + 5,
             *n_big = ctr + 6, *cursor_big = ctr + 7;
    if ((e = launch_tile_rows(n, arcs, off, kWkArcs, ntiles, first_row, st))) return e;
    k_rl_prologue<<<(n + 255) / 256, 256, 0, st>>>(n, rank, rowlen, perm, err);
    k_rl_keep<<<(ntiles + kWkWarps - 1) / kWkWarps, kWkWarps * 32, 0, st>>>(n, arcs, off, cols, rank, first_row,
                                                                         ntiles, kept, rowlen, err, vec4);
    k_scan_rowlen<<<sc_tiles, kScThreads, 0, st>>>(n, rowlen, dag_off, sc_tiles, sc_status, ticket,
                                                   max_len, err, wait_cfg());
    uint32_t grid = (uint32_t)(((uint64_t)n + kFiWarps * 32 - 1) / (kFiWarps * 32));
    if (grid > (uint32_t)num_sms * 8) grid = (uint32_t)num_sms * 8;
    k_rl_fill<<<grid, kFiWarps * 32, 0, st>>>(n, arcs, off, perm, kept, dag_off, dag_cols, arcs / 2,
                                              mid_rows, n_mid, err);
    k_rl_fill_mid<256, kFmMidBlocks><<<(uint32_t)num_sms * kFmMidBlocks, kFmWarps * 32, 0, st>>>(
        perm, kept, off, dag_off, dag_cols, mid_rows, n_mid, cursor, big_rows, n_big, err);
    k_rl_fill_mid<1024, 4><<<(uint32_t)num_sms * 4, kFmWarps * 32, 0, st>>>(
        perm, kept, off, dag_off, dag_cols, big_rows, n_big, cursor_big, long_rows, n_long, err);
    const uint32_t cap_bytes = kLongCap * sizeof(uint32_t);
    if ((e = cudaFuncSetAttribute(k_rl_fill_long, cudaFuncAttributeMaxDynamicSharedMemorySize, cap_bytes)))
        return e;
    k_rl_fill_long<<<(uint32_t)num_sms, 1024, cap_bytes, st>>>(n, arcs, off, perm, kept, dag_off, dag_cols,
                                                               arcs / 2, long_rows, n_long, kLongCap, err);
    note_launches(7);
    if (d_max_outdeg)
        if ((e = cudaMemcpyAsync(d_max_outdeg, max_len, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)))
            return e;
    return cudaGetLastError();
}

}  // namespace citron_host
