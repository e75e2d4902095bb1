// list.cu -- k-clique listing: the counting recursion (Algorithm Counting, Sec. III, over CITRON's
// subgraphs, Sec. V-B) walked down to its last level so that every clique is written out once
// instead of counted (the extension Sec. VIII describes).
//
// A k-clique is written as k ids in recursion order: its first vertex u in the DAG order, the
// out-neighbour a of the edge task (u, a), then the vertices chosen level by level, which follow
// the DAG's row order (ascending ids of a DAG with sorted rows).  With d_map the ids are mapped
// through it (the inverse rank of a relabelled DAG gives input vertex ids).
//
// One block per root (roots taken from a counter), as in the counting phase's bitmap path: the
// block loads N+(u), builds the local subgraph as D bitmap rows of D bits in shared memory
// (row i = N+(u) ∩ N+(a_i) by binary search), and its warps take the root's edge tasks.  A warp
// holds a candidate set one 32-bit word per lane and walks its members warp-uniformly; at the last
// level it compacts the members into a list, reserves their rows in the output with one atomic,
// and writes the rows as consecutive words so that every store of the warp is coalesced.  The
// output is the bound: k * 4 bytes per clique.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace citron {

constexpr int kLsWarps = 16;
constexpr int kMaxListK = CITRON_MAX_K;
constexpr uint32_t kLsCap = 1024;  // largest out-degree the listing path holds in shared memory
constexpr uint32_t kStage3Rows = 96;  // k = 3: triangles staged per warp before one flush

struct ListCtx {
    const uint32_t *sL;     // N+(u), DAG ids
    const uint32_t *rows;   // D x RS bitmap
    uint32_t RS, W;
    uint16_t *elem;         // the warp's member list (last level)
    uint32_t *prefix;       // the warp's chosen vertices (output ids)
    const uint32_t *map;
    uint32_t *out;
    unsigned long long *cursor;
    unsigned long long capacity;
};

__device__ __forceinline__ uint32_t out_id(const uint32_t *map, uint32_t v)
{
    return map ? map[v] : v;
}

// Write every member of the warp's candidate set as the last vertex of a K-clique.
template <int K>
__device__ __forceinline__ void emit(const ListCtx &x, uint32_t c, int lane)
{
    const uint32_t cnt = __popc(c);
    const uint32_t incl = warp_incl_scan(cnt);
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    uint32_t pos = incl - cnt;
    for (uint32_t b = c; b; b &= b - 1) x.elem[pos++] = (uint16_t)(lane * 32 + __ffs(b) - 1);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(x.cursor, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 0);
    __syncwarp();
    if (base >= x.capacity) return;
    unsigned long long rows = total;
    if (rows > x.capacity - base) rows = x.capacity - base;
    uint32_t *dst = x.out + base * K;
    const uint32_t words = (uint32_t)rows * K;
    for (uint32_t g = lane; g < words; g += 32) {
        const uint32_t r = g / K, col = g - r * K;
        dst[g] = col < K - 1 ? x.prefix[col] : out_id(x.map, x.sL[x.elem[r]]);
    }
    __syncwarp();
}

// Walk the R-cliques of candidate set c (lane word), R >= 1; x.prefix holds K - R vertices.
// Members are taken in index order; each one's next set is c ∩ row (the whole set c: in a DAG
// that keeps vertex ids a row can hold lower indices).
template <int K, int R>
__device__ void walk(const ListCtx &x, uint32_t c, int lane)
{
    if constexpr (R == 1) {
        emit<K>(x, c, lane);
    } else {
        uint32_t rem = c;
        for (;;) {
            const uint32_t have = __ballot_sync(kFull, rem != 0);
            if (!have) break;
            const int l = __ffs(have) - 1;
            const uint32_t word = __shfl_sync(kFull, rem, l);
            const uint32_t j = (uint32_t)l * 32 + __ffs(word) - 1;
            if (lane == l) rem &= rem - 1;
            const uint32_t nc = lane < (int)x.W ? (c & x.rows[j * x.RS + lane]) : 0u;
            if (__reduce_add_sync(kFull, __popc(nc)) >= (uint32_t)(R - 1)) {
                if (lane == 0) x.prefix[K - R] = out_id(x.map, x.sL[j]);
                __syncwarp();
                walk<K, R - 1>(x, nc, lane);
            }
        }
    }
}

// Writes the warp's staged triangles (3 ids each) to the output: one atomic reserves the rows,
// then the warp copies consecutive words (coalesced).
__device__ __forceinline__ void flush3(const uint32_t *stage, uint32_t slen, uint32_t *out,
                                       unsigned long long capacity, unsigned long long *cursor,
                                       int lane)
{
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)slen);
    base = __shfl_sync(kFull, base, 0);
    if (base < capacity) {
        unsigned long long rows = slen;
        if (rows > capacity - base) rows = capacity - base;
        uint32_t *dst = out + base * 3;
        for (uint32_t g = lane; g < (uint32_t)rows * 3; g += 32) dst[g] = stage[g];
    }
    __syncwarp();
}

template <int K>
__global__ __launch_bounds__(kLsWarps * 32) void k_list(
    uint32_t n, const uint64_t *__restrict__ dag_off, const uint32_t *__restrict__ dag_cols,
    const uint32_t *__restrict__ map, uint32_t dcap, uint32_t *next, uint32_t *out,
    unsigned long long capacity, unsigned long long *cursor, uint32_t *err)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t rs_cap = (dcap / 32) | 1;
    uint32_t *sL = smem;
    uint32_t *rows = smem + dcap;
    uint32_t *wsc = rows + (size_t)dcap * rs_cap;
    __shared__ uint32_t s_u, s_task;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    ListCtx x;
    x.sL = sL;
    x.rows = rows;
    x.elem = reinterpret_cast<uint16_t *>(wsc + (size_t)w * (dcap / 2 + 1 + kMaxListK));
    x.prefix = wsc + (size_t)w * (dcap / 2 + 1 + kMaxListK) + dcap / 2 + 1;
    x.map = map;
    x.out = out;
    x.cursor = cursor;
    x.capacity = capacity;
    uint32_t *stage = rows + (size_t)w * kStage3Rows * 3;  // k = 3 only (no bitmap rows then)
    uint32_t slen = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            s_u = atomicAdd(next, 1u);
            s_task = 0;
        }
        __syncthreads();
        const uint32_t u = s_u;
        if (u >= n) break;
        const uint64_t base = dag_off[u];
        const uint64_t d64 = dag_off[u + 1] - base;
        if (d64 > dcap) {
            if (threadIdx.x == 0) set_error(err, kDevScratch);
            __syncthreads();
            continue;
        }
        const uint32_t D = (uint32_t)d64;
        if (D < K - 1) {
            __syncthreads();
            continue;
        }
        const uint32_t W = (D + 31) >> 5, RS = W | 1;
        for (uint32_t i = threadIdx.x; i < D; i += blockDim.x) sL[i] = dag_cols[base + i];
        if (K > 3)
            for (uint32_t i = threadIdx.x; i < D * RS; i += blockDim.x) rows[i] = 0;
        __syncthreads();
        const uint32_t lmax = sL[D - 1];
        const uint32_t mu = out_id(map, u);
        for (uint32_t i = w; i < D; i += nw) {  // row i = N+(u) ∩ N+(a_i)
            const uint32_t a = sL[i];
            if (a >= n) {
                if (lane == 0) set_error(err, kDevBadInput);
                continue;
            }
            const uint32_t ma = K == 3 ? out_id(map, a) : 0u;
            const uint64_t b = dag_off[a], e = dag_off[a + 1];
            for (uint64_t p = b; p < e; p += 32) {
                const uint32_t y = p + lane < e ? dag_cols[p + lane] : 0xffffffffu;
                if (__shfl_sync(kFull, y, 0) > lmax) break;
                bool hit = false;
                uint32_t lo = 0;
                if (y <= lmax) {
                    uint32_t len = D;
                    while (len > 0) {
                        const uint32_t half = len >> 1;
                        if (sL[lo + half] < y) {
                            lo += half + 1;
                            len -= half + 1;
                        } else {
                            len = half;
                        }
                    }
                    hit = lo < D && sL[lo] == y;
                }
                if constexpr (K == 3) {
                    // the triangle (u, a_i, y) goes straight to the warp's stage
                    const uint32_t mask = __ballot_sync(kFull, hit);
                    if (hit) {
                        uint32_t *row = stage + 3 * (slen + __popc(mask & lanemask_lt()));
                        row[0] = mu;
                        row[1] = ma;
                        row[2] = out_id(map, y);
                    }
                    slen += __popc(mask);
                    if (slen > kStage3Rows - 32) {
                        flush3(stage, slen, out, capacity, cursor, lane);
                        slen = 0;
                    }
                } else if (hit) {
                    atomicOr(&rows[i * RS + (lo >> 5)], 1u << (lo & 31));
                }
            }
        }
        __syncthreads();
        if constexpr (K == 3) continue;
        x.RS = RS;
        x.W = W;
        for (;;) {  // edge tasks (u, a_t)
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(&s_task, 1u);
            t = __shfl_sync(kFull, t, 0);
            if (t >= D) break;
            const uint32_t c = lane < (int)W ? rows[t * RS + lane] : 0u;
            if (__reduce_add_sync(kFull, __popc(c)) < (uint32_t)(K - 2)) continue;
            if (lane == 0) {
                x.prefix[0] = out_id(map, u);
                x.prefix[1] = out_id(map, sL[t]);
            }
            __syncwarp();
            walk<K, K - 2>(x, c, lane);
        }
        __syncthreads();
    }
    if constexpr (K == 3)
        if (slen) flush3(stage, slen, out, capacity, cursor, lane);
}

// k = 1: every vertex; k = 2: every arc (row vertex, column).
__global__ void k_list_trivial(uint32_t n, uint32_t k, const uint64_t *__restrict__ dag_off,
                               const uint32_t *__restrict__ dag_cols, const uint32_t *__restrict__ map,
                               uint32_t *out, unsigned long long capacity)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t u = gw; u < n; u += nwarps) {
        if (k == 1) {
            if (lane == 0 && u < capacity) out[u] = out_id(map, u);
            continue;
        }
        const uint32_t mu = out_id(map, u);
        for (uint64_t e = dag_off[u] + lane; e < dag_off[u + 1]; e += 32) {
            if (e >= capacity) break;
            out[2 * e] = mu;
            out[2 * e + 1] = out_id(map, dag_cols[e]);
        }
    }
}

__global__ void k_list_maxdeg(uint32_t n, const uint64_t *off, uint32_t *out)
{
    uint32_t best = 0;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        best = max(best, (uint32_t)min(off[u + 1] - off[u], (uint64_t)0xffffffffull));
    best = __reduce_max_sync(kFull, best);
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

}  // namespace citron

namespace citron_host {

using namespace citron;

size_t list_ws_bytes()
{
    Sizer s;
    s.take<uint32_t>(8);
    s.take<unsigned long long>(1);
    return s.used;
}

static size_t list_smem(uint32_t dcap, uint32_t k)
{
    const uint32_t rs_cap = (dcap / 32) | 1;
    size_t rows = (size_t)dcap * rs_cap;
    const size_t stages = (size_t)kLsWarps * kStage3Rows * 3;
    if (k == 3 && rows < stages) rows = stages;
    return sizeof(uint32_t) * ((size_t)dcap + rows + (size_t)kLsWarps * (dcap / 2 + 1 + kMaxListK));
}

template <int K>
static cudaError_t launch_list_k(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_cols,
                                 const uint32_t *map, uint32_t dcap, uint32_t *next, uint32_t *out,
                                 unsigned long long capacity, unsigned long long *cursor,
                                 uint32_t *err, cudaStream_t st, int num_sms)
{
    const size_t smem = list_smem(dcap, K);
    // a fixed upper bound (the device's largest), so that concurrent callers cannot undercut it
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!e && (size_t)(optin - 1024) < smem) e = cudaErrorInvalidValue;
    if (!e) e = cudaFuncSetAttribute(k_list<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
    int per_sm = 0;
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_list<K>, kLsWarps * 32, smem);
    if (e) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    k_list<K><<<num_sms * per_sm, kLsWarps * 32, smem, st>>>(n, dag_off, dag_cols, map, dcap, next,
                                                              out, capacity, cursor, err);
    note_launches(1);
    return cudaGetLastError();
}

// Synchronous: returns the number of k-cliques in *h_total; writes min(total, capacity) rows.
cudaError_t run_list(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_cols, uint32_t k,
                     const uint32_t *map, uint32_t *out, unsigned long long capacity,
                     unsigned long long *h_total, bool *too_wide, uint32_t *err, Carver &c,
                     cudaStream_t st, int num_sms)
{
    uint32_t *scal = c.take<uint32_t>(8);
    unsigned long long *cursor = c.take<unsigned long long>(1);
    if (!c.ok) return cudaErrorMemoryAllocation;
    *h_total = 0;
    *too_wide = false;
    if (n == 0) return cudaSuccess;
    cudaError_t e;
    if (k <= 2) {
        unsigned long long total = n;
        if (k == 2) {
            uint64_t m = 0;
            if ((e = cudaMemcpyAsync(&m, dag_off + n, sizeof(m), cudaMemcpyDeviceToHost, st))) return e;
            if ((e = cudaStreamSynchronize(st))) return e;
            total = m;
        }
        if (capacity && out) {
            k_list_trivial<<<num_sms * 8, 256, 0, st>>>(n, k, dag_off, dag_cols, map, out, capacity);
            note_launches(1);
            if ((e = cudaGetLastError())) return e;
        }
        *h_total = total;
        return cudaStreamSynchronize(st);
    }
    if ((e = cudaMemsetAsync(scal, 0, 8 * sizeof(uint32_t), st))) return e;
    if ((e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st))) return e;
    k_list_maxdeg<<<num_sms * 4, 256, 0, st>>>(n, dag_off, scal + 1);
    note_launches(1);
    uint32_t dmax = 0;
    if ((e = cudaMemcpyAsync(&dmax, scal + 1, sizeof(dmax), cudaMemcpyDeviceToHost, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    if (dmax > kLsCap) {
        *too_wide = true;
        return cudaSuccess;
    }
    if (dmax + 1 < k) return cudaSuccess;  // no k-clique can exist
    const uint32_t dcap = (dmax + 31) & ~31u;
    switch (k) {
#define CITRON_LIST_CASE(KK)                                                                     \
    case KK:                                                                                     \
        e = launch_list_k<KK>(n, dag_off, dag_cols, map, dcap, scal, out, capacity, cursor, err, \
                              st, num_sms);                                                      \
        break;
        CITRON_LIST_CASE(3)
        CITRON_LIST_CASE(4)
        CITRON_LIST_CASE(5)
        CITRON_LIST_CASE(6)
        CITRON_LIST_CASE(7)
        CITRON_LIST_CASE(8)
        CITRON_LIST_CASE(9)
        CITRON_LIST_CASE(10)
        CITRON_LIST_CASE(11)
        CITRON_LIST_CASE(12)
#undef CITRON_LIST_CASE
        default: return cudaErrorInvalidValue;
    }
    if (e) return e;
    if ((e = cudaMemcpyAsync(h_total, cursor, sizeof(*h_total), cudaMemcpyDeviceToHost, st))) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace citron_host
