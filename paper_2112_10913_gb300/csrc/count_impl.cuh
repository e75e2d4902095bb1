// count_impl.cuh -- device templates of the counting phase (included by count.cu and by the
// per-k translation units count_k*.cu, which instantiate them in parallel builds).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace citron {


constexpr int kMaxK = CITRON_MAX_K;
constexpr uint32_t kBitmapCap = 1024;  // largest root handled by the bitmap path
constexpr int kSmallWarps = 8;         // warps per block of k_count_small
constexpr int kListWarps = 4;          // warps per block of k_count_list

struct CountStats {
    uint32_t n_small, n_mid, n_big;
    uint32_t max_mid, max_big, max_all;
    uint32_t pad[2];
};

// ------------------------------------------------------------------------------------------
// Warp-register path (D <= 32).

// Number of R-cliques inside the warp-uniform candidate mask `cand` (bit j = j-th out-neighbour
// of the root); lane i holds row i of the local subgraph.  Adds lane-partial sums to acc.
template <int R>
__device__ __forceinline__ void small_dfs(uint32_t cand, uint32_t myrow, int lane,
                                          unsigned long long &acc)
{
    if constexpr (R == 1) {
        if (lane == 0) acc += __popc(cand);
    } else if constexpr (R == 2) {
        if ((cand >> lane) & 1) acc += __popc(cand & myrow);
    } else {
        uint32_t c = cand;
        while (c) {
            const int a = __ffs(c) - 1;
            c &= c - 1;
            const uint32_t c2 = cand & __shfl_sync(kFull, myrow, a);
            if (__popc(c2) >= R - 1) small_dfs<R - 1>(c2, myrow, lane, acc);
        }
    }
}

__device__ __forceinline__ uint32_t lower_bound_smem(const uint32_t *a, uint32_t n, uint32_t x)
{
    uint32_t lo = 0, len = n;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if (a[lo + half] < x) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

template <int K>
__global__ __launch_bounds__(kSmallWarps * 32) void k_count_small(
    const uint64_t *__restrict__ dag_off, const uint32_t *__restrict__ dag_cols,
    const uint32_t *__restrict__ list, const CountStats *st, unsigned long long *result,
    RootSink sink, Budget budget, uint32_t *err)
{
    __shared__ uint32_t sL[kSmallWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nlist = st->n_small;
    const uint32_t gw = blockIdx.x * kSmallWarps + w, nwarps = gridDim.x * kSmallWarps;
    unsigned long long total = 0;
    for (uint32_t idx = gw; idx < nlist; idx += nwarps) {
        int stop = 0;
        if (lane == 0) stop = budget.over(err);
        if (__shfl_sync(kFull, stop, 0)) break;
        const uint32_t u = list[idx];
        const uint64_t base = dag_off[u];
        const uint32_t D = (uint32_t)(dag_off[u + 1] - base);
        const uint32_t x = lane < D ? dag_cols[base + lane] : 0xffffffffu;
        sL[w][lane] = x;
        __syncwarp();
        const uint32_t lmax = __shfl_sync(kFull, x, D - 1);
        uint64_t rb = 0, re = 0;
        if (lane < D) {
            rb = dag_off[x];
            re = dag_off[x + 1];
        }
        uint32_t myrow = 0;
        for (uint32_t i = 0; i < D; i++) {
            const uint64_t b = __shfl_sync(kFull, rb, i), e = __shfl_sync(kFull, re, i);
            uint32_t bits = 0;
            for (uint64_t p = b; p < e; p += 32) {
                const uint32_t y = p + lane < e ? dag_cols[p + lane] : 0xffffffffu;
                if (__shfl_sync(kFull, y, 0) > lmax) break;
                if (y <= lmax) {
                    const uint32_t j = lower_bound_smem(sL[w], D, y);
                    if (sL[w][j] == y) bits |= 1u << j;
                }
            }
            bits = __reduce_or_sync(kFull, bits);
            if (lane == i) myrow = bits;
        }
        unsigned long long acc = 0;
        const uint32_t all = D == 32 ? kFull : ((1u << D) - 1);
        if (sink.per_arc) {
            // debug output: the root's edge tasks one at a time, each (K-2)-clique count of
            // N+(u) ∩ N+(a) stored for its arc
            for (uint32_t a = 0; a < D; a++) {
                const uint32_t c2 = all & __shfl_sync(kFull, myrow, a);
                unsigned long long t = 0;
                if (__popc(c2) >= K - 2) small_dfs<K - 2>(c2, myrow, lane, t);
                const unsigned long long tt = warp_sum_u64(t, err);
                if (lane == 0) sink.per_arc[base + a] = tt;
                acc += t;
            }
        } else {
            small_dfs<K - 1>(all, myrow, lane, acc);
        }
        if (sink.wants_root_total()) {
            const unsigned long long r = warp_sum_u64(acc, err);
            if (lane == 0) sink.put(u, r, err);
        }
        total += acc;
        __syncwarp();
    }
    total = warp_sum_u64(total, err);
    if (lane == 0) add_checked(result, total, err);
}

// ------------------------------------------------------------------------------------------
// Shared-memory bitmap path (small_max < D <= 1024).

// Per-warp view of the block's local subgraph and the warp's private scratch.
//   rows : D x RS words, row i = bits j with L[j] in N+(L[i]) (RS odd: column reads by
//          different rows fall in different banks)
//   tri  : every row only has bits above its own index (true for a DAG relabelled to ranks, whose
//          rows are sorted in the DAG order); lets the loops skip the words below an element.
//   elem : the current candidate set as a list of indices (compaction buffer)
//   cbuf : the current candidate set's words
//   lbuf : one candidate set per lane, word-major ([w * 32 + lane]), so that lanes reading
//          their own word w always hit 32 different banks

struct WarpCtx {
    const uint32_t *rows;
    uint32_t RS, W;
    bool tri;
    uint16_t *elem;
    uint32_t *cbuf;
    uint32_t *lbuf;
    uint32_t *mv;    // compress masks: 5 per candidate word, then the member prefix per word
    uint32_t *mbuf;  // compact rows, 4 words each (16-byte aligned); aliases lbuf
    uint32_t compact_max;  // largest candidate set re-encoded compactly (0 or 128)
    uint32_t compact3_max; // same for the R = 3 level, which also takes packed 5- and 6-word rows
    uint32_t pair_cap;     // uint16 entries of elem
};

// Carry-save accumulation of bit counts (a full adder per bit position): the bits of
// ones + a + b are kept as a new `ones` word and a carry word of weight two (two LOP3s), so that
// one POPC counts two words.  POPC and the bit scans share the narrow XU pipe, which bounds the
// leaves; the LOP3s go to the wider ALU pipe.  The running total is s + popc(ones): every user
// adds popc(ones) once at the end.
__device__ __forceinline__ void csa_add(uint32_t &ones, uint32_t a, uint32_t b, uint32_t &s)
{
    const uint32_t u = ones ^ a;
    const uint32_t carry = (ones & a) | (u & b);
    ones = u ^ b;
    s += 2u * (uint32_t)__popc(carry);
}

// Number of DAG arcs inside the lane's own candidate set lb (words [lo, hi)): the penultimate
// level of Counting, which only adds subgraph degrees.  WORK adds the 32-bit word operations
// (AND + POPC) performed to `work`.
template <bool WORK>
__device__ __forceinline__ uint32_t lane_arcs(const WarpCtx &x, const uint32_t *lb, int lo, int hi,
                                              unsigned long long &work)
{
    uint32_t s = 0, ones = 0;
    for (int w = lo; w < hi; w++) {
        uint32_t y = lb[w * 32];
        if (WORK) work += (unsigned long long)__popc(y) * (uint32_t)(hi - (x.tri ? w : lo));
        // two members per step (the highest and the lowest bit): independent scans and loads
        while (y & (y - 1u)) {
            const uint32_t b1 = 31u - __clz(y);
            const uint32_t lbit = y & (0u - y);
            const uint32_t b2 = 31u - __clz(lbit);
            y ^= (1u << b1) | lbit;
            const uint32_t *r1 = x.rows + ((uint32_t)(w << 5) + b1) * x.RS;
            const uint32_t *r2 = x.rows + ((uint32_t)(w << 5) + b2) * x.RS;
            for (int w2 = x.tri ? w : lo; w2 < hi; w2++) {
                const uint32_t l = lb[w2 * 32];
                csa_add(ones, l & r1[w2], l & r2[w2], s);
            }
        }
        if (y) {
            const uint32_t b = (uint32_t)(w << 5) + 31u - __clz(y);
            const uint32_t *rb = x.rows + b * x.RS;
            int w2 = x.tri ? w : lo;
            for (; w2 + 1 < hi; w2 += 2) csa_add(ones, lb[w2 * 32] & rb[w2], lb[w2 * 32 + 32] & rb[w2 + 1], s);
            if (w2 < hi) s += __popc(lb[w2 * 32] & rb[w2]);
        }
    }
    return s + __popc(ones);
}

// Writes the candidate set (lane word c) to cbuf and its member indices to elem; returns the
// member count and the range [clo, chi) of its non-zero words.
__device__ __forceinline__ uint32_t compact(const WarpCtx &x, uint32_t c, int lane, int &clo, int &chi)
{
    const uint32_t pc = __popc(c);
    const uint32_t incl = warp_incl_scan(pc);
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    uint32_t pos = incl - pc;
    if (lane < (int)x.W) x.cbuf[lane] = c;
    uint32_t y = c;
    while (y) {
        x.elem[pos++] = (uint16_t)((lane << 5) + __ffs(y) - 1);
        y &= y - 1;
    }
    const uint32_t nz = __ballot_sync(kFull, c != 0);
    clo = nz ? __ffs(nz) - 1 : 0;
    chi = nz ? 32 - __clz(nz) : 0;
    __syncwarp();
    return total;
}

// Triangular layout only (every row holds bits above its own index).  Sum over the members
// b = elem[j], j in [j0, total), that lie in the candidate words cw (broadcast-readable shared
// words) of |cw ∧ row_b|, restricted to words below hi.  Members are taken 32 at a time in
// index order; within such a round every lane loops over the same words [word(first), hi):
// rows have no bits below their own word, so the lanes whose member starts higher only add
// zeros, and the loop stays uniform (no divergence).  Consecutive members sit in different
// banks because the row stride is odd.  MASK: members outside cw contribute nothing.
template <bool MASK, bool WORK>
__device__ __forceinline__ uint32_t tri_rounds(const WarpCtx &x, const uint32_t *cw, uint32_t j0,
                                               uint32_t total, int hi, int lane,
                                               unsigned long long &work)
{
    uint32_t s = 0, ones = 0;
    const uint32_t lim = (uint32_t)hi << 5;
    for (; j0 < total; j0 += 32) {
        const uint32_t j = j0 + lane;
        const uint32_t b = j < total ? x.elem[j] : 0xffffu;
        const uint32_t first = __shfl_sync(kFull, b, 0);
        if (first >= lim) break;
        bool in = b < lim;
        if (MASK && in) in = (cw[b >> 5] >> (b & 31)) & 1;
        if (WORK && in) work += (uint32_t)(hi - (int)(b >> 5));
        const uint32_t *rb = x.rows + (in ? b : first) * x.RS;
        int w = (int)(first >> 5);
        for (; w + 1 < hi; w += 2) {
            const uint32_t r0 = in ? rb[w] : 0u, r1 = in ? rb[w + 1] : 0u;
            csa_add(ones, cw[w] & r0, cw[w + 1] & r1, s);
        }
        if (w < hi) s += __popc(cw[w] & (in ? rb[w] : 0u));
    }
    return s + __popc(ones);
}

// ---- Compact re-encoding of a small candidate set ------------------------------------------
// A candidate set with s <= 128 members (listed in elem) is re-encoded as the s x s adjacency of
// its induced sub-DAG: row i = the members j that are out-neighbours of member i, packed into
// CW = ceil(s/32) <= 4 words ("compact rows"; upper-triangular when the DAG is relabelled to its
// order).  The remaining levels of the recursion then work on at most 4 words per set instead
// of the root-wide span; a row is one 16-byte shared-memory load.  At R = 3, sets of 129..192
// members take packed rows of 5 or 6 words (below); wider sets stay on the root-wide bitmap
// (full 8-word rows for every level were measured slower on R-MAT 20).
//
// Bits are gathered word by word with the parallel-suffix "compress" of H. S. Warren, Hacker's
// Delight (2nd ed., Sec. 7-4): for a mask m the five move masks depend on m only, so they are
// computed once per candidate word (lane-parallel) and shared by every row.
__device__ __forceinline__ void compress_masks(uint32_t m, uint32_t mv[5])
{
    uint32_t mk = ~m << 1;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        uint32_t mp = mk ^ (mk << 1);
        mp ^= mp << 2;
        mp ^= mp << 4;
        mp ^= mp << 8;
        mp ^= mp << 16;
        const uint32_t v = mp & m;
        mv[i] = v;
        m = (m ^ v) | (v >> (1 << i));
        mk &= ~mp;
    }
}

__device__ __forceinline__ uint32_t compress_with(uint32_t x, uint32_t m, const uint32_t *mv)
{
    x &= m;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const uint32_t t = x & mv[i];
        x = (x ^ t) | (t >> (1 << i));
    }
    return x;
}

// o[q] |= lo, o[q + 1] |= hi for a warp-uniform q (the member prefix of a candidate word is the
// same on every lane): a uniform branch instead of a select per output word.
template <int NW>
__device__ __forceinline__ void place_piece(uint32_t (&o)[NW], uint32_t q, uint32_t lo, uint32_t hi)
{
#pragma unroll
    for (int t = 0; t < NW; t++) {
        if (q == (uint32_t)t) {
            o[t] |= lo;
            if (t + 1 < NW) o[t + 1] |= hi;
        }
    }
}

// Builds the compact rows of the s members of the candidate set (words in cbuf, members in
// elem, non-zero words [clo, chi)).  NW = 4 output words per row (one uint4) is the width in
// use; NW = 8 (two uint4 per row) is also supported.
template <int NW>
__device__ __forceinline__ void build_compact(const WarpCtx &x, uint32_t s, int clo, int chi, int lane)
{
    // per candidate word w (lane w): compress masks and the number of members before word w
    {
        const uint32_t m = (lane < chi && lane >= clo) ? x.cbuf[lane] : 0u;
        uint32_t mv[5];
        compress_masks(m, mv);
        const uint32_t pc = __popc(m);
        const uint32_t pre = warp_incl_scan(pc) - pc;
#pragma unroll
        for (int i = 0; i < 5; i++) x.mv[i * 32 + lane] = mv[i];
        x.mv[160 + lane] = pre;
    }
    __syncwarp();
    uint4 *out = reinterpret_cast<uint4 *>(x.mbuf);
    for (uint32_t i0 = 0; i0 < s; i0 += 32) {
        const uint32_t i = i0 + lane;
        const bool act = i < s;
        const uint32_t ei = act ? x.elem[i] : x.elem[i0];
        const uint32_t *row = x.rows + ei * x.RS;
        uint32_t o[NW];
#pragma unroll
        for (int t = 0; t < NW; t++) o[t] = 0;
        // triangular rows hold bits above their own member only: start at the word of the
        // round's first member
        for (int w = x.tri ? (int)(x.elem[i0] >> 5) : clo; w < chi; w++) {
            const uint32_t m = x.cbuf[w];
            if (!m) continue;
            uint32_t mv[5];
#pragma unroll
            for (int t = 0; t < 5; t++) mv[t] = x.mv[t * 32 + w];
            const uint32_t pre = x.mv[160 + w];
            const uint32_t piece = compress_with(row[w], m, mv);
            const uint32_t q = pre >> 5, sh = pre & 31;
            const uint32_t lo = piece << sh, hi = sh ? (piece >> (32 - sh)) : 0u;
            place_piece<NW>(o, q, lo, hi);
        }
        if (act) {
            if (NW == 4) {
                out[i] = make_uint4(o[0], o[1], o[2], o[3]);
            } else {
                out[2 * i] = make_uint4(o[0], o[1], o[2], o[3]);
                out[2 * i + 1] = make_uint4(o[4 % NW], o[5 % NW], o[6 % NW], o[7 % NW]);
            }
        }
    }
    __syncwarp();
}

// Iteration mask of a leaf set: its members except the highest one.  In the triangular layout a
// member's row has no bits at or below its own index, so the highest member of a set adds no
// arc inside it and is not visited.
template <int CW>
__device__ __forceinline__ void drop_top(uint32_t (&Y)[CW])
{
    bool done = false;
#pragma unroll
    for (int q = CW - 1; q >= 0; q--) {
        if (!done && Y[q]) {
            Y[q] &= ~(0x80000000u >> __clz(Y[q]));
            done = true;
        }
    }
}

// Packed triangular compact rows for R = 3 sets of 129..192 members (CW = 5 or 6 words): the row
// of member i holds only its words q = i/32 .. CW-1 (the words below are zero in an
// upper-triangular sub-DAG), so 192 rows take 672 words instead of 1152 and fit the warp's
// scratch.  Rows of the members of word q start at packed_base(q) and are (CW - q) words long.
template <int CW>
__host__ __device__ constexpr uint32_t packed_base(int q)
{
    return q <= 0 ? 0u : packed_base<CW>(q - 1) + 32u * (uint32_t)(CW - (q - 1));
}

__host__ __device__ constexpr uint32_t packed_words(int cw) { return 16u * (uint32_t)(cw * (cw + 1)); }

template <int CW>
__device__ __forceinline__ void build_packed(const WarpCtx &x, uint32_t s, int clo, int chi, int lane)
{
    {
        const uint32_t m = (lane < chi && lane >= clo) ? x.cbuf[lane] : 0u;
        uint32_t mv[5];
        compress_masks(m, mv);
        const uint32_t pc = __popc(m);
        const uint32_t pre = warp_incl_scan(pc) - pc;
#pragma unroll
        for (int i = 0; i < 5; i++) x.mv[i * 32 + lane] = mv[i];
        x.mv[160 + lane] = pre;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < CW; q++) {
        const uint32_t i0 = (uint32_t)q * 32;
        if (i0 >= s) break;
        const uint32_t i = i0 + lane;
        const bool act = i < s;
        const uint32_t ei = act ? x.elem[i] : x.elem[i0];
        const uint32_t *row = x.rows + ei * x.RS;
        uint32_t o[CW];
#pragma unroll
        for (int t = 0; t < CW; t++) o[t] = 0;
        for (int w = (int)(x.elem[i0] >> 5); w < chi; w++) {
            const uint32_t m = x.cbuf[w];
            if (!m) continue;
            uint32_t mv[5];
#pragma unroll
            for (int t = 0; t < 5; t++) mv[t] = x.mv[t * 32 + w];
            const uint32_t pre = x.mv[160 + w];
            const uint32_t piece = compress_with(row[w], m, mv);
            const uint32_t qq = pre >> 5, sh = pre & 31;
            const uint32_t lo = piece << sh, hi = sh ? (piece >> (32 - sh)) : 0u;
            place_piece<CW>(o, qq, lo, hi);
        }
        if (act) {
            uint32_t *dst = x.mbuf + packed_base<CW>(q) + (uint32_t)lane * (CW - q);
#pragma unroll
            for (int t = q; t < CW; t++) dst[t - q] = o[t];
        }
    }
    __syncwarp();
}

// Arcs inside the lane's set D (CW words; zero below word Q2) on packed rows; Y = the members
// to visit (D without its highest member).
template <int CW, bool WORK, int Q2>
__device__ __forceinline__ void packed_leaf(const uint32_t *P, const uint32_t (&D)[CW],
                                            const uint32_t (&Y)[CW], uint32_t &ones, uint32_t &s,
                                            unsigned long long &work)
{
    if constexpr (Q2 < CW) {
        uint32_t y = Y[Q2];
        if (WORK) work += (unsigned long long)__popc(y) * (CW - Q2);
        // two members per step (the highest and the lowest), their words paired in the adder
        while (y & (y - 1u)) {
            const uint32_t j1 = 31u - __clz(y);
            const uint32_t lb = y & (0u - y);
            const uint32_t j2 = 31u - __clz(lb);
            y ^= (1u << j1) | lb;
            const uint32_t *r1 = P + packed_base<CW>(Q2) + j1 * (CW - Q2);
            const uint32_t *r2 = P + packed_base<CW>(Q2) + j2 * (CW - Q2);
#pragma unroll
            for (int w = Q2; w < CW; w++) csa_add(ones, D[w] & r1[w - Q2], D[w] & r2[w - Q2], s);
        }
        if (y) {
            const uint32_t *rj = P + packed_base<CW>(Q2) + (31u - __clz(y)) * (CW - Q2);
#pragma unroll
            for (int w = Q2; w + 1 < CW; w += 2) csa_add(ones, D[w] & rj[w - Q2], D[w + 1] & rj[w + 1 - Q2], s);
            if ((CW - Q2) & 1) s += __popc(D[CW - 1] & rj[CW - 1 - Q2]);
        }
        packed_leaf<CW, WORK, Q2 + 1>(P, D, Y, ones, s, work);
    }
}

// Triangles of a dense compact set of s members (members 0..s-1) on packed rows: lane l takes
// member 32q + l of each word q, forms D = C ∧ row and adds the arcs inside D.
template <int CW, bool WORK, int Q>
__device__ __forceinline__ void packed_r3(const uint32_t *P, uint32_t s_members, int lane,
                                          uint32_t &s, unsigned long long &work)
{
    if constexpr (Q < CW) {
        const uint32_t m = (uint32_t)Q * 32 + lane;
        if (m < s_members) {
            const uint32_t *rm = P + packed_base<CW>(Q) + (uint32_t)lane * (CW - Q);
            uint32_t D[CW];
#pragma unroll
            for (int w = 0; w < CW; w++) {
                const uint32_t cw = (uint32_t)w * 32 >= s_members ? 0u
                                    : (s_members >= (uint32_t)w * 32 + 32 ? kFull : ((1u << (s_members - w * 32)) - 1));
                D[w] = w < Q ? 0u : (cw & rm[w - Q]);
            }
            uint32_t Y[CW];
#pragma unroll
            for (int w = 0; w < CW; w++) Y[w] = D[w];
            drop_top<CW>(Y);
            uint32_t ones = 0, t = 0;
            packed_leaf<CW, WORK, Q>(P, D, Y, ones, t, work);
            s += t + __popc(ones);
        }
        packed_r3<CW, WORK, Q + 1>(P, s_members, lane, s, work);
    }
}

// Sum of popc(a[w] & b[w]) over words w in [FROM, CW).
template <int CW, int FROM>
__device__ __forceinline__ uint32_t popc_and(const uint32_t (&a)[CW], const uint4 &b)
{
    uint32_t s = 0;
    if (FROM <= 0) s += __popc(a[0] & b.x);
    if (CW > 1 && FROM <= 1) s += __popc(a[1] & b.y);
    if (CW > 2 && FROM <= 2) s += __popc(a[2] & b.z);
    if (CW > 3 && FROM <= 3) s += __popc(a[3] & b.w);
    return s;
}

// popc_and with carry-save pairs: words [FROM, CW) of a & b, two at a time.
template <int CW, int FROM>
__device__ __forceinline__ void popc_and_csa(const uint32_t (&a)[CW], const uint4 &b, uint32_t &ones, uint32_t &s)
{
    const uint32_t bw[4] = {b.x, b.y, b.z, b.w};
    int w = FROM;
#pragma unroll
    for (int p = 0; p < 2; p++) {
        if (w + 1 < CW) {
            csa_add(ones, a[w] & bw[w], a[w + 1] & bw[w + 1], s);
            w += 2;
        }
    }
    if (w < CW) s += __popc(a[w] & bw[w]);
}

// Two leaf members at once: words [FROM, CW) of D & b1 and of D & b2 paired in the carry-save
// adder (one POPC per word pair).
template <int CW, int FROM>
__device__ __forceinline__ void popc_and_csa2(const uint32_t (&a)[CW], const uint4 &b1, const uint4 &b2,
                                              uint32_t &ones, uint32_t &s)
{
    const uint32_t v1[4] = {b1.x, b1.y, b1.z, b1.w}, v2[4] = {b2.x, b2.y, b2.z, b2.w};
#pragma unroll
    for (int w = FROM; w < CW; w++) csa_add(ones, a[w] & v1[w], a[w] & v2[w], s);
}

// Arcs from the members y of word q2 (FROM = q2 on triangular rows, else 0) into D, on compact
// rows M: two members per step, the highest and the lowest, whose bit scans and row loads are
// independent of each other.
template <int CW, int FROM>
__device__ __forceinline__ void leaf_word(const uint4 *M, const uint32_t (&D)[CW], uint32_t y, uint32_t base,
                                          uint32_t &ones, uint32_t &s)
{
    while (y & (y - 1u)) {
        const uint32_t b1 = 31u - __clz(y);
        const uint32_t lb = y & (0u - y);
        const uint32_t b2 = 31u - __clz(lb);
        y ^= (1u << b1) | lb;
        popc_and_csa2<CW, FROM>(D, M[base + b1], M[base + b2], ones, s);
    }
    if (y) popc_and_csa<CW, FROM>(D, M[base + 31u - __clz(y)], ones, s);
}

template <int CW, bool TRI>
__device__ __forceinline__ void leaf_word_any(const uint4 *M, const uint32_t (&D)[CW], uint32_t y, int q2,
                                              uint32_t &ones, uint32_t &s)
{
    const uint32_t base = (uint32_t)q2 << 5;
    if (!TRI || q2 == 0) leaf_word<CW, 0>(M, D, y, base, ones, s);
    else if (q2 == 1) leaf_word<CW, (CW > 1 ? 1 : 0)>(M, D, y, base, ones, s);
    else if (q2 == 2) leaf_word<CW, (CW > 2 ? 2 : 0)>(M, D, y, base, ones, s);
    else leaf_word<CW, (CW > 3 ? 3 : 0)>(M, D, y, base, ones, s);
}

// Word q of the members' bits: for R = 2 and 3 lanes take the members of word q (lane l <->
// member 32q + l).  TRI: compact rows are upper-triangular, so a member's row (and any set
// derived from it) has no bits in words below the member's own word; those words are skipped
// at compile time.
template <int R, int CW, bool TRI, bool WORK, int Q>
__device__ __forceinline__ void cdfs_word(const uint4 *M, const uint32_t (&C)[CW], int lane,
                                          uint32_t &s, uint32_t &ones, unsigned long long &work)
{
    if constexpr (Q < CW) {
        if ((C[Q] >> lane) & 1) {
            const uint4 mi = M[Q * 32 + lane];
            if constexpr (R == 2) {
                s += popc_and<CW, TRI ? Q : 0>(C, mi);
                if (WORK) work += TRI ? CW - Q : CW;
            } else {
                uint32_t D[CW];
                D[0] = C[0] & mi.x;
                if (CW > 1) D[1] = C[1] & mi.y;
                if (CW > 2) D[2] = C[2] & mi.z;
                if (CW > 3) D[3] = C[3] & mi.w;
                uint32_t Y[CW];
#pragma unroll
                for (int w = 0; w < CW; w++) Y[w] = D[w];
                if (TRI) drop_top<CW>(Y);
#pragma unroll
                for (int q2 = TRI ? Q : 0; q2 < CW; q2++) {
                    uint32_t y = Y[q2];
                    if (WORK) work += (unsigned long long)__popc(y) * (TRI ? CW - q2 : CW);
                    leaf_word_any<CW, TRI>(M, D, y, q2, ones, s);
                }
            }
        }
        cdfs_word<R, CW, TRI, WORK, Q + 1>(M, C, lane, s, ones, work);
    }
}

// Triangles (R = 3) inside a compact set C whose members are scattered over its CW words (a set
// derived from a wider one, C ∧ row).  Member m_r (in index order) goes to lane r mod 32, so that
// every lane of a round holds a member (dealing by bit position would leave the lanes of the
// absent members idle); lane r forms D = C ∧ row(m_r) and adds the arcs inside D.
template <int CW, bool TRI, bool WORK>
__device__ __forceinline__ void cdfs3_dealt(const WarpCtx &x, const uint32_t (&C)[CW], int lane,
                                            unsigned long long &acc, unsigned long long &work)
{
    const uint4 *M = reinterpret_cast<const uint4 *>(x.mbuf);
    uint32_t total = 0;
#pragma unroll
    for (int q = 0; q < CW; q++) {
        if ((C[q] >> lane) & 1) x.elem[total + __popc(C[q] & lanemask_lt())] = (uint16_t)(q * 32 + lane);
        total += __popc(C[q]);
    }
    __syncwarp();
    uint32_t s = 0, ones = 0;
    for (uint32_t r0 = 0; r0 < total; r0 += 32) {
        if (r0 + lane < total) {
            const uint32_t m = x.elem[r0 + lane];
            const uint4 mi = M[m];
            uint32_t D[CW];
            D[0] = C[0] & mi.x;
            if (CW > 1) D[1] = C[1] & mi.y;
            if (CW > 2) D[2] = C[2] & mi.z;
            if (CW > 3) D[3] = C[3] & mi.w;
            uint32_t Y[CW];
#pragma unroll
            for (int w = 0; w < CW; w++) Y[w] = D[w];
            if (TRI) drop_top<CW>(Y);
#pragma unroll
            for (int q2 = 0; q2 < CW; q2++) {
                uint32_t y = Y[q2];  // zero below the member's own word when TRI
                if (WORK) work += (unsigned long long)__popc(y) * (TRI ? CW - q2 : CW);
                leaf_word_any<CW, TRI>(M, D, y, q2, ones, s);
            }
        }
    }
    acc += s + __popc(ones);
    __syncwarp();
}

// R-cliques inside the compact set C (CW words, the same on every lane); rows in mbuf.
template <int R, int CW, bool TRI, bool WORK>
__device__ __forceinline__ void cdfs(const WarpCtx &x, const uint32_t (&C)[CW], int lane,
                                     unsigned long long &acc, unsigned long long &work)
{
    const uint4 *M = reinterpret_cast<const uint4 *>(x.mbuf);
    if constexpr (R == 1) {
        if (lane == 0) {
            uint32_t t = 0;
#pragma unroll
            for (int q = 0; q < CW; q++) t += __popc(C[q]);
            acc += t;
        }
    } else if constexpr (R == 2 || R == 3) {
        uint32_t s = 0, ones = 0;
        cdfs_word<R, CW, TRI, WORK, 0>(M, C, lane, s, ones, work);
        acc += s + __popc(ones);
    } else {
        // members in order; one recursive call site per level keeps the code linear in R
        uint32_t rem[CW];
#pragma unroll
        for (int t = 0; t < CW; t++) rem[t] = C[t];
        for (;;) {
            int q = -1;
            uint32_t word = 0;
#pragma unroll
            for (int t = CW - 1; t >= 0; t--)
                if (rem[t]) {
                    q = t;
                    word = rem[t];
                }
            if (q < 0) break;
            const uint32_t i = (uint32_t)(q << 5) + __ffs(word) - 1;
#pragma unroll
            for (int t = 0; t < CW; t++)
                if (t == q) rem[t] &= rem[t] - 1;
            const uint4 mi = M[i];
            uint32_t C2[CW];
            C2[0] = C[0] & mi.x;
            if (CW > 1) C2[1] = C[1] & mi.y;
            if (CW > 2) C2[2] = C[2] & mi.z;
            if (CW > 3) C2[3] = C[3] & mi.w;
            uint32_t cnt = 0;
#pragma unroll
            for (int t = 0; t < CW; t++) cnt += __popc(C2[t]);
            if (WORK && lane == 0) work += CW;
            if (cnt >= R - 1) {
                if constexpr (R == 4) cdfs3_dealt<CW, TRI, WORK>(x, C2, lane, acc, work);
                else cdfs<R - 1, CW, TRI, WORK>(x, C2, lane, acc, work);
            }
        }
    }
}

// 4-cliques of a dense compact set of s members (upper-triangular rows M): every arc (i, j) of
// the set is a pair queued in elem (i << 8 | j), and the queue is worked 32 pairs at a time, lane
// p forming D = M[i] ∧ M[j] and adding the arcs inside D.  Dealing the members of each C ∧ M[i]
// on its own leaves the lanes above |C ∧ M[i]| idle; pairs of many i fill every lane.
template <int CW, bool WORK>
__device__ __forceinline__ void cdfs4_pairs(const WarpCtx &x, uint32_t s, uint32_t cap, int lane,
                                            unsigned long long &acc, unsigned long long &work)
{
    const uint4 *M = reinterpret_cast<const uint4 *>(x.mbuf);
    uint16_t *pairs = x.elem;
    uint32_t sum = 0, ones = 0, n = 0;
    auto drain = [&]() {
        __syncwarp();
        for (uint32_t r0 = 0; r0 < n; r0 += 32) {
            if (r0 + lane < n) {
                const uint32_t p = pairs[r0 + lane];
                const uint4 mi = M[p >> 8], mj = M[p & 255u];
                uint32_t D[CW];
                D[0] = mi.x & mj.x;
                if (CW > 1) D[1] = mi.y & mj.y;
                if (CW > 2) D[2] = mi.z & mj.z;
                if (CW > 3) D[3] = mi.w & mj.w;
                uint32_t Y[CW];
#pragma unroll
                for (int w = 0; w < CW; w++) Y[w] = D[w];
                drop_top<CW>(Y);
#pragma unroll
                for (int q2 = 0; q2 < CW; q2++) {
                    uint32_t y = Y[q2];
                    if (WORK) work += (unsigned long long)__popc(y) * (CW - q2);
                    leaf_word_any<CW, true>(M, D, y, q2, ones, sum);
                }
            }
        }
        __syncwarp();
        n = 0;
    };
    for (uint32_t i = 0; i + 3 < s; i++) {  // a 4-clique needs three members above i
        if (n + s > cap) drain();
        const uint4 mi = M[i];
        const uint32_t w4[4] = {mi.x, mi.y, mi.z, mi.w};
        if (WORK && lane == 0) work += CW;
        uint32_t cnt = 0;
#pragma unroll
        for (int q = 0; q < CW; q++) cnt += __popc(w4[q]);
        if (cnt < 3) continue;  // prune: fewer than three members above i
#pragma unroll
        for (int q = 0; q < CW; q++) {
            const uint32_t m = w4[q];
            if ((m >> lane) & 1) pairs[n + __popc(m & lanemask_lt())] = (uint16_t)((i << 8) | (uint32_t)(q * 32 + lane));
            n += __popc(m);
        }
    }
    drain();
    acc += sum + __popc(ones);
}

template <int R, int CW, bool TRI, bool WORK>
__device__ __forceinline__ void cdfs_all(const WarpCtx &x, uint32_t s, int lane,
                                         unsigned long long &acc, unsigned long long &work)
{
    uint32_t C[CW];
#pragma unroll
    for (int q = 0; q < CW; q++) {
        const uint32_t lo = q * 32;
        C[q] = s >= lo + 32 ? kFull : (s > lo ? ((1u << (s - lo)) - 1) : 0u);
    }
    if constexpr (R == 4 && TRI) cdfs4_pairs<CW, WORK>(x, s, x.pair_cap, lane, acc, work);
    else cdfs<R, CW, TRI, WORK>(x, C, lane, acc, work);
}

// Entry for a candidate set of at most compact_max members (lane word c), triangular layout.
template <int R, bool WORK>
__device__ __forceinline__ void compact_entry(const WarpCtx &x, uint32_t c, int lane,
                                              unsigned long long &acc, unsigned long long &work)
{
    int clo, chi;
    const uint32_t s = compact(x, c, lane, clo, chi);
    if (s <= 128) {
        build_compact<4>(x, s, clo, chi, lane);
        if (s <= 32) cdfs_all<R, 1, true, WORK>(x, s, lane, acc, work);
        else if (s <= 64) cdfs_all<R, 2, true, WORK>(x, s, lane, acc, work);
        else if (s <= 96) cdfs_all<R, 3, true, WORK>(x, s, lane, acc, work);
        else cdfs_all<R, 4, true, WORK>(x, s, lane, acc, work);
    } else if constexpr (R == 3) {
        uint32_t t = 0;
        if (s <= 160) {
            build_packed<5>(x, s, clo, chi, lane);
            packed_r3<5, WORK, 0>(x.mbuf, s, lane, t, work);
        } else {
            build_packed<6>(x, s, clo, chi, lane);
            packed_r3<6, WORK, 0>(x.mbuf, s, lane, t, work);
        }
        acc += t;
    }
    __syncwarp();
}

// Counts the R-cliques inside the candidate set whose word w sits in lane w (words >= W are
// zero); adds lane-partial sums to acc.
//   R >= 3, triangular layout, at most compact_max (R >= 4) or compact3_max (R == 3) members:
//           re-encoded compactly (compact_entry) and finished on the compact rows.
//   R >= 4: warp-uniform walk over the members a; the next candidate set c ∧ row_a is again
//           spread over the lanes (one shared-memory load per lane).
//   R == 3: members are compacted and dealt to lanes; each lane builds its own c ∧ row_a and
//           sums its arcs (the last two levels run lane-parallel).
//   R == 2: members dealt to lanes, each adds |c ∧ row_a|.
template <int R, bool WORK>
__device__ __forceinline__ void warp_dfs(const WarpCtx &x, uint32_t c, int lane,
                                         unsigned long long &acc, unsigned long long &work)
{
    if constexpr (R >= 3) {
        if (x.tri && __reduce_add_sync(kFull, __popc(c)) <= (R == 3 ? x.compact3_max : x.compact_max)) {
            compact_entry<R, WORK>(x, c, lane, acc, work);
            return;
        }
    }
    if constexpr (R == 1) {
        acc += __popc(c);
    } else if constexpr (R == 2) {
        const uint32_t nz = __ballot_sync(kFull, c != 0);
        if (__popc(nz) <= 4) {
            // few words: lane l takes bit l of each non-zero word in turn
            if (lane < (int)x.W) x.cbuf[lane] = c;
            __syncwarp();
            const int chi = 32 - __clz(nz);
            uint32_t outer = nz, s = 0;
            while (outer) {
                const int w = __ffs(outer) - 1;
                outer &= outer - 1;
                const uint32_t cw = x.cbuf[w];
                if ((cw >> lane) & 1) {
                    const uint32_t *ra = x.rows + (uint32_t)(w * 32 + lane) * x.RS;
                    const int w0 = x.tri ? w : (__ffs(nz) - 1);
                    if (WORK) work += (uint32_t)(chi - w0);
                    for (int w2 = w0; w2 < chi; w2++) s += __popc(x.cbuf[w2] & ra[w2]);
                }
            }
            acc += s;
            __syncwarp();
        } else if (x.tri) {
            int clo, chi;
            const uint32_t total = compact(x, c, lane, clo, chi);
            acc += tri_rounds<false, WORK>(x, x.cbuf, 0, total, chi, lane, work);
            __syncwarp();
        } else {
            int clo, chi;
            const uint32_t total = compact(x, c, lane, clo, chi);
            uint32_t s = 0;
            for (uint32_t i = lane; i < total; i += 32) {
                const uint32_t a = x.elem[i];
                const uint32_t *ra = x.rows + a * x.RS;
                const int w0 = x.tri ? (int)(a >> 5) : clo;
                if (WORK) work += (uint32_t)(chi - w0);
                for (int w = w0; w < chi; w++) s += __popc(x.cbuf[w] & ra[w]);
            }
            acc += s;
            __syncwarp();
        }
    } else if constexpr (R == 3) {
        int clo, chi;
        const uint32_t total = compact(x, c, lane, clo, chi);
        uint32_t *lb = x.lbuf + lane;
        for (uint32_t i = lane; i < total; i += 32) {
            const uint32_t a = x.elem[i];
            const uint32_t *ra = x.rows + a * x.RS;
            uint32_t cnt = 0;
            int nlo = 32, nhi = 0;
            const int w0 = x.tri ? (int)(a >> 5) : clo;
            if (WORK) work += (uint32_t)(chi - w0);
            for (int w = w0; w < chi; w++) {
                const uint32_t v = x.cbuf[w] & ra[w];
                lb[w * 32] = v;
                if (v) {
                    cnt += __popc(v);
                    nlo = min(nlo, w);
                    nhi = w + 1;
                }
            }
            if (cnt >= 2) acc += lane_arcs<WORK>(x, lb, nlo, nhi, work);
        }
        __syncwarp();
    } else {
        uint32_t rem = c;
        for (;;) {
            const uint32_t nz = __ballot_sync(kFull, rem != 0);
            if (!nz) break;
            const int wl = __ffs(nz) - 1;
            const uint32_t word = __shfl_sync(kFull, rem, wl);
            const uint32_t a = wl * 32 + __ffs(word) - 1;
            if (lane == wl) rem &= rem - 1;
            const uint32_t c2 = lane < (int)x.W ? (c & x.rows[a * x.RS + lane]) : 0u;
            if (WORK && lane < (int)x.W) work += 1;
            const uint32_t cnt = __reduce_add_sync(kFull, __popc(c2));
            if (cnt >= R - 1) warp_dfs<R - 1, WORK>(x, c2, lane, acc, work);
        }
    }
}

// Shared-memory words one warp needs for roots of out-degree <= dcap (dcap multiple of 32).
// Layout: elem (dcap uint16) | cbuf (32) | compress masks + prefixes (192) | lbuf/mbuf, where
// mbuf holds compact_max rows of 4 words or the packed rows of an R = 3 set of up to 192 members.
__host__ __device__ __forceinline__ uint32_t warp_scratch_words(uint32_t dcap, uint32_t compact_max)
{
    const uint32_t m = compact_max ? (compact_max * 4 > packed_words(6) ? compact_max * 4 : packed_words(6)) : 0u;
    return dcap / 2 + 32 + 192 + (dcap > m ? dcap : m);
}

constexpr int kMidMaxWarps = 32;
constexpr uint32_t kSplitMembers = 128;  // k >= 6: rows above this many members split per member
constexpr uint32_t kNoHelpSlot = 0xffffffffu;
constexpr uint32_t kHelpSlots = 8192;    // heavy roots that can take help, per launch

// Position of the r-th (from 0) set bit of x (r < popc(x)).
__device__ __forceinline__ uint32_t select_bit(uint32_t x, uint32_t r)
{
    uint32_t pos = 0;
#pragma unroll
    for (int width = 16; width > 0; width >>= 1) {
        const uint32_t low = __popc(x & ((1u << width) - 1u));
        if (r >= low) {
            r -= low;
            x >>= width;
            pos += width;
        }
    }
    return pos;
}

// Warp 0: the published heavy root with the most units left (kNoHelpSlot when none has any).
__device__ __forceinline__ uint32_t pick_help_slot(const HelpTable &ht, int lane)
{
    const uint32_t ns = min(*(volatile uint32_t *)ht.nslots, ht.cap);
    uint32_t best = kNoHelpSlot, best_rem = 0;
    for (uint32_t s0 = 0; s0 < ns; s0 += 32) {
        const uint32_t sl = s0 + lane;
        uint32_t rem = 0;
        if (sl < ns) {
            cuda::atomic_ref<uint32_t, cuda::thread_scope_device> ready(ht.slots[sl].ready);
            if (ready.load(cuda::memory_order_acquire)) {
                const uint32_t units = ht.slots[sl].units;
                const uint32_t cur = *(volatile uint32_t *)&ht.slots[sl].cursor;
                rem = cur < units ? units - cur : 0u;
            }
        }
        uint32_t bsl = sl;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint32_t r2 = __shfl_xor_sync(kFull, rem, o), s2 = __shfl_xor_sync(kFull, bsl, o);
            if (r2 > rem || (r2 == rem && s2 < bsl)) {
                rem = r2;
                bsl = s2;
            }
        }
        if (rem > best_rem) {
            best_rem = rem;
            best = bsl;
        }
    }
    return best;
}

// Bitmap path (small_max < D <= dcap): one block per root, roots taken largest-D first from the
// queue.  The block builds the root's local subgraph as D x D bitmap rows in shared memory
// (row i = V(g_u) ∩ N+(a_i), Algorithm GenSub-CITRON by sorted-list intersection) and its warps
// count the (K-2)-cliques of every row.
//   D < split_min: the rows (edge tasks (u, a_t)) are taken from a counter in shared memory.
//   D >= split_min (heavy roots, K >= 6): the root's work is a space of units -- one per edge
//       task, or one per member b of a row of more than 128 members (the edge sub-task
//       (u, a_t, b): the (K-3)-cliques of row_t ∧ row_b) -- taken from a cursor in a global
//       table.  Blocks that find the root queue empty pick the published heavy root with the
//       most units left, rebuild its rows and take units from the same cursor (work stealing
//       across blocks); every block adds its own part of the root's count.
// block_ns (optional): each block's start and end on the global timer.
template <int K, bool WORK>
__global__ __launch_bounds__(kMidMaxWarps * 32, 1) void k_count_mid(
    const uint64_t *__restrict__ dag_off, const uint32_t *__restrict__ dag_cols,
    const uint32_t *__restrict__ list, const CountStats *st, uint32_t *next, uint32_t dcap,
    uint32_t compact_max, uint32_t split_min, HelpTable ht, unsigned long long *result,
    RootSink sink, unsigned long long *work_out, unsigned long long *block_ns, Budget budget,
    uint32_t *err)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t rs_cap = (dcap / 32) | 1;
    uint32_t *sL = smem;
    uint32_t *rows = smem + dcap;
    __shared__ uint32_t s_idx, s_task, s_tri, s_slot, s_u, s_units;
    __shared__ unsigned long long s_acc[32], s_arc[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t wsw = warp_scratch_words(dcap, compact_max);
    uint32_t *wscr = rows + (size_t)dcap * rs_cap + (size_t)w * wsw;
    // unit prefix of a heavy root's rows: it reuses sL, which is dead once the rows are built
    uint32_t *s_upre = sL;
    WarpCtx x;
    x.rows = rows;
    x.elem = reinterpret_cast<uint16_t *>(wscr);
    x.cbuf = wscr + dcap / 2;
    x.mv = wscr + dcap / 2 + 32;
    x.lbuf = wscr + dcap / 2 + 32 + 192;
    x.mbuf = x.lbuf;
    x.compact_max = compact_max;
    x.compact3_max = compact_max ? 192u : 0u;
    x.pair_cap = dcap;
    const uint32_t nlist = st->n_mid;
    if (WORK && lane == 0) s_arc[w] = 0;
    if (block_ns && threadIdx.x == 0) block_ns[2 * blockIdx.x] = global_ns();
    unsigned long long block_total = 0;  // meaningful in thread 0
    bool queue_empty = false;
    for (;;) {
        if (threadIdx.x == 0) {
            s_idx = queue_empty || budget.over(err) ? 0xfffffffeu : atomicAdd(next, 1u);
            s_task = 0;
            s_tri = 1;
            s_slot = kNoHelpSlot;
        }
        __syncthreads();
        const uint32_t idx = s_idx;
        const bool owner = idx < nlist;
        if (!owner) {
            queue_empty = true;
            if (K < 6 || ht.slots == nullptr || idx == 0xfffffffeu) break;
            if (w == 0) {
                const uint32_t sl = pick_help_slot(ht, lane);
                if (lane == 0) {
                    s_slot = sl;
                    if (sl != kNoHelpSlot) s_u = ht.slots[sl].u;
                }
            }
            __syncthreads();
            if (s_slot == kNoHelpSlot) break;
        }
        const uint32_t u = owner ? list[idx] : s_u;
        const uint64_t base = dag_off[u];
        const uint32_t D = (uint32_t)(dag_off[u + 1] - base);
        if (D > dcap || D == 0) {  // a root is never larger than the launch's capacity
            if (threadIdx.x == 0) set_error(err, kDevBadInput);
            break;
        }
        const bool heavy = K >= 6 && (!owner || D >= split_min);
        const uint32_t W = (D + 31) >> 5, RS = W | 1;
        for (uint32_t i = threadIdx.x; i < D; i += blockDim.x) sL[i] = dag_cols[base + i];
        if (K > 3)
            for (uint32_t i = threadIdx.x; i < D * RS; i += blockDim.x) rows[i] = 0;
        __syncthreads();
        const uint32_t lmax = sL[D - 1];
        unsigned long long acc = 0, work = 0;
        // Build the local subgraph: row i = V(g_u) ∩ N+(a_i) (CITRON's GenSubgraph).  Each step
        // loads 64 entries of N+(a_i) (two per lane) so that two loads are in flight.  (A block
        // helping with a heavy root rebuilds the same rows; its triangles are not counted here.)
        bool tri = true;
        for (uint32_t i = w; i < D; i += nw) {
            const uint32_t a = sL[i];
            const uint64_t b = dag_off[a], e = dag_off[a + 1];
            for (uint64_t p = b; p < e; p += 64) {
                const uint32_t y0 = p + lane < e ? dag_cols[p + lane] : 0xffffffffu;
                const uint32_t y1 = p + 32 + lane < e ? dag_cols[p + 32 + lane] : 0xffffffffu;
                if (__shfl_sync(kFull, y0, 0) > lmax) break;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t y = h ? y1 : y0;
                    if (y <= lmax) {
                        const uint32_t j = lower_bound_smem(sL, D, y);
                        if (sL[j] == y) {
                            if (K == 3) {
                                acc += 1;
                                if (WORK && sink.per_arc) atomicAdd(&sink.per_arc[base + i], 1ull);
                            } else {
                                atomicOr(&rows[i * RS + (j >> 5)], 1u << (j & 31));
                                tri &= j > i;
                            }
                        }
                    }
                }
            }
        }
        if (K > 3) {
            if (!__all_sync(kFull, tri) && lane == 0) s_tri = 0;
            __syncthreads();
            x.RS = RS;
            x.W = W;
            x.tri = s_tri != 0;
            // Units: edge tasks (u, a_t) -- count (K-2)-cliques in row t -- one per row for a light
            // root; for a heavy root the unit space of its rows (prefix in s_upre), shared with
            // helping blocks through its slot.
            uint32_t U = D;
            if (heavy) {
                for (uint32_t t = w; t < D; t += nw) {
                    const uint32_t c = lane < W ? rows[t * RS + lane] : 0u;
                    const uint32_t m = __reduce_add_sync(kFull, __popc(c));
                    if (lane == 0)
                        s_upre[t] = m < (uint32_t)(K - 2) ? 0u : ((K >= 6 && m > kSplitMembers) ? m : 1u);
                }
                __syncthreads();
                if (w == 0) {
                    uint32_t run = 0;
                    for (uint32_t t0 = 0; t0 < D; t0 += 32) {
                        const uint32_t v = t0 + lane < D ? s_upre[t0 + lane] : 0u;
                        const uint32_t inc = warp_incl_scan(v);
                        if (t0 + lane < D) s_upre[t0 + lane] = run + inc - v;
                        run += __shfl_sync(kFull, inc, 31);
                    }
                    if (lane == 0) s_units = run;
                }
                __syncthreads();
                U = s_units;
                if (threadIdx.x == 0) {
                    if (owner && ht.slots) {
                        const uint32_t sl = atomicAdd(ht.nslots, 1u);
                        if (sl < ht.cap) {
                            ht.slots[sl].u = u;
                            ht.slots[sl].units = U;
                            ht.slots[sl].cursor = 0;
                            cuda::atomic_ref<uint32_t, cuda::thread_scope_device> ready(ht.slots[sl].ready);
                            ready.store(1u, cuda::memory_order_release);
                            s_slot = sl;
                        }
                    } else if (!owner && ht.slots[s_slot].units != U) {
                        set_error(err, kDevBadInput);  // the rebuilt root differs from the published one
                        s_task = U;                    // take nothing
                    }
                }
                __syncthreads();
            }
            // the units of a published heavy root come from its slot's cursor in global memory,
            // the others from the block's counter in shared memory
            uint32_t *gcursor = (s_slot != kNoHelpSlot && (owner || s_task == 0)) ? &ht.slots[s_slot].cursor
                                                                                    : nullptr;
            // a warp claims its next unit before it works on the current one, so that the
            // atomic's round trip (global memory for a published heavy root) overlaps the work
            auto claim = [&]() -> uint32_t {
                uint32_t v = 0;
                if (lane == 0)
                    v = heavy && budget.over(err) ? U : (gcursor ? atomicAdd(gcursor, 1u) : atomicAdd(&s_task, 1u));
                return v;
            };
            uint32_t next_i = claim();
            for (;;) {
                const uint32_t i = __shfl_sync(kFull, next_i, 0);
                if (i >= U) break;
                next_i = claim();
                uint32_t t = i, j = 0;
                bool whole = true;
                if (heavy) {
                    // the row of unit i: the last t with s_upre[t] <= i
                    uint32_t lo = 0, hi = D - 1;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (s_upre[mid] <= i) lo = mid;
                        else hi = mid - 1;
                    }
                    t = lo;
                    j = i - s_upre[t];
                    whole = (t + 1 < D ? s_upre[t + 1] : U) - s_upre[t] == 1u;
                }
                const uint32_t c = lane < W ? rows[t * RS + lane] : 0u;
                if (whole) {
                    const uint32_t cnt = __reduce_add_sync(kFull, __popc(c));
                    if (cnt >= K - 2) warp_dfs<K - 2, WORK>(x, c, lane, acc, work);
                } else if constexpr (K >= 6) {
                    // the j-th member b of row t: the sub-task (u, a_t, b)
                    const uint32_t pc = __popc(c);
                    const uint32_t incl = warp_incl_scan(pc);
                    const int wl = __ffs(__ballot_sync(kFull, incl > j)) - 1;
                    const uint32_t before = __shfl_sync(kFull, incl - pc, wl);
                    const uint32_t word = __shfl_sync(kFull, c, wl);
                    const uint32_t b = (uint32_t)wl * 32 + select_bit(word, j - before);
                    const uint32_t c2 = lane < W ? (c & rows[b * RS + lane]) : 0u;
                    if (WORK && lane < (int)W) work += 1;
                    const uint32_t cnt = __reduce_add_sync(kFull, __popc(c2));
                    if (cnt >= K - 3) warp_dfs<K - 3, WORK>(x, c2, lane, acc, work);
                }
                if (WORK && sink.per_arc) {
                    // debug output (instrumented kernel only): acc holds this unit's part of edge
                    // task t alone (it restarts from zero after every unit; the warp's running
                    // sum is kept in s_arc)
                    const unsigned long long d = warp_sum_u64(acc, err);
                    if (lane == 0) {
                        if (d) atomicAdd(&sink.per_arc[base + t], d);
                        s_arc[w] += d;
                    }
                    acc = 0;
                }
            }
        }
        if (WORK) {
            const unsigned long long wsum = warp_sum_u64(work, err);
            if (lane == 0 && wsum) atomicAdd(work_out, wsum);
        }
        const unsigned long long ws = warp_sum_u64(acc, err);
        if (lane == 0) {
            s_acc[w] = ws;
            if (WORK) {  // the per-arc mode's running sum (zero without it)
                s_acc[w] += s_arc[w];
                s_arc[w] = 0;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long r = 0;
            bool wrapped = false;
            for (int i = 0; i < nw; i++) {
                const unsigned long long s2 = r + s_acc[i];
                wrapped |= s2 < r;
                r = s2;
            }
            if (wrapped) set_error(err, kDevOverflow);
            if (sink.wants_root_total()) {
                if (heavy) sink.add(u, r, err);
                else sink.put(u, r, err);
            }
            const unsigned long long s2 = block_total + r;
            if (s2 < block_total) set_error(err, kDevOverflow);
            block_total = s2;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        add_checked(result, block_total, err);
        if (block_ns) block_ns[2 * blockIdx.x + 1] = global_ns();
    }
}

// ------------------------------------------------------------------------------------------
// Sorted-list path (D > bitmap_max).

// R-cliques inside the sorted candidate list C[0..len); buf holds one list per deeper level.
template <int R>
__device__ void list_dfs(const uint64_t *__restrict__ dag_off, const uint32_t *__restrict__ cols,
                         const uint32_t *C, uint32_t len, uint32_t *buf, uint32_t stride, int lane,
                         unsigned long long &acc)
{
    if (len < (uint32_t)R) return;
    if constexpr (R == 1) {
        if (lane == 0) acc += len;
    } else {
        for (uint32_t i = 0; i < len; i++) {
            const uint32_t a = C[i];
            const uint64_t ab = dag_off[a], ae = dag_off[a + 1];
            uint32_t out = 0;
            for (uint32_t p = 0; p < len; p += 32) {
                bool hit = false;
                uint32_t x = 0;
                if (p + lane < len) {
                    x = C[p + lane];
                    uint64_t lo = ab, hi = ae;
                    while (lo < hi) {
                        const uint64_t mid = lo + (hi - lo) / 2;
                        if (cols[mid] < x) lo = mid + 1;
                        else hi = mid;
                    }
                    hit = lo < ae && cols[lo] == x;
                }
                const uint32_t bal = __ballot_sync(kFull, hit);
                if constexpr (R == 2) {
                    if (lane == 0) acc += __popc(bal);
                } else {
                    if (hit) buf[out + __popc(bal & lanemask_lt())] = x;
                }
                out += __popc(bal);
            }
            if constexpr (R >= 3) {
                __syncwarp();
                if (out >= (uint32_t)(R - 1))
                    list_dfs<R - 1>(dag_off, cols, buf, out, buf + stride, stride, lane, acc);
                __syncwarp();
            }
        }
    }
}

template <int K>
__global__ __launch_bounds__(kListWarps * 32) void k_count_list(
    const uint64_t *__restrict__ dag_off, const uint32_t *__restrict__ dag_cols,
    const uint32_t *__restrict__ list, const CountStats *st, uint32_t *next, uint32_t *scratch,
    uint32_t stride, unsigned long long *result, RootSink sink, Budget budget, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    const uint32_t gw = blockIdx.x * kListWarps + (threadIdx.x >> 5);
    uint32_t *buf = scratch + (size_t)gw * stride * (K > 3 ? K - 3 : 1);
    const uint32_t nlist = st->n_big;
    unsigned long long total = 0;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = budget.over(err) ? nlist : atomicAdd(next, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= nlist) break;
        const uint32_t u = list[idx];
        const uint64_t base = dag_off[u];
        const uint32_t D = (uint32_t)(dag_off[u + 1] - base);
        if (D > stride) {
            if (lane == 0) set_error(err, kDevScratch);
            continue;
        }
        unsigned long long acc = 0;
        if (sink.per_arc) {
            // debug output: the root's edge tasks one at a time (list_dfs's first level, with
            // the intersection N+(u) ∩ N+(a) always listed in buf)
            const uint32_t *C = dag_cols + base;
            for (uint32_t i = 0; i < D; i++) {
                const uint32_t a = C[i];
                const uint64_t ab = dag_off[a], ae = dag_off[a + 1];
                uint32_t out = 0;
                for (uint32_t p = 0; p < D; p += 32) {
                    bool hit = false;
                    uint32_t y = 0;
                    if (p + lane < D) {
                        y = C[p + lane];
                        uint64_t lo = ab, hi = ae;
                        while (lo < hi) {
                            const uint64_t mid = lo + (hi - lo) / 2;
                            if (dag_cols[mid] < y) lo = mid + 1;
                            else hi = mid;
                        }
                        hit = lo < ae && dag_cols[lo] == y;
                    }
                    const uint32_t bal = __ballot_sync(kFull, hit);
                    if (hit) buf[out + __popc(bal & lanemask_lt())] = y;
                    out += __popc(bal);
                }
                __syncwarp();
                unsigned long long t = 0;
                list_dfs<K - 2>(dag_off, dag_cols, buf, out, buf + stride, stride, lane, t);
                __syncwarp();
                const unsigned long long tt = warp_sum_u64(t, err);
                if (lane == 0) sink.per_arc[base + i] = tt;
                acc += t;
            }
        } else {
            list_dfs<K - 1>(dag_off, dag_cols, dag_cols + base, D, buf, stride, lane, acc);
        }
        if (sink.wants_root_total()) {
            const unsigned long long r = warp_sum_u64(acc, err);
            if (lane == 0) sink.put(u, r, err);
        }
        total += acc;
    }
    total = warp_sum_u64(total, err);
    if (lane == 0) add_checked(result, total, err);
}

}  // namespace citron

namespace citron_host {
using namespace citron;

// Global-memory helpers of the bitmap kernel: the help table of heavy roots and the per-block
// start/end times (2 words per block, kMidBlocksPerSmCap blocks per SM at most).
constexpr uint32_t kMidBlocksPerSmCap = 8;
struct MidAux {
    HelpTable help;
    unsigned long long *block_ns = nullptr;
    Budget budget;  // the count's time budget (all of its launches)
};

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    bool on;
    cudaStream_t s;
    Timer(bool enable, cudaStream_t st) : on(enable), s(st)
    {
        if (on && (cudaEventCreate(&a) || cudaEventCreate(&b))) on = false;
        if (on) cudaEventRecord(a, s);
    }
    void stop() { if (on) cudaEventRecord(b, s); }
    float ms()
    {
        float t = 0;
        if (on && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&t, a, b);
        return t;
    }
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

template <int K, bool WORK>
static cudaError_t launch_mid(uint32_t grid_cap, uint32_t block_cap, uint32_t dcap,
                              uint32_t compact_max, uint32_t split_min, const HelpTable &ht,
                              uint32_t warps, size_t smem, const uint64_t *dag_off,
                              const uint32_t *dag_cols, const uint32_t *mid_list,
                              const CountStats *st, uint32_t *next, unsigned long long *result,
                              RootSink sink, unsigned long long *work, unsigned long long *block_ns,
                              Budget budget, uint32_t *grid_out, uint32_t *err, cudaStream_t s,
                              int num_sms)
{
    cudaError_t e;
    // the attribute is an upper bound on the launches' dynamic shared memory; it is always set to
    // the device's largest value, because host threads that count concurrently would otherwise
    // overwrite each other's smaller setting between the set and the launch
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    if ((size_t)(optin - 1024) < smem) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(k_count_mid<K, WORK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - 1024)))
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_mid<K, WORK>, warps * 32,
                                                           smem)))
        return e;
    if (per_sm < 1) per_sm = 1;
    uint32_t grid = (uint32_t)(num_sms * per_sm);
    if (grid > grid_cap) grid = grid_cap;
    if (block_cap && grid > block_cap) grid = block_cap;
    if (grid > (uint32_t)num_sms * kMidBlocksPerSmCap) grid = (uint32_t)num_sms * kMidBlocksPerSmCap;
    *grid_out = grid;
    k_count_mid<K, WORK><<<grid, warps * 32, smem, s>>>(dag_off, dag_cols, mid_list, st, next, dcap,
                                                        compact_max, split_min, ht, result, sink,
                                                        work, block_ns, budget, err);
    note_launches(1);
    return cudaGetLastError();
}

template <int K>
static cudaError_t launch_count_k(CountRun &run, const uint64_t *dag_off, const uint32_t *dag_cols,
                                  const CountStats &hs, const CountStats *st,
                                  const uint32_t *small_list, const uint32_t *mid_list,
                                  const uint32_t *big_list, uint32_t *next, uint32_t *list_scratch,
                                  size_t list_scratch_words, unsigned long long *result,
                                  unsigned long long *work, const MidAux &aux, uint32_t *err,
                                  cudaStream_t s, int num_sms)
{
    cudaError_t e = cudaSuccess;
    const CountPlan &plan = run.plan;
    if (hs.n_mid) {
        const uint32_t dcap = (hs.max_mid + 31) & ~31u;
        const uint32_t rs = (dcap / 32) | 1;
        int smem_cap = 0, dev = 0;
        cudaGetDevice(&dev);
        if ((e = cudaDeviceGetAttribute(&smem_cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)))
            return e;
        smem_cap -= 1024;  // static shared memory of the kernel
        auto smem_for = [&](uint32_t warps) {
            return ((size_t)dcap +
                    (K > 3 ? (size_t)dcap * rs + (size_t)warps * warp_scratch_words(dcap, plan.compact_max) : 0)) *
                   sizeof(uint32_t);
        };
        uint32_t warps = plan.warps_per_cta > (uint32_t)kMidMaxWarps ? kMidMaxWarps : plan.warps_per_cta;
        while (warps > 1 && smem_for(warps) > (size_t)smem_cap) warps--;
        Timer t(run.time_kernels, s);
        unsigned long long *block_ns = run.balance ? aux.block_ns : nullptr;
        uint32_t grid = 0;
        // the instrumented kernel also serves the per-arc debug output (its code is compiled out
        // of the plain kernel)
        if (run.count_work || run.sink.per_arc) {
            if constexpr (K <= (int)kInstrumentedMaxK)
                e = launch_mid<K, true>(hs.n_mid, plan.max_blocks, dcap, plan.compact_max, plan.split_min,
                                        aux.help, warps, smem_for(warps), dag_off, dag_cols, mid_list, st,
                                        next + 0, result, run.sink, work, block_ns, aux.budget, &grid, err,
                                        s, num_sms);
            else
                e = cudaErrorNotSupported;  // refused by citron_count_ex before any launch
        } else
            e = launch_mid<K, false>(hs.n_mid, plan.max_blocks, dcap, plan.compact_max, plan.split_min,
                                     aux.help, warps, smem_for(warps), dag_off, dag_cols, mid_list, st,
                                     next + 0, result, run.sink, work, block_ns, aux.budget, &grid, err, s,
                                    num_sms);
        if (e) return e;
        t.stop();
        run.kernel_ms[1] = t.ms();
        if (block_ns && grid) {
            // span = first block start .. last block end; tail = first block end .. last block end
            unsigned long long h[2 * kMidBlocksPerSmCap * 256];
            const size_t cnt = 2 * (size_t)grid;
            if (cnt <= sizeof(h) / sizeof(h[0])) {
                e = cudaMemcpyAsync(h, block_ns, cnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
                if (!e) e = cudaStreamSynchronize(s);
                if (e) return e;
                unsigned long long s0 = ~0ull, e0 = ~0ull, e1 = 0;
                for (uint32_t b = 0; b < grid; b++) {
                    s0 = h[2 * b] < s0 ? h[2 * b] : s0;
                    e0 = h[2 * b + 1] < e0 ? h[2 * b + 1] : e0;
                    e1 = h[2 * b + 1] > e1 ? h[2 * b + 1] : e1;
                }
                run.busy_ms[0] = (float)((e1 - s0) * 1e-6);
                run.busy_ms[1] = (float)((e1 - e0) * 1e-6);
            }
        }
    }
    if (hs.n_small) {
        uint32_t grid = (hs.n_small + kSmallWarps - 1) / kSmallWarps;
        uint32_t cap = (uint32_t)num_sms * 16;
        if (plan.max_blocks && cap > plan.max_blocks * 4) cap = plan.max_blocks * 4;
        if (grid > cap) grid = cap;
        Timer t(run.time_kernels, s);
        k_count_small<K><<<grid, kSmallWarps * 32, 0, s>>>(dag_off, dag_cols, small_list, st, result,
                                                           run.sink, aux.budget, err);
        note_launches(1);
        if ((e = cudaGetLastError())) return e;
        t.stop();
        run.kernel_ms[0] = t.ms();
    }
    if (hs.n_big) {
        const size_t per_warp = (size_t)hs.max_big * (K > 3 ? K - 3 : 1);
        size_t warps = per_warp ? list_scratch_words / per_warp : 0;
        if (warps < kListWarps) return cudaErrorMemoryAllocation;
        uint32_t grid = (uint32_t)(warps / kListWarps);
        uint32_t cap = (uint32_t)num_sms;
        if (plan.max_blocks && cap > plan.max_blocks) cap = plan.max_blocks;
        if (grid > cap) grid = cap;
        if (grid > (hs.n_big + kListWarps - 1) / kListWarps) grid = (hs.n_big + kListWarps - 1) / kListWarps;
        Timer t(run.time_kernels, s);
        k_count_list<K><<<grid, kListWarps * 32, 0, s>>>(dag_off, dag_cols, big_list, st, next + 1,
                                                         list_scratch, hs.max_big, result,
                                                         run.sink, aux.budget, err);
        note_launches(1);
        if ((e = cudaGetLastError())) return e;
        t.stop();
        run.kernel_ms[2] = t.ms();
    }
    return cudaSuccess;
}

// Per-k launchers, each compiled in its own translation unit (count_k*.cu).
#define CITRON_LAUNCH_K_DECL(KK)                                                                     \
    cudaError_t launch_count_##KK(CountRun &run, const uint64_t *dag_off, const uint32_t *dag_cols,  \
                                  const CountStats &hs, const CountStats *st,                       \
                                  const uint32_t *small_list, const uint32_t *mid_list,             \
                                  const uint32_t *big_list, uint32_t *next, uint32_t *list_scratch, \
                                  size_t list_scratch_words, unsigned long long *result,            \
                                  unsigned long long *work, const MidAux &aux, uint32_t *err,       \
                                  cudaStream_t s, int num_sms)
#define CITRON_LAUNCH_K_DEF(KK)                                                                      \
    CITRON_LAUNCH_K_DECL(KK)                                                                         \
    {                                                                                                \
        return launch_count_k<KK>(run, dag_off, dag_cols, hs, st, small_list, mid_list, big_list,   \
                                  next, list_scratch, list_scratch_words, result, work, aux, err,   \
                                  s, num_sms);                                                      \
    }
CITRON_LAUNCH_K_DECL(3);
CITRON_LAUNCH_K_DECL(4);
CITRON_LAUNCH_K_DECL(5);
CITRON_LAUNCH_K_DECL(6);
CITRON_LAUNCH_K_DECL(7);
CITRON_LAUNCH_K_DECL(8);
CITRON_LAUNCH_K_DECL(9);
CITRON_LAUNCH_K_DECL(10);
CITRON_LAUNCH_K_DECL(11);
CITRON_LAUNCH_K_DECL(12);

}  // namespace citron_host
