/*
 * citron.h -- C ABI of the GB300 (sm_103a) k-clique counter.
 *
 * The method is the ordering-based k-clique counter of "Accelerating Clique Counting in Sparse
 * Real-World Graphs via Communication-Reducing Optimizations" (CITRON, arXiv 2112.10913):
 *   ordering phase  -- degree ordering (Sec. II, Sec. IV) and the DAG it induces
 *                      (Algorithm GenOrdering, Sec. IV);
 *   counting phase  -- the recursion of Algorithm Counting (Sec. III) over subgraphs induced by
 *                      out-neighbour sets, built by sorted-set intersection (Sec. V-B), with the
 *                      prune and the penultimate-level shortcut (Sec. V-B, other optimizations).
 *
 * Conventions shared by every entry point
 *   - Graphs are CSR.  `off` has n+1 uint64 entries (off[0] = 0, non-decreasing), `cols` has
 *     off[n] uint32 entries, every row sorted strictly ascending.  An undirected input graph
 *     holds each edge {u,v} as the two arcs u->v and v->u (symmetrised, Sec. VI-B), no self-loops,
 *     no duplicates (Sec. V-B).  n must be below 2^32 - 1.
 *   - Pointers named d_* are DEVICE pointers, h_* are HOST pointers.  All memory belongs to the
 *     caller; the library never allocates, frees or keeps a pointer after a call returns.
 *   - `ws` is a device workspace of at least citron_workspace_bytes(...) bytes, 256-byte aligned.
 *     Its contents are scratch: nothing survives from one call to the next.  Two calls that
 *     overlap in time must not share a workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls that
 *     return only device results are asynchronous on `stream`; calls that return a host value
 *     (h_*) synchronise `stream` before returning.
 *   - Errors are returned, never raised: no abort, no trap, no device assert.  Device kernels
 *     record the first error in the workspace; the call that owns them reports it.
 */
#ifndef CITRON_H
#define CITRON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CITRON_OK = 0,
    CITRON_E_INVALID = 1,     /* bad argument or input that breaks the CSR contract */
    CITRON_E_WORKSPACE = 2,   /* workspace missing, misaligned or smaller than required */
    CITRON_E_CUDA = 3,        /* a CUDA runtime call failed (launch, copy, sync) */
    CITRON_E_OVERFLOW = 4,    /* the exact count does not fit in uint64 */
    CITRON_E_TIMEOUT = 5,     /* a bounded device wait gave up (the result is not valid) */
    CITRON_E_UNSUPPORTED = 6, /* the input exceeds a documented size limit of this build */
    CITRON_E_BUDGET = 7       /* the count's time budget ran out before it finished (no result) */
} citron_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *citron_status_str(citron_status s);

/* Name of the CUDA runtime error behind the most recent CITRON_E_CUDA returned to this thread
 * (static string, never NULL; "none" when there was none). */
const char *citron_last_cuda_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int citron_version(void);

/*
 * Workspace size in bytes that is enough for every entry point below on a graph with n vertices,
 * `arcs` = off[n] input arcs and a DAG whose largest out-degree is at most `max_outdeg`
 * (pass 0 when unknown: the bound min(n-1, arcs/2) is then used, which can be large).
 */
size_t citron_workspace_bytes(uint32_t n, uint64_t arcs, uint32_t max_outdeg);

/*
 * citron_validate -- check the CSR contract on the device: offsets start at 0 and never
 * decrease, ids < n, rows strictly ascending (sorted, no duplicates), no self-loops, and every
 * arc u->v has its reverse v->u (symmetrised input, Sec. VI-B).
 *   returns CITRON_OK or CITRON_E_INVALID; *h_bad (optional) receives a code 1..5 for the first
 *   kind of defect found (1 offsets, 2 range, 3 order/duplicate, 4 self-loop, 5 asymmetric).
 * Synchronises `stream`.
 */
citron_status citron_validate(uint32_t n, uint64_t arcs, const uint64_t *d_off,
                              const uint32_t *d_cols, uint32_t *h_bad, void *ws, size_t ws_bytes,
                              void *stream);

/*
 * citron_order -- the degree ordering of Sec. II / Sec. IV: vertices sorted by (d(u), u) with
 * d(u) = off[u+1] - off[u], lower degree first, lower id first on equal degree.
 *   d_rank[u] (device, n entries, written) = position of u in that order (a permutation);
 *   d_perm[i] (device, n entries, optional, may be NULL) = the vertex at position i.
 * Implemented as a stable LSD radix sort of the ids by degree (ids start ascending, so stability
 * gives the id tie-break).  Asynchronous.
 */
citron_status citron_order(uint32_t n, const uint64_t *d_off, uint32_t *d_rank, uint32_t *d_perm,
                           void *ws, size_t ws_bytes, void *stream);

/*
 * citron_order_grouped -- the degree ordering of every graph of a batch at once.  The input is
 * the disjoint union of the graphs (d_off as for citron_order) with d_group[u] (device, n
 * entries) = the graph of vertex u, below ngroups.  The vertices are sorted by (d_group[u], d(u),
 * u): every graph's vertices get a contiguous range of positions, in the graph's own degree
 * order (Sec. II, Sec. IV).  The DAG citron_build_dag relabels with this rank is therefore the
 * concatenation of the graphs' own relabelled DAGs (ranks shifted by the graph's first
 * position), so each graph's DAG is a contiguous slice of it.  Outputs as for citron_order.
 * Asynchronous.
 */
citron_status citron_order_grouped(uint32_t n, const uint64_t *d_off, const uint32_t *d_group,
                                   uint32_t ngroups, uint32_t *d_rank, uint32_t *d_perm, void *ws,
                                   size_t ws_bytes, void *stream);

/*
 * citron_core_order -- the core ordering of Algorithm OrdCore (Sec. III), computed in
 * synchronous peeling rounds: each round raises a level to the smallest remaining degree (it
 * never falls) and removes, together, every remaining vertex whose remaining degree is at most
 * the level; then their neighbours' remaining degrees drop.  The order is (removal round, id).
 * As with the paper's one-vertex-at-a-time removal, orienting edges from earlier to later vertices
 * gives a DAG whose maximum out-degree is the degeneracy (the smallest possible, Sec. III and
 * Table II); the order itself can differ from the sequential one.
 *   d_off[n+1], d_cols[arcs] (device): the undirected graph, as for citron_build_dag.
 *   d_rank[u] (device, n entries, written) = position of u; d_perm (optional) = the inverse.
 *   h_degeneracy, h_rounds (host, optional): the final level (the degeneracy) and the number of
 *   rounds.
 * One cooperative kernel runs all rounds (grid barriers with a bounded wait; a wait that gives
 * up returns CITRON_E_TIMEOUT), then a radix sort by round.  Synchronises `stream`.  Returns
 * CITRON_E_UNSUPPORTED on a device without cooperative launch.  Pass the rank to
 * citron_build_dag for the core-ordered DAG.
 */
citron_status citron_core_order(uint32_t n, uint64_t arcs, const uint64_t *d_off,
                                const uint32_t *d_cols, uint32_t *d_rank, uint32_t *d_perm,
                                uint32_t *h_degeneracy, uint32_t *h_rounds, void *ws,
                                size_t ws_bytes, void *stream);

/*
 * citron_build_dag -- directionalise the graph (Sec. II) into a DAG in CSR form.
 *   d_rank == NULL: Algorithm GenOrdering (Sec. IV): the arc u->v is kept iff
 *       d(u) < d(v) or (d(u) == d(v) and u < v); vertex ids are unchanged and each row keeps the
 *       input's ascending order.  One fused pass: keep-test, prefix sum and fill.
 *   d_rank != NULL: any total order given as a permutation rank[0..n): u->v kept iff
 *       rank[u] < rank[v], and the DAG is RELABELLED: row r belongs to the vertex of rank r and
 *       holds the ranks of its out-neighbours, sorted ascending.  With the rank of citron_order
 *       this is the degree-ordered DAG in rank space.  Limit: a row longer than 32768 is reported
 *       as CITRON_E_UNSUPPORTED (by this call when it synchronises, else by the next one that does).
 *   Output (device, caller-allocated): d_dag_off[n+1] (uint64), d_dag_cols[arcs/2] (uint32).
 *   h_max_outdeg (optional host pointer): receives the largest row length of the DAG; when
 *   given, the call synchronises `stream`, otherwise it is asynchronous.
 */
citron_status citron_build_dag(uint32_t n, uint64_t arcs, const uint64_t *d_off,
                               const uint32_t *d_cols, const uint32_t *d_rank,
                               uint64_t *d_dag_off, uint32_t *d_dag_cols, uint32_t *h_max_outdeg,
                               void *ws, size_t ws_bytes, void *stream);

/*
 * citron_count -- exact number of k-cliques (Sec. II) of the undirected graph whose DAG is given
 * (any acyclic orientation with sorted rows: the count does not depend on the ordering).
 *   k = 0 -> CITRON_E_INVALID; k = 1 -> n; k = 2 -> number of arcs of the DAG; k >= 3 -> the
 *   counting phase (Algorithm Counting with CITRON's subgraphs, Sec. III and Sec. V-B).
 *   Supported k: 1..CITRON_MAX_K.
 *   max_outdeg: largest DAG row length if known (from citron_build_dag), else 0 (computed here).
 *   *h_count (host) receives the count.  A count above 2^64-1 returns CITRON_E_OVERFLOW.
 *   d_per_root (device, optional, n uint64 entries): when not NULL, receives for every vertex u
 *   the number of k-cliques whose first vertex in the DAG order is u (for localising errors).
 * Synchronises `stream`.
 */
#define CITRON_MAX_K 12
citron_status citron_count(uint32_t n, const uint64_t *d_dag_off, const uint32_t *d_dag_cols,
                           uint32_t k, uint32_t max_outdeg, uint64_t *h_count,
                           uint64_t *d_per_root, void *ws, size_t ws_bytes, void *stream);

/*
 * citron_list -- write out every k-clique instead of counting it (the extension of the counting
 * recursion that Sec. VIII describes).  Each clique is one row of k uint32 ids in recursion
 * order: its first vertex in the DAG order, then the vertex of its edge task, then the vertices
 * chosen level by level (ascending DAG ids for a DAG relabelled to ranks).
 *   d_map (device, optional): ids are written as d_map[id] (pass the inverse rank, i.e. the
 *       d_perm of citron_order, to get input vertex ids from a relabelled DAG); NULL writes DAG ids.
 *   d_out (device, capacity * k uint32, caller-allocated): the rows, in no particular order.
 *   capacity: rows d_out can hold; 0 (with d_out NULL) only counts.
 *   *h_total (host, required): the number of k-cliques.  When *h_total > capacity, only
 *       `capacity` rows were written, an unspecified subset: call again with a larger buffer.
 * Limits: k <= CITRON_MAX_K; a DAG row longer than 1024 returns CITRON_E_UNSUPPORTED (the rows
 * of a root's local subgraph are held in shared memory).  Synchronises `stream`.
 */
citron_status citron_list(uint32_t n, const uint64_t *d_dag_off, const uint32_t *d_dag_cols,
                          uint32_t k, const uint32_t *d_map, uint32_t *d_out, uint64_t capacity,
                          uint64_t *h_total, void *ws, size_t ws_bytes, void *stream);

/*
 * citron_count_ex -- citron_count with options: the internal path thresholds (for tests that must
 * reach every path on small graphs, and for tuning), device timing of the counting kernels, and
 * a count of the word operations the bitmap path performs (for roofline accounting).
 *   opts (host, required): see citron_count_opts; its "in" fields are read, its "out" fields
 *   written.  Same count as citron_count.  Synchronises `stream`.
 */
#define CITRON_COUNT_TIME_KERNELS 1u /* fill kernel_ms (events on `stream`) */
#define CITRON_COUNT_WORK 2u         /* fill work_ops (a separately compiled, instrumented kernel,
                                        built for k <= 8: larger k returns CITRON_E_UNSUPPORTED) */
#define CITRON_COUNT_BALANCE 4u      /* fill busy_ms (each bitmap-path block's start and end) */
typedef struct {
    uint32_t small_max;      /* in: warp-register path for out-degree <= small_max, 0..32 (0: 32) */
    uint32_t bitmap_max;     /* in: shared-memory bitmap path up to this out-degree, <= 1024
                                (0: 1024); larger roots take the sorted-list path */
    uint32_t warps_per_cta;  /* in: warps per bitmap-path block, 1..32 (0: 32); fewer are used
                                when the block's shared memory would not fit */
    uint32_t flags;          /* in: CITRON_COUNT_* bits */
    uint32_t compact_max;    /* in: candidate sets of the bitmap path with at most this many
                                members are re-encoded as compact bitmaps: 0 or 128 mean 128,
                                1 means never */
    uint32_t max_blocks;     /* in: cap on the blocks of each counting launch, so that work on
                                other streams keeps some SMs (0: no cap) */
    uint64_t *d_per_root;    /* in: optional device array of n uint64, as in citron_count */
    uint64_t work_ops;       /* out: 32-bit AND+POPC word operations of the bitmap path */
    float kernel_ms[3];      /* out: device ms of the warp-register, bitmap, sorted-list kernels */
    uint32_t split_min;      /* in: for k >= 6, bitmap-path roots of at least this out-degree
                                share their work with idle blocks (heavy-edge splitting,
                                Sec. VII-C): their edge tasks, and the sub-tasks (u, a_t, b) of
                                rows above 128 members, are taken from a global cursor, which
                                blocks that find the root queue empty join after rebuilding the
                                root's subgraph.  0: default (384); 1: never; else the threshold */
    float busy_ms[2];        /* out (CITRON_COUNT_BALANCE): bitmap kernel's span from the first
                                block start to the last block end, and its tail from the first
                                block end to the last */
    uint32_t budget_ms;      /* in: device time the count may take (0: no limit); when it runs
                                out, the blocks stop taking work and the call returns
                                CITRON_E_BUDGET */
    uint64_t *d_per_arc;     /* in: optional device array of one uint64 per DAG arc (dag_off[n]
                                entries; k >= 3, else CITRON_E_INVALID).  When not NULL it
                                receives, for every arc e = (u, v), the number of k-cliques whose
                                first two vertices in the DAG order are u then v (a clique is
                                counted once, at its first vertex, Sec. II; inside that root by
                                its second): the count of the edge task (u, v), for localising
                                a difference inside a root.  A debug mode: it runs the
                                instrumented bitmap-path kernel (as CITRON_COUNT_WORK does, and
                                fills work_ops; k <= 8, else CITRON_E_UNSUPPORTED), and the edge
                                tasks of small and sorted-list roots one at a time. */
} citron_count_opts;

citron_status citron_count_ex(uint32_t n, const uint64_t *d_dag_off, const uint32_t *d_dag_cols,
                              uint32_t k, uint32_t max_outdeg, citron_count_opts *opts,
                              uint64_t *h_count, void *ws, size_t ws_bytes, void *stream);

/* Number of CUDA kernels this library has launched since it was loaded (all threads). */
uint64_t citron_kernel_launches(void);

/*
 * citron_count_host -- the whole hot path from HOST buffers: copies the CSR (h_off[n+1],
 * h_cols[arcs]) to the device buffer d_buf, orders (citron_order), builds the relabelled DAG
 * (citron_build_dag with that rank) and counts every k in h_ks[0..nk) into h_counts[0..nk).
 * d_buf must hold citron_host_buffer_bytes(n, arcs) bytes; ws as above.  Host buffers should be
 * pinned for full copy speed (pageable memory works, slower).  Synchronises `stream`.
 */
size_t citron_host_buffer_bytes(uint32_t n, uint64_t arcs);
citron_status citron_count_host(uint32_t n, uint64_t arcs, const uint64_t *h_off,
                                const uint32_t *h_cols, const uint32_t *h_ks, uint32_t nk,
                                uint64_t *h_counts, void *d_buf, size_t buf_bytes, void *ws,
                                size_t ws_bytes, void *stream);

/*
 * citron_count_batch -- exact counts of many graphs at once, each graph ("group") with its own
 * k.  The graphs are given as ONE DAG: the DAG of their disjoint union (citron_build_dag over
 * the union CSR; edges never cross graphs, so this is the union of the graphs' DAGs).  Each
 * k-clique lies inside one graph and is counted once, at its first vertex (Sec. II); that
 * root's count goes to its graph's total.  One counting pass runs per k present.
 *   d_rank: the rank the DAG was relabelled with (NULL if the DAG keeps vertex ids).
 *   d_group_of_vertex[v] (device, n): graph of input vertex v, < ngroups.
 *   d_group_k[g] (device, ngroups): the k of graph g, 1..CITRON_MAX_K.
 *   kmask (host): bit k set for every k that occurs in d_group_k (passes for other k are skipped).
 *   max_outdeg: largest DAG row (from citron_build_dag); launch sizes derive from it.
 *   opts: optional path thresholds (only small_max, bitmap_max, warps_per_cta, compact_max,
 *         max_blocks are read); NULL for the defaults.
 *   d_counts[g] (device, ngroups uint64, written).
 * The call is ASYNCHRONOUS and never synchronises the host, so it can be captured into a CUDA
 * graph and replayed; device errors stay in the workspace until citron_workspace_status.
 */
citron_status citron_count_batch(uint32_t n, const uint64_t *d_dag_off, const uint32_t *d_dag_cols,
                                 const uint32_t *d_rank, const uint32_t *d_group_of_vertex,
                                 const uint32_t *d_group_k, uint32_t ngroups, uint32_t kmask,
                                 uint32_t max_outdeg, const citron_count_opts *opts,
                                 uint64_t *d_counts, void *ws, size_t ws_bytes, void *stream);

/*
 * citron_dag_append -- copies the DAG of one graph into another DAG at a new place: the rows
 * src_row .. src_row+n-1 of a source DAG (d_src_off holds those rows' n+1 offsets into
 * d_src_cols; the columns are ids of the source's id space) become rows dst_row .. dst_row+n-1 of
 * the destination, whose arcs start at dst_arc:
 *   d_dst_off[i] = d_src_off[i] - d_src_off[0] + dst_arc            (i = 0..n, n+1 entries)
 *   d_dst_cols[dst_arc + e] = d_src_cols[d_src_off[0] + e] - src_row + dst_row
 * (the graph's arcs must point inside its own rows, as every graph of a disjoint union does).
 * With it a batch is assembled from the DAGs of graphs counted before (kept on the device by a
 * serving loop) without ordering them again, and a graph's DAG is cut out of a batch's union
 * DAG.  The paper has no counterpart: this is data movement for batching.  Asynchronous.
 */
citron_status citron_dag_append(uint32_t n, const uint64_t *d_src_off, const uint32_t *d_src_cols,
                                uint32_t src_row, uint64_t *d_dst_off, uint32_t *d_dst_cols,
                                uint32_t dst_row, uint64_t dst_arc, void *stream);

/* Synchronises `stream` and reports (then clears) the device error word of the workspace:
 * errors recorded by asynchronous calls such as citron_count_batch or citron_build_dag. */
citron_status citron_workspace_status(void *ws, void *stream);

/*
 * citron_probe_word_ops -- measures the device's peak rate of the counting phase's unit of work,
 * the 32-bit word operation (one AND, one POPC and one add on register operands), for the
 * roofline of the counting kernels (the paper has no counterpart: this is measurement).  A
 * kernel of blocks_per_sm x (number of SMs) blocks of 1024 threads runs `iters` iterations of 8
 * independent word operations per thread; *h_ops_per_s receives word operations per second and
 * *h_ms the kernel's device time (CUDA events on `stream`).  Synchronises `stream`.
 */
citron_status citron_probe_word_ops(uint32_t blocks_per_sm, uint32_t iters, double *h_ops_per_s,
                                    float *h_ms, void *stream);

/*
 * citron_set_faults -- fault injection for tests of the error paths (the paper has no
 * counterpart: the method itself never fails).  Process-wide; applies to every call made after it
 * on any device until it is called again; NULL restores normal operation.  Nothing here faults
 * a GPU: every injected failure is a wait that nothing will end, which the library's own bounded
 * waits must turn into CITRON_E_TIMEOUT, or a seeded sum that must report CITRON_E_OVERFLOW.
 *   lookback_spin_limit : probes a decoupled look-back makes before it gives up (0: 2^22);
 *   lookback_stall_tile : tile index + 1 whose look-back never publishes its prefix, so that
 *                         the next tile's wait must run out (0: none);
 *   barrier_wait_ns     : time a grid barrier of the core ordering waits (0: 4 s);
 *   barrier_absent_block: block index + 1 of the core ordering that never arrives at the first
 *                         grid barrier, so that the others' wait must run out (0: none);
 *   count_seed          : initial value of the device totals of counting passes (citron_count
 *                         and its variants: the grand total; citron_count_batch: every graph's
 *                         total); a count that carries it past 2^64 - 1 reports
 *                         CITRON_E_OVERFLOW (0: none).
 * Results computed while a fault is injected are not valid; calls still return a status.
 */
typedef struct {
    uint32_t lookback_spin_limit;
    uint32_t lookback_stall_tile;
    uint64_t barrier_wait_ns;
    uint32_t barrier_absent_block;
    uint32_t reserved;
    uint64_t count_seed;
} citron_faults;

citron_status citron_set_faults(const citron_faults *faults);

/*
 * citron_count_noalloc -- citron_count for callers that cannot allocate device memory.  (The
 * paper has no counterpart: this is an interface choice of this library.)
 *   Who needs it: host applications or plugin frameworks that own the device heap and forbid
 *   allocation after start-up, real-time loops that cannot take the implicit synchronisation of
 *   cudaMalloc/cudaFree, and C callers with no allocator of their own.  They still pass the DAG
 *   (input) and receive the count (output); no workspace is needed.
 *   How: the scratch lives in one fixed file-scope device array of 1 MiB that every GPU loading
 *   this library holds until the process exits.  No cudaMalloc, cudaFree or allocating library
 *   routine is called.  The first call on a device (with that device current) looks up the
 *   array's device address; make that first call before any stream capture.
 *   Limits: n <= 65536 vertices (larger n returns CITRON_E_UNSUPPORTED); roots with out-degree
 *   above 1024 take the sorted-list path, whose scratch may not fit (CITRON_E_WORKSPACE).
 *   Every call shares the one array and clears what it needs: calls that overlap on the GPU
 *   (different streams or threads on the same device) race and must not be issued.
 *   Same arguments and results as citron_count otherwise.  Synchronises `stream`.
 */
citron_status citron_count_noalloc(uint32_t n, const uint64_t *d_dag_off,
                                   const uint32_t *d_dag_cols, uint32_t k, uint64_t *h_count,
                                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CITRON_H */
