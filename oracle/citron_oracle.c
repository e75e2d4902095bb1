/*
 * citron_oracle.c -- the ORACLE: plain, slow, obviously correct CPU restatement of the
 * ordering-based k-clique counter of "Accelerating Clique Counting in Sparse Real-World Graphs
 * via Communication-Reducing Optimizations" (CITRON, arXiv 2112.10913).
 *
 * This file is TEST INFRASTRUCTURE.  Only the tests, the smoke check and the bench's CPU-baseline
 * leg may build, load or call it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (Sec. II): the number of k-vertex subsets of V that are pairwise adjacent.
 * How (the paper's method, step by step, no blocking or reordering beyond it):
 *   1. degrees d(u) = |N(u)|                                            (Sec. II)
 *   2. degree ordering: u before v iff (d(u), u) < (d(v), v)            (Sec. II, Sec. IV)
 *   3. DAG by Algorithm "GenOrdering": count kept arcs, prefix sum, fill (Sec. IV)
 *   4. counting by the kClist recursion "Counting" (Sec. III), with CITRON's subgraph build by
 *      sorted-set intersection (Sec. V-B), the prune of candidate sets too small to hold the
 *      clique size still needed
 *      (Sec. V-B, other optimizations) and the penultimate-level shortcut that only adds
 *      subgraph degrees (Sec. V-B, last paragraph; Counting's l = 2 branch).
 *   Also: core ordering by Algorithm "OrdCore" (Matula-Beck smallest-last, Sec. III) and the DAG
 *   of an arbitrary total order, both used to check that the count does not depend on the order.
 *
 * Every count is an exact uint64; any addition that overflows is reported, never wrapped.
 * Parity status: every function below is pinned by tests (brute force, closed forms, trace,
 * ordering invariance, the Fig. 1 worked example); none is "parity unpinned".
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_E_OFFSETS 1
#define ORACLE_E_RANGE 2
#define ORACLE_E_UNSORTED 3
#define ORACLE_E_LOOP 4
#define ORACLE_E_ASYMMETRIC 5
#define ORACLE_E_OVERFLOW 6
#define ORACLE_E_NOMEM 7
#define ORACLE_E_ARG 8

/* ------------------------------------------------------------------------------------------ */
/* Input checks (Sec. VI-B: symmetrised, unweighted; Sec. V-B: no duplicate edges).           */

static int row_contains(const uint64_t *off, const uint32_t *cols, uint32_t row, uint32_t x)
{
    uint64_t lo = off[row], hi = off[row + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (cols[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo < off[row + 1] && cols[lo] == x;
}

int oracle_validate(uint32_t n, const uint64_t *off, const uint32_t *cols)
{
    if (off[0] != 0) return ORACLE_E_OFFSETS;
    for (uint32_t u = 0; u < n; u++)
        if (off[u + 1] < off[u]) return ORACLE_E_OFFSETS;
    for (uint32_t u = 0; u < n; u++) {
        for (uint64_t e = off[u]; e < off[u + 1]; e++) {
            uint32_t v = cols[e];
            if (v >= n) return ORACLE_E_RANGE;
            if (v == u) return ORACLE_E_LOOP;
            if (e > off[u] && cols[e - 1] >= v) return ORACLE_E_UNSORTED;
        }
    }
    for (uint32_t u = 0; u < n; u++)
        for (uint64_t e = off[u]; e < off[u + 1]; e++)
            if (!row_contains(off, cols, cols[e], u)) return ORACLE_E_ASYMMETRIC;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Degree ordering (Sec. II; Algorithm GenOrdering's test, Sec. IV).                          */

static uint64_t degree(const uint64_t *off, uint32_t u) { return off[u + 1] - off[u]; }

/* u comes before v in the degree ordering: lower degree first, lower id on equal degree. */
static int degree_before(const uint64_t *off, uint32_t u, uint32_t v)
{
    uint64_t du = degree(off, u), dv = degree(off, v);
    return du < dv || (du == dv && u < v);
}

static const uint64_t *g_sort_off; /* comparator context for qsort (single-threaded use) */

static int cmp_degree_order(const void *a, const void *b)
{
    uint32_t u = *(const uint32_t *)a, v = *(const uint32_t *)b;
    if (u == v) return 0;
    return degree_before(g_sort_off, u, v) ? -1 : 1;
}

/* rank[u] = position of u when all vertices are sorted by (d(u), u); a library sort is the step. */
void oracle_degree_rank(uint32_t n, const uint64_t *off, uint32_t *rank)
{
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t u = 0; u < n; u++) perm[u] = u;
    g_sort_off = off;
    qsort(perm, n, sizeof(uint32_t), cmp_degree_order);
    for (uint32_t i = 0; i < n; i++) rank[perm[i]] = i;
    free(perm);
}

/* Algorithm GenOrdering (Sec. IV): first loop counts kept arcs per vertex, PrefixSum gives the
 * offsets, second loop fills the neighbours in the input's (ascending) order.  The fill loop runs
 * over N(u): the listing's N->(u) there names the list being built (reading noted in the docs). */
void oracle_gen_ordering(uint32_t n, const uint64_t *off, const uint32_t *cols,
                         uint64_t *dag_off, uint32_t *dag_cols)
{
    uint64_t *count = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    for (uint32_t u = 0; u < n; u++)
        for (uint64_t e = off[u]; e < off[u + 1]; e++)
            if (degree_before(off, u, cols[e])) count[u] += 1;
    dag_off[0] = 0;
    for (uint32_t u = 0; u < n; u++) dag_off[u + 1] = dag_off[u] + count[u];
    for (uint32_t u = 0; u < n; u++) {
        uint64_t pos = dag_off[u];
        for (uint64_t e = off[u]; e < off[u + 1]; e++)
            if (degree_before(off, u, cols[e])) dag_cols[pos++] = cols[e];
    }
    free(count);
}

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* DAG of an arbitrary total order given as rank[] (a permutation of 0..n-1): the edge {u,v}
 * becomes u -> v iff rank[u] < rank[v] (Sec. II, directionalizing).  relabel = 0 keeps vertex
 * ids (rows sorted by id); relabel = 1 renames every vertex to its rank, so row r belongs to the
 * vertex of rank r and holds the ranks of its out-neighbours, sorted. */
void oracle_dag_by_rank(uint32_t n, const uint64_t *off, const uint32_t *cols, const uint32_t *rank,
                        int relabel, uint64_t *dag_off, uint32_t *dag_cols)
{
    uint64_t *count = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    for (uint32_t u = 0; u < n; u++) {
        uint32_t row = relabel ? rank[u] : u;
        for (uint64_t e = off[u]; e < off[u + 1]; e++)
            if (rank[u] < rank[cols[e]]) count[row] += 1;
    }
    dag_off[0] = 0;
    for (uint32_t r = 0; r < n; r++) dag_off[r + 1] = dag_off[r] + count[r];
    for (uint32_t u = 0; u < n; u++) {
        uint32_t row = relabel ? rank[u] : u;
        uint64_t pos = dag_off[row];
        for (uint64_t e = off[u]; e < off[u + 1]; e++) {
            uint32_t v = cols[e];
            if (rank[u] < rank[v]) dag_cols[pos++] = relabel ? rank[v] : v;
        }
        if (relabel)
            qsort(dag_cols + dag_off[row], (size_t)(dag_off[row + 1] - dag_off[row]),
                  sizeof(uint32_t), cmp_u32);
    }
    free(count);
}

/* Algorithm OrdCore (Sec. III), Matula-Beck smallest-last: repeatedly take the remaining vertex
 * of smallest remaining degree (smallest id on ties), remove it and lower its neighbours' degrees.
 * rank[u] = the step at which u was removed (0 for the first).  Orienting every edge from the
 * earlier-removed to the later-removed endpoint (rank[u] < rank[v]) gives each vertex exactly the
 * neighbours still present at its removal as out-neighbours, which is what makes the maximum
 * out-degree the smallest possible (the property the paper attributes to this ordering).
 * Plain O(n^2 + m): for the small graphs of the ordering-invariance checks. */
void oracle_core_rank(uint32_t n, const uint64_t *off, const uint32_t *cols, uint32_t *rank)
{
    uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    char *gone = (char *)calloc(n ? n : 1, 1);
    for (uint32_t u = 0; u < n; u++) cur[u] = degree(off, u);
    for (uint32_t step = 0; step < n; step++) {
        uint32_t best = UINT32_MAX;
        for (uint32_t u = 0; u < n; u++)
            if (!gone[u] && (best == UINT32_MAX || cur[u] < cur[best])) best = u;
        rank[best] = step;
        gone[best] = 1;
        for (uint64_t e = off[best]; e < off[best + 1]; e++)
            if (!gone[cols[e]]) cur[cols[e]] -= 1;
    }
    free(cur);
    free(gone);
}

/* Core ordering by synchronous peeling rounds: the parallel form of Algorithm OrdCore that the
 * GPU computes.  level starts at 0; every round first raises level to the smallest remaining
 * degree (it never falls), then removes ALL remaining vertices whose remaining degree is at most
 * level, together, and only then lowers their remaining neighbours' degrees.  rank[u] orders the
 * vertices by (removal round, id).  A vertex's out-neighbours (rank[u] < rank[v]) were all
 * present when its round began, so its out-degree is at most the level of that round, which never
 * exceeds the degeneracy: the maximum out-degree is the degeneracy, as with the sequential order.
 * The final level (the degeneracy) and the number of rounds are returned.  Plain O(rounds * n + m). */
void oracle_core_rank_rounds(uint32_t n, const uint64_t *off, const uint32_t *cols, uint32_t *rank,
                             uint32_t *out_level, uint32_t *out_rounds)
{
    uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    char *gone = (char *)calloc(n ? n : 1, 1);
    char *now = (char *)calloc(n ? n : 1, 1);
    uint64_t level = 0;
    uint32_t removed = 0, rounds = 0;
    for (uint32_t u = 0; u < n; u++) cur[u] = degree(off, u);
    while (removed < n) {
        uint64_t least = UINT64_MAX;
        for (uint32_t u = 0; u < n; u++)
            if (!gone[u] && cur[u] < least) least = cur[u];
        if (least > level) level = least;
        for (uint32_t u = 0; u < n; u++) /* this round's vertices, in id order */
            if (!gone[u] && cur[u] <= level) {
                now[u] = 1;
                rank[u] = removed++;
            }
        for (uint32_t u = 0; u < n; u++)
            if (now[u]) gone[u] = 1;
        for (uint32_t u = 0; u < n; u++)
            if (now[u]) {
                for (uint64_t e = off[u]; e < off[u + 1]; e++)
                    if (!gone[cols[e]]) cur[cols[e]] -= 1;
                now[u] = 0;
            }
        rounds++;
    }
    if (out_level) *out_level = (uint32_t)level;
    if (out_rounds) *out_rounds = rounds;
    free(cur);
    free(gone);
    free(now);
}

/* ------------------------------------------------------------------------------------------ */
/* Counting phase (Sec. III Algorithm "Counting"; Sec. V-B subgraph build and heuristics).    */

typedef struct {
    uint32_t n;
    const uint64_t *off; /* DAG offsets [n+1] */
    const uint32_t *adj; /* DAG out-neighbours, each row sorted ascending */
} dag_t;

/* |A ∩ B| and, when out != NULL, the intersection itself, by a merge of two sorted lists
 * (the intersections of sorted neighbour lists of Sec. V-B). */
static uint32_t intersect(const uint32_t *a, uint32_t na, const uint32_t *b, uint64_t nb,
                          uint32_t *out)
{
    uint32_t i = 0, c = 0;
    uint64_t j = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) i++;
        else if (a[i] > b[j]) j++;
        else {
            if (out) out[c] = a[i];
            c++;
            i++;
            j++;
        }
    }
    return c;
}

/* cnt(C, r): the number of r-cliques of the DAG whose vertices all lie in the candidate list C
 * (the vertex set of the current induced subgraph).
 *   r = 1: every vertex is a 1-clique.
 *   r = 2: the penultimate level only needs subgraph degrees: sum over a in C of |C ∩ N+(a)|.
 *   r > 2: for each a in C build the next subgraph's vertex set C ∩ N+(a) and recurse with r-1.
 *   A candidate list shorter than r cannot hold an r-clique and is skipped (the prune).
 * levels[] holds one buffer per recursion level, each at least as long as the root list.
 * Returns 0, or ORACLE_E_OVERFLOW when a sum leaves uint64. */
static int cnt(const dag_t *g, const uint32_t *C, uint32_t len, int r, uint32_t **levels,
               uint64_t *out)
{
    *out = 0;
    if (len < (uint32_t)r) return ORACLE_OK;
    if (r == 1) {
        *out = len;
        return ORACLE_OK;
    }
    uint64_t total = 0;
    for (uint32_t i = 0; i < len; i++) {
        uint32_t a = C[i];
        const uint32_t *na = g->adj + g->off[a];
        uint64_t da = g->off[a + 1] - g->off[a];
        uint64_t part;
        if (r == 2) {
            part = intersect(C, len, na, da, NULL);
        } else {
            uint32_t *next = levels[0];
            uint32_t len2 = intersect(C, len, na, da, next);
            int st = cnt(g, next, len2, r - 1, levels + 1, &part);
            if (st) return st;
        }
        if (__builtin_add_overflow(total, part, &total)) return ORACLE_E_OVERFLOW;
    }
    *out = total;
    return ORACLE_OK;
}

static uint32_t max_row(const dag_t *g)
{
    uint64_t best = 0;
    for (uint32_t u = 0; u < g->n; u++)
        if (g->off[u + 1] - g->off[u] > best) best = g->off[u + 1] - g->off[u];
    return (uint32_t)best;
}

/* Worker pool: vertex-parallel over roots with a shared counter and task size 1 (Sec. VII-C). */
typedef struct {
    const dag_t *g;
    int k;
    const uint32_t *roots; /* NULL: all vertices */
    uint64_t nroots;
    uint64_t *per_root;    /* optional: count per root */
    atomic_uint_fast64_t next;
    atomic_int status;
    uint32_t width;
    pthread_mutex_t lock;
    uint64_t total;
} pool_t;

static void *worker(void *arg)
{
    pool_t *p = (pool_t *)arg;
    int depth = p->k > 2 ? p->k - 2 : 1;
    uint32_t **levels = (uint32_t **)malloc(sizeof(uint32_t *) * (size_t)depth);
    uint32_t *store = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)p->width + 1) * depth);
    for (int i = 0; i < depth; i++) levels[i] = store + (size_t)i * (p->width + 1);
    uint64_t mine = 0;
    int st = ORACLE_OK;
    for (;;) {
        uint64_t t = atomic_fetch_add(&p->next, 1);
        if (t >= p->nroots || atomic_load(&p->status)) break;
        uint32_t u = p->roots ? p->roots[t] : (uint32_t)t;
        const uint32_t *nu = p->g->adj + p->g->off[u];
        uint32_t du = (uint32_t)(p->g->off[u + 1] - p->g->off[u]);
        uint64_t c;
        st = cnt(p->g, nu, du, p->k - 1, levels, &c);
        if (st) break;
        if (p->per_root) p->per_root[t] = c;
        if (__builtin_add_overflow(mine, c, &mine)) {
            st = ORACLE_E_OVERFLOW;
            break;
        }
    }
    pthread_mutex_lock(&p->lock);
    if (st) atomic_store(&p->status, st);
    else if (__builtin_add_overflow(p->total, mine, &p->total)) atomic_store(&p->status, ORACLE_E_OVERFLOW);
    pthread_mutex_unlock(&p->lock);
    free(store);
    free(levels);
    return NULL;
}

/* Sum over roots u of cnt(N+(u), k-1): every k-clique is counted once, at its first vertex in
 * the DAG order (Sec. II).  k = 1 gives n.  roots == NULL means all vertices. */
static int count_roots(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_adj, int k,
                       const uint32_t *roots, uint64_t nroots, int threads, uint64_t *per_root,
                       uint64_t *out)
{
    *out = 0;
    if (k < 1) return ORACLE_E_ARG;
    if (k == 1) {
        *out = roots ? nroots : n;
        if (per_root)
            for (uint64_t i = 0; i < (roots ? nroots : n); i++) per_root[i] = 1;
        return ORACLE_OK;
    }
    dag_t g = {n, dag_off, dag_adj};
    pool_t p;
    p.g = &g;
    p.k = k;
    p.roots = roots;
    p.nroots = roots ? nroots : n;
    p.per_root = per_root;
    atomic_init(&p.next, 0);
    atomic_init(&p.status, 0);
    p.width = max_row(&g);
    pthread_mutex_init(&p.lock, NULL);
    p.total = 0;
    if (threads < 1) threads = 1;
    if (threads > 512) threads = 512;
    pthread_t tid[512];
    for (int i = 0; i < threads; i++) pthread_create(&tid[i], NULL, worker, &p);
    for (int i = 0; i < threads; i++) pthread_join(tid[i], NULL);
    pthread_mutex_destroy(&p.lock);
    *out = p.total;
    return atomic_load(&p.status);
}

int oracle_count(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_adj, int k, int threads,
                 uint64_t *out)
{
    return count_roots(n, dag_off, dag_adj, k, NULL, 0, threads, NULL, out);
}

int oracle_count_roots(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_adj, int k,
                       const uint32_t *roots, uint64_t nroots, int threads, uint64_t *per_root,
                       uint64_t *out)
{
    return count_roots(n, dag_off, dag_adj, k, roots, nroots, threads, per_root, out);
}

/* Listing instead of counting (Sec. VIII: the counting recursion enumerates each clique once).
 * Every k-clique is written as k DAG ids in recursion order: its first vertex u, then the
 * vertices chosen level by level (for a DAG whose rows are sorted, ascending order along the
 * DAG's order).  The recursion is cnt()'s with the r = 2 shortcut replaced by a walk over the
 * last level's members.  Writes at most `capacity` cliques; *total receives how many exist. */
typedef struct {
    const dag_t *g;
    int k;
    uint32_t *out;
    uint64_t capacity, total;
    uint32_t *prefix;
} lister_t;

static void list_rec(lister_t *L, const uint32_t *C, uint32_t len, int r, uint32_t **levels)
{
    if (len < (uint32_t)r) return;
    int depth = L->k - r; /* vertices already chosen */
    for (uint32_t i = 0; i < len; i++) {
        uint32_t a = C[i];
        L->prefix[depth] = a;
        if (r == 1) {
            if (L->total < L->capacity)
                memcpy(L->out + L->total * (uint64_t)L->k, L->prefix, sizeof(uint32_t) * (size_t)L->k);
            L->total++;
            continue;
        }
        const uint32_t *na = L->g->adj + L->g->off[a];
        uint64_t da = L->g->off[a + 1] - L->g->off[a];
        uint32_t *next = levels[0];
        uint32_t len2 = intersect(C, len, na, da, next);
        list_rec(L, next, len2, r - 1, levels + 1);
    }
}

int oracle_list(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_adj, int k, uint32_t *out,
                uint64_t capacity, uint64_t *total)
{
    *total = 0;
    if (k < 1 || k > 64) return ORACLE_E_ARG;
    dag_t g = {n, dag_off, dag_adj};
    uint32_t width = max_row(&g);
    uint32_t *store = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)width + 1) * (size_t)k);
    uint32_t **levels = (uint32_t **)malloc(sizeof(uint32_t *) * (size_t)k);
    uint32_t prefix[64];
    if (!store || !levels) {
        free(store);
        free(levels);
        return ORACLE_E_NOMEM;
    }
    for (int i = 0; i < k; i++) levels[i] = store + (size_t)i * (width + 1);
    lister_t L = {&g, k, out, capacity, 0, prefix};
    for (uint32_t u = 0; u < n; u++) {
        prefix[0] = u; /* the root; its candidates are N+(u) */
        if (k == 1) {
            if (L.total < capacity) out[L.total] = u;
            L.total++;
            continue;
        }
        list_rec(&L, dag_adj + dag_off[u], (uint32_t)(dag_off[u + 1] - dag_off[u]), k - 1, levels);
    }
    *total = L.total;
    free(store);
    free(levels);
    return ORACLE_OK;
}

/* Edge-level form used to localise differences: for DAG arc e = (u, v), the number of k-cliques
 * whose first two vertices in the DAG order are u then v, i.e. cnt(N+(u) ∩ N+(v), k-2) (k >= 3). */
int oracle_count_per_edge(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_adj, int k,
                          uint64_t *per_edge)
{
    if (k < 3) return ORACLE_E_ARG;
    dag_t g = {n, dag_off, dag_adj};
    uint32_t width = max_row(&g);
    int depth = k - 2;
    uint32_t *store = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)width + 1) * (depth + 1));
    uint32_t **levels = (uint32_t **)malloc(sizeof(uint32_t *) * (size_t)(depth + 1));
    if (!store || !levels) {
        free(store);
        free(levels);
        return ORACLE_E_NOMEM;
    }
    for (int i = 0; i <= depth; i++) levels[i] = store + (size_t)i * (width + 1);
    int st = ORACLE_OK;
    for (uint32_t u = 0; u < n && !st; u++) {
        const uint32_t *nu = dag_adj + dag_off[u];
        uint32_t du = (uint32_t)(dag_off[u + 1] - dag_off[u]);
        for (uint64_t e = dag_off[u]; e < dag_off[u + 1] && !st; e++) {
            uint32_t v = dag_adj[e];
            uint32_t len = intersect(nu, du, dag_adj + dag_off[v], dag_off[v + 1] - dag_off[v],
                                     levels[0]);
            st = cnt(&g, levels[0], len, k - 2, levels + 1, &per_edge[e]);
        }
    }
    free(store);
    free(levels);
    return st;
}

/* The same edge-level form for a listed subset of arcs: per_arc[i] = the number of k-cliques
 * whose first two vertices in the DAG order are the ends (u, v) of DAG arc arcs[i] (k >= 3), and
 * *out their sum.  The row u owning an arc index is found by binary search in dag_off.  One
 * thread; used to time a sample of edge tasks (the units of the edge-parallel form). */
int oracle_count_arcs(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_adj, int k,
                      const uint64_t *arcs, uint64_t narcs, uint64_t *per_arc, uint64_t *out)
{
    *out = 0;
    if (k < 3) return ORACLE_E_ARG;
    dag_t g = {n, dag_off, dag_adj};
    uint32_t width = max_row(&g);
    int depth = k - 2;
    uint32_t *store = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)width + 1) * (depth + 1));
    uint32_t **levels = (uint32_t **)malloc(sizeof(uint32_t *) * (size_t)(depth + 1));
    if (!store || !levels) {
        free(store);
        free(levels);
        return ORACLE_E_NOMEM;
    }
    for (int i = 0; i <= depth; i++) levels[i] = store + (size_t)i * (width + 1);
    int st = ORACLE_OK;
    uint64_t total = 0;
    for (uint64_t i = 0; i < narcs && !st; i++) {
        uint64_t e = arcs[i];
        if (e >= dag_off[n]) {
            st = ORACLE_E_ARG;
            break;
        }
        /* u = the last row with dag_off[u] <= e (rows may be empty) */
        uint32_t lo = 0, hi = n - 1;
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo + 1) / 2;
            if (dag_off[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        uint32_t u = lo, v = dag_adj[e];
        const uint32_t *nu = dag_adj + dag_off[u];
        uint32_t du = (uint32_t)(dag_off[u + 1] - dag_off[u]);
        uint32_t len = intersect(nu, du, dag_adj + dag_off[v], dag_off[v + 1] - dag_off[v], levels[0]);
        uint64_t c;
        st = cnt(&g, levels[0], len, k - 2, levels + 1, &c);
        if (st) break;
        if (per_arc) per_arc[i] = c;
        if (__builtin_add_overflow(total, c, &total)) st = ORACLE_E_OVERFLOW;
    }
    *out = total;
    free(store);
    free(levels);
    return st;
}
