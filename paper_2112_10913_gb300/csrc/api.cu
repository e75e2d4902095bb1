// api.cu -- the C ABI (include/citron.h): argument checks, workspace layout, kernel sequencing,
// error mapping.  Every step of the hot path runs in the kernels of order.cu and count.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "citron.h"
#include "common.cuh"

namespace citron_host {
size_t order_ws_bytes(uint32_t n);
size_t dag_ws_bytes(uint32_t n, uint64_t arcs);
cudaError_t launch_order(uint32_t n, const uint64_t *off, uint32_t *rank, uint32_t *perm,
                         uint32_t *err, Carver &c, cudaStream_t st);
cudaError_t launch_order_grouped(uint32_t n, const uint64_t *off, const uint32_t *group,
                                 uint32_t ngroups, uint32_t *rank, uint32_t *perm, uint32_t *err,
                                 Carver &c, cudaStream_t st);
cudaError_t launch_build_dag(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                             const uint32_t *rank, uint64_t *dag_off, uint32_t *dag_cols,
                             uint32_t *d_max_outdeg, uint32_t *err, Carver &c, cudaStream_t st,
                             int num_sms);
size_t core_ws_bytes(uint32_t n);
size_t list_ws_bytes();
cudaError_t run_list(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_cols, uint32_t k,
                     const uint32_t *map, uint32_t *out, unsigned long long capacity,
                     unsigned long long *h_total, bool *too_wide, uint32_t *err, Carver &c,
                     cudaStream_t st, int num_sms);
cudaError_t launch_core_order(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                              uint32_t *rank, uint32_t *perm, uint32_t *h_level,
                              uint32_t *h_rounds, uint32_t *err, Carver &c, cudaStream_t st,
                              int num_sms);
cudaError_t launch_validate(uint32_t n, uint64_t arcs, const uint64_t *off, const uint32_t *cols,
                            uint32_t *bad, cudaStream_t st, int num_sms);
size_t count_ws_bytes(uint32_t n, uint32_t max_outdeg, int num_sms);
cudaError_t run_count(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_cols, uint32_t k,
                      CountRun &run, uint32_t *err, Carver &c, cudaStream_t s, int num_sms,
                      unsigned long long *h_result);

static std::atomic<unsigned long long> g_launches{0};
void note_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }

static std::mutex g_fault_mutex;
static citron_faults g_faults = {};
citron_faults injected_faults()
{
    std::lock_guard<std::mutex> lock(g_fault_mutex);
    return g_faults;
}
cudaError_t seed_totals(unsigned long long *p, uint32_t count, cudaStream_t s);
cudaError_t launch_dag_append(uint32_t n, const uint64_t *src_off, const uint32_t *src_cols,
                              uint32_t src_row, uint64_t *dst_off, uint32_t *dst_cols,
                              uint32_t dst_row, uint64_t dst_arc, cudaStream_t s);
cudaError_t launch_per_root_trivial(uint32_t n, const uint64_t *dag_off, uint32_t k,
                                    unsigned long long *per_root, cudaStream_t s);
cudaError_t run_count_async(uint32_t n, const uint64_t *dag_off, const uint32_t *dag_cols, uint32_t k,
                            uint32_t max_outdeg, CountRun &run, uint32_t *err, Carver &c,
                            cudaStream_t s, int num_sms);
cudaError_t launch_batch_rows(uint32_t n, const uint32_t *rank, const uint32_t *group_of_vertex,
                              uint32_t *group_of_row, uint32_t *err, cudaStream_t s);
cudaError_t launch_batch_trivial(uint32_t n, const uint64_t *dag_off, const uint32_t *group_of_row,
                                 const uint32_t *group_k, uint32_t ngroups,
                                 unsigned long long *counts, uint32_t *err, cudaStream_t s);
}  // namespace citron_host

using namespace citron_host;

namespace {

// Workspace header: [0] device error word, [1] validation code, [2] max out-degree, rest unused.
constexpr size_t kHeader = 256;

int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 132;
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 132;
        cache[dev] = v;
    }
    return cache[dev];
}

uint32_t *err_word(void *ws) { return (uint32_t *)ws; }

thread_local const char *t_last_cuda_error = "none";

citron_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return CITRON_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return CITRON_E_WORKSPACE;
    }
    t_last_cuda_error = cudaGetErrorName(e);
    return CITRON_E_CUDA;
}

citron_status from_device(uint32_t code)
{
    switch (code) {
        case citron::kDevOk: return CITRON_OK;
        case citron::kDevTimeout: return CITRON_E_TIMEOUT;
        case citron::kDevOverflow: return CITRON_E_OVERFLOW;
        case citron::kDevTooLong: return CITRON_E_UNSUPPORTED;
        case citron::kDevBadInput: return CITRON_E_INVALID;
        case citron::kDevScratch: return CITRON_E_WORKSPACE;
        case citron::kDevBudget: return CITRON_E_BUDGET;
        default: return CITRON_E_CUDA;
    }
}

bool ws_ok(void *ws, size_t bytes, size_t need)
{
    return ws && ((uintptr_t)ws % 256) == 0 && bytes >= need;
}

// Synchronous calls report (and then clear) the device error word, including errors left by
// earlier asynchronous calls on the same workspace.
citron_status finish_sync(void *ws, cudaStream_t s, citron_status st)
{
    uint32_t code = 0;
    cudaError_t e = cudaMemcpyAsync(&code, err_word(ws), sizeof(code), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return CITRON_E_CUDA;
    if (code) {
        cudaMemsetAsync(err_word(ws), 0, sizeof(uint32_t), s);
        cudaStreamSynchronize(s);
        if (st == CITRON_OK) st = from_device(code);
    }
    return st;
}

}  // namespace

extern "C" {

const char *citron_status_str(citron_status s)
{
    switch (s) {
        case CITRON_OK: return "ok";
        case CITRON_E_INVALID: return "invalid argument or input";
        case CITRON_E_WORKSPACE: return "workspace missing, misaligned or too small";
        case CITRON_E_CUDA: return "CUDA runtime error";
        case CITRON_E_OVERFLOW: return "count exceeds uint64";
        case CITRON_E_TIMEOUT: return "bounded device wait gave up";
        case CITRON_E_UNSUPPORTED: return "input exceeds a size limit of this build";
        case CITRON_E_BUDGET: return "time budget ran out before the count finished";
    }
    return "unknown status";
}

int citron_version(void) { return 200; }

const char *citron_last_cuda_error(void) { return t_last_cuda_error; }

static bool plan_from_opts(const citron_count_opts *opts, CountPlan &plan)
{
    if (!opts) return true;
    if (opts->small_max > 32 || opts->bitmap_max > 1024 || opts->warps_per_cta > 32) return false;
    if (opts->compact_max != 0 && opts->compact_max != 1 && opts->compact_max != 128) return false;
    if (opts->small_max) plan.small_max = opts->small_max;
    if (opts->bitmap_max) plan.bitmap_max = opts->bitmap_max;
    if (opts->warps_per_cta) plan.warps_per_cta = opts->warps_per_cta;
    if (opts->compact_max) plan.compact_max = opts->compact_max == 1 ? 0 : opts->compact_max;
    if (opts->split_min) plan.split_min = opts->split_min == 1 ? 0xffffffffu : opts->split_min;
    plan.max_blocks = opts->max_blocks;
    if (plan.bitmap_max < plan.small_max) plan.bitmap_max = plan.small_max;
    return true;
}

size_t citron_workspace_bytes(uint32_t n, uint64_t arcs, uint32_t max_outdeg)
{
    if (max_outdeg == 0) {
        uint64_t b = arcs / 2;
        if (n && b > (uint64_t)n - 1) b = (uint64_t)n - 1;
        max_outdeg = (uint32_t)(b > 0xffffffffull ? 0xffffffffull : b);
    }
    size_t need = order_ws_bytes(n);
    size_t d = dag_ws_bytes(n, arcs);
    if (d > need) need = d;
    d = core_ws_bytes(n);
    if (d > need) need = d;
    size_t c = count_ws_bytes(n, max_outdeg, sm_count()) + (((size_t)n + 1) * 4 + 255) / 256 * 256;
    if (c > need) need = c;
    return kHeader + need;
}

citron_status citron_validate(uint32_t n, uint64_t arcs, const uint64_t *d_off,
                              const uint32_t *d_cols, uint32_t *h_bad, void *ws, size_t ws_bytes,
                              void *stream)
{
    if (n == 0xffffffffu || !d_off || (arcs && !d_cols)) return CITRON_E_INVALID;
    if (!ws_ok(ws, ws_bytes, kHeader)) return CITRON_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *bad = err_word(ws) + 1;
    cudaError_t e = cudaMemsetAsync(bad, 0xff, sizeof(uint32_t), s);
    if (!e) e = launch_validate(n, arcs, d_off, d_cols, bad, s, sm_count());
    uint32_t code = 0xffffffffu;
    if (!e) e = cudaMemcpyAsync(&code, bad, sizeof(code), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return from_cuda(e);
    if (h_bad) *h_bad = code == 0xffffffffu ? 0 : code;
    return code == 0xffffffffu ? CITRON_OK : CITRON_E_INVALID;
}

citron_status citron_order(uint32_t n, const uint64_t *d_off, uint32_t *d_rank, uint32_t *d_perm,
                           void *ws, size_t ws_bytes, void *stream)
{
    if (n == 0xffffffffu || !d_off || (n && !d_rank)) return CITRON_E_INVALID;
    if (!ws_ok(ws, ws_bytes, kHeader + order_ws_bytes(n))) return CITRON_E_WORKSPACE;
    Carver c((char *)ws + kHeader, ws_bytes - kHeader);
    return from_cuda(launch_order(n, d_off, d_rank, d_perm, err_word(ws), c, (cudaStream_t)stream));
}

citron_status citron_order_grouped(uint32_t n, const uint64_t *d_off, const uint32_t *d_group,
                                   uint32_t ngroups, uint32_t *d_rank, uint32_t *d_perm, void *ws,
                                   size_t ws_bytes, void *stream)
{
    if (n == 0xffffffffu || !d_off || (n && (!d_rank || !d_group))) return CITRON_E_INVALID;
    if (!ws_ok(ws, ws_bytes, kHeader + order_ws_bytes(n))) return CITRON_E_WORKSPACE;
    Carver c((char *)ws + kHeader, ws_bytes - kHeader);
    return from_cuda(launch_order_grouped(n, d_off, d_group, ngroups, d_rank, d_perm, err_word(ws), c,
                                          (cudaStream_t)stream));
}

citron_status citron_core_order(uint32_t n, uint64_t arcs, const uint64_t *d_off,
                                const uint32_t *d_cols, uint32_t *d_rank, uint32_t *d_perm,
                                uint32_t *h_degeneracy, uint32_t *h_rounds, void *ws,
                                size_t ws_bytes, void *stream)
{
    if (n == 0xffffffffu || !d_off || (n && !d_rank) || (arcs && !d_cols) || (arcs & 1))
        return CITRON_E_INVALID;
    if (!ws_ok(ws, ws_bytes, kHeader + core_ws_bytes(n))) return CITRON_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Carver c((char *)ws + kHeader, ws_bytes - kHeader);
    cudaError_t e = launch_core_order(n, arcs, d_off, d_cols, d_rank, d_perm, h_degeneracy, h_rounds,
                                      err_word(ws), c, s, sm_count());
    if (e == cudaErrorNotSupported) {
        cudaGetLastError();
        return CITRON_E_UNSUPPORTED;
    }
    if (e) return from_cuda(e);
    return finish_sync(ws, s, CITRON_OK);
}

citron_status citron_build_dag(uint32_t n, uint64_t arcs, const uint64_t *d_off,
                               const uint32_t *d_cols, const uint32_t *d_rank,
                               uint64_t *d_dag_off, uint32_t *d_dag_cols, uint32_t *h_max_outdeg,
                               void *ws, size_t ws_bytes, void *stream)
{
    if (n == 0xffffffffu || !d_off || !d_dag_off || (arcs && (!d_cols || !d_dag_cols)) ||
        (arcs & 1))
        return CITRON_E_INVALID;
    if (!ws_ok(ws, ws_bytes, kHeader + dag_ws_bytes(n, arcs))) return CITRON_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *d_max = h_max_outdeg ? err_word(ws) + 2 : nullptr;
    cudaError_t e = cudaSuccess;
    if (d_max) e = cudaMemsetAsync(d_max, 0, sizeof(uint32_t), s);
    Carver c((char *)ws + kHeader, ws_bytes - kHeader);
    if (!e)
        e = launch_build_dag(n, arcs, d_off, d_cols, d_rank, d_dag_off, d_dag_cols, d_max,
                             err_word(ws), c, s, sm_count());
    if (e) return from_cuda(e);
    if (!h_max_outdeg) return CITRON_OK;
    e = cudaMemcpyAsync(h_max_outdeg, d_max, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e) return from_cuda(e);
    return finish_sync(ws, s, CITRON_OK);
}

citron_status citron_count_ex(uint32_t n, const uint64_t *d_dag_off, const uint32_t *d_dag_cols,
                              uint32_t k, uint32_t max_outdeg, citron_count_opts *opts,
                              uint64_t *h_count, void *ws, size_t ws_bytes, void *stream)
{
    (void)max_outdeg;  // the count derives every size it needs from the DAG itself
    if (!h_count || !opts || !d_dag_off || n == 0xffffffffu || k == 0) return CITRON_E_INVALID;
    if (k > CITRON_MAX_K) return CITRON_E_UNSUPPORTED;
    CountRun run;
    if (!plan_from_opts(opts, run.plan)) return CITRON_E_INVALID;
    run.sink.per_root = (unsigned long long *)opts->d_per_root;
    run.sink.per_arc = (unsigned long long *)opts->d_per_arc;
    if (run.sink.per_arc && k < 3) return CITRON_E_INVALID;
    run.time_kernels = (opts->flags & CITRON_COUNT_TIME_KERNELS) != 0;
    run.count_work = (opts->flags & CITRON_COUNT_WORK) != 0;
    if ((run.count_work || run.sink.per_arc) && k > kInstrumentedMaxK) return CITRON_E_UNSUPPORTED;
    run.balance = (opts->flags & CITRON_COUNT_BALANCE) != 0;
    run.budget_ns = (unsigned long long)opts->budget_ms * 1000000ull;
    opts->work_ops = 0;
    opts->kernel_ms[0] = opts->kernel_ms[1] = opts->kernel_ms[2] = 0.f;
    opts->busy_ms[0] = opts->busy_ms[1] = 0.f;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ws_ok(ws, ws_bytes, kHeader)) return CITRON_E_WORKSPACE;
    if (k <= 2) {
        cudaError_t e = cudaSuccess;
        if (k == 1) {
            *h_count = n;
        } else {
            uint64_t m = 0;
            e = cudaMemcpyAsync(&m, d_dag_off + n, sizeof(m), cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaStreamSynchronize(s);
            *h_count = m;
        }
        if (!e && run.sink.per_root)
            e = launch_per_root_trivial(n, d_dag_off, k, run.sink.per_root, s);
        if (e) return from_cuda(e);
        return finish_sync(ws, s, CITRON_OK);
    }
    if (n && !d_dag_cols) return CITRON_E_INVALID;
    Carver c((char *)ws + kHeader, ws_bytes - kHeader);
    unsigned long long result = 0;
    cudaError_t e = run_count(n, d_dag_off, d_dag_cols, k, run, err_word(ws), c, s, sm_count(),
                              &result);
    if (e) return from_cuda(e);
    citron_status st = finish_sync(ws, s, CITRON_OK);
    if (st == CITRON_OK) *h_count = result;
    opts->work_ops = run.work;
    for (int i = 0; i < 3; i++) opts->kernel_ms[i] = run.kernel_ms[i];
    opts->busy_ms[0] = run.busy_ms[0];
    opts->busy_ms[1] = run.busy_ms[1];
    return st;
}

citron_status citron_list(uint32_t n, const uint64_t *d_dag_off, const uint32_t *d_dag_cols,
                          uint32_t k, const uint32_t *d_map, uint32_t *d_out, uint64_t capacity,
                          uint64_t *h_total, void *ws, size_t ws_bytes, void *stream)
{
    if (!h_total || !d_dag_off || n == 0xffffffffu || k == 0 || (capacity && !d_out) ||
        (k >= 2 && n && !d_dag_cols))
        return CITRON_E_INVALID;
    if (k > CITRON_MAX_K) return CITRON_E_UNSUPPORTED;
    if (!ws_ok(ws, ws_bytes, kHeader + list_ws_bytes())) return CITRON_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Carver c((char *)ws + kHeader, ws_bytes - kHeader);
    unsigned long long total = 0;
    bool too_wide = false;
    cudaError_t e = run_list(n, d_dag_off, d_dag_cols, k, d_map, d_out, capacity, &total, &too_wide,
                             err_word(ws), c, s, sm_count());
    if (e) return from_cuda(e);
    citron_status st = finish_sync(ws, s, too_wide ? CITRON_E_UNSUPPORTED : CITRON_OK);
    if (st == CITRON_OK) *h_total = total;
    return st;
}

citron_status citron_count(uint32_t n, const uint64_t *d_dag_off, const uint32_t *d_dag_cols,
                           uint32_t k, uint32_t max_outdeg, uint64_t *h_count,
                           uint64_t *d_per_root, void *ws, size_t ws_bytes, void *stream)
{
    citron_count_opts o = {};
    o.d_per_root = d_per_root;
    return citron_count_ex(n, d_dag_off, d_dag_cols, k, max_outdeg, &o, h_count, ws, ws_bytes,
                           stream);
}

uint64_t citron_kernel_launches(void) { return launches(); }

citron_status citron_count_batch(uint32_t n, const uint64_t *d_dag_off, const uint32_t *d_dag_cols,
                                 const uint32_t *d_rank, const uint32_t *d_group_of_vertex,
                                 const uint32_t *d_group_k, uint32_t ngroups, uint32_t kmask,
                                 uint32_t max_outdeg, const citron_count_opts *opts,
                                 uint64_t *d_counts, void *ws, size_t ws_bytes, void *stream)
{
    if (n == 0xffffffffu || !d_dag_off || (n && (!d_dag_cols || !d_group_of_vertex)) ||
        (ngroups && (!d_group_k || !d_counts)))
        return CITRON_E_INVALID;
    if (kmask & ~(((2u << CITRON_MAX_K) - 1) & ~1u)) return CITRON_E_UNSUPPORTED;
    CountPlan plan;
    if (!plan_from_opts(opts, plan)) return CITRON_E_INVALID;
    if (!ws_ok(ws, ws_bytes, kHeader)) return CITRON_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    Carver c((char *)ws + kHeader, ws_bytes - kHeader);
    uint32_t *group_of_row = c.take<uint32_t>((size_t)n + 1);
    if (!c.ok) return CITRON_E_WORKSPACE;
    unsigned long long *counts = (unsigned long long *)d_counts;
    cudaError_t e = ngroups ? cudaMemsetAsync(counts, 0, (size_t)ngroups * 8, s) : cudaSuccess;
    if (!e) e = seed_totals(counts, ngroups, s);
    const uint32_t *gor = d_group_of_vertex;
    if (!e && d_rank) {
        e = launch_batch_rows(n, d_rank, d_group_of_vertex, group_of_row, err_word(ws), s);
        gor = group_of_row;
    }
    if (!e && (kmask & 6u))
        e = launch_batch_trivial(n, d_dag_off, gor, d_group_k, ngroups, counts, err_word(ws), s);
    for (uint32_t k = 3; !e && k <= CITRON_MAX_K; k++) {
        if (!((kmask >> k) & 1)) continue;
        CountRun run;
        run.plan = plan;
        run.filter.group_of_row = gor;
        run.filter.group_k = d_group_k;
        run.filter.ngroups = ngroups;
        run.filter.k = k;
        run.sink.group_of_row = gor;
        run.sink.group_counts = counts;
        run.sink.ngroups = ngroups;
        Carver cc = c;  // every pass reuses the same regions (stream-ordered)
        e = run_count_async(n, d_dag_off, d_dag_cols, k, max_outdeg, run, err_word(ws), cc, s,
                            sm_count());
    }
    return from_cuda(e);
}

citron_status citron_dag_append(uint32_t n, const uint64_t *d_src_off, const uint32_t *d_src_cols,
                                uint32_t src_row, uint64_t *d_dst_off, uint32_t *d_dst_cols,
                                uint32_t dst_row, uint64_t dst_arc, void *stream)
{
    if (!d_src_off || !d_dst_off || (n && (!d_src_cols || !d_dst_cols))) return CITRON_E_INVALID;
    return from_cuda(launch_dag_append(n, d_src_off, d_src_cols, src_row, d_dst_off, d_dst_cols,
                                       dst_row, dst_arc, (cudaStream_t)stream));
}

citron_status citron_set_faults(const citron_faults *faults)
{
    std::lock_guard<std::mutex> lock(g_fault_mutex);
    g_faults = faults ? *faults : citron_faults{};
    return CITRON_OK;
}

citron_status citron_workspace_status(void *ws, void *stream)
{
    if (!ws) return CITRON_E_WORKSPACE;
    return finish_sync(ws, (cudaStream_t)stream, CITRON_OK);
}

size_t citron_host_buffer_bytes(uint32_t n, uint64_t arcs)
{
    Sizer z;
    z.take<uint64_t>((size_t)n + 1);  // off
    z.take<uint32_t>(arcs + 1);       // cols
    z.take<uint32_t>((size_t)n + 1);  // rank
    z.take<uint64_t>((size_t)n + 1);  // dag_off
    z.take<uint32_t>(arcs / 2 + 1);   // dag_cols
    return z.used;
}

citron_status citron_count_host(uint32_t n, uint64_t arcs, const uint64_t *h_off,
                                const uint32_t *h_cols, const uint32_t *h_ks, uint32_t nk,
                                uint64_t *h_counts, void *d_buf, size_t buf_bytes, void *ws,
                                size_t ws_bytes, void *stream)
{
    if (n == 0xffffffffu || !h_off || (arcs && !h_cols) || (nk && (!h_ks || !h_counts)))
        return CITRON_E_INVALID;
    if (!d_buf || buf_bytes < citron_host_buffer_bytes(n, arcs)) return CITRON_E_WORKSPACE;
    Carver b(d_buf, buf_bytes);
    uint64_t *off = b.take<uint64_t>((size_t)n + 1);
    uint32_t *cols = b.take<uint32_t>(arcs + 1);
    uint32_t *rank = b.take<uint32_t>((size_t)n + 1);
    uint64_t *dag_off = b.take<uint64_t>((size_t)n + 1);
    uint32_t *dag_cols = b.take<uint32_t>(arcs / 2 + 1);
    if (!b.ok) return CITRON_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(off, h_off, ((size_t)n + 1) * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, s);
    if (!e && arcs) e = cudaMemcpyAsync(cols, h_cols, arcs * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e) return from_cuda(e);
    citron_status st = citron_order(n, off, rank, nullptr, ws, ws_bytes, stream);
    if (st) return st;
    uint32_t max_outdeg = 0;
    st = citron_build_dag(n, arcs, off, cols, rank, dag_off, dag_cols, &max_outdeg, ws, ws_bytes,
                          stream);
    if (st) return st;
    for (uint32_t i = 0; i < nk; i++) {
        st = citron_count(n, dag_off, dag_cols, h_ks[i], max_outdeg, &h_counts[i], nullptr, ws,
                          ws_bytes, stream);
        if (st) return st;
    }
    return CITRON_OK;
}

}  // extern "C"
