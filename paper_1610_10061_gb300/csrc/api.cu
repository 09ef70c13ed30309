// C ABI: instances, population evaluation, status strings (include/pm.h).

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "pm_alloc.h"
#include "pm_common.cuh"

void pm_note_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    static const bool verbose = std::getenv("PM_VERBOSE") != nullptr;
    if (verbose)
        std::fprintf(stderr, "libpmgpu: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
}

// Injected allocation failure (pm_debug_fail_alloc): the number of allocations still to succeed before one
// fails, or -1 when none is armed.
static std::atomic<long long> g_fail_after{-1};

static bool injected_failure()
{
    long long k = g_fail_after.load();
    while (k >= 0) {
        if (g_fail_after.compare_exchange_weak(k, k - 1))
            return k == 0;  // this allocation is the one that fails; the counter is now -1 (disarmed)
    }
    return false;
}

// The library's device memory comes from one memory pool per device, which keeps up to kPoolKeepBytes of
// released memory mapped for the next allocations: cudaMalloc and cudaFree cost tens of microseconds each on
// GB300, a pool allocation or release a few.  Memory above that amount goes back to the driver at the next
// synchronisation.  A device without memory pools falls back to cudaMalloc / cudaFree.
constexpr size_t kPoolKeepBytes = (size_t)256 << 20;
constexpr int kMaxDevices = 64;

namespace {
struct DevicePool {
    bool tried = false;
    cudaMemPool_t pool = nullptr;  // null: this device allocates with cudaMalloc
    cudaStream_t stream = nullptr;  // allocations and releases of pm_dbuf memory are ordered on it
};
std::mutex g_pool_mu;
DevicePool g_pools[kMaxDevices];
}  // namespace

// The current device's pool (created on first use; never destroyed: it lives as long as the process).
static DevicePool *device_pool()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(g_pool_mu);
    DevicePool &dp = g_pools[dev];
    if (!dp.tried) {
        dp.tried = true;
        int supported = 0;
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        cudaStream_t st = nullptr;
        uint64_t keep = kPoolKeepBytes;
        const char *env = std::getenv("PM_POOL");  // PM_POOL=0: cudaMalloc / cudaFree (for comparison)
        bool ok = !(env && env[0] == '0') &&
                  cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev) == cudaSuccess &&
                  supported && cudaMemPoolCreate(&pool, &props) == cudaSuccess;
        ok = ok && cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) {
            dp.pool = pool;
            dp.stream = st;
        } else {
            if (st)
                (void)cudaStreamDestroy(st);
            if (pool)
                (void)cudaMemPoolDestroy(pool);
            (void)cudaGetLastError();
        }
    }
    return &dp;
}

cudaError_t pm_device_malloc(void **ptr, size_t bytes)
{
    if (injected_failure()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    DevicePool *dp = device_pool();
    if (!dp || !dp->pool)
        return cudaMalloc(ptr, bytes);
    // ordered on the pool's stream, then waited for: the memory is ready for any stream, as cudaMalloc's is
    cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, dp->pool, dp->stream);
    if (e != cudaSuccess)
        return e;
    e = cudaStreamSynchronize(dp->stream);
    if (e != cudaSuccess) {
        (void)cudaFreeAsync(*ptr, dp->stream);
        *ptr = nullptr;
    }
    return e;
}

void pm_device_free(void *ptr)
{
    if (!ptr)
        return;
    int cur = 0, dev = 0;
    cudaPointerAttributes a;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    dev = a.device;
    if (dev != cur && cudaSetDevice(dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    DevicePool *dp = device_pool();
    if (!dp || !dp->pool) {
        pm_clear_error(cudaFree(ptr));
    } else {
        // as cudaFree does, wait for every launch that may still use the memory, then return it to the pool
        pm_clear_error(cudaDeviceSynchronize());
        pm_clear_error(cudaFreeAsync(ptr, dp->stream));
    }
    if (dev != cur)
        pm_clear_error(cudaSetDevice(cur));
}

cudaError_t pm_device_malloc_async(void **ptr, size_t bytes, cudaStream_t s)
{
    if (injected_failure()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    DevicePool *dp = device_pool();
    if (!dp || !dp->pool)
        return cudaMallocAsync(ptr, bytes, s);
    return cudaMallocFromPoolAsync(ptr, bytes, dp->pool, s);
}

extern "C" pm_status pm_debug_fail_alloc(int64_t after, int64_t *pending)
{
    const long long prev = g_fail_after.exchange(after < 0 ? -1 : (long long)after);
    if (pending)
        *pending = (int64_t)prev;
    return PM_OK;
}

pm_status pm_dbuf::reserve(size_t want, bool *fresh)
{
    if (fresh)
        *fresh = false;
    if (want <= bytes && ptr)
        return PM_OK;
    release();
    size_t sz = want < 256 ? 256 : want;
    cudaError_t e = pm_device_malloc(&ptr, sz);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        pm_note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        return e == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;
    }
    bytes = sz;
    if (fresh)
        *fresh = true;
    return PM_OK;
}

void pm_dbuf::release()
{
    if (ptr && !borrowed)
        pm_device_free(ptr);
    ptr = nullptr;
    bytes = 0;
    borrowed = false;
}

pm_status pm_carve(pm_dbuf &arena, const pm_part *parts, int count)
{
    size_t total = 0;
    for (int k = 0; k < count; ++k) {
        parts[k].buf->release();
        total += (std::max<size_t>(parts[k].bytes, 256) + 255) & ~size_t(255);
    }
    arena.release();
    PM_TRY(arena.reserve(total));
    char *base = static_cast<char *>(arena.ptr);
    size_t off = 0;
    for (int k = 0; k < count; ++k) {
        const size_t sz = std::max<size_t>(parts[k].bytes, 256);
        parts[k].buf->ptr = base + off;
        parts[k].buf->bytes = sz;
        parts[k].buf->borrowed = true;
        off += (sz + 255) & ~size_t(255);
    }
    return PM_OK;
}

bool pm_is_device_ptr(const void *p)
{
    if (!p)
        return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" const char *pm_strerror(pm_status s)
{
    switch (s) {
    case PM_OK:
        return "PM_OK";
    case PM_ERR_INVALID_ARG:
        return "PM_ERR_INVALID_ARG: argument out of range";
    case PM_ERR_NEGATIVE_DIST:
        return "PM_ERR_NEGATIVE_DIST: the distance matrix has a negative entry";
    case PM_ERR_UNSUPPORTED:
        return "PM_ERR_UNSUPPORTED: m exceeds 65535";
    case PM_ERR_MASK:
        return "PM_ERR_MASK: a bitset does not have exactly p open facilities";
    case PM_ERR_CUDA:
        return "PM_ERR_CUDA: a CUDA runtime call failed";
    case PM_ERR_OOM:
        return "PM_ERR_OOM: out of memory";
    case PM_ERR_TIMEOUT:
        return "PM_ERR_TIMEOUT: a bounded device wait gave up";
    }
    return "unknown pm_status";
}

static void destroy_instance(pm_instance *inst)
{
    if (!inst)
        return;
    pm_clear_error(cudaSetDevice(inst->device));
    inst->stage_masks.release();
    inst->stage_costs.release();
    inst->partials.release();
    inst->tickets.release();
    inst->columns.release();
    inst->flag.release();
    inst->err.release();
    inst->tab_arena.release();  // the tables, err and flag
    inst->dsorted.release();
    delete inst;
}

static pm_status create_impl(const int32_t *d, int64_t n, int64_t m, int64_t p, int device, cudaStream_t stream,
                             pm_instance *inst)
{
    PM_CUDA(cudaSetDevice(device));
    inst->device = device;
    inst->n = n;
    inst->m = m;
    inst->p = p;
    inst->L = m - p + 1;
    inst->W = pm_ceil_div(m, 32);
    inst->stride = pm_round_up(inst->L, 32);
    int v = 0;
    PM_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device));
    inst->sm_count = v;
    PM_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    inst->smem_optin = (size_t)v;
    const size_t tab = (size_t)n * (size_t)inst->stride;
    pm_dbuf dbuf, pbuf;
    const pm_part parts[] = {{&inst->err, 256}, {&inst->flag, 256}, {&dbuf, tab * sizeof(int32_t)},
                             {&pbuf, tab * sizeof(uint16_t)}};
    PM_TRY(pm_carve(inst->tab_arena, parts, 4));
    inst->delta = static_cast<int32_t *>(dbuf.ptr);
    inst->pi = static_cast<uint16_t *>(pbuf.ptr);
    PM_CUDA(cudaMemsetAsync(inst->err.ptr, 0, 256, stream));
    PM_TRY(pm_fitness_init(inst));
    const int32_t *d_dev = d;
    int32_t *tmp = nullptr;
    if (!pm_is_device_ptr(d)) {
        const size_t bytes = (size_t)n * (size_t)m * sizeof(int32_t);
        PM_CUDA(pm_device_malloc_async(reinterpret_cast<void **>(&tmp), bytes, stream));
        cudaError_t e = cudaMemcpyAsync(tmp, d, bytes, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(tmp, stream);
            PM_CUDA(e);
        }
        d_dev = tmp;
    }
    pm_status st = pm_build_tables(inst, d_dev, stream);
    if (tmp)
        cudaFreeAsync(tmp, stream);
    PM_TRY(st);
    PM_CUDA(cudaStreamSynchronize(stream));
    return PM_OK;
}

extern "C" pm_status pm_instance_create_ex(const int32_t *d, int64_t n, int64_t m, int64_t p, int device,
                                           void *stream, uint32_t flags, pm_instance **out)
{
    if (!out)
        return PM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d || n < 1 || m < 2 || p < 1 || p >= m || device < 0 || (flags & ~PM_TABLES_CUMULATIVE) != 0)
        return PM_ERR_INVALID_ARG;
    if (m > 65535)
        return PM_ERR_UNSUPPORTED;
    if (n > ((int64_t)1 << 40) / m)
        return PM_ERR_INVALID_ARG;
    pm_instance *inst = new (std::nothrow) pm_instance();
    if (!inst)
        return PM_ERR_OOM;
    inst->cum = (flags & PM_TABLES_CUMULATIVE) != 0;
    pm_status st = create_impl(d, n, m, p, device, static_cast<cudaStream_t>(stream), inst);
    if (st != PM_OK) {
        destroy_instance(inst);
        return st;
    }
    *out = inst;
    return PM_OK;
}

extern "C" pm_status pm_instance_create(const int32_t *d, int64_t n, int64_t m, int64_t p, int device, void *stream,
                                        pm_instance **out)
{
    return pm_instance_create_ex(d, n, m, p, device, stream, 0u, out);
}

extern "C" pm_status pm_instance_flags(const pm_instance *inst, uint32_t *flags)
{
    if (!inst || !flags)
        return PM_ERR_INVALID_ARG;
    *flags = inst->cum ? PM_TABLES_CUMULATIVE : 0u;
    return PM_OK;
}

extern "C" pm_status pm_instance_destroy(pm_instance *inst)
{
    destroy_instance(inst);
    return PM_OK;
}

extern "C" pm_status pm_instance_info(const pm_instance *inst, int64_t *n, int64_t *m, int64_t *p, int64_t *L,
                                      int64_t *W, int64_t *row_stride)
{
    if (!inst)
        return PM_ERR_INVALID_ARG;
    if (n)
        *n = inst->n;
    if (m)
        *m = inst->m;
    if (p)
        *p = inst->p;
    if (L)
        *L = inst->L;
    if (W)
        *W = inst->W;
    if (row_stride)
        *row_stride = inst->stride;
    return PM_OK;
}

extern "C" pm_status pm_instance_tables(const pm_instance *inst, uint16_t *pi_out, int32_t *delta_out, void *stream)
{
    if (!inst || (!pi_out && !delta_out))
        return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(inst->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (pi_out)
        PM_CUDA(cudaMemcpy2DAsync(pi_out, inst->L * sizeof(uint16_t), inst->pi, inst->stride * sizeof(uint16_t),
                                  inst->L * sizeof(uint16_t), inst->n, cudaMemcpyDefault, s));
    if (delta_out && !inst->cum)
        PM_CUDA(cudaMemcpy2DAsync(delta_out, inst->L * sizeof(int32_t), inst->delta, inst->stride * sizeof(int32_t),
                                  inst->L * sizeof(int32_t), inst->n, cudaMemcpyDefault, s));
    if (delta_out && inst->cum) {
        // the instance holds D': its consecutive differences are Delta'
        const size_t bytes = (size_t)inst->n * (size_t)inst->L * sizeof(int32_t);
        if (pm_is_device_ptr(delta_out)) {
            PM_TRY(pm_launch_increments(inst, delta_out, s));
        } else {
            int32_t *tmp = nullptr;
            PM_CUDA(pm_device_malloc_async(reinterpret_cast<void **>(&tmp), bytes, s));
            pm_status st = pm_launch_increments(inst, tmp, s);
            cudaError_t e = st == PM_OK ? cudaMemcpyAsync(delta_out, tmp, bytes, cudaMemcpyDeviceToHost, s)
                                        : cudaSuccess;
            cudaFreeAsync(tmp, s);
            PM_TRY(st);
            PM_CUDA(e);
        }
    }
    PM_CUDA(cudaStreamSynchronize(s));
    return PM_OK;
}

extern "C" pm_status pm_columns_layout(pm_instance *inst, int64_t pop, int32_t *groups, int64_t *words)
{
    if (!inst || pop < 1)
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(inst->lock);
    const pm_eval_plan plan = pm_plan_eval(inst, pop);
    if (groups)
        *groups = plan.groups;
    if (words)
        *words = plan.groups ? (int64_t)(pm_plan_column_bytes(inst, plan) / 4) : 0;
    return plan.groups ? PM_OK : PM_ERR_UNSUPPORTED;
}

extern "C" pm_status pm_population_columns(pm_instance *inst, const uint32_t *masks, int64_t pop, uint32_t *cols,
                                           void *stream)
{
    pm_clear_stale_error();
    if (!inst || pop < 1 || !masks || !cols || !pm_is_device_ptr(masks) || !pm_is_device_ptr(cols))
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(inst->lock);
    PM_CUDA(cudaSetDevice(inst->device));
    return pm_launch_columns(inst, pm_plan_eval(inst, pop), masks, pop, cols, static_cast<cudaStream_t>(stream));
}

extern "C" pm_status pm_eval_columns(pm_instance *inst, const uint32_t *cols, int64_t pop, int64_t *costs,
                                     void *stream)
{
    pm_clear_stale_error();
    if (!inst || pop < 1 || !cols || !costs || !pm_is_device_ptr(cols) || !pm_is_device_ptr(costs))
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(inst->lock);
    PM_CUDA(cudaSetDevice(inst->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const pm_eval_plan plan = pm_plan_eval(inst, pop);
    if (!plan.groups)
        return PM_ERR_UNSUPPORTED;
    bool fresh = false;
    PM_TRY(inst->partials.reserve(pm_plan_partial_bytes(plan, pop), &fresh));
    if (fresh)  // accumulators start at zero; launches leave them zero
        PM_CUDA(cudaMemsetAsync(inst->partials.ptr, 0, inst->partials.bytes, s));
    PM_TRY(inst->tickets.reserve(pm_plan_ticket_bytes(plan), &fresh));
    if (fresh)
        PM_CUDA(cudaMemsetAsync(inst->tickets.ptr, 0, inst->tickets.bytes, s));
    pm_accept_args acc;
    acc.columns_ready = true;  // the scan reads `cols` as they are; no transpose
    return pm_launch_eval(inst, plan, nullptr, pop, nullptr, costs, static_cast<int64_t *>(inst->partials.ptr),
                          static_cast<int *>(inst->tickets.ptr), const_cast<uint32_t *>(cols),
                          static_cast<int *>(inst->err.ptr), acc, s);
}

extern "C" pm_status pm_eval_population(pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *costs,
                                        int checked, void *stream)
{
    pm_clear_stale_error();
    if (!inst || pop < 0)
        return PM_ERR_INVALID_ARG;
    if (pop == 0)
        return PM_OK;
    if (!masks || !costs)
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(inst->lock);
    PM_CUDA(cudaSetDevice(inst->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t mask_bytes = (size_t)pop * (size_t)inst->W * sizeof(uint32_t);
    const size_t cost_bytes = (size_t)pop * sizeof(int64_t);
    const bool masks_dev = pm_is_device_ptr(masks);
    const bool costs_dev = pm_is_device_ptr(costs);
    const uint32_t *m_dev = masks;
    int64_t *c_dev = costs;
    if (!masks_dev) {
        PM_TRY(inst->stage_masks.reserve(mask_bytes));
        PM_CUDA(cudaMemcpyAsync(inst->stage_masks.ptr, masks, mask_bytes, cudaMemcpyHostToDevice, s));
        m_dev = static_cast<const uint32_t *>(inst->stage_masks.ptr);
    }
    if (!costs_dev) {
        PM_TRY(inst->stage_costs.reserve(cost_bytes));
        c_dev = static_cast<int64_t *>(inst->stage_costs.ptr);
    }
    if (checked) {
        PM_TRY(inst->flag.reserve(64));
        int *flag = static_cast<int *>(inst->flag.ptr);
        PM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
        PM_TRY(pm_launch_mask_check(inst, m_dev, pop, flag, s));
        int bad = 0;
        PM_CUDA(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaStreamSynchronize(s));
        if (bad)
            return PM_ERR_MASK;
    }
    const pm_eval_plan plan = pm_plan_eval(inst, pop);
    bool fresh = false;
    PM_TRY(inst->partials.reserve(pm_plan_partial_bytes(plan, pop), &fresh));
    if (fresh)  // column-kernel accumulators start at zero; launches leave them zero
        PM_CUDA(cudaMemsetAsync(inst->partials.ptr, 0, inst->partials.bytes, s));
    PM_TRY(inst->tickets.reserve(pm_plan_ticket_bytes(plan), &fresh));
    if (fresh)
        PM_CUDA(cudaMemsetAsync(inst->tickets.ptr, 0, inst->tickets.bytes, s));
    PM_TRY(inst->columns.reserve(std::max<size_t>(pm_plan_column_bytes(inst, plan), 256)));
    pm_accept_args acc;
    PM_TRY(pm_launch_eval(inst, plan, m_dev, pop, nullptr, c_dev, static_cast<int64_t *>(inst->partials.ptr),
                          static_cast<int *>(inst->tickets.ptr), static_cast<uint32_t *>(inst->columns.ptr),
                          static_cast<int *>(inst->err.ptr), acc, s));
    if (!costs_dev || checked) {
        if (!costs_dev)
            PM_CUDA(cudaMemcpyAsync(costs, c_dev, cost_bytes, cudaMemcpyDeviceToHost, s));
        int err = 0;
        PM_CUDA(cudaMemcpyAsync(&err, inst->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaStreamSynchronize(s));
        if (err) {
            PM_TRY(pm_reset_eval_scratch(inst, s));
            return (pm_status)err;
        }
    }
    return PM_OK;
}

pm_status pm_reset_eval_scratch(pm_instance *inst, cudaStream_t s)
{
    // a CTA that gave up left its split's sums (and maybe a tile ticket) behind
    pm_dbuf *bufs[] = {&inst->err, &inst->partials, &inst->tickets};
    for (pm_dbuf *b : bufs)
        if (b->ptr)
            PM_CUDA(cudaMemsetAsync(b->ptr, 0, b->bytes, s));
    PM_CUDA(cudaStreamSynchronize(s));
    return PM_OK;
}
