// Shared definitions of libpmgpu's translation units (device helpers, the
// instance object and launch configuration).  Nothing here is visible at the
// C ABI except through include/pm.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstdlib>
#include <utility>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "pm.h"

#define PM_FULL_MASK 0xffffffffu

// Evaluate a CUDA runtime call; on failure return PM_ERR_CUDA (or OOM).
#define PM_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            pm_note_cuda_error(e_, #call, __FILE__, __LINE__);                                         \
            return (e_ == cudaErrorMemoryAllocation) ? PM_ERR_OOM : PM_ERR_CUDA;                       \
        }                                                                                              \
    } while (0)

#define PM_TRY(expr)                                                                                   \
    do {                                                                                               \
        pm_status s_ = (expr);                                                                         \
        if (s_ != PM_OK)                                                                               \
            return s_;                                                                                 \
    } while (0)

void pm_note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// A failed CUDA runtime call leaves its (non-sticky) error for the next cudaGetLastError of the thread, where
// it would be taken for a failed launch.  Calls whose result is not needed (releases, device selection in
// destroy paths) clear it; entry points that launch clear what other code left before their first launch.
inline void pm_clear_error(cudaError_t e)
{
    if (e != cudaSuccess)
        (void)cudaGetLastError();
}
inline void pm_clear_stale_error() { (void)cudaGetLastError(); }

// A device buffer owned by the library that grows on demand, or a slice of
// another buffer (pm_carve), which release() only forgets.
struct pm_dbuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    bool borrowed = false;
    // Grow to at least `want` bytes; *fresh (optional) tells whether new memory was allocated.  A slice that is
    // too small is forgotten and replaced by memory of its own.
    pm_status reserve(size_t want, bool *fresh = nullptr);
    void release();
};

// One device allocation (`arena`, replacing what it held) laid out as consecutive 256-byte aligned slices of
// at least max(size, 256) bytes, handed to the parts as borrowed buffers: one cudaMalloc and, at release, one
// cudaFree for a group of buffers that live and die together.  The parts' previous memory is released first.
struct pm_part {
    pm_dbuf *buf;
    size_t bytes;
};
pm_status pm_carve(pm_dbuf &arena, const pm_part *parts, int count);

// Scratch for one fitness launch configuration (partial sums per client split).
struct pm_eval_plan {
    int groups = 4;       // G: 32-individual groups per CTA
    int warps = 16;       // warps per CTA
    int splits = 1;       // CTAs per individual tile along the client axis
    int64_t tiles = 0;    // ceil(pop / (32 G))
    int64_t grid = 0;     // CTAs launched (column kernel: persistent over tiles x splits items)
    int bytes = 0;        // row kernel only: each warp's bitset expanded to one byte per facility (byte masks)
};

// One instance inside an evaluation launch (host and device).  Individuals
// of the launch are numbered globally: instance k owns [ind_base, ind_base +
// pop), ind_base a multiple of 32; its bitset rows start at word word_base;
// its facility-major tiles at word col_base.  Work items (tile, split) of
// instance k are item_base .. item_base + tiles * splits - 1 (split-major).
struct pm_prob {
    const uint16_t *pi;
    const int32_t *delta;  // Delta', or D' (running sums) when cum
    int64_t n, stride;
    int32_t L, W, m, p;
    int32_t cum;
    int32_t packed;  // split sums and a split count share one 64-bit word (see pm_packed_reduction_ok)
    int64_t pop;
    int64_t ind_base;   // accumulators, active bits, GA per-individual arrays
    int64_t out_base;   // caller's cost array
    int64_t word_base;  // bitset rows
    int64_t col_base;   // facility-major tiles
    int64_t tiles, tile_base;
    int64_t splits, cps;  // client splits and clients per split
    int64_t item_base;
    int64_t job_base;     // transpose jobs (tiles * G * W per instance)
};

// Programmatic dependent launch.  Kernels of the GA generation and of the
// evaluation are launched with programmatic stream serialisation, so the next
// kernel of the stream is scheduled while the current one still runs; every
// such kernel first waits for the completion (and memory) of the grid before
// it, then lets its own successor be scheduled.  Without the launch attribute
// the wait returns at once.  PM_PDL=0 in the environment turns the attribute off.
__device__ __forceinline__ void pm_grid_dependency_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

inline bool pm_pdl_enabled()
{
    static const bool on = [] {
        const char *e = std::getenv("PM_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

template <typename... KArgs, typename... Args>
cudaError_t pm_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pm_pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

struct pm_instance {
    int device = 0;
    int64_t n = 0, m = 0, p = 0, L = 0, W = 0, stride = 0;
    int32_t max_d = 0;
    bool cum = false;           // PM_TABLES_CUMULATIVE: delta holds D' (running sums of Delta') instead
    uint16_t *pi = nullptr;     // n x stride, Pi' (0-based facility ids)
    int32_t *delta = nullptr;   // n x stride, Delta'
    int sm_count = 0;
    size_t smem_optin = 0;
    // staging and scratch for pm_eval_population
    pm_dbuf stage_masks, stage_costs, partials, tickets, columns, flag, err;
    pm_dbuf tab_arena;  // one allocation holding delta, pi, err and flag
    // Delta' instances: the running sums D' (the sorted distances), built once on the first request for swap
    // statistics, which then read distances directly instead of re-summing increments
    mutable pm_dbuf dsorted;
    mutable std::mutex dsorted_mu;
    std::mutex lock;
    // evaluation plans chosen by the autotuner, by population size
    mutable std::mutex plan_mu;
    std::map<int64_t, pm_eval_plan> tuned;
};

// ---------------------------------------------------------------------------
// Fitness evaluation (fitness.cu)
// ---------------------------------------------------------------------------

// Choose the tile configuration for `pop` individuals on `inst` (the tuned
// plan if the autotuner has run for this size, else a heuristic).
pm_eval_plan pm_plan_eval(const pm_instance *inst, int64_t pop);
// A plan with explicit groups (0 = row kernel), warps per CTA and client
// splits (0 = one full wave).
pm_eval_plan pm_plan_eval_with(const pm_instance *inst, int64_t pop, int G, int warps, int splits_hint);
// Bytes of per-tile tickets the plan needs (zero before the first launch;
// every launch leaves them zero, whatever the plan).
size_t pm_plan_ticket_bytes(const pm_eval_plan &plan);
// The packed split reduction holds a partial cost below 2^48 and a split
// count below 2^16 in one 64-bit word: usable when every cost is below 2^47
// (n * max d) and there are fewer than 2^16 splits.
static inline bool pm_packed_reduction_ok(const pm_instance *inst, int64_t splits)
{
    const double bound = (double)inst->n * (double)std::max<int32_t>(inst->max_d, 1);
    return splits < 65536 && bound < 140737488355328.0;  // 2^47
}
// Bytes of int64 partial sums (one per client split and individual).
size_t pm_plan_partial_bytes(const pm_eval_plan &plan, int64_t pop);

// Epilogue applied after the per-individual sums are formed.
//   mode 0: costs[t] = sum.
//   mode 1 (accept): if active(t) and sum < cur_cost[t]: cur_cost[t] = sum,
//           copy cand row t into cur row t, set improved[t] = 1.
struct pm_accept_args {
    int mode = 0;
    int64_t *cur_cost = nullptr;
    uint32_t *cur_masks = nullptr;
    const uint32_t *cand_masks = nullptr;
    uint8_t *improved = nullptr;
    bool columns_ready = false;  // the caller already wrote the facility-major copy
};

// A scan launch over one or more instances.
struct pm_scan_launch {
    int groups = 4, warps = 16;
    int64_t grid = 0;
    int K = 1;
    const pm_prob *probs_dev = nullptr;  // K > 1: device table
    pm_prob one{};                       // K == 1: passed by value
    int64_t items = 0, jobs = 0;
    const uint32_t *masks = nullptr;     // rows, for the transpose (when !columns_ready)
    uint32_t *colT = nullptr;
    const uint32_t *active = nullptr;    // bit per global individual, nullable
    int64_t *accum = nullptr;            // one int64 per global individual, zero at rest
    int *tickets = nullptr;              // one per global tile, zero at rest
    int *err = nullptr;
};
pm_status pm_launch_scan(const pm_scan_launch &L, const pm_accept_args &acc, int64_t *costs, size_t smem,
                         cudaStream_t stream);
// The single-instance launch of `plan` (K = 1, all bases 0).
pm_prob pm_single_prob(const pm_instance *inst, const pm_eval_plan &plan, int64_t pop);

// Enqueue the scan over (masks, pop) -> partials -> sums (+ epilogue).
// active: nullable, bit (t & 31) of word t >> 5 marks individual t as
// evaluated; inactive individuals get no cost written.
pm_status pm_launch_eval(const pm_instance *inst, const pm_eval_plan &plan, const uint32_t *masks, int64_t pop,
                         const uint32_t *active, int64_t *costs, int64_t *partials, int *tickets, uint32_t *colT,
                         int *err, const pm_accept_args &acc, cudaStream_t stream);
// The facility-major copy of (masks, pop) for the column kernel of `plan` (PM_ERR_UNSUPPORTED for the row
// kernel): the first of the two launches of pm_launch_eval.
pm_status pm_launch_columns(const pm_instance *inst, const pm_eval_plan &plan, const uint32_t *masks, int64_t pop,
                            uint32_t *colT, cudaStream_t stream);
// Bytes of the facility-major copy of the population the plan needs.
size_t pm_plan_column_bytes(const pm_instance *inst, const pm_eval_plan &plan);
// One-time per-process kernel attributes (dynamic shared memory opt-in).
pm_status pm_fitness_init(const pm_instance *inst);
// Consume one launch armed by pm_debug_scan_timeout (true if one was armed).
bool pm_take_scan_stall();
// After a device-side failure of an evaluation on inst (its error word set): clear the error word and bring
// the accumulators and tickets back to zero, so later evaluations start from a clean state.  Synchronises s.
pm_status pm_reset_eval_scratch(pm_instance *inst, cudaStream_t s);

// Checked mode: count bitsets with popcount != p or stray high bits into *flag.
pm_status pm_launch_mask_check(const pm_instance *inst, const uint32_t *masks, int64_t pop, int *flag,
                               cudaStream_t stream);

// Uniform random p-subsets (Floyd sampling, fixed seed) for tuning (ga.cu).
pm_status pm_launch_random_population(const pm_instance *inst, uint64_t seed, int64_t pop, uint32_t *masks,
                                      cudaStream_t s);

// A scan plan over several instances (batch.cu): one tile shape for all,
// per-instance splits, global numbering of individuals, rows, tiles.
struct pm_multi_plan {
    int groups = 4, warps = 16;
    int64_t grid = 0, items = 0, jobs = 0;
    int64_t tiles_total = 0, ind_total = 0, words_total = 0, cols_total = 0;
    size_t smem = 0;  // tile bytes of the widest instance
    std::vector<pm_prob> probs;
};
// Plan for `insts` with pops[k] individuals each; items_per_slot work items per
// resident CTA (splits apportioned by an estimate of each instance's scan work).
pm_status pm_plan_multi(const std::vector<const pm_instance *> &insts, const std::vector<int64_t> &pops, int G,
                        int warps, int items_per_slot, pm_multi_plan &out);
// The same layout for one instance under a single-instance plan.
pm_multi_plan pm_plan_from_single(const pm_instance *inst, const pm_eval_plan &plan, int64_t pop);
// Fill L from a multi plan (probs_dev: the plan's table on the device, or null when K == 1).
void pm_scan_launch_from(const pm_multi_plan &mp, const pm_prob *probs_dev, pm_scan_launch &L);

// ---------------------------------------------------------------------------
// Tables (tables.cu)
// ---------------------------------------------------------------------------
pm_status pm_build_tables(pm_instance *inst, const int32_t *d_dev, cudaStream_t stream);
// Delta' of a cumulative instance (differences of its D' rows) into out (n x L, device).
pm_status pm_launch_increments(const pm_instance *inst, int32_t *out, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
bool pm_is_device_ptr(const void *p);

static inline int64_t pm_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t pm_round_up(int64_t a, int64_t b) { return pm_ceil_div(a, b) * b; }

// 32 x 32 bit-matrix transpose across a warp: on entry lane l holds row l
// (bit c = element (l, c)); on exit lane c holds column c (bit l = element
// (l, c)).  Five butterfly exchanges; in exchange j (16, 8, 4, 2, 1) with the
// partner lane l ^ j, the lane with bit j set keeps the upper j bits of each
// 2j-bit block and takes the partner's upper j bits into the lower ones, the
// other lane the reverse.  Rotating the partner's word by j (right for the
// first lane, left for the second) puts exactly those bits in place, so an
// exchange is a shuffle, a rotation by a per-lane amount and one masked merge.
__device__ __forceinline__ uint32_t pm_transpose32(uint32_t x, int lane)
{
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int j = 16 >> s;
        const bool up = (lane & j) != 0;
        const uint32_t keep = up ? ~masks[s] : masks[s];
        const uint32_t y = __shfl_xor_sync(PM_FULL_MASK, x, j);
        const uint32_t r = __funnelshift_l(y, y, up ? 32 - j : j);  // y rotated right (up) or left by j
        x = (x & keep) | (r & ~keep);
    }
    return x;
}
