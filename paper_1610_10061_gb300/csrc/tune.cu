// Autotuner for the evaluation tile shape (pm_tune_eval in include/pm.h).
//
// The scan's best shape depends on the instance: for short scans (many open
// facilities) an evaluation is a few microseconds of dependent shuffles per
// client and wants many small CTAs; for long scans it is issue-bound and
// wants large tiles that share each staged row chunk among 128 individuals.
// The candidates cover both mask layouts: facility-major bit columns (the
// column kernel, G x 32 individuals per shared-memory load) and
// individual-major bitsets (the row kernel, one individual per warp).
// Rather than model that, the tuner times the candidate shapes on the
// instance itself and keeps the fastest per population size.

#include <algorithm>
#include <vector>

#include "pm_common.cuh"

// Timed repetitions per autotuner candidate (after one warm-up); the median decides.  Each repetition is a
// sequence of kTuneChain back-to-back launches, as the GA chains its evaluations (programmatic dependent launch
// overlaps a launch's start with the previous one's end), and counts as its mean.
static constexpr int kTuneReps = 5;
static constexpr int kTuneChain = 8;

namespace {
bool same_shape(const pm_eval_plan &a, const pm_eval_plan &b)
{
    return a.groups == b.groups && a.warps == b.warps && a.splits == b.splits && a.bytes == b.bytes;
}

// The shape as the ABI reports it: groups -1 is the row kernel with byte masks.
int32_t abi_groups(const pm_eval_plan &p) { return p.groups == 0 && p.bytes ? -1 : p.groups; }
}  // namespace

extern "C" pm_status pm_tune_eval(pm_instance *inst, int64_t pop, void *stream, pm_eval_shape *chosen)
{
    if (!inst || pop < 1 || pop > ((int64_t)1 << 31))
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(inst->lock);
    PM_CUDA(cudaSetDevice(inst->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // candidate shapes
    std::vector<pm_eval_plan> cands;
    const size_t budget = inst->smem_optin > 4096 ? inst->smem_optin - 4096 : 0;
    for (int G : {4, 2, 1}) {
        if ((size_t)inst->W * 32 * G * 4 > budget)
            continue;
        for (int warps : {8, 16, 32}) {
            const pm_eval_plan base = pm_plan_eval_with(inst, pop, G, warps, 0);
            if (base.groups != G)
                continue;
            for (int sp : {std::max(1, base.splits / 2), base.splits, base.splits * 2}) {
                const pm_eval_plan pl = pm_plan_eval_with(inst, pop, G, warps, sp);
                bool dup = false;
                for (const auto &c : cands)
                    dup = dup || same_shape(c, pl);
                if (!dup)
                    cands.push_back(pl);
            }
        }
    }
    // the other mask layouts: individual-major bitsets, one warp per individual (the row kernel), and the same
    // with each bitset expanded to one byte per facility (byte masks)
    if ((size_t)8 * inst->W * 4 + 1024 <= inst->smem_optin)
        cands.push_back(pm_plan_eval_with(inst, pop, 0, 8, 0));
    if ((size_t)8 * inst->W * 32 + 1024 <= inst->smem_optin)
        cands.push_back(pm_plan_eval_with(inst, pop, -1, 8, 0));
    if (cands.empty())
        cands.push_back(pm_plan_eval_with(inst, pop, 0, 8, 0));

    // scratch for the largest candidate and a random population
    size_t part = 0, tick = 0, cols = 0;
    for (const auto &c : cands) {
        part = std::max(part, pm_plan_partial_bytes(c, pop));
        tick = std::max(tick, pm_plan_ticket_bytes(c));
        cols = std::max(cols, pm_plan_column_bytes(inst, c));
    }
    bool fresh = false;
    PM_TRY(inst->partials.reserve(part, &fresh));
    if (fresh)
        PM_CUDA(cudaMemsetAsync(inst->partials.ptr, 0, inst->partials.bytes, s));
    PM_TRY(inst->tickets.reserve(tick, &fresh));
    if (fresh)
        PM_CUDA(cudaMemsetAsync(inst->tickets.ptr, 0, inst->tickets.bytes, s));
    PM_TRY(inst->columns.reserve(std::max<size_t>(cols, 256)));
    PM_TRY(inst->stage_masks.reserve((size_t)pop * inst->W * 4));
    PM_TRY(inst->stage_costs.reserve((size_t)pop * 8));
    uint32_t *masks = static_cast<uint32_t *>(inst->stage_masks.ptr);
    int64_t *costs = static_cast<int64_t *>(inst->stage_costs.ptr);
    PM_TRY(pm_launch_random_population(inst, 0x5EEDull, pop, masks, s));

    cudaEvent_t e0, e1;
    PM_CUDA(cudaEventCreate(&e0));
    PM_CUDA(cudaEventCreate(&e1));
    pm_accept_args acc;
    int best = -1;
    double best_ms = 1e30;
    pm_status st = PM_OK;
    for (size_t k = 0; k < cands.size() && st == PM_OK; ++k) {
        const pm_eval_plan &pl = cands[k];
        auto run = [&]() {
            return pm_launch_eval(inst, pl, masks, pop, nullptr, costs, static_cast<int64_t *>(inst->partials.ptr),
                                  static_cast<int *>(inst->tickets.ptr), static_cast<uint32_t *>(inst->columns.ptr),
                                  static_cast<int *>(inst->err.ptr), acc, s);
        };
        st = run();  // warm-up
        float t[kTuneReps];
        for (int r = 0; r < kTuneReps && st == PM_OK; ++r) {
            cudaEventRecord(e0, s);
            for (int c = 0; c < kTuneChain && st == PM_OK; ++c)
                st = run();
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess)
                st = PM_ERR_CUDA;
            t[r] /= (float)kTuneChain;
        }
        if (st != PM_OK)
            break;
        std::sort(t, t + kTuneReps);
        if (t[kTuneReps / 2] < best_ms) {
            best_ms = t[kTuneReps / 2];
            best = (int)k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    PM_TRY(st);
    int err = 0;
    PM_CUDA(cudaMemcpyAsync(&err, inst->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaStreamSynchronize(s));
    if (err)
        return (pm_status)err;
    {
        std::lock_guard<std::mutex> g(inst->plan_mu);
        inst->tuned[pop] = cands[best];
    }
    if (chosen) {
        chosen->groups = abi_groups(cands[best]);
        chosen->warps = cands[best].warps;
        chosen->splits = cands[best].splits;
        chosen->grid = (int32_t)cands[best].grid;
        chosen->ms = best_ms;
        chosen->candidates = (int32_t)cands.size();
        chosen->reserved = 0;
    }
    return PM_OK;
}

extern "C" pm_status pm_set_eval_shape(pm_instance *inst, int64_t pop, const pm_eval_shape *shape)
{
    if (!inst || !shape || pop < 1 || pop > ((int64_t)1 << 31))
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(inst->lock);
    PM_CUDA(cudaSetDevice(inst->device));
    pm_eval_plan pl;
    if (shape->groups == 0 || shape->groups == -1) {
        pl = pm_plan_eval_with(inst, pop, shape->groups, 8, std::max(0, shape->splits));
        if (shape->groups == -1 && !pl.bytes)
            return PM_ERR_UNSUPPORTED;  // the byte masks of 8 warps do not fit in shared memory
    } else {
        if (shape->groups != 1 && shape->groups != 2 && shape->groups != 4)
            return PM_ERR_INVALID_ARG;
        if (shape->warps < 1 || shape->warps > 32)
            return PM_ERR_INVALID_ARG;
        pl = pm_plan_eval_with(inst, pop, shape->groups, shape->warps, std::max(0, shape->splits));
        if (pl.groups != shape->groups)
            return PM_ERR_UNSUPPORTED;
    }
    // scratch for the new shape (tickets and accumulators start at zero)
    bool fresh = false;
    PM_TRY(inst->partials.reserve(pm_plan_partial_bytes(pl, pop), &fresh));
    if (fresh)
        PM_CUDA(cudaMemset(inst->partials.ptr, 0, inst->partials.bytes));
    PM_TRY(inst->tickets.reserve(pm_plan_ticket_bytes(pl), &fresh));
    if (fresh)
        PM_CUDA(cudaMemset(inst->tickets.ptr, 0, inst->tickets.bytes));
    std::lock_guard<std::mutex> g(inst->plan_mu);
    inst->tuned[pop] = pl;
    return PM_OK;
}
