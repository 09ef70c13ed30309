// Several instances in one evaluation launch (the batched mode): planning,
// the pm_batch_* ABI and its autotuner.
//
// All instances of a launch share one tile shape (groups G, warps); each gets
// its own number of client splits so that the work items -- (instance, tile,
// split) -- are of similar size.  The scan kernel walks the items
// persistently, so uneven instances (n = m from 100 to 5000, p from 5 to
// n/10) fill the GPU in one launch.

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "pm_common.cuh"

// Timed launches per autotuner candidate (after one warm-up); the median decides.
static constexpr int kTuneReps = 5;

static size_t tile_bytes(int64_t W, int G) { return (size_t)W * 32 * G * 4; }

pm_status pm_plan_multi(const std::vector<const pm_instance *> &insts, const std::vector<int64_t> &pops, int G,
                        int warps, int items_per_slot, pm_multi_plan &out)
{
    const int K = (int)insts.size();
    if (K < 1 || (int)pops.size() != K || (G != 1 && G != 2 && G != 4))
        return PM_ERR_INVALID_ARG;
    out = pm_multi_plan();
    out.groups = G;
    out.warps = warps;
    const pm_instance *i0 = insts[0];
    for (const pm_instance *in : insts)
        out.smem = std::max(out.smem, tile_bytes(in->W, G));
    const size_t budget = i0->smem_optin > 4096 ? i0->smem_optin - 4096 : 0;
    if (out.smem > budget)
        return PM_ERR_UNSUPPORTED;
    int slots_per_sm = 0;
    // resident CTAs per SM for this shape and shared memory
    {
        const int by_smem = (int)std::max<size_t>(1, i0->smem_optin / std::max<size_t>(out.smem + 2048, 1));
        const int by_threads = std::max(1, 2048 / (warps * 32));
        slots_per_sm = std::max(1, std::min(by_smem, by_threads));
        // register limit: ~56 registers per thread
        const int by_regs = std::max(1, 65536 / (warps * 32 * 56));
        slots_per_sm = std::min(slots_per_sm, by_regs);
    }
    const int64_t slots = (int64_t)i0->sm_count * slots_per_sm;
    // scan work estimate per instance: tiles x clients x expected 32-rank steps of a 128-individual tile
    std::vector<double> work(K);
    double total = 0.0;
    for (int k = 0; k < K; ++k) {
        const pm_instance *in = insts[k];
        const double tiles = (double)pm_ceil_div(pops[k], 32 * G);
        const double steps = 1.0 + 5.4 * (double)(in->m + 1) / (double)(in->p + 1) / 32.0;
        work[k] = tiles * (double)in->n * steps;
        total += work[k];
    }
    const double target_items = (double)slots * std::max(1, items_per_slot);
    int64_t ind = 0, words = 0, cols = 0, tiles_acc = 0, items = 0, jobs = 0;
    out.probs.resize(K);
    for (int k = 0; k < K; ++k) {
        const pm_instance *in = insts[k];
        pm_prob &pr = out.probs[k];
        pr = pm_prob{};
        pr.pi = in->pi;
        pr.delta = in->delta;
        pr.n = in->n;
        pr.stride = in->stride;
        pr.L = (int32_t)in->L;
        pr.W = (int32_t)in->W;
        pr.m = (int32_t)in->m;
        pr.p = (int32_t)in->p;
        pr.cum = in->cum ? 1 : 0;
        pr.pop = pops[k];
        pr.tiles = std::max<int64_t>(1, pm_ceil_div(pops[k], 32 * G));
        const double want_items = total > 0 ? target_items * work[k] / total : 1.0;
        int64_t splits = (int64_t)std::ceil(want_items / (double)pr.tiles);
        splits = std::max<int64_t>(1, std::min<int64_t>(splits, std::max<int64_t>(1, in->n / warps)));
        pr.splits = splits;
        pr.cps = pm_ceil_div(in->n, splits);
        pr.packed = pm_packed_reduction_ok(in, splits) ? 1 : 0;
        pr.ind_base = ind;
        pr.out_base = 0;  // set by the caller for packed outputs
        pr.word_base = words;
        pr.col_base = cols;
        pr.tile_base = tiles_acc;
        pr.item_base = items;
        pr.job_base = jobs;
        ind += pm_round_up(std::max<int64_t>(pops[k], 1), 32);
        words += pops[k] * in->W;
        cols += pr.tiles * in->W * 32 * G;
        tiles_acc += pr.tiles;
        items += pr.tiles * splits;
        jobs += pr.tiles * G * in->W;
    }
    out.ind_total = ind;
    out.words_total = words;
    out.cols_total = cols;
    out.tiles_total = tiles_acc;
    out.items = items;
    out.jobs = jobs;
    out.grid = std::min<int64_t>(items, slots);
    return PM_OK;
}

pm_multi_plan pm_plan_from_single(const pm_instance *inst, const pm_eval_plan &plan, int64_t pop)
{
    pm_multi_plan mp;
    mp.groups = plan.groups;
    mp.warps = plan.warps;
    mp.grid = plan.grid;
    mp.probs.push_back(pm_single_prob(inst, plan, pop));
    mp.items = plan.tiles * plan.splits;
    mp.jobs = plan.tiles * std::max(plan.groups, 1) * inst->W;
    mp.tiles_total = plan.tiles;
    mp.ind_total = pm_round_up(std::max<int64_t>(pop, 1), 32);
    mp.words_total = pop * inst->W;
    mp.cols_total = plan.groups ? plan.tiles * inst->W * 32 * plan.groups : 0;
    mp.smem = plan.groups ? tile_bytes(inst->W, plan.groups) : 0;
    return mp;
}

void pm_scan_launch_from(const pm_multi_plan &mp, const pm_prob *probs_dev, pm_scan_launch &L)
{
    L.groups = mp.groups;
    L.warps = mp.warps;
    L.grid = mp.grid;
    L.K = (int)mp.probs.size();
    L.one = mp.probs[0];
    L.probs_dev = L.K > 1 ? probs_dev : nullptr;
    L.items = mp.items;
    L.jobs = mp.jobs;
}

// ---------------------------------------------------------------------------
// pm_batch ABI
// ---------------------------------------------------------------------------

struct pm_batch {
    std::vector<const pm_instance *> insts;
    int device = 0;
    // the current plan and its device table, keyed by the population sizes
    std::vector<int64_t> plan_pops;
    pm_multi_plan plan;
    bool have_plan = false;
    std::vector<int64_t> tuned_pops;
    int tuned_G = 0, tuned_warps = 0, tuned_ips = 0;
    pm_dbuf probs, accum, tickets, columns, err, stage_masks, stage_costs;
    std::mutex lock;
};

static pm_status batch_plan(pm_batch *b, const std::vector<int64_t> &pops, int G, int warps, int ips, cudaStream_t s)
{
    pm_multi_plan mp;
    PM_TRY(pm_plan_multi(b->insts, pops, G, warps, ips, mp));
    int64_t out = 0;
    for (auto &pr : mp.probs) {
        pr.out_base = out;
        out += pr.pop;
    }
    PM_TRY(b->probs.reserve(mp.probs.size() * sizeof(pm_prob)));
    PM_CUDA(cudaMemcpyAsync(b->probs.ptr, mp.probs.data(), mp.probs.size() * sizeof(pm_prob), cudaMemcpyHostToDevice,
                            s));
    bool fresh = false;
    PM_TRY(b->accum.reserve((size_t)mp.ind_total * 8, &fresh));
    if (fresh)
        PM_CUDA(cudaMemsetAsync(b->accum.ptr, 0, b->accum.bytes, s));
    PM_TRY(b->tickets.reserve((size_t)pm_round_up(mp.tiles_total * 4, 256), &fresh));
    if (fresh)
        PM_CUDA(cudaMemsetAsync(b->tickets.ptr, 0, b->tickets.bytes, s));
    PM_TRY(b->columns.reserve(std::max<size_t>((size_t)mp.cols_total * 4, 256)));
    b->plan = mp;
    b->plan_pops = pops;
    b->have_plan = true;
    return PM_OK;
}

static void default_shape(const pm_batch *b, int &G, int &warps, int &ips)
{
    const size_t budget = b->insts[0]->smem_optin > 4096 ? b->insts[0]->smem_optin - 4096 : 0;
    int64_t Wmax = 0;
    for (auto *in : b->insts)
        Wmax = std::max<int64_t>(Wmax, in->W);
    G = 4;
    while (G > 1 && tile_bytes(Wmax, G) > budget)
        G /= 2;
    warps = 2 * tile_bytes(Wmax, G) + 8192 > b->insts[0]->smem_optin ? 32 : 16;
    ips = 4;
}

extern "C" pm_status pm_batch_create(pm_instance *const *insts, int64_t k, pm_batch **out)
{
    if (!out || !insts || k < 1 || k > (1 << 20))
        return PM_ERR_INVALID_ARG;
    *out = nullptr;
    for (int64_t i = 0; i < k; ++i)
        if (!insts[i] || insts[i]->device != insts[0]->device)
            return PM_ERR_INVALID_ARG;
    const size_t budget = insts[0]->smem_optin > 4096 ? insts[0]->smem_optin - 4096 : 0;
    for (int64_t i = 0; i < k; ++i)
        if (tile_bytes(insts[i]->W, 1) > budget)
            return PM_ERR_UNSUPPORTED;  // batched mode needs facility-major tiles (m up to ~56000)
    pm_batch *b = new (std::nothrow) pm_batch();
    if (!b)
        return PM_ERR_OOM;
    b->insts.assign(insts, insts + k);
    b->device = insts[0]->device;
    *out = b;
    return PM_OK;
}

extern "C" pm_status pm_batch_destroy(pm_batch *b)
{
    if (!b)
        return PM_OK;
    pm_clear_error(cudaSetDevice(b->device));
    pm_dbuf *bufs[] = {&b->probs, &b->accum, &b->tickets, &b->columns, &b->err, &b->stage_masks, &b->stage_costs};
    for (pm_dbuf *x : bufs)
        x->release();
    delete b;
    return PM_OK;
}

static pm_status batch_eval_impl(pm_batch *b, const uint32_t *masks, const std::vector<int64_t> &pops, int64_t *costs,
                                 cudaStream_t s)
{
    int G, warps, ips;
    if (b->tuned_pops == pops) {
        G = b->tuned_G;
        warps = b->tuned_warps;
        ips = b->tuned_ips;
    } else {
        default_shape(b, G, warps, ips);
    }
    if (!b->have_plan || b->plan_pops != pops || b->plan.groups != G || b->plan.warps != warps)
        PM_TRY(batch_plan(b, pops, G, warps, ips, s));
    PM_TRY(b->err.reserve(256));
    pm_scan_launch L;
    pm_scan_launch_from(b->plan, static_cast<const pm_prob *>(b->probs.ptr), L);
    L.masks = masks;
    L.colT = static_cast<uint32_t *>(b->columns.ptr);
    L.accum = static_cast<int64_t *>(b->accum.ptr);
    L.tickets = static_cast<int *>(b->tickets.ptr);
    L.err = static_cast<int *>(b->err.ptr);
    pm_accept_args acc;
    // the epilogue writes costs[out_base + t]; masks rows start at word_base (packed, as the caller lays them out)
    return pm_launch_scan(L, acc, costs, b->plan.smem, s);
}

extern "C" pm_status pm_batch_eval(pm_batch *b, const uint32_t *masks, const int64_t *pops, int64_t *costs,
                                   void *stream)
{
    if (!b || !masks || !pops || !costs)
        return PM_ERR_INVALID_ARG;
    std::vector<int64_t> pv(b->insts.size());
    int64_t total = 0;
    for (size_t k = 0; k < pv.size(); ++k) {
        if (pops[k] < 1 || pops[k] > ((int64_t)1 << 31))
            return PM_ERR_INVALID_ARG;
        pv[k] = pops[k];
        total += pops[k];
    }
    if (!pm_is_device_ptr(masks) || !pm_is_device_ptr(costs))
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(b->lock);
    PM_CUDA(cudaSetDevice(b->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!b->err.ptr) {
        PM_TRY(b->err.reserve(256));
        PM_CUDA(cudaMemsetAsync(b->err.ptr, 0, 256, s));
    }
    (void)total;
    return batch_eval_impl(b, masks, pv, costs, s);
}

extern "C" pm_status pm_batch_tune(pm_batch *b, const int64_t *pops, void *stream, pm_eval_shape *chosen)
{
    if (!b || !pops)
        return PM_ERR_INVALID_ARG;
    std::vector<int64_t> pv(b->insts.size());
    int64_t words = 0, total = 0;
    for (size_t k = 0; k < pv.size(); ++k) {
        if (pops[k] < 1 || pops[k] > ((int64_t)1 << 31))
            return PM_ERR_INVALID_ARG;
        pv[k] = pops[k];
        words += pops[k] * b->insts[k]->W;
        total += pops[k];
    }
    std::lock_guard<std::mutex> guard(b->lock);
    PM_CUDA(cudaSetDevice(b->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_TRY(b->err.reserve(256));
    PM_CUDA(cudaMemsetAsync(b->err.ptr, 0, 256, s));
    PM_TRY(b->stage_masks.reserve((size_t)words * 4));
    PM_TRY(b->stage_costs.reserve((size_t)total * 8));
    uint32_t *masks = static_cast<uint32_t *>(b->stage_masks.ptr);
    {
        int64_t wb = 0;
        for (size_t k = 0; k < pv.size(); ++k) {
            PM_TRY(pm_launch_random_population(b->insts[k], 0x5EEDull + k, pv[k], masks + wb, s));
            wb += pv[k] * b->insts[k]->W;
        }
    }
    int64_t Wmax = 0;
    for (auto *in : b->insts)
        Wmax = std::max<int64_t>(Wmax, in->W);
    const size_t budget = b->insts[0]->smem_optin > 4096 ? b->insts[0]->smem_optin - 4096 : 0;
    cudaEvent_t e0, e1;
    PM_CUDA(cudaEventCreate(&e0));
    PM_CUDA(cudaEventCreate(&e1));
    double best_ms = 1e30;
    int bG = 0, bw = 0, bi = 0, ncand = 0;
    int64_t bgrid = 0;
    pm_status st = PM_OK;
    for (int G : {4, 2, 1}) {
        if (tile_bytes(Wmax, G) > budget)
            continue;
        for (int warps : {16, 32}) {
            for (int ips : {2, 4, 8}) {
                b->tuned_pops = pv;
                b->tuned_G = G;
                b->tuned_warps = warps;
                b->tuned_ips = ips;
                b->have_plan = false;
                float t[kTuneReps];
                st = batch_eval_impl(b, masks, pv, static_cast<int64_t *>(b->stage_costs.ptr), s);
                for (int r = 0; r < kTuneReps && st == PM_OK; ++r) {
                    cudaEventRecord(e0, s);
                    st = batch_eval_impl(b, masks, pv, static_cast<int64_t *>(b->stage_costs.ptr), s);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess)
                        st = PM_ERR_CUDA;
                }
                if (st != PM_OK)
                    break;
                ++ncand;
                std::sort(t, t + kTuneReps);
                if (t[kTuneReps / 2] < best_ms) {
                    best_ms = t[1];
                    bG = G;
                    bw = warps;
                    bi = ips;
                    bgrid = b->plan.grid;
                }
            }
            if (st != PM_OK)
                break;
        }
        if (st != PM_OK)
            break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    PM_TRY(st);
    if (ncand == 0)
        return PM_ERR_UNSUPPORTED;
    b->tuned_pops = pv;
    b->tuned_G = bG;
    b->tuned_warps = bw;
    b->tuned_ips = bi;
    b->have_plan = false;
    int err = 0;
    PM_CUDA(cudaMemcpyAsync(&err, b->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaStreamSynchronize(s));
    if (err)
        return (pm_status)err;
    if (chosen) {
        chosen->groups = bG;
        chosen->warps = bw;
        chosen->splits = bi;  // work items per resident CTA slot
        chosen->grid = (int32_t)bgrid;
        chosen->ms = best_ms;
        chosen->candidates = ncand;
        chosen->reserved = 0;
    }
    return PM_OK;
}

// Plan used by a batched GA (batch.cu owns the shape choice).
pm_status pm_batch_ga_plan(pm_batch *b, int64_t pop, pm_multi_plan &out)
{
    std::vector<int64_t> pv(b->insts.size(), pop);
    int G, warps, ips;
    if (b->tuned_pops == pv) {
        G = b->tuned_G;
        warps = b->tuned_warps;
        ips = b->tuned_ips;
    } else {
        default_shape(b, G, warps, ips);
    }
    PM_TRY(pm_plan_multi(b->insts, pv, G, warps, ips, out));
    for (auto &pr : out.probs)
        pr.out_base = pr.ind_base;  // GA costs are indexed by the padded individual number
    return PM_OK;
}

// The speculative mutation cycle's candidates of a batched GA: popQ = Q x pop per instance, planned with the
// tile shape the GA's own scans use (tuned for pop, or the default); costs indexed like the GA's.
pm_status pm_batch_ga_plan_candidates(pm_batch *b, int64_t pop, int64_t popQ, pm_multi_plan &out)
{
    std::vector<int64_t> pv(b->insts.size(), pop), pq(b->insts.size(), popQ);
    int G, warps, ips;
    if (b->tuned_pops == pv) {
        G = b->tuned_G;
        warps = b->tuned_warps;
        ips = b->tuned_ips;
    } else {
        default_shape(b, G, warps, ips);
    }
    PM_TRY(pm_plan_multi(b->insts, pq, G, warps, ips, out));
    for (auto &pr : out.probs)
        pr.out_base = pr.ind_base;
    return PM_OK;
}

const std::vector<const pm_instance *> &pm_batch_instances(const pm_batch *b) { return b->insts; }
