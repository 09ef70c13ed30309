// Population fitness evaluation -- the paper's Fitness function (Section 4.2)
// over the truncated tables Pi' and Delta' (Section 2.1), for a whole
// population at once.
//
// For individual t and client i the cost term is sum_{s <= k} Delta'_i[s],
// where k is the first rank whose facility Pi'_i[k] is open in t; the cost
// of t is the sum over clients (Eq. 6).
//
// GB300 design ("column" kernel):
//  * The population is first transposed into a facility-major layout: for a
//    tile of 32*G individuals, word (j, g) holds bit b = "individual
//    tile*32G + 32g + b has facility j open".  One 32-bit shared-memory load
//    then tests one facility for 32 individuals.
//  * A CTA owns one tile; its m x G words are brought into shared memory with
//    one TMA bulk copy (cp.async.bulk + mbarrier).  Grid.y splits the clients.
//  * A warp takes one client at a time and walks its row 32 ranks per step:
//    lane r loads Pi'[r] and Delta'[r] (coalesced), a warp scan turns the
//    increments into running sums (the prefix of Delta' up to rank r), and
//    for each group g lane r loads the 32-individual word of facility
//    Pi'[r].  The 32x32 bit block (rank x individual) is transposed with
//    five shuffles, so lane b finds its individual's first open rank with one
//    find-first-set and takes that rank's running sum with one shuffle.
//    Individuals resolved in a step leave the active set; the row walk ends
//    when no individual of the tile is active.  Steps where no active
//    individual has an open facility cost one load, one AND and one vote.
//  * Per-lane int64 sums are combined in shared memory and written as one
//    partial sum per (client split, individual); a second kernel adds the
//    splits (integer, so the order does not matter) and applies the
//    epilogue (plain store, or the GA's strict-improvement acceptance).
//
// For very large m (the facility-major tile does not fit in shared memory)
// a "row" kernel keeps each individual's own bitset in shared memory and
// resolves one individual per warp step with a ballot.

#include <cstdio>

#include "pm_common.cuh"

namespace {

constexpr int kMaxG = 4;
constexpr uint32_t kSpinLimit = 1u << 22;  // bounded mbarrier wait (a few seconds at most)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Row-major population -> facility-major tiles.
// colT[tile][j][g] (j < 32W) = bits over individuals tile*32G + 32g + b.
// One warp per (tile, g, w); grid-stride over those jobs.
// ---------------------------------------------------------------------------
__global__ void k_pop_to_columns(const uint32_t *__restrict__ masks, int64_t pop, int32_t W, int32_t G,
                                 int64_t tiles, uint32_t *__restrict__ colT)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t jobs = tiles * G * W;
    for (int64_t job = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); job < jobs;
         job += warps_total) {
        const int32_t w = (int32_t)(job % W);
        const int64_t tg = job / W;
        const int32_t g = (int32_t)(tg % G);
        const int64_t tile = tg / G;
        const int64_t t = tile * 32 * G + 32 * g + lane;
        const uint32_t x = (t < pop) ? __ldg(masks + t * W + w) : 0u;
        const uint32_t col = pm_transpose32(x, lane);
        colT[(tile * (int64_t)W * 32 + (int64_t)w * 32 + lane) * G + g] = col;
    }
}

// ---------------------------------------------------------------------------
// The column scan kernel.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(1024) k_scan_columns(const uint16_t *__restrict__ pi,
                                                       const int32_t *__restrict__ delta, int64_t n, int32_t L,
                                                       int64_t stride, const uint32_t *__restrict__ colT,
                                                       int32_t W, int64_t pop, const uint32_t *__restrict__ active,
                                                       int64_t clients_per_split,
                                                       unsigned long long *__restrict__ partial,
                                                       int *__restrict__ err)
{
    extern __shared__ __align__(128) uint32_t colbits[];  // [32W][G]
    __shared__ unsigned long long acc_s[G * 32];
    __shared__ uint32_t a0_s[G];
    __shared__ __align__(8) uint64_t bar;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int64_t tile = blockIdx.x;
    const int split = blockIdx.y;
    const int64_t ind0 = tile * 32 * G;
    const uint32_t tile_bytes = (uint32_t)W * 32u * G * 4u;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, tile_bytes);
        const char *src = reinterpret_cast<const char *>(colT + tile * (int64_t)W * 32 * G);
        char *dst = reinterpret_cast<char *>(colbits);
        for (uint32_t off = 0; off < tile_bytes; off += 32768u) {
            const uint32_t sz = (tile_bytes - off) < 32768u ? (tile_bytes - off) : 32768u;
            bulk_g2s(dst + off, src + off, sz, &bar);
        }
    }
    if (warp < G) {
        const int64_t t = ind0 + 32 * warp + lane;
        const bool on = (t < pop) && (active == nullptr || ((__ldg(active + (t >> 5)) >> (t & 31)) & 1u));
        const uint32_t b = __ballot_sync(PM_FULL_MASK, on);
        if (lane == 0)
            a0_s[warp] = b;
    }
    for (int i = threadIdx.x; i < G * 32; i += blockDim.x)
        acc_s[i] = 0ull;
    // bounded wait for the tile (every thread waits; phase 0)
    {
        uint32_t spins = 0;
        while (!mbar_try_wait(&bar, 0)) {
            if (++spins > kSpinLimit) {
                if (threadIdx.x == 0)
                    atomicExch(err, (int)PM_ERR_TIMEOUT);
                // the copy may still land: wait once more, again bounded, then leave
                uint32_t extra = 0;
                while (!mbar_try_wait(&bar, 0) && ++extra < kSpinLimit) {
                }
                return;
            }
        }
    }
    __syncthreads();

    uint32_t a0[G];
    uint32_t any0 = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        a0[g] = a0_s[g];
        any0 |= a0[g];
    }
    unsigned long long acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g)
        acc[g] = 0ull;

    const int64_t c_begin = (int64_t)split * clients_per_split;
    const int64_t c_end = (c_begin + clients_per_split < n) ? c_begin + clients_per_split : n;
    if (any0) {
        for (int64_t c = c_begin + warp; c < c_end; c += nwarps) {
            const uint16_t *prow = pi + c * stride;
            const int32_t *drow = delta + c * stride;
            uint32_t a[G];
#pragma unroll
            for (int g = 0; g < G; ++g)
                a[g] = a0[g];
            int32_t carry = 0;
            for (int base = 0; base < L; base += 32) {
                const int r = base + lane;
                uint32_t j = 0;
                int32_t dl = 0;
                if (r < L) {
                    j = __ldg(prow + r);
                    dl = __ldg(drow + r);
                }
                // running sum of Delta' up to rank r: the sorted distance at rank r
                int32_t cs = dl;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(PM_FULL_MASK, cs, o);
                    if (lane >= o)
                        cs += y;
                }
                cs += carry;
                carry = __shfl_sync(PM_FULL_MASK, cs, 31);
                uint32_t left = 0;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (a[g] == 0u)
                        continue;
                    const uint32_t w = (r < L) ? (colbits[j * G + g] & a[g]) : 0u;
                    if (!__any_sync(PM_FULL_MASK, w != 0u)) {
                        left |= a[g];
                        continue;
                    }
                    const uint32_t T = pm_transpose32(w, lane);
                    const int f = __ffs(T) - 1;
                    const int32_t v = __shfl_sync(PM_FULL_MASK, cs, f & 31);
                    if (T)
                        acc[g] += (unsigned long long)(uint32_t)v;
                    a[g] &= ~__ballot_sync(PM_FULL_MASK, T != 0u);
                    left |= a[g];
                }
                if (left == 0u)
                    break;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g)
        if (acc[g])
            atomicAdd(&acc_s[g * 32 + lane], acc[g]);
    __syncthreads();
    for (int i = threadIdx.x; i < G * 32; i += blockDim.x) {
        const int64_t t = ind0 + i;
        if (t < pop)
            partial[(int64_t)split * pop + t] = acc_s[i];
    }
}

// ---------------------------------------------------------------------------
// Row kernel (fallback for m too large for facility-major tiles): one warp
// per individual, the individual's bitset in shared memory, one ballot per
// 32 ranks.  Grid: (ceil(pop / warps), splits).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scan_rows(const uint16_t *__restrict__ pi, const int32_t *__restrict__ delta,
                                                   int64_t n, int32_t L, int64_t stride,
                                                   const uint32_t *__restrict__ masks, int32_t W, int64_t pop,
                                                   const uint32_t *__restrict__ active, int64_t clients_per_split,
                                                   unsigned long long *__restrict__ partial)
{
    extern __shared__ __align__(16) uint32_t rowbits[];  // [warps][W]
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * nwarps + warp;
    const int split = blockIdx.y;
    if (t >= pop)
        return;
    if (active != nullptr && !((__ldg(active + (t >> 5)) >> (t & 31)) & 1u))
        return;
    uint32_t *x = rowbits + (int64_t)warp * W;
    for (int w = lane; w < W; w += 32)
        x[w] = __ldg(masks + t * W + w);
    __syncwarp();
    const int64_t c_begin = (int64_t)split * clients_per_split;
    const int64_t c_end = (c_begin + clients_per_split < n) ? c_begin + clients_per_split : n;
    unsigned long long acc = 0ull;
    for (int64_t c = c_begin; c < c_end; ++c) {
        const uint16_t *prow = pi + c * stride;
        const int32_t *drow = delta + c * stride;
        int32_t carry = 0;
        for (int base = 0; base < L; base += 32) {
            const int r = base + lane;
            uint32_t j = 0;
            int32_t dl = 0;
            if (r < L) {
                j = __ldg(prow + r);
                dl = __ldg(drow + r);
            }
            const bool open = (r < L) && ((x[j >> 5] >> (j & 31)) & 1u);
            int32_t cs = dl;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(PM_FULL_MASK, cs, o);
                if (lane >= o)
                    cs += y;
            }
            cs += carry;
            const uint32_t hit = __ballot_sync(PM_FULL_MASK, open);
            if (hit) {
                acc += (unsigned long long)(uint32_t)__shfl_sync(PM_FULL_MASK, cs, __ffs(hit) - 1);
                break;
            }
            carry = __shfl_sync(PM_FULL_MASK, cs, 31);
        }
    }
    if (lane == 0)
        partial[(int64_t)split * pop + t] = acc;
}

// ---------------------------------------------------------------------------
// Sum the splits and apply the epilogue.  One warp per individual.
// ---------------------------------------------------------------------------
__global__ void k_reduce_accept(const unsigned long long *__restrict__ partial, int splits, int64_t pop,
                                const uint32_t *__restrict__ active, int64_t *__restrict__ costs, int mode,
                                int64_t *__restrict__ cur_cost, uint32_t *__restrict__ cur_masks,
                                const uint32_t *__restrict__ cand_masks, uint8_t *__restrict__ improved, int32_t W)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= pop)
        return;
    if (active != nullptr && !((__ldg(active + (t >> 5)) >> (t & 31)) & 1u))
        return;
    unsigned long long s = 0ull;
    for (int k = lane; k < splits; k += 32)
        s += partial[(int64_t)k * pop + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(PM_FULL_MASK, s, o);
    const int64_t sum = (int64_t)s;
    if (costs != nullptr && lane == 0)
        costs[t] = sum;
    if (mode == 1) {
        const bool better = sum < cur_cost[t];
        if (better) {
            for (int w = lane; w < W; w += 32)
                cur_masks[t * W + w] = cand_masks[t * W + w];
            if (lane == 0) {
                cur_cost[t] = sum;
                if (improved)
                    improved[t] = 1;
            }
        }
    }
}

__global__ void k_mask_check(const uint32_t *__restrict__ masks, int64_t pop, int32_t W, int32_t m, int32_t p,
                             int *__restrict__ flag)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pop)
        return;
    int cnt = 0;
    for (int w = 0; w < W; ++w)
        cnt += __popc(masks[t * W + w]);
    const int tail = m & 31;
    const bool stray = tail && (masks[t * W + W - 1] >> tail) != 0u;
    if (cnt != p || stray)
        atomicAdd(flag, 1);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static size_t column_smem_bytes(int64_t W, int G) { return (size_t)W * 32 * G * 4; }

pm_eval_plan pm_plan_eval(const pm_instance *inst, int64_t pop)
{
    pm_eval_plan plan;
    const size_t budget = inst->smem_optin > 4096 ? inst->smem_optin - 4096 : 0;
    int G = kMaxG;
    // fewer groups for small populations (keep >= 8 tiles) or when the tile does not fit
    while (G > 1 && (pop <= (int64_t)32 * (G / 2) * 8 || column_smem_bytes(inst->W, G) > budget))
        G /= 2;
    int64_t ctas_per_sm;
    if (column_smem_bytes(inst->W, G) > budget) {
        plan.groups = 0;  // row kernel
        plan.warps = 8;
        plan.tiles = pm_ceil_div(pop, plan.warps);
        ctas_per_sm = 8;
    } else {
        plan.groups = G;
        const size_t smem = column_smem_bytes(inst->W, G);
        plan.warps = smem > budget / 2 ? 32 : 16;
        plan.tiles = pm_ceil_div(pop, 32 * G);
        ctas_per_sm = std::min<int64_t>(64 / plan.warps, (int64_t)(budget / std::max<size_t>(smem, 1)));
        ctas_per_sm = std::max<int64_t>(ctas_per_sm, 1);
    }
    const int64_t target = (int64_t)inst->sm_count * ctas_per_sm;
    int64_t splits = pm_ceil_div(target, std::max<int64_t>(1, plan.tiles));
    const int64_t max_splits = std::max<int64_t>(1, inst->n / (plan.groups ? plan.warps : 1));
    splits = std::min<int64_t>(std::max<int64_t>(1, splits), std::min<int64_t>(max_splits, 65535));
    plan.splits = (int)splits;
    return plan;
}

pm_status pm_fitness_init(const pm_instance *inst)
{
    const int cap = (int)(inst->smem_optin > 2048 ? inst->smem_optin - 2048 : inst->smem_optin);
    PM_CUDA(cudaFuncSetAttribute(k_scan_columns<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    PM_CUDA(cudaFuncSetAttribute(k_scan_columns<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    PM_CUDA(cudaFuncSetAttribute(k_scan_columns<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    PM_CUDA(cudaFuncSetAttribute(k_scan_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    return PM_OK;
}

size_t pm_plan_partial_bytes(const pm_eval_plan &plan, int64_t pop)
{
    size_t part = (size_t)plan.splits * (size_t)std::max<int64_t>(pop, 1) * sizeof(unsigned long long);
    return part;
}

size_t pm_plan_column_bytes(const pm_instance *inst, const pm_eval_plan &plan)
{
    if (!plan.groups)
        return 0;
    return (size_t)plan.tiles * column_smem_bytes(inst->W, plan.groups);
}

pm_status pm_launch_eval(const pm_instance *inst, const pm_eval_plan &plan, const uint32_t *masks, int64_t pop,
                         const uint32_t *active, int64_t *costs, int64_t *partials_i64, uint32_t *colT,
                         int *err, const pm_accept_args &acc, cudaStream_t stream)
{
    if (pop <= 0)
        return PM_OK;
    unsigned long long *partials = reinterpret_cast<unsigned long long *>(partials_i64);
    const int64_t cps = pm_ceil_div(inst->n, plan.splits);
    if (plan.groups) {
        const int G = plan.groups;
        const int64_t jobs = plan.tiles * G * inst->W;
        const int threads = 256;
        const int64_t blocks = std::min<int64_t>(pm_ceil_div(jobs, threads / 32), (int64_t)inst->sm_count * 16);
        k_pop_to_columns<<<(unsigned)blocks, threads, 0, stream>>>(masks, pop, (int32_t)inst->W, G, plan.tiles,
                                                                   colT);
        PM_CUDA(cudaGetLastError());
        const size_t smem = column_smem_bytes(inst->W, G);
        dim3 grid((unsigned)plan.tiles, (unsigned)plan.splits);
        const int threadsc = plan.warps * 32;
        switch (G) {
        case 1:
            k_scan_columns<1><<<grid, threadsc, smem, stream>>>(inst->pi, inst->delta, inst->n, (int32_t)inst->L,
                                                               inst->stride, colT, (int32_t)inst->W, pop, active,
                                                               cps, partials, err);
            break;
        case 2:
            k_scan_columns<2><<<grid, threadsc, smem, stream>>>(inst->pi, inst->delta, inst->n, (int32_t)inst->L,
                                                               inst->stride, colT, (int32_t)inst->W, pop, active,
                                                               cps, partials, err);
            break;
        default:
            k_scan_columns<4><<<grid, threadsc, smem, stream>>>(inst->pi, inst->delta, inst->n, (int32_t)inst->L,
                                                               inst->stride, colT, (int32_t)inst->W, pop, active,
                                                               cps, partials, err);
            break;
        }
        PM_CUDA(cudaGetLastError());
    } else {
        const size_t smem = (size_t)plan.warps * inst->W * 4;
        dim3 grid((unsigned)plan.tiles, (unsigned)plan.splits);
        k_scan_rows<<<grid, plan.warps * 32, smem, stream>>>(inst->pi, inst->delta, inst->n, (int32_t)inst->L,
                                                             inst->stride, masks, (int32_t)inst->W, pop, active,
                                                             cps, partials);
        PM_CUDA(cudaGetLastError());
    }
    const int64_t threads = 256;
    const int64_t blocks = pm_ceil_div(pop * 32, threads);
    k_reduce_accept<<<(unsigned)blocks, (unsigned)threads, 0, stream>>>(
        partials, plan.splits, pop, active, costs, acc.mode, acc.cur_cost, acc.cur_masks, acc.cand_masks,
        acc.improved, (int32_t)inst->W);
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

pm_status pm_launch_mask_check(const pm_instance *inst, const uint32_t *masks, int64_t pop, int *flag,
                               cudaStream_t stream)
{
    if (pop <= 0)
        return PM_OK;
    k_mask_check<<<(unsigned)pm_ceil_div(pop, 256), 256, 0, stream>>>(masks, pop, (int32_t)inst->W,
                                                                      (int32_t)inst->m, (int32_t)inst->p, flag);
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

// ---------------------------------------------------------------------------
// Evaluation that allocates nothing (no counterpart in the paper): the
// scratch of pm_launch_eval lives in a fixed array compiled into the library.
// Layout inside the array: [0, 256) error word, then the facility-major
// population copy, then the partial sums, each 256-byte aligned.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per GPU
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` (which must be current);
// looked up once per device.
pm_status noalloc_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= kNoAllocMaxDevices)
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            pm_note_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            return PM_ERR_CUDA;
        }
        g_noalloc_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_addr[device]);
    return PM_OK;
}
}  // namespace

extern "C" pm_status pm_eval_population_noalloc(pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *costs,
                                                void *stream)
{
    if (!inst || pop < 0)
        return PM_ERR_INVALID_ARG;
    if (pop == 0)
        return PM_OK;
    if (!masks || !costs || !pm_is_device_ptr(masks) || !pm_is_device_ptr(costs))
        return PM_ERR_INVALID_ARG;
    const pm_eval_plan plan = pm_plan_eval(inst, pop);
    const size_t cols = (size_t)pm_round_up((int64_t)pm_plan_column_bytes(inst, plan), 256);
    const size_t part = (size_t)pm_round_up((int64_t)pm_plan_partial_bytes(plan, pop), 256);
    if (256 + cols + part > kNoAllocScratchBytes)
        return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(inst->device));
    unsigned char *base = nullptr;
    PM_TRY(noalloc_scratch(inst->device, &base));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *err = reinterpret_cast<int *>(base);
    uint32_t *colT = reinterpret_cast<uint32_t *>(base + 256);
    int64_t *partials = reinterpret_cast<int64_t *>(base + 256 + cols);
    // the array keeps the previous call's contents: the error word must start at zero
    PM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    pm_accept_args acc;
    return pm_launch_eval(inst, plan, masks, pop, nullptr, costs, partials, colT, err, acc, s);
}
