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
//    tile*32G + 32g + b has facility j open".  One shared-memory load of the
//    G words of facility j (128 bits for G = 4) tests 32G individuals.
//  * Work items are (client split, tile) pairs, split-major, walked by a
//    persistent grid so that CTAs running at the same time stream the same
//    rows through L2.  A CTA brings its tile's 32W x G words into shared
//    memory with TMA bulk copies (cp.async.bulk + mbarrier, bounded wait)
//    and keeps them while consecutive items share the tile.
//  * A warp takes one client at a time and walks its row 32 ranks per step:
//    lane r holds Pi'[r] and Delta'[r] (coalesced loads, the next step and
//    the next client's first step prefetched into registers).  If no still
//    active individual of the tile has facility Pi'[r] open at any lane, the
//    step only adds the 32 increments to a running carry (one warp
//    reduction).  Otherwise a warp scan turns the increments into running
//    sums (the sum of Delta' up to rank r), and each group with hits
//    resolves its individuals' first open ranks: with few hit lanes by
//    walking those lanes in rank order, else by transposing the 32 x 32 bit
//    block (rank x individual) with five shuffles so lane b finds its
//    individual's first open rank with one find-first-set.  Resolved
//    individuals leave the active set; the walk ends when none is left.
//  * Per-lane int64 sums are combined in shared memory.  With one client
//    split the CTA applies the epilogue itself.  Otherwise each split adds
//    its sum and a count of one into a single 64-bit word per individual
//    (sum in bits 0..47, count above); the split whose atomic completes the
//    count holds the total, zeroes the word for the next launch and applies
//    that individual's epilogue -- a plain store of the cost, or the GA's
//    acceptance (replace the current individual iff the candidate is
//    strictly cheaper).  Integer sums do not depend on the order of the
//    additions.  Where n * max d could reach 2^47 the splits add plain int64
//    sums and the last CTA of the tile (an atomic ticket) applies the
//    epilogues.
//
// For very large m (the facility-major tile does not fit in shared memory)
// a "row" kernel keeps each individual's own bitset in shared memory and
// resolves one individual per warp step with a ballot; a separate kernel
// adds its splits.

#include <atomic>
#include <cstdio>

#include "pm_common.cuh"
#include "scan_walk.cuh"

namespace {

constexpr int kMaxG = 4;
constexpr uint32_t kSpinLimit = 1u << 22;  // bounded mbarrier wait (a few seconds at most)
constexpr uint32_t kStallSpinLimit = 1u << 14;  // the poll limit of a launch armed by pm_debug_scan_timeout
constexpr int kCountShift = 48;            // packed split reduction: count in bits 48..63, sum below

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

// Largest k in [0, K) with base(k) <= x (bases ascending, base(0) = 0).
template <typename F>
__device__ __forceinline__ int find_prob(int K, int64_t x, F base)
{
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base(mid) <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Row-major population -> facility-major tiles, for every instance of the
// launch.  colT[col_base + (tile*32W + j)*G + g] (j < 32W) = bits over
// individuals tile*32G + 32g + b of that instance.  One warp per (instance,
// tile, g, w) job; grid-stride over the jobs.
// ---------------------------------------------------------------------------
__global__ void k_pop_to_columns(const uint32_t *__restrict__ masks, const pm_prob *__restrict__ probs, int K,
                                 pm_prob one, int64_t jobs, int32_t G, uint32_t *__restrict__ colT)
{
    pm_grid_dependency_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t job = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); job < jobs;
         job += warps_total) {
        const pm_prob *pr = &one;
        if (K > 1)
            pr = probs + find_prob(K, job, [&](int k) { return probs[k].job_base; });
        const int64_t lj = job - pr->job_base;
        const int32_t W = pr->W;
        const int32_t w = (int32_t)(lj % W);
        const int64_t tg = lj / W;
        const int32_t g = (int32_t)(tg % G);
        const int64_t tile = tg / G;
        const int64_t t = tile * 32 * G + 32 * g + lane;
        const uint32_t x = (t < pr->pop) ? __ldg(masks + pr->word_base + t * W + w) : 0u;
        const uint32_t col = pm_transpose32(x, lane);
        colT[pr->col_base + (tile * (int64_t)W * 32 + (int64_t)w * 32 + lane) * G + g] = col;
    }
}

struct ScanEpilogue {
    int mode;                    // 0: store costs; 1: accept strictly cheaper candidates
    int64_t *costs;              // mode 0 (and optionally mode 1): candidate costs
    int64_t *cur_cost;           // mode 1
    uint32_t *cur_masks;         // mode 1
    const uint32_t *cand_masks;  // mode 1
    uint8_t *improved;           // mode 1, nullable
};

// The epilogue of one tile's individuals marked in fin_s (bit i of word i/32),
// one warp per individual: store the cost, or
// accept the candidate (copy its bitset, cost and improved flag) when it is
// strictly cheaper than the current individual.
template <int G>
__device__ __forceinline__ void apply_epilogue(const unsigned long long *acc_s, const uint32_t *fin_s, const pm_prob &pr,
                                               int64_t ind0, int warp, int nwarps, int lane, const ScanEpilogue &ep)
{
    const int32_t W = pr.W;
    for (int i = warp; i < G * 32; i += nwarps) {
        const int64_t t = ind0 + i;
        if (t >= pr.pop)
            break;
        if (!((fin_s[i >> 5] >> (i & 31)) & 1u))
            continue;
        const int64_t sum = (int64_t)acc_s[i];
        if (ep.costs != nullptr && lane == 0)
            ep.costs[pr.out_base + t] = sum;
        if (ep.mode == 1 && sum < ep.cur_cost[pr.ind_base + t]) {
            const int64_t row = pr.word_base + t * W;
            for (int q = lane; q < W; q += 32)
                ep.cur_masks[row + q] = ep.cand_masks[row + q];
            if (lane == 0) {
                ep.cur_cost[pr.ind_base + t] = sum;
                if (ep.improved)
                    ep.improved[pr.ind_base + t] = 1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The column scan kernel (with the split reduction and epilogue fused), over
// every instance of the launch.  Persistent: CTA b takes work items b, b +
// gridDim.x, ...; within an instance item = split * tiles + tile, so the CTAs
// running at the same time walk the same clients for different tiles and
// the rows they stream are shared through L2.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(1024) k_scan_columns(const pm_prob *__restrict__ probs, int K, pm_prob one,
                                                       int64_t items, const uint32_t *__restrict__ colT,
                                                       const uint32_t *__restrict__ active,
                                                       unsigned long long *__restrict__ accum,
                                                       int *__restrict__ tickets, int *__restrict__ err,
                                                       ScanEpilogue ep, uint32_t stall)
{
    // the previous kernel of the stream may still run until pm_grid_dependency_wait(): before it only the
    // constant tables (Pi', Delta', the launch's problem table) are read
    extern __shared__ __align__(128) uint32_t colbits[];  // [32W][G]
    __shared__ unsigned long long acc_s[G * 32];
    __shared__ uint32_t a0_s[G], fin_s[G];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int last_s;
    __shared__ pm_prob pr_s;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    // a launch armed by pm_debug_scan_timeout stalls its odd-numbered CTAs; the even ones finish their items, so
    // the stalled launch leaves partial sums (and tile tickets) behind, as a real timeout would
    const bool stalled = stall != 0u && (blockIdx.x & 1u) != 0u;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t phase = 0;
    int64_t loaded_tile = -1;  // global tile index of the tile in shared memory
    bool waited = false;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        if (threadIdx.x == 0)
            pr_s = (K > 1) ? probs[find_prob(K, item, [&](int k) { return probs[k].item_base; })] : one;
        __syncthreads();
        const pm_prob &pr = pr_s;
        const int64_t li = item - pr.item_base;
        const int64_t tile = li % pr.tiles;
        const int64_t split = li / pr.tiles;
        const int64_t gtile = pr.tile_base + tile;
        const int64_t ind0 = tile * 32 * G;  // first individual of the tile, within the instance
        const int32_t W = pr.W, L = pr.L;
        const int64_t pop = pr.pop, stride = pr.stride;
        const uint16_t *__restrict__ pi = pr.pi;
        const int32_t *__restrict__ delta = pr.delta;
        const bool reload = gtile != loaded_tile;

        // first steps of this warp's first two clients (constant tables), loaded while the tile lands
        const int64_t c_begin = split * pr.cps;
        const int64_t c_end = (c_begin + pr.cps < pr.n) ? c_begin + pr.cps : pr.n;
        auto load = [&](int64_t cc, int base, uint32_t &j, int32_t &dl) {
            const int r = base + lane;
            if (cc < c_end && r < L) {
                j = __ldg(pi + cc * stride + r);
                dl = __ldg(delta + cc * stride + r);
            } else {
                j = 0;
                dl = 0;
            }
        };
        int64_t c = c_begin + warp;
        uint32_t j_cur, j_nxt, j_nc, j_nc1;
        int32_t d_cur, d_nxt, d_nc, d_nc1;
        load(c, 0, j_cur, d_cur);
        load(c, 32, j_nxt, d_nxt);
        load(c + nwarps, 0, j_nc, d_nc);
        load(c + nwarps, 32, j_nc1, d_nc1);
        if (!waited) {  // from here on: the columns, active bits and accumulators of the previous kernels
            pm_grid_dependency_wait();
            waited = true;
        }

        // stalled (failure-detection tests only): no copy is issued and nothing arrives on the barrier, so the
        // bounded wait below runs out with nothing in flight
        if (reload && threadIdx.x == 0 && !stalled) {
            const uint32_t tile_bytes = (uint32_t)W * 32u * G * 4u;
            mbar_arrive_expect_tx(&bar, tile_bytes);
            const char *src = reinterpret_cast<const char *>(colT + pr.col_base + tile * (int64_t)W * 32 * G);
            char *dst = reinterpret_cast<char *>(colbits);
            for (uint32_t off = 0; off < tile_bytes; off += 32768u) {
                const uint32_t sz = (tile_bytes - off) < 32768u ? (tile_bytes - off) : 32768u;
                bulk_g2s(dst + off, src + off, sz, &bar);
            }
        }
        if (warp < G) {
            const int64_t t = ind0 + 32 * warp + lane;
            const int64_t tg = pr.ind_base + t;
            const bool on = (t < pop) && (active == nullptr || ((__ldg(active + (tg >> 5)) >> (tg & 31)) & 1u));
            const uint32_t b = __ballot_sync(PM_FULL_MASK, on);
            if (lane == 0)
                a0_s[warp] = b;
        }
        for (int i = threadIdx.x; i < G * 32; i += blockDim.x)
            acc_s[i] = 0ull;

        if (reload) {
            // bounded wait for the tile (every thread waits)
            const uint32_t limit = stalled ? kStallSpinLimit : kSpinLimit;
            uint32_t spins = 0;
            while (!mbar_try_wait(&bar, phase)) {
                if (++spins > limit) {
                    if (threadIdx.x == 0)
                        atomicExch(err, (int)PM_ERR_TIMEOUT);
                    uint32_t extra = 0;  // the copy may still land: wait once more, bounded, then leave
                    while (!mbar_try_wait(&bar, phase) && ++extra < limit) {
                    }
                    return;
                }
            }
            phase ^= 1u;
            loaded_tile = gtile;
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

        if (any0 && c < c_end)
            scan_clients<G>(colbits, a0, c, c_end, nwarps, L, lane, pr.cum != 0, load, j_cur, d_cur, j_nxt, d_nxt, j_nc,
                            d_nc, j_nc1, d_nc1, acc);
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (acc[g])
                atomicAdd(&acc_s[g * 32 + lane], acc[g]);
        __syncthreads();

        bool finish = true;
        const uint32_t *fin = a0_s;  // individuals whose epilogue this CTA applies
        if (pr.splits > 1 && pr.packed) {
            // one atomic per individual carries the split's sum plus one count in the top 16 bits; the split
            // that brings the count to `splits` holds the total, applies that individual's epilogue and leaves
            // the word zero for the next launch -- no fences, no tile ticket
            for (int i = threadIdx.x; i < G * 32; i += blockDim.x) {
                const int64_t t = ind0 + i;
                bool last = false;
                if (t < pop && ((a0_s[i >> 5] >> (i & 31)) & 1u)) {
                    const unsigned long long add = acc_s[i] + (1ull << kCountShift);
                    const unsigned long long old = atomicAdd(accum + pr.ind_base + t, add);
                    if ((old >> kCountShift) == (unsigned long long)(pr.splits - 1)) {
                        acc_s[i] = (old + add) & ((1ull << kCountShift) - 1ull);
                        accum[pr.ind_base + t] = 0ull;
                        last = true;
                    }
                }
                const uint32_t b = __ballot_sync(PM_FULL_MASK, last);
                if ((i & 31) == 0)
                    fin_s[i >> 5] = b;
            }
            __syncthreads();
            fin = fin_s;
        } else if (pr.splits > 1) {
            // add this split's sums into the instance's accumulators; the last split of the tile
            // (atomic ticket) reads the totals and leaves the accumulators zero again
            for (int i = threadIdx.x; i < G * 32; i += blockDim.x) {
                const int64_t t = ind0 + i;
                if (t < pop && acc_s[i] != 0ull)
                    atomicAdd(accum + pr.ind_base + t, acc_s[i]);
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0)
                last_s = (atomicAdd(tickets + gtile, 1) == (int)pr.splits - 1) ? 1 : 0;
            __syncthreads();
            finish = last_s != 0;
            if (finish) {
                __threadfence();
                for (int i = threadIdx.x; i < G * 32; i += blockDim.x) {
                    const int64_t t = ind0 + i;
                    if (t < pop) {
                        acc_s[i] = __ldcg(accum + pr.ind_base + t);
                        accum[pr.ind_base + t] = 0ull;
                    }
                }
                if (threadIdx.x == 0)
                    tickets[gtile] = 0;  // every CTA of the tile has taken its ticket: reset for the next launch
                __syncthreads();
            }
        }
        if (finish)
            apply_epilogue<G>(acc_s, fin, pr, ind0, warp, nwarps, lane, ep);
        __syncthreads();  // shared state (tile, acc_s, a0_s, pr_s) is reused by the next item
    }
}

// ---------------------------------------------------------------------------
// Row kernel (fallback for m too large for facility-major tiles): one warp
// per individual, the individual's mask in shared memory, one ballot per
// 32 ranks.  Grid: (ceil(pop / warps), splits).  The mask is the bitset
// (W words per warp) or, with kBytes, the bitset expanded to one byte per
// facility (32 W bytes per warp; a facility's test is one byte load instead
// of a word load, a shift and a mask) -- the byte-mask layout the autotuner
// weighs against the bit layouts.
// ---------------------------------------------------------------------------
template <bool kBytes>
__global__ void __launch_bounds__(256) k_scan_rows(const uint16_t *__restrict__ pi, const int32_t *__restrict__ delta,
                                                   int64_t n, int32_t L, int64_t stride,
                                                   const uint32_t *__restrict__ masks, int32_t W, int64_t pop,
                                                   const uint32_t *__restrict__ active, int64_t clients_per_split,
                                                   int cum, unsigned long long *__restrict__ partial)
{
    pm_grid_dependency_wait();
    extern __shared__ __align__(16) uint32_t rowbits[];  // [warps][W] words, or [warps][8W] words of bytes
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * nwarps + warp;
    const int split = blockIdx.y;
    if (t >= pop)
        return;
    if (active != nullptr && !((__ldg(active + (t >> 5)) >> (t & 31)) & 1u))
        return;
    uint32_t *x = rowbits + (int64_t)warp * W * (kBytes ? 8 : 1);
    for (int w = lane; w < W; w += 32) {
        const uint32_t v = __ldg(masks + t * W + w);
        if constexpr (kBytes) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // facilities 32w + 4q .. 32w + 4q + 3 -> bytes 0..3 of word 8w + q
                const uint32_t b = v >> (4 * q);
                x[8 * w + q] = (b & 1u) | ((b & 2u) << 7) | ((b & 4u) << 14) | ((b & 8u) << 21);
            }
        } else {
            x[w] = v;
        }
    }
    __syncwarp();
    const uint8_t *xb = reinterpret_cast<const uint8_t *>(x);
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
            bool open;
            if constexpr (kBytes)
                open = (r < L) && xb[j] != 0;
            else
                open = (r < L) && ((x[j >> 5] >> (j & 31)) & 1u);
            const uint32_t hit = __ballot_sync(PM_FULL_MASK, open);
            if (!hit) {
                if (!cum)
                    carry += __reduce_add_sync(PM_FULL_MASK, dl);
                continue;
            }
            int32_t cs = dl;  // cumulative tables: already the running sum
            if (!cum) {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(PM_FULL_MASK, cs, o);
                    if (lane >= o)
                        cs += y;
                }
                cs += carry;
            }
            acc += (unsigned long long)(uint32_t)__shfl_sync(PM_FULL_MASK, cs, __ffs(hit) - 1);
            break;
        }
    }
    if (lane == 0)
        partial[(int64_t)split * pop + t] = acc;
}

// ---------------------------------------------------------------------------
// Sum the splits of the row kernel and apply the epilogue (one warp per
// individual).
// ---------------------------------------------------------------------------
__global__ void k_reduce_accept(unsigned long long *__restrict__ partial, int splits, int64_t pop,
                                const uint32_t *__restrict__ active, ScanEpilogue ep, int32_t W)
{
    pm_grid_dependency_wait();
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= pop)
        return;
    if (active != nullptr && !((__ldg(active + (t >> 5)) >> (t & 31)) & 1u))
        return;
    unsigned long long s = 0ull;
    for (int k = lane; k < splits; k += 32) {
        s += partial[(int64_t)k * pop + t];
        partial[(int64_t)k * pop + t] = 0ull;  // leave the scratch zero, as the column kernel does
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(PM_FULL_MASK, s, o);
    const int64_t sum = (int64_t)s;
    if (ep.costs != nullptr && lane == 0)
        ep.costs[t] = sum;
    if (ep.mode == 1 && sum < ep.cur_cost[t]) {
        for (int w = lane; w < W; w += 32)
            ep.cur_masks[t * W + w] = ep.cand_masks[t * W + w];
        if (lane == 0) {
            ep.cur_cost[t] = sum;
            if (ep.improved)
                ep.improved[t] = 1;
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

// Self-test of the bounded wait: an mbarrier that nothing arrives on (a flag
// nothing sets).  The wait gives up after `limit` polls, records
// PM_ERR_TIMEOUT and returns -- the same exit the scan kernel takes.
__global__ void k_wait_selftest(int *__restrict__ err, uint32_t limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t spins = 0;
    while (!mbar_try_wait(&bar, 0)) {
        if (++spins > limit) {
            if (threadIdx.x == 0)
                atomicExch(err, (int)PM_ERR_TIMEOUT);
            return;
        }
    }
}

template <int G>
const void *scan_fn()
{
    return reinterpret_cast<const void *>(k_scan_columns<G>);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

static size_t column_smem_bytes(int64_t W, int G) { return (size_t)W * 32 * G * 4; }

// Let `fn` take all the opt-in shared memory its static shared memory leaves.
template <typename F>
static pm_status allow_dynamic_smem(const pm_instance *inst, F *fn)
{
    cudaFuncAttributes fa;
    PM_CUDA(cudaFuncGetAttributes(&fa, fn));
    const size_t cap = inst->smem_optin > fa.sharedSizeBytes ? inst->smem_optin - fa.sharedSizeBytes : 0;
    PM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
    return PM_OK;
}

pm_status pm_fitness_init(const pm_instance *inst)
{
    PM_TRY(allow_dynamic_smem(inst, k_scan_columns<1>));
    PM_TRY(allow_dynamic_smem(inst, k_scan_columns<2>));
    PM_TRY(allow_dynamic_smem(inst, k_scan_columns<4>));
    PM_TRY(allow_dynamic_smem(inst, k_scan_rows<false>));
    PM_TRY(allow_dynamic_smem(inst, k_scan_rows<true>));
    return PM_OK;
}


// Resident CTAs per SM of the column kernel for (G, warps) at this instance's W.
static int column_ctas_per_sm(const pm_instance *inst, int G, int warps)
{
    const size_t smem = column_smem_bytes(inst->W, G);
    int nb = 0;
    const void *fn = G == 4 ? scan_fn<4>() : (G == 2 ? scan_fn<2>() : scan_fn<1>());
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, warps * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

pm_eval_plan pm_plan_eval_with(const pm_instance *inst, int64_t pop, int G, int warps, int splits_hint)
{
    pm_eval_plan plan;
    const size_t budget = inst->smem_optin > 4096 ? inst->smem_optin - 4096 : 0;
    int64_t ctas_per_sm = 0;
    if (G > 0 && column_smem_bytes(inst->W, G) <= budget)
        ctas_per_sm = column_ctas_per_sm(inst, G, warps);
    if (G <= 0 || ctas_per_sm <= 0) {
        plan.groups = 0;  // row kernel
        plan.warps = 8;
        plan.tiles = pm_ceil_div(pop, plan.warps);
        plan.bytes = (G < 0 && (size_t)plan.warps * inst->W * 32 + 1024 <= inst->smem_optin) ? 1 : 0;
        ctas_per_sm = 8;
    } else {
        plan.groups = G;
        plan.warps = warps;
        plan.tiles = pm_ceil_div(pop, 32 * G);
    }
    const int64_t slots = (int64_t)inst->sm_count * ctas_per_sm;
    // default: about four work items per resident CTA slot; every warp gets at least one client
    const int64_t max_splits = std::max<int64_t>(1, inst->n / (plan.groups ? plan.warps : 1));
    int64_t splits = splits_hint > 0 ? splits_hint : pm_ceil_div(4 * slots, std::max<int64_t>(1, plan.tiles));
    if (splits_hint <= 0 && splits > max_splits)  // too few clients for that: one item per slot instead
        splits = std::max<int64_t>(1, std::min<int64_t>(max_splits, slots / std::max<int64_t>(1, plan.tiles)));
    splits = std::min<int64_t>(std::max<int64_t>(1, splits), std::min<int64_t>(max_splits, 65535));
    plan.splits = (int)splits;
    plan.grid = plan.groups ? std::min<int64_t>(plan.tiles * splits, slots) : plan.tiles;
    return plan;
}

pm_eval_plan pm_plan_eval(const pm_instance *inst, int64_t pop)
{
    {
        std::lock_guard<std::mutex> g(inst->plan_mu);
        auto it = inst->tuned.find(pop);
        if (it != inst->tuned.end())
            return it->second;
    }
    const size_t budget = inst->smem_optin > 4096 ? inst->smem_optin - 4096 : 0;
    int G = kMaxG;
    // fewer groups for small populations or when the tile does not fit: keep >= 8 tiles, or >= 16 where a
    // client's walk is short (expected first open rank (m+1)/(p+1) below 32: one or two steps, so the
    // launch's fixed costs weigh more than the per-step savings of wide tiles)
    const int64_t min_tiles = (inst->m + 1) < 32 * (inst->p + 1) ? 16 : 8;
    while (G > 1 && (pop <= (int64_t)32 * (G / 2) * min_tiles || column_smem_bytes(inst->W, G) > budget))
        G /= 2;
    // 32 warps when only one CTA fits per SM, else 16
    const int warps = 2 * column_smem_bytes(inst->W, G) + 8192 > inst->smem_optin ? 32 : 16;
    return pm_plan_eval_with(inst, pop, G, warps, 0);
}

size_t pm_plan_partial_bytes(const pm_eval_plan &plan, int64_t pop)
{
    // column kernel: one self-resetting accumulator per individual; row kernel: one sum per split and individual
    const int64_t per = plan.groups ? 1 : plan.splits;
    return (size_t)pm_round_up(per * std::max<int64_t>(pop, 1) * 8, 256);
}

size_t pm_plan_ticket_bytes(const pm_eval_plan &plan) { return (size_t)pm_round_up(plan.tiles * 4, 256); }

size_t pm_plan_column_bytes(const pm_instance *inst, const pm_eval_plan &plan)
{
    if (!plan.groups)
        return 0;
    return (size_t)plan.tiles * column_smem_bytes(inst->W, plan.groups);
}

pm_prob pm_single_prob(const pm_instance *inst, const pm_eval_plan &plan, int64_t pop)
{
    pm_prob pr{};
    pr.pi = inst->pi;
    pr.delta = inst->delta;
    pr.n = inst->n;
    pr.stride = inst->stride;
    pr.L = (int32_t)inst->L;
    pr.W = (int32_t)inst->W;
    pr.m = (int32_t)inst->m;
    pr.p = (int32_t)inst->p;
    pr.cum = inst->cum ? 1 : 0;
    pr.packed = pm_packed_reduction_ok(inst, plan.splits) ? 1 : 0;
    pr.pop = pop;
    pr.tiles = plan.tiles;
    pr.splits = plan.splits;
    pr.cps = pm_ceil_div(inst->n, plan.splits);
    return pr;  // every base 0
}

// Scan launches still to be armed by pm_debug_scan_timeout.
static std::atomic<long long> g_scan_stall{0};

static bool take_stall()
{
    return pm_take_scan_stall();
}

bool pm_take_scan_stall()
{
    long long k = g_scan_stall.load();
    while (k > 0) {
        if (g_scan_stall.compare_exchange_weak(k, k - 1))
            return true;
    }
    return false;
}

extern "C" pm_status pm_debug_scan_timeout(int64_t launches, int64_t *pending)
{
    const long long prev = g_scan_stall.exchange(launches > 0 ? (long long)launches : 0);
    if (pending)
        *pending = (int64_t)prev;
    return PM_OK;
}

// Enqueue the transpose (unless the caller wrote the columns) and the column
// scan of a launch; smem = the tile bytes of the launch's widest instance.
static pm_status launch_transpose(const uint32_t *masks, const pm_prob *probs, int K, const pm_prob &one, int64_t jobs,
                                  int G, uint32_t *colT, cudaStream_t stream)
{
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>(pm_ceil_div(jobs, threads / 32), (int64_t)2048);
    PM_CUDA(pm_launch(k_pop_to_columns, (unsigned)blocks, threads, 0, stream, masks, probs, K, one, jobs, G, colT));
    return PM_OK;
}

pm_status pm_launch_columns(const pm_instance *inst, const pm_eval_plan &plan, const uint32_t *masks, int64_t pop,
                            uint32_t *colT, cudaStream_t stream)
{
    if (pop <= 0)
        return PM_OK;
    if (plan.groups == 0)
        return PM_ERR_UNSUPPORTED;
    return launch_transpose(masks, nullptr, 1, pm_single_prob(inst, plan, pop), plan.tiles * plan.groups * inst->W,
                            plan.groups, colT, stream);
}

pm_status pm_launch_scan(const pm_scan_launch &L, const pm_accept_args &acc, int64_t *costs, size_t smem,
                         cudaStream_t stream)
{
    if (L.items <= 0)
        return PM_OK;
    ScanEpilogue ep;
    ep.mode = acc.mode;
    ep.costs = costs;
    ep.cur_cost = acc.cur_cost;
    ep.cur_masks = acc.cur_masks;
    ep.cand_masks = acc.cand_masks;
    ep.improved = acc.improved;
    const int G = L.groups;
    if (!acc.columns_ready)
        PM_TRY(launch_transpose(L.masks, L.probs_dev, L.K, L.one, L.jobs, G, L.colT, stream));
    const int threads = L.warps * 32;
    const unsigned grid = (unsigned)L.grid;
    unsigned long long *accum = reinterpret_cast<unsigned long long *>(L.accum);
    const uint32_t stall = take_stall() ? 1u : 0u;
#define PM_SCAN_ARGS L.probs_dev, L.K, L.one, L.items, L.colT, L.active, accum, L.tickets, L.err, ep, stall
    switch (G) {
    case 1:
        PM_CUDA(pm_launch(k_scan_columns<1>, grid, threads, smem, stream, PM_SCAN_ARGS));
        break;
    case 2:
        PM_CUDA(pm_launch(k_scan_columns<2>, grid, threads, smem, stream, PM_SCAN_ARGS));
        break;
    default:
        PM_CUDA(pm_launch(k_scan_columns<4>, grid, threads, smem, stream, PM_SCAN_ARGS));
        break;
    }
#undef PM_SCAN_ARGS
    return PM_OK;
}

pm_status pm_launch_eval(const pm_instance *inst, const pm_eval_plan &plan, const uint32_t *masks, int64_t pop,
                         const uint32_t *active, int64_t *costs, int64_t *partials_i64, int *tickets, uint32_t *colT,
                         int *err, const pm_accept_args &acc, cudaStream_t stream)
{
    if (pop <= 0)
        return PM_OK;
    unsigned long long *partials = reinterpret_cast<unsigned long long *>(partials_i64);
    if (plan.groups) {
        pm_scan_launch L;
        L.groups = plan.groups;
        L.warps = plan.warps;
        L.grid = plan.grid;
        L.K = 1;
        L.one = pm_single_prob(inst, plan, pop);
        L.items = plan.tiles * plan.splits;
        L.jobs = plan.tiles * plan.groups * inst->W;
        L.masks = masks;
        L.colT = colT;
        L.active = active;
        L.accum = partials_i64;
        L.tickets = tickets;
        L.err = err;
        return pm_launch_scan(L, acc, costs, column_smem_bytes(inst->W, plan.groups), stream);
    }
    ScanEpilogue ep;
    ep.mode = acc.mode;
    ep.costs = costs;
    ep.cur_cost = acc.cur_cost;
    ep.cur_masks = acc.cur_masks;
    ep.cand_masks = acc.cand_masks;
    ep.improved = acc.improved;
    const int64_t cps = pm_ceil_div(inst->n, plan.splits);
    const size_t smem = (size_t)plan.warps * inst->W * 4 * (plan.bytes ? 8 : 1);
    dim3 grid((unsigned)plan.tiles, (unsigned)plan.splits);
    if (plan.bytes)
        PM_CUDA(pm_launch(k_scan_rows<true>, grid, plan.warps * 32, smem, stream, inst->pi, inst->delta, inst->n,
                          (int32_t)inst->L, inst->stride, masks, (int32_t)inst->W, pop, active, cps,
                          inst->cum ? 1 : 0, partials));
    else
        PM_CUDA(pm_launch(k_scan_rows<false>, grid, plan.warps * 32, smem, stream, inst->pi, inst->delta, inst->n,
                          (int32_t)inst->L, inst->stride, masks, (int32_t)inst->W, pop, active, cps,
                          inst->cum ? 1 : 0, partials));
    const int64_t threads = 256;
    const int64_t blocks = pm_ceil_div(pop * 32, threads);
    PM_CUDA(pm_launch(k_reduce_accept, (unsigned)blocks, (unsigned)threads, 0, stream, partials, plan.splits, pop,
                      active, ep, (int32_t)inst->W));
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
// Layout inside the array: [0, 256) error word, then the tile tickets, the
// facility-major population copy and the partial sums, each 256-byte
// aligned.
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
    const size_t tick = pm_plan_ticket_bytes(plan);
    const size_t cols = (size_t)pm_round_up((int64_t)pm_plan_column_bytes(inst, plan), 256);
    const size_t part = pm_plan_partial_bytes(plan, pop);
    if (256 + tick + cols + part > kNoAllocScratchBytes)
        return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(inst->device));
    unsigned char *base = nullptr;
    PM_TRY(noalloc_scratch(inst->device, &base));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *err = reinterpret_cast<int *>(base);
    int *tickets = reinterpret_cast<int *>(base + 256);
    uint32_t *colT = reinterpret_cast<uint32_t *>(base + 256 + tick);
    int64_t *partials = reinterpret_cast<int64_t *>(base + 256 + tick + cols);
    // the array keeps the previous call's contents: the tile tickets and the
    // accumulators must start at zero.  The error word is not cleared here: it
    // keeps the first failure until pm_eval_status reads and clears it (it is
    // zero when the library is loaded).
    PM_CUDA(cudaMemsetAsync(base + 256, 0, tick, s));
    PM_CUDA(cudaMemsetAsync(partials, 0, part, s));
    pm_accept_args acc;
    return pm_launch_eval(inst, plan, masks, pop, nullptr, costs, partials, tickets, colT, err, acc, s);
}

extern "C" pm_status pm_eval_status(pm_instance *inst, void *stream)
{
    if (!inst)
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> guard(inst->lock);
    PM_CUDA(cudaSetDevice(inst->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *na = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (inst->device < kNoAllocMaxDevices)
            na = static_cast<unsigned char *>(g_noalloc_addr[inst->device]);
    }
    int words[2] = {0, 0};
    PM_CUDA(cudaMemcpyAsync(&words[0], inst->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (na)
        PM_CUDA(cudaMemcpyAsync(&words[1], na, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaStreamSynchronize(s));
    if (words[0])
        PM_TRY(pm_reset_eval_scratch(inst, s));
    if (words[1]) {
        PM_CUDA(cudaMemsetAsync(na, 0, 256, s));
        PM_CUDA(cudaStreamSynchronize(s));
    }
    return (pm_status)(words[0] ? words[0] : words[1]);
}

extern "C" pm_status pm_selftest_bounded_wait(int device, void *stream)
{
    if (device < 0)
        return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *err = nullptr;
    PM_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&err), sizeof(int), s));
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32, 0, s>>>(err, 1u << 14);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(err, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    PM_CUDA(e);
    return (pm_status)h;
}
