// The genetic algorithm of Sections 3.1, 3.2.2 and 4.3-4.5, run entirely on
// the device, for one instance or for a batch of instances at once (every
// kernel below covers all instances of the GA in one launch).
//
// One generation (the paper's Evolve call plus the host's population
// renewal and migration):
//   k_ga_init_warp   fresh random population by Floyd sampling of a p-subset
//                    (k_ga_init where its shared memory does not fit), or with
//                    k_ga_init_comb the paper's generation (Section 4.1): a
//                    uniform multi-word rank below C(m, p) and the combination
//                    of that rank in lexicographic order; for generation g > 0
//                    slot 0 of every deme gets that deme's best of generation
//                    g-1 (Section 4.5, variant (i); variant (ii) puts every
//                    deme's best into deme 0).
//   evaluate         the column scan (fitness.cu, Section 4.2).
//   crossover r      k_ga_crossover builds every child (butterfly partner
//                    t XOR (D >> (1 + r mod lg D)), Section 3.2.2 step 3), the
//                    scan evaluates the children and replaces a parent by its
//                    child iff strictly cheaper.  Children are built from the
//                    population as it was when the round started.
//   mutation q       k_ga_mutate rotates the whole bitset or a block of it
//                    (Section 4.4) for individuals not yet improved in this
//                    generation; the first strictly cheaper mutant replaces
//                    the individual (Section 3.2.2 step 5).  For one instance
//                    on the column path all tries are built and evaluated at
//                    once (k_ga_mutate_all, one scan, k_ga_mutate_accept).
//   k_ga_generation_end  lowest (cost, index) per deme (Section 3.2.2 step
//                    7); the last deme of an instance updates its global best
//                    (strict improvement), saturation counter, trace and
//                    counters; the last instance sets the loop condition
//                    (k_ga_generation_end_one: the same for one instance in
//                    one CTA).
// The operators also write the facility-major copy of their output that the
// scan reads, so no evaluation needs a separate transpose.  A call of several
// generations is one CUDA graph: a gate kernel and a conditional while-node
// whose body is one generation; a call of one generation launches a plain
// graph of the body (pm_ga_run, a single call, captures only the one it
// launches).  An instance that reached its saturation limit stops: its
// kernels do nothing while the others go on.  A GA's device buffers (and the
// speculative cycle's candidates) are slices of one allocation.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), stateless, keyed by
// (seed) with counter (generation, unit, op * 2^16 + slot / 4, stream id);
// draw `slot` is word slot & 3.  U[0, N) = floor(u * N / 2^32).  Instance k
// of a batch uses stream id (base + k).

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pm_alloc.h"
#include "pm_common.cuh"
#include "scan_walk.cuh"

// batch.cu
pm_status pm_batch_ga_plan(pm_batch *b, int64_t pop, pm_multi_plan &out);
pm_status pm_batch_ga_plan_candidates(pm_batch *b, int64_t pop, int64_t popQ, pm_multi_plan &out);
// learn.cu
pm_status pm_learn_prepare(const pm_instance *inst, cudaStream_t s);
pm_status pm_launch_swap_stats(const pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *gain,
                               int32_t *cap, int64_t *loss, int32_t *assign, cudaStream_t s);
// the two above in one kernel when the statistics fit in shared memory (the arrays are then left unwritten)
pm_status pm_launch_learned_candidates(const pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *gain,
                                       int32_t *cap, int64_t *loss, int32_t *assign, const int64_t *costs, int T,
                                       int32_t *moves, uint16_t *x, cudaStream_t s);
pm_status pm_launch_candidates(const pm_instance *inst, const uint32_t *masks, int64_t pop, const int64_t *gain,
                               const int32_t *cap, const int64_t *loss, const int32_t *assign, const int64_t *costs,
                               int T, int32_t *moves, uint16_t *x, cudaStream_t s);
pm_status pm_model_forward_dev(pm_model *md, const void *x_dev, int64_t rows, float *y_dev, cudaStream_t s);
const std::vector<const pm_instance *> &pm_batch_instances(const pm_batch *b);

namespace {

constexpr uint32_t OP_INIT = 0x001u;
constexpr uint32_t OP_COMB = 0x002u;  // combinadic rank words (Section 4.1)
constexpr int kCombTries = 64;        // rejection tries for a uniform rank below C(m, p)
constexpr uint32_t OP_XOVER = 0x100u;
constexpr uint32_t OP_MUT = 0x200u;

struct ga_dev {            // per instance
    long long gen;         // index of the next generation
    long long best_cost;   // -1 until the first generation finishes
    long long sat;         // generations since the best last improved
    long long evals;       // fitness evaluations so far
    long long total_gens;  // generations run since creation
    long long saturation;  // S (0 = off)
    long long *trace;      // this instance's trace for the current step
    int stop;              // saturation reached
    int deme_ticket;       // k_ga_generation_end: demes done this generation (zero at rest)
};

struct ga_glob {
    long long remaining;  // generations left in the current step
    long long step_gens;  // generations run in the current step
    int alive;            // instances not stopped
    int done;             // k_ga_generation_end tickets (instances done this generation)
};

struct ga_prob {  // per instance layout of the GA arrays
    int64_t pop, D, NB;
    int32_t W, m, p, lgD;
    int64_t ind_base;    // cost, improved, active bits (multiple of 32)
    int64_t word_base;   // X, Xc rows
    int64_t grp_base;    // first 32-individual group
    int64_t deme_base;   // deme_cost index
    int64_t dword_base;  // deme_best rows
    int64_t best_base;   // best bitset
    int64_t col_base;    // facility-major tiles
    uint32_t sid;
    uint32_t team;  // migration variant (ii): all deme bests into deme 0
};

// ----------------------------- Philox4x32-10 --------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw_block(uint64_t seed, uint32_t gen, uint32_t unit, uint32_t op, uint32_t blk,
                                            uint32_t sid)
{
    return philox10(make_uint4(gen, unit, (op << 16) + blk, sid), (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, uint32_t i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

__device__ __forceinline__ uint32_t uniform_below(uint32_t u, uint32_t N)
{
    return (uint32_t)(((unsigned long long)u * N) >> 32);
}

__device__ __forceinline__ uint32_t lowest_bits(uint32_t x, int k)
{
    if (__popc(x) <= k)
        return x;
    uint32_t r = 0;
    for (int q = 0; q < k; ++q) {
        const uint32_t low = x & (0u - x);
        r |= low;
        x ^= low;
    }
    return r;
}

// Loads of data another CTA may have written earlier in the same kernel (the
// persistent generation kernel) go through L2 (kCG); the per-phase kernels
// read data of earlier launches and keep their usual loads.
template <bool kCG>
__device__ __forceinline__ uint32_t ld_row(const uint32_t *p)
{
    if constexpr (kCG)
        return __ldcg(p);
    else
        return *p;
}

template <bool kCG>
__device__ __forceinline__ uint32_t ld_ro(const uint32_t *p)
{
    if constexpr (kCG)
        return __ldcg(p);
    else
        return __ldg(p);
}

// Largest k with base(k) <= x.
template <typename F>
__device__ __forceinline__ int find_k(int K, int64_t x, F base)
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

// The instance owning 32-individual group `grp` (by value).
__device__ __forceinline__ ga_prob prob_of_group(const ga_prob *gps, int K, const ga_prob &one, int64_t grp, int &k)
{
    if (K == 1) {
        k = 0;
        return one;
    }
    k = find_k(K, grp, [&](int i) { return gps[i].grp_base; });
    return gps[k];
}

// Where the operator kernels write the facility-major copy the scan reads
// (colT == nullptr: the evaluation uses the row kernel and needs none).
struct ColumnsOut {
    uint32_t *colT;
    int32_t G;
};

// Transpose 32 rows (individuals t0 .. t0+31 of one instance, row r at
// rows + r*rs) into that instance's tiles; rows of individuals >= pop read
// as zero.  One warp, words w_begin, w_begin + w_step, ...
__device__ __forceinline__ void write_columns(const uint32_t *rows, int64_t rs, int64_t t0, const ga_prob &gp,
                                              ColumnsOut co, int lane, int w_begin, int w_step)
{
    if (co.colT == nullptr)
        return;
    const int32_t W = gp.W;
    const int64_t tile = t0 / (32 * co.G);
    const int32_t g = (int32_t)((t0 / 32) % co.G);
    for (int w = w_begin; w < W; w += w_step) {
        const uint32_t x = (t0 + lane < gp.pop) ? rows[(int64_t)lane * rs + w] : 0u;
        const uint32_t col = pm_transpose32(x, lane);
        co.colT[gp.col_base + (tile * (int64_t)W * 32 + (int64_t)w * 32 + lane) * co.G + g] = col;
    }
}

// The first 64 ranks of every row of one instance's tables (n = 0: none).
struct TablePrefix {
    const uint16_t *pi;
    const int32_t *delta;
    int64_t n, stride;
};

// ------------------------------- kernels -----------------------------------

__global__ void k_ga_begin(ga_glob *glob, ga_dev *st, int K, long long gens, long long *trace, unsigned *bar)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K)
        st[k].trace = trace ? trace + (long long)k * gens : nullptr;
    if (k == 0) {
        glob->remaining = gens;
        glob->step_gens = 0;
        if (bar)
            bar[0] = 0u;  // the persistent kernel's barrier starts with no arrivals, whatever a failed launch left
    }
}

__global__ void k_ga_gate(const ga_glob *glob, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, (glob->remaining > 0 && glob->alive > 0) ? 1u : 0u);
}

// Floyd sampling + migration, one warp per 32 individuals (lane = individual,
// the bitsets in shared memory when they fit, else in place in X); also
// clears the improved flags, sets the active bits and writes the columns.
__global__ void __launch_bounds__(32) k_ga_init(const ga_prob *__restrict__ gps, int K, ga_prob one,
                                                uint32_t *__restrict__ X, uint8_t *__restrict__ improved,
                                                uint32_t *__restrict__ active, const uint32_t *__restrict__ deme_best,
                                                uint64_t seed, const ga_dev *__restrict__ st, ColumnsOut co,
                                                int rows_in_smem)
{
    pm_grid_dependency_wait();
    extern __shared__ uint32_t rows_s[];  // [32][Ws], Ws = W | 1 (odd stride: conflict-free transposes)
    int k;
    const ga_prob gp = prob_of_group(gps, K, one, blockIdx.x, k);
    const int lane = threadIdx.x;
    const int64_t t0 = (blockIdx.x - gp.grp_base) * 32;
    const int64_t t = t0 + lane;
    const int32_t W = gp.W, Ws = W | 1;
    if (st[k].stop) {
        if (lane == 0)
            active[(gp.ind_base + t0) >> 5] = 0u;
        return;
    }
    const uint32_t gen = (uint32_t)st[k].gen;
    uint32_t *row = rows_in_smem ? rows_s + (int64_t)lane * Ws : X + gp.word_base + t * W;
    if (t < gp.pop) {
        improved[gp.ind_base + t] = 0;
        // migration (Section 4.5): variant (i) puts deme b's best of the previous generation into slot 0 of
        // deme b; variant (ii) puts all of them into deme 0, deme b's best into slot b
        const bool migrant = gen > 0 && (gp.team ? t < gp.NB : (t % gp.D) == 0);
        if (migrant) {
            const uint32_t *src = deme_best + gp.dword_base + (gp.team ? t : t / gp.D) * W;
            for (int w = 0; w < W; ++w)
                row[w] = src[w];
        } else {
            for (int w = 0; w < W; ++w)
                row[w] = 0u;
            uint4 v = make_uint4(0, 0, 0, 0);
            for (int q = 0; q < gp.p; ++q) {
                if ((q & 3) == 0)
                    v = draw_block(seed, gen, (uint32_t)t, OP_INIT, (uint32_t)q >> 2, gp.sid);
                const uint32_t j = (uint32_t)(gp.m - gp.p + q);
                const uint32_t c = uniform_below(word_of(v, q & 3), j + 1);
                const uint32_t pick = ((row[c >> 5] >> (c & 31)) & 1u) ? j : c;
                row[pick >> 5] |= 1u << (pick & 31);
            }
        }
    }
    const uint32_t on = __ballot_sync(PM_FULL_MASK, t < gp.pop);
    if (lane == 0)
        active[(gp.ind_base + t0) >> 5] = on;
    __syncwarp();
    if (rows_in_smem) {
        // copy the 32 rows out (rows of consecutive individuals are contiguous in X)
        const int64_t nrows = (gp.pop - t0) < 32 ? (gp.pop - t0) : 32;
        for (int64_t idx = lane; idx < nrows * W; idx += 32)
            X[gp.word_base + t0 * W + idx] = rows_s[(idx / W) * Ws + (idx % W)];
        write_columns(rows_s, Ws, t0, gp, co, lane, 0, 1);
    } else {
        write_columns(X + gp.word_base + t0 * W, W, t0, gp, co, lane, 0, 1);
    }
}

// Individual t of generation gen into the W-word row `row` (shared memory), by
// one warp: a migrant (Section 4.5) copies its deme's best of the previous
// generation; any other individual is a fresh p-subset by Floyd's sampling,
// the lanes computing the p Philox draws in parallel (lane l the counter
// blocks l, l + 32, ...; draw q is uniform below m - p + q + 1) into `draws`
// (p words, shared).  Floyd's insertions are sequential -- draw q takes c_q
// unless c_q is already in the set, else m - p + q -- and are resolved 32 at
// a time, lane l taking draw q0 + l: against the set of the earlier batches
// by one bit test, against the earlier lanes of its batch by iterating
// "take m - p + q iff c_q is in the set or is an earlier lane's current
// pick" to its fixed point (after iteration i lanes 0..i hold the sequential
// picks, so at most 32 iterations, usually one).  The picks are distinct
// (m - p + q exceeds every earlier pick), so the batch is inserted with one
// atomic OR per lane.
template <bool kCG>
__device__ __forceinline__ void fresh_individual(const ga_prob &gp, int64_t t, uint32_t gen, uint64_t seed,
                                                 const uint32_t *__restrict__ deme_best, uint32_t *row,
                                                 uint32_t *draws, int lane)
{
    const int32_t W = gp.W, m = gp.m, p = gp.p;
    const bool migrant = gen > 0 && (gp.team ? t < gp.NB : (t % gp.D) == 0);
    if (migrant) {
        const uint32_t *src = deme_best + gp.dword_base + (gp.team ? t : t / gp.D) * W;
        for (int w = lane; w < W; w += 32)
            row[w] = ld_row<kCG>(src + w);
    } else {
        for (int w = lane; w < W; w += 32)
            row[w] = 0u;
        for (int b = lane; 4 * b < p; b += 32) {
            const uint4 v = draw_block(seed, gen, (uint32_t)t, OP_INIT, (uint32_t)b, gp.sid);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int q = 4 * b + i;
                if (q < p)
                    draws[q] = uniform_below(word_of(v, (uint32_t)i), (uint32_t)(m - p + q + 1));
            }
        }
        __syncwarp();
        for (int q0 = 0; q0 < p; q0 += 32) {
            const int q = q0 + lane;
            const bool live = q < p;
            const int nb = (p - q0) < 32 ? (p - q0) : 32;
            const uint32_t c = live ? draws[q] : 0u;
            const uint32_t jj = (uint32_t)(m - p + q);
            const bool inset = live && ((row[c >> 5] >> (c & 31)) & 1u) != 0u;
            uint32_t pick = inset ? jj : c;
            for (int it = 0; it < nb; ++it) {
                bool taken = false;  // c is the current pick of an earlier lane of the batch
                for (int l = 0; l < nb; ++l) {
                    const uint32_t pl = __shfl_sync(PM_FULL_MASK, pick, l);
                    taken |= (l < lane) && (pl == c);
                }
                const uint32_t np = (inset || taken) ? jj : c;
                const bool changed = __any_sync(PM_FULL_MASK, live && np != pick);
                pick = np;
                if (!changed)
                    break;
            }
            if (live)
                atomicOr(&row[pick >> 5], 1u << (pick & 31));
            __syncwarp();
        }
    }
    __syncwarp();
}

// The same fresh population as k_ga_init with one warp per individual
// (fresh_individual: the lanes compute the p Philox draws of Floyd's sampling
// in parallel and resolve its insertions 32 at a time on the warp's bitset in
// shared memory).  CTA = 32 warps = 32 individuals; needs 32 * (W + p) words
// of shared memory.
__global__ void __launch_bounds__(1024) k_ga_init_warp(const ga_prob *__restrict__ gps, int K, ga_prob one,
                                                       uint32_t *__restrict__ X, uint8_t *__restrict__ improved,
                                                       uint32_t *__restrict__ active,
                                                       const uint32_t *__restrict__ deme_best, uint64_t seed,
                                                       const ga_dev *__restrict__ st, ColumnsOut co,
                                                       TablePrefix tp)
{
    // the tables are constant: their rows' first ranks go to L2 while the previous kernel finishes, for the
    // generation's first scan (the only one that may find them evicted)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tp.n; i += (int64_t)gridDim.x * blockDim.x) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(tp.pi + i * tp.stride));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(tp.delta + i * tp.stride));
        if (tp.stride > 32)  // the row's second 128-byte line of Delta' (rows are padded to a multiple of 32)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(tp.delta + i * tp.stride + 32));
    }
    pm_grid_dependency_wait();
    extern __shared__ uint32_t wrows[];  // [32][W] bitsets, then [32][p] draws
    __shared__ uint32_t on_s;
    int k;
    const ga_prob gp = prob_of_group(gps, K, one, blockIdx.x, k);
    const int lane = threadIdx.x & 31;
    const int j = threadIdx.x >> 5;
    const int64_t t0 = (blockIdx.x - gp.grp_base) * 32;
    const int64_t t = t0 + j;
    const int32_t W = gp.W, m = gp.m, p = gp.p;
    if (st[k].stop) {
        if (threadIdx.x == 0)
            active[(gp.ind_base + t0) >> 5] = 0u;
        return;
    }
    if (threadIdx.x == 0)
        on_s = 0u;
    __syncthreads();
    const uint32_t gen = (uint32_t)st[k].gen;
    uint32_t *row = wrows + (int64_t)j * W;
    uint32_t *draws = wrows + (int64_t)32 * W + (int64_t)j * p;
    if (t < gp.pop) {
        if (lane == 0) {
            improved[gp.ind_base + t] = 0;
            atomicOr(&on_s, 1u << j);
        }
        fresh_individual<false>(gp, t, gen, seed, deme_best, row, draws, lane);
        for (int w = lane; w < W; w += 32)
            X[gp.word_base + t * W + w] = row[w];
    }
    __syncthreads();
    if (threadIdx.x == 0)
        active[(gp.ind_base + t0) >> 5] = on_s;
    write_columns(wrows, W, t0, gp, co, lane, j, 32);
}

// ------------------- combinadic chromosome generation -----------------------
// Section 4.1 draws a chromosome as the i-th p-combination of {0..m-1} in
// lexicographic order for a random i below C(m, p).  C(900, 90) is about
// 2^418, so ranks are multi-word integers: K words, least significant
// first.  A warp holds one such integer with Q = K/32 (rounded up to a power
// of two) consecutive words per lane, lane l words [lQ, lQ + Q).
//
// Binomial table: the unranking below only meets C(b + d, b) with b <= p
// and d <= m - p (b = choices left, d = positions left minus choices left);
// entry (b, d) sits at word ((b * (m - p + 1)) + d) * K.  Every entry is at
// most C(m, p), so K words (the host's estimate of bits(C(m, p)) / 32, plus a
// spare word) hold it.  After the entries, one 64-bit head per entry, same
// index: (bit length << 32) | the entry's 32 most significant bits (the entry
// itself below 2^32).  Heads order like the values they head, and equal heads
// below 2^32 mean equal values.

// word offset of the heads: after the entries' words, rounded up to 8 bytes
static inline size_t comb_head_offset(size_t entries, int32_t K) { return (entries * (size_t)K + 1) & ~(size_t)1; }

__device__ __forceinline__ uint64_t big_head(uint32_t top_word, uint32_t below, int32_t wtop)
{
    const int32_t r = 32 - __clz(top_word);  // bits used in the top word (top_word != 0)
    const int32_t bits = 32 * wtop + r;
    const uint32_t t32 = (wtop == 0 || r == 32) ? top_word : ((top_word << (32 - r)) | (below >> r));
    return ((uint64_t)(uint32_t)bits << 32) | t32;
}

// Pascal's rule along anti-diagonals s = b + d (each entry needs (b - 1, d)
// and (b, d - 1) of the diagonal before): one CTA, a barrier per diagonal.
// *overflow is set if a sum ever carries out of K words.
__global__ void __launch_bounds__(1024) k_comb_table(uint32_t *__restrict__ T, uint64_t *__restrict__ H, int32_t m,
                                                     int32_t p, int32_t K, int *__restrict__ overflow)
{
    const int64_t D1 = (int64_t)m - p + 1;
    for (int32_t s = 0; s <= m; ++s) {
        const int32_t b_lo = s - (m - p) > 0 ? s - (m - p) : 0;
        const int32_t b_hi = s < p ? s : p;
        for (int32_t b = b_lo + (int32_t)threadIdx.x; b <= b_hi; b += (int32_t)blockDim.x) {
            const int32_t d = s - b;
            uint32_t *out = T + ((int64_t)b * D1 + d) * K;
            if (b == 0 || d == 0) {
                out[0] = 1u;
                for (int32_t w = 1; w < K; ++w)
                    out[w] = 0u;
            } else {
                const uint32_t *x = T + ((int64_t)(b - 1) * D1 + d) * K;
                const uint32_t *y = T + ((int64_t)b * D1 + d - 1) * K;
                uint32_t carry = 0;
                for (int32_t w = 0; w < K; ++w) {
                    const unsigned long long v = (unsigned long long)x[w] + y[w] + carry;
                    out[w] = (uint32_t)v;
                    carry = (uint32_t)(v >> 32);
                }
                if (carry)
                    atomicExch(overflow, 1);
            }
            int32_t wt = K - 1;  // every entry is at least 1
            while (wt > 0 && out[wt] == 0u)
                --wt;
            H[(int64_t)b * D1 + d] = big_head(out[wt], wt > 0 ? out[wt - 1] : 0u, wt);
        }
        __syncthreads();
    }
}

template <int Q>
__device__ __forceinline__ void big_load(const uint32_t *__restrict__ e, int32_t K, int lane, uint32_t (&v)[Q])
{
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int32_t w = lane * Q + q;
        v[q] = w < K ? __ldg(e + w) : 0u;
    }
}

// x < y for warp-held integers.
template <int Q>
__device__ __forceinline__ bool big_less(const uint32_t (&x)[Q], const uint32_t (&y)[Q])
{
    int cmp = 0;
#pragma unroll
    for (int q = Q - 1; q >= 0; --q)
        if (cmp == 0 && x[q] != y[q])
            cmp = x[q] < y[q] ? -1 : 1;
    const uint32_t ne = __ballot_sync(PM_FULL_MASK, cmp != 0);
    if (ne == 0u)
        return false;
    return __shfl_sync(PM_FULL_MASK, cmp, 31 - __clz(ne)) < 0;
}

// Word w (the same for every lane) of a warp-held integer.
template <int Q>
__device__ __forceinline__ uint32_t big_word(const uint32_t (&x)[Q], int32_t w)
{
    uint32_t v = 0u;
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (q == (w % Q))
            v = x[q];
    return __shfl_sync(PM_FULL_MASK, v, w / Q);
}

// Head (as in the binomial table) of a nonzero warp-held integer, and its most significant nonzero word.
template <int Q>
__device__ __forceinline__ uint64_t big_head_warp(const uint32_t (&x)[Q], int32_t &wtop)
{
    int hiq = -1;
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (x[q] != 0u)
            hiq = q;
    const uint32_t nz = __ballot_sync(PM_FULL_MASK, hiq >= 0);
    const int top = 31 - __clz(nz);
    wtop = top * Q + __shfl_sync(PM_FULL_MASK, hiq, top);
    const uint32_t top_word = big_word<Q>(x, wtop);
    const uint32_t below = wtop > 0 ? big_word<Q>(x, wtop - 1) : 0u;
    return big_head(top_word, below, wtop);
}

// x -= y for warp-held integers with x >= y.  Each lane subtracts its words;
// a lane passes a borrow up if it generated one, or if it received one and
// its difference is zero.  Those two lane masks G and P give the borrow into
// every lane at once: the carries of the 32-bit sum G + (G | P).
template <int Q>
__device__ __forceinline__ void big_sub(uint32_t (&x)[Q], const uint32_t (&y)[Q], int lane)
{
    uint32_t borrow = 0;
    bool zero = true;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint32_t a = x[q], b = y[q];
        const uint32_t d = a - b - borrow;
        borrow = (a < b || (a == b && borrow)) ? 1u : 0u;
        x[q] = d;
        zero = zero && d == 0u;
    }
    const uint32_t G = __ballot_sync(PM_FULL_MASK, borrow != 0u);
    const uint32_t P = __ballot_sync(PM_FULL_MASK, zero);
    const uint32_t in = (G + (G | P)) ^ G ^ (G | P);
    if ((in >> lane) & 1u) {
        uint32_t b = 1u;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const uint32_t a = x[q];
            x[q] = a - b;
            b = (a < b) ? 1u : 0u;
        }
    }
}

// Fresh chromosomes by Section 4.1 (rank by bounded rejection on Philox
// words, then lexicographic unranking) + migration, for single-instance GAs.
// CTA = 32 warps = 32 individuals; warp j builds individual t0 + j's row in
// X, then the CTA writes the columns.
template <int Q>
__global__ void __launch_bounds__(1024) k_ga_init_comb(ga_prob gp, uint32_t *__restrict__ X,
                                                       uint8_t *__restrict__ improved, uint32_t *__restrict__ active,
                                                       const uint32_t *__restrict__ deme_best,
                                                       const uint32_t *__restrict__ T,
                                                       const uint64_t *__restrict__ H, int32_t K, uint64_t seed,
                                                       const ga_dev *__restrict__ st, ColumnsOut co)
{
    pm_grid_dependency_wait();
    __shared__ uint32_t on_s;
    const int lane = threadIdx.x & 31;
    const int j = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * 32;
    const int64_t t = t0 + j;
    const int32_t W = gp.W, m = gp.m, p = gp.p;
    if (st[0].stop) {
        if (threadIdx.x == 0)
            active[t0 >> 5] = 0u;
        return;
    }
    if (threadIdx.x == 0)
        on_s = 0u;
    __syncthreads();
    const uint32_t gen = (uint32_t)st[0].gen;
    if (t < gp.pop) {
        if (lane == 0) {
            improved[t] = 0;
            atomicOr(&on_s, 1u << j);
        }
        uint32_t *row = X + gp.word_base + t * W;
        const bool migrant = gen > 0 && (gp.team ? t < gp.NB : (t % gp.D) == 0);
        if (migrant) {
            const uint32_t *src = deme_best + gp.dword_base + (gp.team ? t : t / gp.D) * W;
            for (int w = lane; w < W; w += 32)
                row[w] = src[w];
        } else {
            const int64_t D1 = (int64_t)m - p + 1;
            auto entry = [&](int32_t b, int32_t d) { return T + ((int64_t)b * D1 + d) * K; };
            // C(m, p), its bit length and exact word count
            uint32_t C[Q];
            big_load<Q>(entry(p, m - p), K, lane, C);
            int hiq = -1;
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (C[q] != 0u)
                    hiq = q;
            const uint32_t nz = __ballot_sync(PM_FULL_MASK, hiq >= 0);
            const int top = 31 - __clz(nz);  // C >= 2, so some word is nonzero
            const int top_q = __shfl_sync(PM_FULL_MASK, hiq, top);
            uint32_t top_word = 0u;
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (q == top_q)
                    top_word = C[q];
            top_word = __shfl_sync(PM_FULL_MASK, top_word, top);
            const int32_t wtop = top * Q + top_q;                  // most significant nonzero word
            const int32_t bits = 32 * wtop + (32 - __clz(top_word));  // bit length of C(m, p)
            const int32_t Kc = wtop + 1;
            const uint32_t topmask = (bits - 32 * wtop) == 32 ? 0xffffffffu : ((1u << (bits - 32 * wtop)) - 1u);
            // rank: try r uses draws r*Kc .. r*Kc + Kc - 1 (word w = draw r*Kc + w)
            uint32_t x[Q];
            bool got = false;
            for (int r = 0; r < kCombTries && !got; ++r) {
                uint32_t u[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const int32_t w = lane * Q + q;
                    u[q] = 0u;
                    if (w < Kc) {
                        const uint32_t slot = (uint32_t)(r * Kc + w);
                        u[q] = word_of(draw_block(seed, gen, (uint32_t)t, OP_COMB, slot >> 2, gp.sid), slot & 3u);
                        if (w == wtop)
                            u[q] &= topmask;
                    }
                }
                if (big_less<Q>(u, C)) {
#pragma unroll
                    for (int q = 0; q < Q; ++q)
                        x[q] = u[q];
                    got = true;
                }
            }
            if (!got) {
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    x[q] = 0u;
            }
            // unrank.  State: next position e, k still to choose, d = m - e - k, and y = C(m - e, k) - x
            // (1 <= y; x = the rank among the combinations of the remaining positions).  Skipping s
            // positions passes over C(m - e, k) - C(m - e - s, k) combinations (hockey stick), so the next
            // element is e + s* with s* the smallest s where C(k + d - s - 1, k) < y; then y loses that
            // binomial, k drops by one and d by s*.  A warp tests 32 values of s at once on the heads.
            for (int w = lane; w < W; w += 32)
                row[w] = 0u;
            __syncwarp();
            int32_t k = p, e = 0, d = m - p;
            int32_t cur_w = 0;
            uint32_t cur = 0u;
            auto take = [&](int32_t pos) {
                if ((pos >> 5) != cur_w) {
                    if (lane == 0 && cur)
                        row[cur_w] = cur;
                    cur_w = pos >> 5;
                    cur = 0u;
                }
                cur |= 1u << (pos & 31);
            };
            uint32_t y[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q)
                y[q] = C[q];
            big_sub<Q>(y, x, lane);
            int32_t ywtop;
            uint64_t hy = big_head_warp<Q>(y, ywtop);
            // heads of the first 32 candidates, C(k + d - 1 - lane, k)
            uint64_t hc = (d - 1 - lane >= 0) ? __ldg(H + (int64_t)k * D1 + (d - 1 - lane)) : 0ull;
            while (k > 0) {
                if (d == 0) {  // as many positions left as choices: take them all
                    for (int32_t q = 0; q < k; ++q)
                        take(e + q);
                    break;
                }
                int32_t s_star = -1;
                for (int32_t s0 = 0; s_star < 0; s0 += 32) {
                    const int32_t dd = d - 1 - (s0 + lane);  // candidate s = s0 + lane tests C(k + dd, k)
                    if (s0 > 0)
                        hc = dd >= 0 ? __ldg(H + (int64_t)k * D1 + dd) : 0ull;
                    // dd < 0: the binomial is 0 < y.  Different heads decide; equal heads below 2^32 mean equal
                    // values; otherwise compare the words from y's top word down (rare)
                    bool less = dd < 0 || hc < hy;
                    bool open = dd >= 0 && hc == hy && (hy >> 32) > 32u;
                    const uint32_t *ew = T + ((int64_t)k * D1 + (dd >= 0 ? dd : 0)) * K;
                    for (int32_t w = ywtop; w >= 0 && __any_sync(PM_FULL_MASK, open); --w) {
                        const uint32_t yw = big_word<Q>(y, w);
                        if (open) {
                            const uint32_t v = __ldg(ew + w);
                            if (v != yw) {
                                less = v < yw;
                                open = false;
                            }
                        }
                    }
                    const uint32_t hit = __ballot_sync(PM_FULL_MASK, less);
                    if (hit)
                        s_star = s0 + __ffs(hit) - 1;
                }
                take(e + s_star);
                const int32_t dsub = d - s_star - 1;  // y loses C(k + dsub, k) (nothing when dsub < 0)
                const int32_t k1 = k - 1, d1 = d - s_star;
                // the next step's first candidates, loaded while y is updated
                hc = (k1 > 0 && d1 - 1 - lane >= 0) ? __ldg(H + (int64_t)k1 * D1 + (d1 - 1 - lane)) : 0ull;
                if (dsub >= 0) {
                    uint32_t c[Q];
                    big_load<Q>(entry(k, dsub), K, lane, c);
                    big_sub<Q>(y, c, lane);
                    hy = big_head_warp<Q>(y, ywtop);
                }
                k = k1;
                d = d1;
                e += s_star + 1;
            }
            if (lane == 0 && cur)
                row[cur_w] = cur;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        active[t0 >> 5] = on_s;
    write_columns(X + gp.word_base + t0 * W, W, t0, gp, co, lane, j, 32);
}

// The child F of C and its couple Kp (W-word rows) for the pair's draws (r1, i), built by one warp (Section
// 4.3, reading R6): the positions r1, r1+1, ... (circularly) are visited as W+1 segments -- word w0 = r1/32 from
// bit r1%32 up, the following words, and word w0 below bit r1%32; a warp scan of the per-segment counts of 0->1
// and 1->0 candidates (C != couple) tells each segment how many of its candidates to take, the lowest bits
// (earliest positions) of a segment first.  Returns whether i candidates of each kind were found (the crossover
// succeeded); the same on every lane.
template <bool kCG>
__device__ __forceinline__ bool crossover_child(const uint32_t *C, const uint32_t *Kp, uint32_t *F, int32_t W,
                                                uint32_t r1, int i, int lane)
{
    const int w0 = (int)(r1 >> 5);
    const uint32_t b0 = r1 & 31u;
    int c01 = 0, c10 = 0;    // candidates in the segments of earlier rounds
    uint32_t w0change = 0u;  // changes to word w0 (first and last segment)
    for (int base = 0; base <= W; base += 32) {
        const int sidx = base + lane;
        uint32_t z = 0u, o = 0u, cw = 0u;
        int w = -1;
        if (sidx <= W) {
            uint32_t seg;
            if (sidx == 0) {
                w = w0;
                seg = 0xffffffffu << b0;
            } else if (sidx < W) {
                w = w0 + sidx;
                if (w >= W)
                    w -= W;
                seg = 0xffffffffu;
            } else {
                w = w0;
                seg = b0 ? ((1u << b0) - 1u) : 0u;
            }
            cw = ld_row<kCG>(C + w);
            const uint32_t kw = ld_row<kCG>(Kp + w);
            z = ~cw & kw & seg;
            o = cw & ~kw & seg;
        }
        // exclusive warp scan of the two counts packed in one word
        const uint32_t nz = __popc(z), no = __popc(o);
        const uint32_t packed = nz | (no << 16);
        uint32_t incl = packed;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(PM_FULL_MASK, incl, off);
            if (lane >= off)
                incl += y;
        }
        const uint32_t excl = incl - packed;
        const int before01 = c01 + (int)(excl & 0xffffu);
        const int before10 = c10 + (int)(excl >> 16);
        const int take01 = min(max(i - before01, 0), (int)nz);
        const int take10 = min(max(i - before10, 0), (int)no);
        const uint32_t change = lowest_bits(z, take01) | lowest_bits(o, take10);
        if (w >= 0) {
            if (sidx == 0 || sidx == W)
                w0change |= change;
            else
                F[w] = cw ^ change;
        }
        const uint32_t tot = __shfl_sync(PM_FULL_MASK, incl, 31);
        c01 += (int)(tot & 0xffffu);
        c10 += (int)(tot >> 16);
    }
    w0change = __reduce_or_sync(PM_FULL_MASK, w0change);
    if (lane == 0)
        F[w0] = ld_row<kCG>(C + w0) ^ w0change;
    return c01 >= i && c10 >= i;
}

// One crossover round (Section 4.3).  CTA = 32 warps = 32 individuals; warp
// j builds the child of individual t0 + j (crossover_child).
__global__ void __launch_bounds__(1024) k_ga_crossover(const ga_prob *__restrict__ gps, int K, ga_prob one,
                                                       const uint32_t *__restrict__ X, uint32_t *__restrict__ Xc,
                                                       uint32_t *__restrict__ active, uint32_t round, uint64_t seed,
                                                       ga_dev *__restrict__ st, ColumnsOut co, int rows_in_smem)
{
    extern __shared__ uint32_t crows[];  // [32][W] the children, when rows_in_smem (transposed from here)
    __shared__ uint32_t valid_s;
    int k;
    const ga_prob gp = prob_of_group(gps, K, one, blockIdx.x, k);
    const int lane = threadIdx.x & 31;
    const int j = threadIdx.x >> 5;
    const int64_t t0 = (blockIdx.x - gp.grp_base) * 32;
    const int64_t t = t0 + j;
    const int32_t W = gp.W;
    // the generation counter and stop flag were written by an earlier generation's end, and the draws depend on
    // nothing else: both are read before waiting for the previous kernel (the evaluation of the last round)
    const bool stopped = st[k].stop != 0;
    const int64_t stride = gp.D >> (1 + ((int)round % gp.lgD));
    const int64_t partner = t ^ stride;
    const uint32_t pair = (uint32_t)(t < partner ? t : partner);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (!stopped && t < gp.pop)
        v = draw_block(seed, (uint32_t)st[k].gen, pair, OP_XOVER + round, 0, gp.sid);
    pm_grid_dependency_wait();
    if (stopped) {
        if (threadIdx.x == 0)
            active[(gp.ind_base + t0) >> 5] = 0u;
        return;
    }
    if (threadIdx.x == 0)
        valid_s = 0u;
    __syncthreads();
    const int p = gp.p;
    if (t < gp.pop) {
        const uint32_t r1 = uniform_below(v.x, (uint32_t)gp.m);
        const int i = 1 + (int)uniform_below(v.y, (uint32_t)(p / 2));
        uint32_t *F = rows_in_smem ? crows + (int64_t)j * W : Xc + gp.word_base + t * W;
        const bool ok = crossover_child<false>(X + gp.word_base + t * W, X + gp.word_base + partner * W, F, W, r1,
                                               i, lane);
        if (rows_in_smem) {
            __syncwarp();
            for (int w = lane; w < W; w += 32)
                Xc[gp.word_base + t * W + w] = F[w];
        }
        if (lane == 0 && p / 2 > 0 && ok)
            atomicOr(&valid_s, 1u << j);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        active[(gp.ind_base + t0) >> 5] = valid_s;
        if (valid_s)
            atomicAdd(reinterpret_cast<unsigned long long *>(&st[k].evals), (unsigned long long)__popc(valid_s));
    }
    if (rows_in_smem)  // rows of individuals past the population were never written: write_columns reads them as 0
        write_columns(crows, W, t0, gp, co, lane, j, 32);
    else
        write_columns(Xc + gp.word_base + t0 * W, W, t0, gp, co, lane, j, 32);
}

// 32 bits of the bitset C starting at bit position s (s may be as low as
// -31; bits read from below position 0 are zero).
template <bool kCG>
__device__ __forceinline__ uint32_t bits_from(const uint32_t *C, int32_t W, int64_t s)
{
    if (s < 0)
        return ld_ro<kCG>(C) << (uint32_t)(-s);
    const int64_t q = s >> 5;
    const uint32_t r = (uint32_t)(s & 31);
    const uint32_t lo = ld_ro<kCG>(C + q);
    const uint32_t hi = (q + 1 < W) ? ld_ro<kCG>(C + q + 1) : 0u;
    return __funnelshift_r(lo, hi, r);
}

__device__ __forceinline__ uint32_t range_mask(int64_t lo, int64_t hi)  // bits [lo, hi) of a word, 0 <= lo <= hi <= 32
{
    const uint32_t upto = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
    const uint32_t below = lo >= 32 ? 0xffffffffu : ((1u << lo) - 1u);
    return upto & ~below;
}

// Try q's shift of individual t: circular or block shift with the draws of
// operation OP_MUT + q -- kind and direction from draws 0 and 1, the circular
// amount or the block's two ends from draws 2 and 3, the block's amount from
// draw 4.  The mutant rotates bits [a, a+len) left by kl: F[a+i] =
// C[a + (i+kl) mod len].  Depends on nothing a kernel of the generation
// writes, so callers may take it before waiting for the previous kernel.
struct MutantShift {
    int64_t a, len, kl;
};

__device__ __forceinline__ MutantShift mutant_shift(int32_t m, uint64_t seed, uint32_t gen, uint32_t t, uint32_t q,
                                                    uint32_t sid)
{
    const uint4 v0 = draw_block(seed, gen, (uint32_t)t, OP_MUT + q, 0, sid);
    const uint32_t kind = uniform_below(v0.x, 2u);
    const uint32_t right = uniform_below(v0.y, 2u);
    int64_t a, len, kk;
    if (kind == 0) {
        a = 0;
        len = m;
        kk = 1 + uniform_below(v0.z, (uint32_t)(m - 1));
    } else {
        const uint4 v1 = draw_block(seed, gen, (uint32_t)t, OP_MUT + q, 1, sid);
        const uint32_t x = uniform_below(v0.z, (uint32_t)m);
        uint32_t y = uniform_below(v0.w, (uint32_t)(m - 1));
        if (y >= x)
            ++y;
        const uint32_t lo = x < y ? x : y, hi = x < y ? y : x;
        a = lo;
        len = hi - lo + 1;
        kk = 1 + uniform_below(v1.x, hi - lo);
    }
    MutantShift ms;
    ms.a = a;
    ms.len = len;
    ms.kl = right ? (len - kk) : kk;  // rotate left by kl, 1 <= kl < len
    return ms;
}

// The mutant F of the W-word row C for a shift, built by a warp (lanes over words).
template <bool kCG = false>
__device__ __forceinline__ void mutant_row_shift(const uint32_t *__restrict__ C, uint32_t *__restrict__ F, int32_t W,
                                                 const MutantShift &ms, int lane)
{
    const int64_t a = ms.a, len = ms.len, kl = ms.kl;
    const int64_t pwrap = a + len - kl;  // positions >= pwrap wrap to the start of the block
    for (int w = lane; w < W; w += 32) {
        const int64_t pos0 = (int64_t)w * 32;
        const int64_t in_lo = a > pos0 ? a : pos0;
        const int64_t in_hi = (a + len) < (pos0 + 32) ? (a + len) : (pos0 + 32);
        const uint32_t cw = ld_ro<kCG>(C + w);
        if (in_lo >= in_hi) {
            F[w] = cw;
            continue;
        }
        uint32_t out = cw & ~range_mask(in_lo - pos0, in_hi - pos0);
        const int64_t e1 = in_hi < pwrap ? in_hi : pwrap;
        if (in_lo < e1)
            out |= bits_from<kCG>(C, W, pos0 + kl) & range_mask(in_lo - pos0, e1 - pos0);
        const int64_t s2 = in_lo > pwrap ? in_lo : pwrap;
        if (s2 < in_hi)
            out |= bits_from<kCG>(C, W, pos0 + kl - len) & range_mask(s2 - pos0, in_hi - pos0);
        F[w] = out;
    }
}

// Try q's mutant F of the W-word row C (m bits) of individual t, built by a warp.
template <bool kCG = false>
__device__ __forceinline__ void mutant_row(const uint32_t *__restrict__ C, uint32_t *__restrict__ F, int32_t W,
                                           int32_t m, uint64_t seed, uint32_t gen, uint32_t t, uint32_t q,
                                           uint32_t sid, int lane)
{
    mutant_row_shift<kCG>(C, F, W, mutant_shift(m, seed, gen, t, q, sid), lane);
}

// One mutation try (Section 4.4).  CTA = 32 warps = 32 individuals; warp j
// rotates individual t0 + j's bits [a, a+len) left by kl: F[a+i] =
// C[a + (i+kl) mod len].  Each output word is at most three pieces, each a
// funnel-shifted 32-bit read of C.
__global__ void __launch_bounds__(1024) k_ga_mutate(const ga_prob *__restrict__ gps, int K, ga_prob one,
                                                    const uint32_t *__restrict__ X, uint32_t *__restrict__ Xc,
                                                    uint32_t *__restrict__ active,
                                                    const uint8_t *__restrict__ improved, uint32_t q, uint64_t seed,
                                                    ga_dev *__restrict__ st, ColumnsOut co)
{
    pm_grid_dependency_wait();
    __shared__ uint32_t on_s;
    int k;
    const ga_prob gp = prob_of_group(gps, K, one, blockIdx.x, k);
    const int lane = threadIdx.x & 31;
    const int j = threadIdx.x >> 5;
    const int64_t t0 = (blockIdx.x - gp.grp_base) * 32;
    const int64_t t = t0 + j;
    const int32_t W = gp.W, m = gp.m;
    if (st[k].stop) {
        if (threadIdx.x == 0)
            active[(gp.ind_base + t0) >> 5] = 0u;
        return;
    }
    if (threadIdx.x == 0)
        on_s = 0u;
    __syncthreads();
    if (t < gp.pop && improved[gp.ind_base + t] == 0) {
        if (lane == 0)
            atomicOr(&on_s, 1u << j);
        mutant_row(X + gp.word_base + t * W, Xc + gp.word_base + t * W, W, m, seed, (uint32_t)st[k].gen, (uint32_t)t,
                   q, gp.sid, lane);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        active[(gp.ind_base + t0) >> 5] = on_s;
        if (on_s)
            atomicAdd(reinterpret_cast<unsigned long long *>(&st[k].evals), (unsigned long long)__popc(on_s));
    }
    write_columns(Xc + gp.word_base + t0 * W, W, t0, gp, co, lane, j, 32);
}

// Speculative mutation cycle (GAs on the column path).  Every try mutates the
// individual as it stood when the cycle began (an individual stops at its
// first strict improvement), so all Q tries of all individuals can be built
// and evaluated at once and the first improving try kept: candidate u =
// q * pop + t of an instance is try q of its individual t.  The result and
// the evaluation count (tries an individual reaches) equal the cycle run try
// by try; the tries after an individual's first improvement are evaluated
// but not counted.  CTA = 32 warps = 32 candidates of one instance; gqs[k]
// (or oneq for one instance) lays out instance k's Q x pop candidates: their
// rows, facility-major tiles, active bits and costs (ind_base), and their
// first 32-candidate group (grp_base).
__global__ void __launch_bounds__(1024, 2) k_ga_mutate_all(const ga_prob *__restrict__ gps,
                                                        const ga_prob *__restrict__ gqs, int K, ga_prob one,
                                                        ga_prob oneq, int32_t Q, const uint32_t *__restrict__ X,
                                                        uint32_t *__restrict__ XQ, uint32_t *__restrict__ activeQ,
                                                        const uint8_t *__restrict__ improved, uint64_t seed,
                                                        const ga_dev *__restrict__ st, ColumnsOut coQ,
                                                        int rows_in_smem)
{
    extern __shared__ uint32_t mrows[];  // [32][W] the mutants, when rows_in_smem (transposed from here)
    __shared__ uint32_t on_s;
    int k = 0;
    ga_prob gp = one, gq = oneq;
    if (K > 1) {
        k = find_k(K, blockIdx.x, [&](int i) { return gqs[i].grp_base; });
        gp = gps[k];
        gq = gqs[k];
    }
    const int lane = threadIdx.x & 31;
    const int j = threadIdx.x >> 5;
    const int64_t u0 = ((int64_t)blockIdx.x - gq.grp_base) * 32;
    const int64_t u = u0 + j;
    const int32_t W = gp.W;
    // the shift's draws depend on the generation counter and the stop flag, written by an earlier generation's
    // end: taken before waiting for the previous kernel (the evaluation of the last crossover round)
    const bool stopped = st[k].stop != 0;
    const int64_t q_u = u / gp.pop, t_u = u - q_u * gp.pop;
    MutantShift ms{0, 1, 0};
    if (!stopped && u < gq.pop)
        ms = mutant_shift(gp.m, seed, (uint32_t)st[k].gen, (uint32_t)t_u, (uint32_t)q_u, gp.sid);
    pm_grid_dependency_wait();
    if (stopped) {
        if (threadIdx.x == 0)
            activeQ[(gq.ind_base + u0) >> 5] = 0u;
        return;
    }
    if (threadIdx.x == 0)
        on_s = 0u;
    __syncthreads();
    if (u < gq.pop) {
        const int64_t t = t_u;
        if (improved[gp.ind_base + t] == 0) {
            if (lane == 0)
                atomicOr(&on_s, 1u << j);
            uint32_t *F = rows_in_smem ? mrows + (int64_t)j * W : XQ + gq.word_base + u * W;
            mutant_row_shift(X + gp.word_base + t * W, F, W, ms, lane);
            if (rows_in_smem) {
                __syncwarp();
                for (int w = lane; w < W; w += 32)
                    XQ[gq.word_base + u * W + w] = F[w];
            }
        } else if (rows_in_smem) {
            for (int w = lane; w < W; w += 32)
                mrows[(int64_t)j * W + w] = 0u;  // not evaluated (inactive); its column bits are masked anyway
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        activeQ[(gq.ind_base + u0) >> 5] = on_s;
    if (rows_in_smem)
        write_columns(mrows, W, u0, gq, coQ, lane, j, 32);
    else
        write_columns(XQ + gq.word_base + u0 * W, W, u0, gq, coQ, lane, j, 32);
}

// Keep each individual's first improving try (warp per individual, 8 per
// CTA, individuals numbered as in the GA's scans: instance k's start at
// gps[k].ind_base) and count the tries it reaches: q + 1 for an improvement
// at try q, else Q; none for an individual already improved in this
// generation.
__global__ void __launch_bounds__(256) k_ga_mutate_accept(const ga_prob *__restrict__ gps,
                                                          const ga_prob *__restrict__ gqs, int K, ga_prob one,
                                                          ga_prob oneq, int32_t Q, uint32_t *__restrict__ X,
                                                          const uint32_t *__restrict__ XQ, int64_t *__restrict__ cost,
                                                          const int64_t *__restrict__ costQ,
                                                          uint8_t *__restrict__ improved, ga_dev *__restrict__ st)
{
    pm_grid_dependency_wait();
    __shared__ unsigned long long tries_s;
    __shared__ int k0_s;
    const int lane = threadIdx.x & 31;
    const int64_t gi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    auto inst_of = [&](int64_t x) { return K > 1 ? find_k(K, x, [&](int i) { return gps[i].ind_base; }) : 0; };
    if (threadIdx.x == 0) {
        tries_s = 0ull;
        k0_s = inst_of((int64_t)blockIdx.x * (blockDim.x >> 5));
    }
    __syncthreads();
    const int k = inst_of(gi);
    const ga_prob gp = K > 1 ? gps[k] : one, gq = K > 1 ? gqs[k] : oneq;
    const int64_t t = gi - gp.ind_base;
    const int32_t W = gp.W;
    if (t < gp.pop && !st[k].stop && improved[gp.ind_base + t] == 0) {
        const int64_t c0 = cost[gp.ind_base + t];
        int qs = Q;  // first improving try; every lane takes the same iterations and the same break
        for (int base = 0; base < Q; base += 32) {
            const int q = base + lane;
            const bool hit = q < Q && costQ[gq.ind_base + (int64_t)q * gp.pop + t] < c0;
            const uint32_t b = __ballot_sync(PM_FULL_MASK, hit);
            if (b) {
                qs = base + __ffs(b) - 1;
                break;
            }
        }
        if (qs < Q) {
            const int64_t u = (int64_t)qs * gp.pop + t;
            for (int w = lane; w < W; w += 32)
                X[gp.word_base + t * W + w] = XQ[gq.word_base + u * W + w];
            if (lane == 0) {
                cost[gp.ind_base + t] = costQ[gq.ind_base + u];
                improved[gp.ind_base + t] = 1;
            }
        }
        if (lane == 0) {
            const unsigned long long tr = (unsigned long long)(qs < Q ? qs + 1 : Q);
            if (k == k0_s)
                atomicAdd(&tries_s, tr);
            else
                atomicAdd(reinterpret_cast<unsigned long long *>(&st[k].evals), tr);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && tries_s)
        atomicAdd(reinterpret_cast<unsigned long long *>(&st[k0_s].evals), tries_s);
}

// Generation end (Section 3.2.2 steps 7-8, Section 3.1 steps 13-14), one CTA
// per deme: the deme's lowest (cost, index) -> deme_best / deme_cost.  The
// last deme CTA of an instance (a ticket in its state, zero at rest) then
// takes that instance's global best, saturation, trace and counters; the last
// instance (a second ticket) advances the step and sets the loop condition.
__global__ void k_ga_generation_end(const ga_prob *__restrict__ gps, int K, ga_prob one,
                                    const uint32_t *__restrict__ X, const int64_t *__restrict__ cost,
                                    uint32_t *__restrict__ deme_best, int64_t *__restrict__ deme_cost,
                                    uint32_t *__restrict__ best, ga_dev *__restrict__ st, ga_glob *__restrict__ glob,
                                    cudaGraphConditionalHandle h, int in_graph)
{
    pm_grid_dependency_wait();
    __shared__ long long sc[32];
    __shared__ long long si[32];
    __shared__ long long win;
    __shared__ int improve, last_deme, last_inst;
    __shared__ int alive_s[32];
    int k = 0;
    ga_prob gp = one;
    if (K > 1) {
        k = find_k(K, blockIdx.x, [&](int i) { return gps[i].deme_base; });
        gp = gps[k];
    }
    ga_dev &s = st[k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const int64_t b = blockIdx.x - gp.deme_base;
    const int32_t W = gp.W;
    const bool running = !s.stop;

    // the deme's best
    if (running) {
        long long bc = 0x7fffffffffffffffLL, bi = 0x7fffffffffffffffLL;
        for (int64_t i = threadIdx.x; i < gp.D; i += blockDim.x) {
            const int64_t t = b * gp.D + i;
            const long long c = cost[gp.ind_base + t];
            if (c < bc || (c == bc && t < bi)) {
                bc = c;
                bi = t;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long oc = __shfl_xor_sync(PM_FULL_MASK, bc, o);
            const long long oi = __shfl_xor_sync(PM_FULL_MASK, bi, o);
            if (oc < bc || (oc == bc && oi < bi)) {
                bc = oc;
                bi = oi;
            }
        }
        if (lane == 0) {
            sc[warp] = bc;
            si[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; ++w)
                if (sc[w] < bc || (sc[w] == bc && si[w] < bi)) {
                    bc = sc[w];
                    bi = si[w];
                }
            win = bi;
            deme_cost[gp.deme_base + b] = bc;
        }
        __syncthreads();
        const int64_t tw = win;
        for (int w = threadIdx.x; w < W; w += blockDim.x)
            deme_best[gp.dword_base + b * W + w] = X[gp.word_base + tw * W + w];
    }

    // the instance's last deme CTA goes on
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_deme = (atomicAdd(&s.deme_ticket, 1) == (int)gp.NB - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!last_deme)
        return;
    __threadfence();
    if (running) {
        long long bc = 0x7fffffffffffffffLL, bi = 0x7fffffffffffffffLL;
        for (int64_t d = threadIdx.x; d < gp.NB; d += blockDim.x) {
            const long long c = __ldcg(reinterpret_cast<const long long *>(deme_cost) + gp.deme_base + d);
            if (c < bc || (c == bc && d < bi)) {
                bc = c;
                bi = d;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long oc = __shfl_xor_sync(PM_FULL_MASK, bc, o);
            const long long oi = __shfl_xor_sync(PM_FULL_MASK, bi, o);
            if (oc < bc || (oc == bc && oi < bi)) {
                bc = oc;
                bi = oi;
            }
        }
        if (lane == 0) {
            sc[warp] = bc;
            si[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; ++w)
                if (sc[w] < bc || (sc[w] == bc && si[w] < bi)) {
                    bc = sc[w];
                    bi = si[w];
                }
            const bool better = s.best_cost < 0 || bc < s.best_cost;
            improve = better ? 1 : 0;
            win = bi;
            if (better) {
                s.best_cost = bc;
                s.sat = 0;
            } else {
                s.sat += 1;
            }
        }
        __syncthreads();
        if (improve)
            for (int w = threadIdx.x; w < W; w += blockDim.x)
                best[gp.best_base + w] = __ldcg(deme_best + gp.dword_base + win * W + w);
        if (threadIdx.x == 0) {
            if (s.trace)
                s.trace[glob->step_gens] = s.best_cost;
            s.evals += gp.pop;
            s.gen += 1;
            s.total_gens += 1;
            s.stop = (s.saturation > 0 && s.sat >= s.saturation) ? 1 : 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s.deme_ticket = 0;  // every deme of the instance has taken its ticket: reset for the next generation
        __threadfence();
        last_inst = (atomicAdd(&glob->done, 1) == K - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!last_inst)
        return;
    __threadfence();
    int alive = 0;
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        alive += (*(volatile int *)&st[i].stop) ? 0 : 1;
    alive = __reduce_add_sync(PM_FULL_MASK, alive);
    if (lane == 0)
        alive_s[warp] = alive;
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0;
        for (int w = 0; w < nw; ++w)
            a += alive_s[w];
        glob->alive = a;
        glob->done = 0;
        glob->step_gens += 1;
        glob->remaining -= 1;
        if (in_graph)
            cudaGraphSetConditional(h, (glob->remaining > 0 && a > 0) ? 1u : 0u);
    }
}

// The generation end of a single-instance GA (same results as
// k_ga_generation_end) in one CTA of 1024 threads, without tickets: each warp
// reduces (cost, index) over its 32 individuals by a butterfly whose first
// lg(min(D, 32)) steps stay inside a deme; demes wider than a warp combine
// their warps' minima in shared memory.  The global best is the lowest
// (cost, index) over all individuals -- the same individual as the lowest
// (cost, deme) over the deme bests.  Rows are copied by all threads.
__global__ void __launch_bounds__(1024) k_ga_generation_end_one(ga_prob gp, const uint32_t *__restrict__ X,
                                                                const int64_t *__restrict__ cost,
                                                                uint32_t *__restrict__ deme_best,
                                                                int64_t *__restrict__ deme_cost,
                                                                uint32_t *__restrict__ best, ga_dev *__restrict__ st,
                                                                ga_glob *__restrict__ glob,
                                                                cudaGraphConditionalHandle h, int in_graph)
{
    pm_grid_dependency_wait();
    __shared__ long long wc[32], wi[32];  // per-warp minima of the current 1024-individual tile
    __shared__ long long gc[32], gi[32];  // per-warp minima over all tiles
    __shared__ int win_s[1024];           // winner of each deme of the tile (D <= 32: one per D lanes)
    __shared__ long long gwin;
    __shared__ int improve;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ga_dev &s = st[0];
    const bool running = !s.stop;
    const int32_t W = gp.W;
    const int64_t D = gp.D;
    const int seg = D < 32 ? (int)D : 32;
    constexpr long long kNone = 0x7fffffffffffffffLL;
    if (running) {
        long long mc = kNone, mi = kNone;  // this warp's minimum over all tiles (lane 0)
        for (int64_t t0 = 0; t0 < gp.pop; t0 += 1024) {
            const int64_t t = t0 + threadIdx.x;
            long long c = kNone, i = kNone;
            if (t < gp.pop) {
                c = cost[gp.ind_base + t];
                i = t;
            }
            long long sc = c, si = i;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long oc = __shfl_xor_sync(PM_FULL_MASK, c, o);
                const long long oi = __shfl_xor_sync(PM_FULL_MASK, i, o);
                if (oc < c || (oc == c && oi < i)) {
                    c = oc;
                    i = oi;
                }
                if (o == seg / 2) {  // the deme's (or the warp's, for D >= 32) minimum
                    sc = c;
                    si = i;
                }
            }
            if (seg == 1) {
                sc = c;
                si = i;
            }
            if (lane == 0) {
                wc[warp] = c;
                wi[warp] = i;
                if (c < mc || (c == mc && i < mi)) {
                    mc = c;
                    mi = i;
                }
            }
            const int nd = (int)((gp.pop - t0) < 1024 ? (gp.pop - t0) : 1024) / (int)D;  // demes of the tile
            if (D <= 32) {
                if ((lane % seg) == 0 && t < gp.pop) {
                    const int64_t d = t / D;
                    deme_cost[gp.deme_base + d] = sc;
                    win_s[threadIdx.x / seg] = (int)(si - t0);
                }
            }
            __syncthreads();
            if (D > 32 && threadIdx.x < nd) {
                const int per = (int)(D >> 5);
                long long bc = kNone, bi = kNone;
                for (int w = threadIdx.x * per; w < (threadIdx.x + 1) * per; ++w)
                    if (wc[w] < bc || (wc[w] == bc && wi[w] < bi)) {
                        bc = wc[w];
                        bi = wi[w];
                    }
                deme_cost[gp.deme_base + t0 / D + threadIdx.x] = bc;
                win_s[threadIdx.x] = (int)(bi - t0);
            }
            __syncthreads();
            for (int64_t x = threadIdx.x; x < (int64_t)nd * W; x += blockDim.x) {
                const int64_t d = x / W, w = x - d * W;
                deme_best[gp.dword_base + (t0 / D + d) * W + w] = X[gp.word_base + (t0 + win_s[d]) * W + w];
            }
            __syncthreads();
        }
        if (lane == 0) {
            gc[warp] = mc;
            gi[warp] = mi;
        }
        __syncthreads();
        if (warp == 0) {
            long long c = gc[lane], i = gi[lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long oc = __shfl_xor_sync(PM_FULL_MASK, c, o);
                const long long oi = __shfl_xor_sync(PM_FULL_MASK, i, o);
                if (oc < c || (oc == c && oi < i)) {
                    c = oc;
                    i = oi;
                }
            }
            if (lane == 0) {
                const bool better = s.best_cost < 0 || c < s.best_cost;
                improve = better ? 1 : 0;
                gwin = i;
                if (better) {
                    s.best_cost = c;
                    s.sat = 0;
                } else {
                    s.sat += 1;
                }
                if (s.trace)
                    s.trace[glob->step_gens] = s.best_cost;
                s.evals += gp.pop;
                s.gen += 1;
                s.total_gens += 1;
                s.stop = (s.saturation > 0 && s.sat >= s.saturation) ? 1 : 0;
            }
        }
        __syncthreads();
        if (improve)
            for (int w = threadIdx.x; w < W; w += blockDim.x)
                best[gp.best_base + w] = X[gp.word_base + gwin * W + w];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int a = s.stop ? 0 : 1;
        glob->alive = a;
        glob->step_gens += 1;
        glob->remaining -= 1;
        if (in_graph)
            cudaGraphSetConditional(h, (glob->remaining > 0 && a > 0) ? 1u : 0u);
    }
}

// The learned mutation try: individual t0 + j (warp j of the CTA) takes the
// candidate swap with the lowest predicted cost change (ties: lowest
// candidate index; a NaN score never wins) -- close moves[.][0], open
// moves[.][1] -- into Xc, unless it already improved in this generation.
__global__ void __launch_bounds__(1024) k_ga_learned_pick(const ga_prob *__restrict__ gps, int K, ga_prob one,
                                                          const uint32_t *__restrict__ X, uint32_t *__restrict__ Xc,
                                                          uint32_t *__restrict__ active,
                                                          const uint8_t *__restrict__ improved,
                                                          const float *__restrict__ scores,
                                                          const int32_t *__restrict__ moves, int64_t C,
                                                          ga_dev *__restrict__ st, ColumnsOut co)
{
    pm_grid_dependency_wait();
    __shared__ uint32_t on_s;
    int k;
    const ga_prob gp = prob_of_group(gps, K, one, blockIdx.x, k);
    const int lane = threadIdx.x & 31;
    const int j = threadIdx.x >> 5;
    const int64_t t0 = (blockIdx.x - gp.grp_base) * 32;
    const int64_t t = t0 + j;
    const int32_t W = gp.W;
    if (st[k].stop) {
        if (threadIdx.x == 0)
            active[(gp.ind_base + t0) >> 5] = 0u;
        return;
    }
    if (threadIdx.x == 0)
        on_s = 0u;
    __syncthreads();
    if (t < gp.pop && improved[gp.ind_base + t] == 0) {
        float bs = __int_as_float(0x7f800000);  // +inf
        int64_t bc = C;
        const float *sc = scores + t * C;
        for (int64_t c = lane; c < C; c += 32) {
            const float v = sc[c];
            if (v < bs) {  // NaN compares false
                bs = v;
                bc = c;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(PM_FULL_MASK, bs, o);
            const int64_t oc = __shfl_xor_sync(PM_FULL_MASK, bc, o);
            if (ov < bs || (ov == bs && oc < bc)) {
                bs = ov;
                bc = oc;
            }
        }
        if (bc < C) {
            const int32_t jc = moves[(t * C + bc) * 2], ko = moves[(t * C + bc) * 2 + 1];
            const uint32_t *src = X + gp.word_base + t * W;
            uint32_t *dst = Xc + gp.word_base + t * W;
            for (int w = lane; w < W; w += 32) {
                uint32_t v = src[w];
                if (w == (jc >> 5))
                    v &= ~(1u << (jc & 31));
                if (w == (ko >> 5))
                    v |= 1u << (ko & 31);
                dst[w] = v;
            }
            if (lane == 0)
                atomicOr(&on_s, 1u << j);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        active[(gp.ind_base + t0) >> 5] = on_s;
        if (on_s)
            atomicAdd(reinterpret_cast<unsigned long long *>(&st[k].evals), (unsigned long long)__popc(on_s));
    }
    write_columns(Xc + gp.word_base + t0 * W, W, t0, gp, co, lane, j, 32);
}

// ---------------------------------------------------------------------------
// The persistent generation kernel.  For one instance evaluated by the column
// scan, with the speculative mutation cycle, Floyd generation and no learned
// try (the default GA), one cooperative launch runs all the generations of a
// pm_ga_step call: the phases of the per-phase kernels above -- population,
// evaluation, lg D x (crossover, evaluation with acceptance), all mutation
// tries, their evaluation, first improving try, deme bests, global best --
// separated by grid-wide barriers instead of kernel boundaries.  A phase
// works on the same per-warp operators (fresh_individual, crossover_child,
// mutant_row) and the same client walk (scan_clients), so the population of
// every generation is the one the per-phase kernels produce.  Data another
// CTA wrote earlier in the launch is read through L2 (ld.cg); tiles are
// copied into shared memory with coherent vector loads.
// ---------------------------------------------------------------------------

constexpr int kFusedThreads = 1024;
constexpr uint64_t kBarrierTimeoutNs = 4000000000ull;  // a grid barrier gives up after 4 s
constexpr uint64_t kStallTimeoutNs = 20000000ull;      // 20 ms in a launch armed by pm_debug_scan_timeout
constexpr uint32_t kBarrierSpinCap = 1u << 23;         // and after this many polls whatever the timer says

struct FusedArgs {
    ga_prob gp;                      // the instance (bases 0)
    ga_prob gq;                      // layout of the Q x pop mutation candidates (pop = Q * pop)
    const uint16_t *pi;
    const int32_t *delta;
    int64_t n, stride;
    int32_t L, cum;
    int64_t tiles, splits, cps;      // the population's scans: tiles of 32 G individuals x client splits
    int64_t tilesQ, splitsQ, cpsQ;   // the candidates' scan
    int32_t R, Q;
    uint64_t seed;
    uint32_t *X, *Xc, *XQ;           // population, crossover children, mutation candidates (rows)
    uint32_t *colT, *colQ;           // facility-major copies of children / candidates
    uint32_t *active, *activeQ;      // bit per individual / candidate: evaluated in this scan
    int64_t *cost, *costQ;
    unsigned long long *accum, *accumQ;  // packed split reduction words, zero at rest
    uint8_t *improved;
    uint32_t *deme_best;
    int64_t *deme_cost;
    uint32_t *best;
    ga_dev *st;
    ga_glob *glob;
    unsigned *bar;                   // [0] arrivals at the current barrier, [1] barriers completed
    int *err;
    uint32_t stall;                  // failure-detection tests: CTA 0 leaves before the first barrier
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of the cooperative launch.  bar[1] counts the barriers completed; every CTA read it once at
// the start of the launch (no barrier completes before every CTA has arrived, so they all read the same value)
// and counts its own barriers in *passed.  Thread 0 of each CTA arrives on bar[0] with a release-ordered atomic;
// the last arrival resets bar[0] and publishes the new count with a release store; the others poll it with
// acquire loads for at most limit_ns (and kBarrierSpinCap polls), then record PM_ERR_TIMEOUT and the CTA leaves
// (false).  Writes before the barrier are visible to loads after it that bypass L1 (ld.cg) or acquire.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, int *ok_s, unsigned *passed,
                                             uint64_t limit_ns = kBarrierTimeoutNs)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = *passed + 1u;
        unsigned old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
        if (old + 1u == gridDim.x) {
            bar[0] = 0u;  // ordered before the release below; nobody arrives again before seeing it
            st_release_u32(bar + 1, target);
        } else {
            const uint64_t t0 = global_ns();
            uint32_t spins = 0;
            while (ld_acquire_u32(bar + 1) != target) {
                if (++spins > kBarrierSpinCap || ((spins & 63u) == 0u && global_ns() - t0 > limit_ns)) {
                    atomicExch(err, (int)PM_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        *passed = target;
        *ok_s = ok;
    }
    __syncthreads();
    return *ok_s != 0;
}

enum FusedScanMode { kScanStore = 0, kScanAccept = 1, kScanCandidates = 2 };

// One scan phase: the (client split, tile) items of the population (kScanStore: costs; kScanAccept: a child
// replaces its parent when strictly cheaper) or of the mutation candidates (kScanCandidates: their costs), with
// the packed split reduction of the column kernel; then the grid barrier.
template <int G>
__device__ __forceinline__ bool fused_scan(const FusedArgs &a, int mode, uint32_t *colbits, unsigned long long *acc_s,
                                           uint32_t *a0_s, uint32_t *fin_s, int *ok_s, unsigned *passed_s)
{
    const bool cand = mode == kScanCandidates;
    const int64_t tiles = cand ? a.tilesQ : a.tiles, splits = cand ? a.splitsQ : a.splits;
    const int64_t cps = cand ? a.cpsQ : a.cps, pop = cand ? a.gq.pop : a.gp.pop;
    const uint32_t *colT = cand ? a.colQ : a.colT;
    const uint32_t *active = cand ? a.activeQ : a.active;
    unsigned long long *accum = cand ? a.accumQ : a.accum;
    const int32_t W = a.gp.W, L = a.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t tile_words = (int64_t)W * 32 * G;
    int64_t loaded = -1;
    for (int64_t item = blockIdx.x; item < tiles * splits; item += gridDim.x) {
        const int64_t tile = item % tiles, split = item / tiles;
        const int64_t ind0 = tile * 32 * G;
        const int64_t c_begin = split * cps;
        const int64_t c_end = (c_begin + cps < a.n) ? c_begin + cps : a.n;
        auto load = [&](int64_t cc, int base, uint32_t &j, int32_t &dl) {
            const int r = base + lane;
            if (cc < c_end && r < L) {
                j = __ldg(a.pi + cc * a.stride + r);
                dl = __ldg(a.delta + cc * a.stride + r);
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
        if (tile != loaded) {
            const uint4 *src = reinterpret_cast<const uint4 *>(colT + tile * tile_words);
            uint4 *dst = reinterpret_cast<uint4 *>(colbits);
            for (int64_t q = threadIdx.x; q < tile_words / 4; q += blockDim.x)
                dst[q] = __ldcg(src + q);
            loaded = tile;
        }
        if (warp < G) {
            const int64_t t = ind0 + 32 * warp + lane;
            const bool on = t < pop && ((__ldcg(active + (t >> 5)) >> (t & 31)) & 1u);
            const uint32_t b = __ballot_sync(PM_FULL_MASK, on);
            if (lane == 0)
                a0_s[warp] = b;
        }
        for (int q = threadIdx.x; q < G * 32; q += blockDim.x)
            acc_s[q] = 0ull;
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
            scan_clients<G>(colbits, a0, c, c_end, nwarps, L, lane, a.cum != 0, load, j_cur, d_cur, j_nxt, d_nxt,
                            j_nc, d_nc, j_nc1, d_nc1, acc);
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (acc[g])
                atomicAdd(&acc_s[g * 32 + lane], acc[g]);
        __syncthreads();
        const uint32_t *fin = a0_s;
        if (splits > 1) {
            // one atomic per individual carries the split's sum and a count of one (bits 48..63); the split that
            // completes the count holds the total and leaves the word zero
            for (int q = threadIdx.x; q < G * 32; q += blockDim.x) {
                const int64_t t = ind0 + q;
                bool last = false;
                if (t < pop && ((a0_s[q >> 5] >> (q & 31)) & 1u)) {
                    const unsigned long long add = acc_s[q] + (1ull << 48);
                    const unsigned long long old = atomicAdd(accum + t, add);
                    if ((old >> 48) == (unsigned long long)(splits - 1)) {
                        acc_s[q] = (old + add) & ((1ull << 48) - 1ull);
                        accum[t] = 0ull;
                        last = true;
                    }
                }
                const uint32_t b = __ballot_sync(PM_FULL_MASK, last);
                if ((q & 31) == 0)
                    fin_s[q >> 5] = b;
            }
            __syncthreads();
            fin = fin_s;
        }
        for (int q = warp; q < G * 32; q += nwarps) {
            const int64_t t = ind0 + q;
            if (t >= pop)
                break;
            if (!((fin[q >> 5] >> (q & 31)) & 1u))
                continue;
            const int64_t sum = (int64_t)acc_s[q];
            if (mode == kScanStore) {
                if (lane == 0)
                    a.cost[t] = sum;
            } else if (mode == kScanCandidates) {
                if (lane == 0)
                    a.costQ[t] = sum;
            } else if (sum < (int64_t)__ldcg(reinterpret_cast<const long long *>(a.cost + t))) {
                for (int w = lane; w < W; w += 32)
                    a.X[t * W + w] = __ldcg(a.Xc + t * W + w);
                if (lane == 0)
                    a.cost[t] = sum;
            }
        }
        __syncthreads();
    }
    return grid_barrier(a.bar, a.err, ok_s, passed_s);
}

template <int G>
__global__ void __launch_bounds__(kFusedThreads, 1) k_ga_fused(const __grid_constant__ FusedArgs a)
{
    extern __shared__ __align__(16) uint32_t fsm[];
    __shared__ unsigned long long acc_s[G * 32];
    __shared__ uint32_t a0_s[G], fin_s[G];
    __shared__ uint32_t on_s;
    __shared__ unsigned long long tries_s;
    __shared__ int ok_s;
    __shared__ long long sc[32], si[32];
    __shared__ long long win_s;
    __shared__ int improve_s;
    __shared__ unsigned passed_s;  // barriers this CTA has passed (thread 0's count; the launch starts at bar[1])
    if (threadIdx.x == 0)
        passed_s = ld_acquire_u32(a.bar + 1);
    const ga_prob &gp = a.gp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int32_t W = gp.W, p = gp.p;
    const int64_t P = gp.pop, QP = a.gq.pop;
    const int64_t groups = (P + 31) / 32, groupsQ = (QP + 31) / 32;
    ga_dev *st = a.st;
    ColumnsOut co{a.colT, G}, coQ{a.colQ, G};
    if (a.stall) {
        // failure-detection tests: CTA 0 never arrives, so the first barrier runs out (after kStallTimeoutNs)
        // in every other CTA, which records PM_ERR_TIMEOUT and leaves; nothing is in flight
        if (blockIdx.x == 0)
            return;
        grid_barrier(a.bar, a.err, &ok_s, &passed_s, kStallTimeoutNs);
        return;
    }
    for (;;) {
        // every CTA reads what the last barrier published (or k_ga_begin, before the launch)
        const long long remaining = __ldcg(&a.glob->remaining);
        const int stop = __ldcg(&st->stop);
        if (remaining <= 0 || stop)
            return;
        const uint32_t gen = (uint32_t)__ldcg(&st->gen);

        // ---- A2: fresh population with migration: rows, facility-major copy, active bits ----
        for (int64_t vb = blockIdx.x; vb < groups; vb += gridDim.x) {
            const int64_t t0 = vb * 32, t = t0 + warp;
            uint32_t *row = fsm + (int64_t)warp * W;
            uint32_t *draws = fsm + (int64_t)32 * W + (int64_t)warp * p;
            if (t < P) {
                if (lane == 0)
                    a.improved[t] = 0;
                fresh_individual<true>(gp, t, gen, a.seed, a.deme_best, row, draws, lane);
                for (int w = lane; w < W; w += 32)
                    a.X[t * W + w] = row[w];
            }
            __syncthreads();
            if (threadIdx.x == 0)
                a.active[vb] = (P - t0 >= 32) ? 0xffffffffu : ((1u << (P - t0)) - 1u);
            write_columns(fsm, W, t0, gp, co, lane, warp, nwarps);
            __syncthreads();
        }
        if (!grid_barrier(a.bar, a.err, &ok_s, &passed_s))
            return;
        // ---- A3: evaluation ----
        if (!fused_scan<G>(a, kScanStore, fsm, acc_s, a0_s, fin_s, &ok_s, &passed_s))
            return;
        // ---- A4: crossover rounds (children from the population as the round starts; acceptance) ----
        if (p / 2 > 0) {
            for (int32_t r = 0; r < a.R; ++r) {
                const int64_t stride = gp.D >> (1 + (r % gp.lgD));
                for (int64_t vb = blockIdx.x; vb < groups; vb += gridDim.x) {
                    const int64_t t0 = vb * 32, t = t0 + warp;
                    uint32_t *row = fsm + (int64_t)warp * W;
                    if (threadIdx.x == 0)
                        on_s = 0u;
                    __syncthreads();
                    if (t < P) {
                        const int64_t partner = t ^ stride;
                        const uint32_t pair = (uint32_t)(t < partner ? t : partner);
                        const uint4 v = draw_block(a.seed, gen, pair, OP_XOVER + (uint32_t)r, 0, gp.sid);
                        const uint32_t r1 = uniform_below(v.x, (uint32_t)gp.m);
                        const int i = 1 + (int)uniform_below(v.y, (uint32_t)(p / 2));
                        const bool ok = crossover_child<true>(a.X + t * W, a.X + partner * W, row, W, r1, i, lane);
                        __syncwarp();
                        for (int w = lane; w < W; w += 32)
                            a.Xc[t * W + w] = row[w];
                        if (lane == 0 && ok)
                            atomicOr(&on_s, 1u << warp);
                    } else {
                        for (int w = lane; w < W; w += 32)
                            row[w] = 0u;
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        a.active[vb] = on_s;
                        if (on_s)
                            atomicAdd(reinterpret_cast<unsigned long long *>(&st->evals),
                                      (unsigned long long)__popc(on_s));
                    }
                    write_columns(fsm, W, t0, gp, co, lane, warp, nwarps);
                    __syncthreads();
                }
                if (!grid_barrier(a.bar, a.err, &ok_s, &passed_s))
                    return;
                if (!fused_scan<G>(a, kScanAccept, fsm, acc_s, a0_s, fin_s, &ok_s, &passed_s))
                    return;
            }
        }
        // ---- A5: every mutation try of every individual, one scan, first improving try ----
        for (int64_t vb = blockIdx.x; vb < groupsQ; vb += gridDim.x) {
            const int64_t u0 = vb * 32, u = u0 + warp;
            uint32_t *row = fsm + (int64_t)warp * W;
            if (threadIdx.x == 0)
                on_s = 0u;
            __syncthreads();
            bool built = false;
            if (u < QP) {
                const int64_t q = u / P, t = u - q * P;
                if (__ldcg(a.improved + t) == 0) {
                    mutant_row<true>(a.X + t * W, row, W, gp.m, a.seed, gen, (uint32_t)t, (uint32_t)q, gp.sid, lane);
                    __syncwarp();
                    for (int w = lane; w < W; w += 32)
                        a.XQ[u * W + w] = row[w];
                    if (lane == 0)
                        atomicOr(&on_s, 1u << warp);
                    built = true;
                }
            }
            if (!built)
                for (int w = lane; w < W; w += 32)
                    row[w] = 0u;
            __syncthreads();
            if (threadIdx.x == 0)
                a.activeQ[vb] = on_s;
            write_columns(fsm, W, u0, a.gq, coQ, lane, warp, nwarps);
            __syncthreads();
        }
        if (!grid_barrier(a.bar, a.err, &ok_s, &passed_s))
            return;
        if (!fused_scan<G>(a, kScanCandidates, fsm, acc_s, a0_s, fin_s, &ok_s, &passed_s))
            return;
        for (int64_t vb = blockIdx.x; vb < groups; vb += gridDim.x) {
            const int64_t t = vb * 32 + warp;
            if (threadIdx.x == 0)
                tries_s = 0ull;
            __syncthreads();
            if (t < P && __ldcg(a.improved + t) == 0) {
                const int64_t c0 = __ldcg(reinterpret_cast<const long long *>(a.cost + t));
                int qs = a.Q;
                for (int base = 0; base < a.Q; base += 32) {
                    const int q = base + lane;
                    const bool hit =
                        q < a.Q && __ldcg(reinterpret_cast<const long long *>(a.costQ + (int64_t)q * P + t)) < c0;
                    const uint32_t b = __ballot_sync(PM_FULL_MASK, hit);
                    if (b) {
                        qs = base + __ffs(b) - 1;
                        break;
                    }
                }
                if (qs < a.Q) {
                    const int64_t u = (int64_t)qs * P + t;
                    for (int w = lane; w < W; w += 32)
                        a.X[t * W + w] = __ldcg(a.XQ + u * W + w);
                    if (lane == 0) {
                        a.cost[t] = __ldcg(reinterpret_cast<const long long *>(a.costQ + u));
                        a.improved[t] = 1;
                    }
                }
                if (lane == 0)
                    atomicAdd(&tries_s, (unsigned long long)(qs < a.Q ? qs + 1 : a.Q));
            }
            __syncthreads();
            if (threadIdx.x == 0 && tries_s)
                atomicAdd(reinterpret_cast<unsigned long long *>(&st->evals), tries_s);
        }
        if (!grid_barrier(a.bar, a.err, &ok_s, &passed_s))
            return;
        // ---- A6: deme bests (lowest cost, then lowest index) ----
        for (int64_t b = blockIdx.x; b < gp.NB; b += gridDim.x) {
            long long bc = 0x7fffffffffffffffLL, bi = 0x7fffffffffffffffLL;
            for (int64_t i = threadIdx.x; i < gp.D; i += blockDim.x) {
                const int64_t t = b * gp.D + i;
                const long long c = __ldcg(reinterpret_cast<const long long *>(a.cost + t));
                if (c < bc || (c == bc && t < bi)) {
                    bc = c;
                    bi = t;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long oc = __shfl_xor_sync(PM_FULL_MASK, bc, o);
                const long long oi = __shfl_xor_sync(PM_FULL_MASK, bi, o);
                if (oc < bc || (oc == bc && oi < bi)) {
                    bc = oc;
                    bi = oi;
                }
            }
            if (lane == 0) {
                sc[warp] = bc;
                si[warp] = bi;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 1; w < nwarps; ++w)
                    if (sc[w] < bc || (sc[w] == bc && si[w] < bi)) {
                        bc = sc[w];
                        bi = si[w];
                    }
                win_s = bi;
                a.deme_cost[b] = bc;
            }
            __syncthreads();
            for (int w = threadIdx.x; w < W; w += blockDim.x)
                a.deme_best[b * W + w] = __ldcg(a.X + win_s * W + w);
            __syncthreads();
        }
        if (!grid_barrier(a.bar, a.err, &ok_s, &passed_s))
            return;
        // ---- global best, saturation, trace, counters (one CTA) ----
        if (blockIdx.x == 0) {
            long long bc = 0x7fffffffffffffffLL, bi = 0x7fffffffffffffffLL;
            for (int64_t d = threadIdx.x; d < gp.NB; d += blockDim.x) {
                const long long c = __ldcg(reinterpret_cast<const long long *>(a.deme_cost) + d);
                if (c < bc || (c == bc && d < bi)) {
                    bc = c;
                    bi = d;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long oc = __shfl_xor_sync(PM_FULL_MASK, bc, o);
                const long long oi = __shfl_xor_sync(PM_FULL_MASK, bi, o);
                if (oc < bc || (oc == bc && oi < bi)) {
                    bc = oc;
                    bi = oi;
                }
            }
            if (lane == 0) {
                sc[warp] = bc;
                si[warp] = bi;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 1; w < nwarps; ++w)
                    if (sc[w] < bc || (sc[w] == bc && si[w] < bi)) {
                        bc = sc[w];
                        bi = si[w];
                    }
                const long long prev = __ldcg(&st->best_cost);
                const bool better = prev < 0 || bc < prev;
                improve_s = better ? 1 : 0;
                win_s = bi;
                long long sat = __ldcg(&st->sat);
                if (better) {
                    st->best_cost = bc;
                    sat = 0;
                } else {
                    sat += 1;
                }
                st->sat = sat;
                const long long step = __ldcg(&a.glob->step_gens);
                if (st->trace)
                    st->trace[step] = better ? bc : prev;
                // the generation's initial evaluation (the crossover and mutation phases added theirs atomically)
                atomicAdd(reinterpret_cast<unsigned long long *>(&st->evals), (unsigned long long)P);
                st->gen = (long long)gen + 1;
                st->total_gens = __ldcg(&st->total_gens) + 1;
                const long long S = st->saturation;
                const int stopped = (S > 0 && sat >= S) ? 1 : 0;
                st->stop = stopped;
                a.glob->alive = stopped ? 0 : 1;
                a.glob->step_gens = step + 1;
                a.glob->remaining = __ldcg(&a.glob->remaining) - 1;
            }
            __syncthreads();
            if (improve_s)
                for (int w = threadIdx.x; w < W; w += blockDim.x)
                    a.best[w] = __ldcg(a.deme_best + win_s * W + w);
        }
        if (!grid_barrier(a.bar, a.err, &ok_s, &passed_s))
            return;
    }
}


// Uniform random p-subsets (Floyd sampling, generation 0, no migration), one
// thread per individual, bitsets written in place.
__global__ void k_random_population(uint32_t *__restrict__ X, int64_t P, int32_t W, int32_t m, int32_t p,
                                    uint64_t seed)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P)
        return;
    uint32_t *row = X + t * W;
    for (int w = 0; w < W; ++w)
        row[w] = 0u;
    uint4 v = make_uint4(0, 0, 0, 0);
    for (int q = 0; q < p; ++q) {
        if ((q & 3) == 0)
            v = draw_block(seed, 0u, (uint32_t)t, OP_INIT, (uint32_t)q >> 2, 0u);
        const uint32_t j = (uint32_t)(m - p + q);
        const uint32_t c = uniform_below(word_of(v, q & 3), j + 1);
        const uint32_t pick = ((row[c >> 5] >> (c & 31)) & 1u) ? j : c;
        row[pick >> 5] |= 1u << (pick & 31);
    }
}

}  // namespace

// ------------------------------- host side ---------------------------------

pm_status pm_launch_random_population(const pm_instance *inst, uint64_t seed, int64_t pop, uint32_t *masks,
                                      cudaStream_t s)
{
    if (pop <= 0)
        return PM_OK;
    k_random_population<<<(unsigned)pm_ceil_div(pop, 128), 128, 0, s>>>(masks, pop, (int32_t)inst->W,
                                                                       (int32_t)inst->m, (int32_t)inst->p, seed);
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

struct pm_ga {
    std::vector<pm_instance *> insts;
    int device = 0;  // the instances' device (kept here: a GA may outlive the handles it was created on)
    int K = 1;
    uint64_t seed = 0;
    int64_t P = 0, D = 0, NB = 0;
    int lgD = 0, R = 0, Q = 0;
    int64_t S = 0;
    uint32_t sid = 0;
    bool team = false;  // migration variant (ii)
    bool comb = false;  // Section 4.1 chromosome generation (combinadic)
    int comb_K = 0, comb_Q = 0;
    size_t comb_entries = 0;
    pm_dbuf comb_tab;
    bool single_row = false;  // one instance whose evaluation uses the row kernel
    // speculative mutation cycle: all Q tries evaluated in one scan (single instance, column path)
    bool spec = false;
    pm_eval_plan spec_single;
    pm_multi_plan spec_plan;
    ga_prob gq{};                // instance 0's candidates
    std::vector<ga_prob> gqs;    // every instance's candidates
    int64_t groupsQ_total = 0;   // 32-candidate groups over all instances
    pm_dbuf XQ, costQ, activeQ, accumQ, ticketsQ, colQ, gqprobs, probsQ;
    pm_eval_plan single;      // K == 1: the single-instance plan
    pm_multi_plan plan;       // the scan plan over all instances
    std::vector<ga_prob> gps;
    int64_t groups_total = 0, demes_total = 0, dwords_total = 0, best_total = 0, Wmax = 0;
    pm_dbuf X, Xc, cost, active, improved, deme_best, deme_cost, best, trace, accum, tickets, columns, st, glob, err,
        probs, gprobs;
    pm_dbuf arena;  // the memory of the buffers above and of the candidates' buffers
    // the persistent generation kernel (one cooperative launch per pm_ga_step) when the GA qualifies
    bool fused = false;
    int fused_G = 4;
    unsigned fused_grid = 0;
    size_t fused_smem = 0;
    int64_t f_tiles = 0, f_splits = 1, f_cps = 0, f_tilesQ = 0, f_splitsQ = 1, f_cpsQ = 0;
    pm_dbuf bar;
    // learned swap proposal (single-instance GAs)
    pm_model *model = nullptr;
    int T = 4;
    pm_dbuf s_gain, s_cap, s_loss, s_assign, moves, xfeat, scores;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;   // gate + conditional while-node over the generation
    cudaGraphExec_t exec1 = nullptr;  // one generation, no loop (calls of one generation)
    cudaGraph_t graph1 = nullptr;     // the graph exec1 was instantiated from
    int graphs = 3;                   // which of the two to build: bit 0 exec, bit 1 exec1 (pm_ga_run: one)
    // the root node of each graph: k_ga_begin, whose arguments (generation budget, trace) each call sets
    cudaGraphNode_t begin_node = nullptr, begin_node1 = nullptr;
};

static void ga_free(pm_ga *ga)
{
    if (!ga)
        return;
    pm_clear_error(cudaSetDevice(ga->device));
    if (ga->exec)
        pm_clear_error(cudaGraphExecDestroy(ga->exec));
    if (ga->exec1)
        pm_clear_error(cudaGraphExecDestroy(ga->exec1));
    if (ga->graph)
        pm_clear_error(cudaGraphDestroy(ga->graph));
    if (ga->graph1)
        pm_clear_error(cudaGraphDestroy(ga->graph1));
    if (ga->cap)
        pm_clear_error(cudaStreamDestroy(ga->cap));
    pm_dbuf *bufs[] = {&ga->X,         &ga->Xc,   &ga->cost,  &ga->active, &ga->improved, &ga->deme_best,
                       &ga->deme_cost, &ga->best, &ga->trace, &ga->accum,  &ga->tickets,  &ga->columns,
                       &ga->st,        &ga->glob, &ga->err,   &ga->probs,  &ga->gprobs,
                       &ga->s_gain,    &ga->s_cap, &ga->s_loss, &ga->s_assign, &ga->moves, &ga->xfeat, &ga->scores,
                       &ga->comb_tab,  &ga->XQ,    &ga->costQ, &ga->activeQ, &ga->accumQ, &ga->ticketsQ, &ga->colQ,
                       &ga->bar,       &ga->gqprobs, &ga->probsQ, &ga->arena};
    for (pm_dbuf *b : bufs)
        b->release();
    delete ga;
}

// PM_GA_GRAPH=0 in the environment selects direct stream launches instead of
// the conditional-while graph (identical results; for profiling).
static bool graph_mode()
{
    const char *v = std::getenv("PM_GA_GRAPH");
    return !(v && v[0] == '0');
}

// PM_GA_SPEC=0 in the environment runs the mutation cycle try by try even where the speculative cycle applies
// (identical results; for comparison).
static bool spec_allowed()
{
    const char *v = std::getenv("PM_GA_SPEC");
    return !(v && v[0] == '0');
}

// PM_GA_SPEC=1: the speculative cycle for batched GAs too.
static bool spec_forced()
{
    const char *v = std::getenv("PM_GA_SPEC");
    return v && v[0] == '1';
}

static pm_status ga_eval(pm_ga *ga, const uint32_t *masks, int64_t *costs, const pm_accept_args &acc,
                         cudaStream_t s)
{
    int64_t *accum = static_cast<int64_t *>(ga->accum.ptr);
    int *tickets = static_cast<int *>(ga->tickets.ptr);
    uint32_t *columns = static_cast<uint32_t *>(ga->columns.ptr);
    int *err = static_cast<int *>(ga->err.ptr);
    const uint32_t *active = static_cast<const uint32_t *>(ga->active.ptr);
    if (ga->single_row)
        return pm_launch_eval(ga->insts[0], ga->single, masks, ga->P, active, costs, accum, tickets, columns, err, acc,
                              s);
    pm_scan_launch L;
    pm_scan_launch_from(ga->plan, static_cast<const pm_prob *>(ga->probs.ptr), L);
    L.masks = masks;
    L.colT = columns;
    L.active = active;
    L.accum = accum;
    L.tickets = tickets;
    L.err = err;
    return pm_launch_scan(L, acc, costs, ga->plan.smem, s);
}

// Enqueue one generation on `s`: under stream capture for the graph body
// (in_graph = 1), or directly on the stream (in_graph = 0).
static pm_status enqueue_generation(pm_ga *ga, cudaStream_t s, cudaGraphConditionalHandle h, int in_graph)
{
    const ga_prob *gps = static_cast<const ga_prob *>(ga->gprobs.ptr);
    const ga_prob one = ga->gps[0];
    const int K = ga->K;
    ga_dev *st = static_cast<ga_dev *>(ga->st.ptr);
    uint32_t *X = static_cast<uint32_t *>(ga->X.ptr);
    uint32_t *Xc = static_cast<uint32_t *>(ga->Xc.ptr);
    int64_t *cost = static_cast<int64_t *>(ga->cost.ptr);
    uint32_t *active = static_cast<uint32_t *>(ga->active.ptr);
    uint8_t *improved = static_cast<uint8_t *>(ga->improved.ptr);
    ColumnsOut co;
    co.colT = ga->single_row ? nullptr : static_cast<uint32_t *>(ga->columns.ptr);
    co.G = ga->single_row ? 1 : ga->plan.groups;
    const unsigned groups = (unsigned)ga->groups_total;
    const size_t init_smem = (size_t)32 * (ga->Wmax | 1) * 4;
    const int rows_in_smem = init_smem <= 48 * 1024 ? 1 : 0;
    int32_t pmax = 1;
    for (const ga_prob &g : ga->gps)
        pmax = std::max(pmax, g.p);
    const size_t warp_init_smem = (size_t)32 * ((size_t)ga->Wmax + (size_t)pmax) * 4;
    // crossover children and mutants are built in shared memory (and transposed from there) when 32 rows fit
    // in the default 48 KB; only the column path has columns to write
    const size_t rows_smem = (!ga->single_row && (size_t)32 * ga->Wmax * 4 <= 48 * 1024) ? (size_t)32 * ga->Wmax * 4 : 0;

    if (ga->comb) {
        const uint32_t *T = static_cast<const uint32_t *>(ga->comb_tab.ptr);
        const uint64_t *Hh = reinterpret_cast<const uint64_t *>(T + comb_head_offset(ga->comb_entries, ga->comb_K));
        const uint32_t *db = static_cast<const uint32_t *>(ga->deme_best.ptr);
        switch (ga->comb_Q) {
        case 1:
            PM_CUDA(pm_launch(k_ga_init_comb<1>, groups, 1024, 0, s, one, X, improved, active, db, T, Hh, ga->comb_K,
                              ga->seed, st, co));
            break;
        case 2:
            PM_CUDA(pm_launch(k_ga_init_comb<2>, groups, 1024, 0, s, one, X, improved, active, db, T, Hh, ga->comb_K,
                              ga->seed, st, co));
            break;
        case 4:
            PM_CUDA(pm_launch(k_ga_init_comb<4>, groups, 1024, 0, s, one, X, improved, active, db, T, Hh, ga->comb_K,
                              ga->seed, st, co));
            break;
        default:
            PM_CUDA(pm_launch(k_ga_init_comb<8>, groups, 1024, 0, s, one, X, improved, active, db, T, Hh, ga->comb_K,
                              ga->seed, st, co));
            break;
        }
    } else if (warp_init_smem <= 200 * 1024) {
        TablePrefix tp{nullptr, nullptr, 0, 0};
        if (K == 1) {
            tp.pi = ga->insts[0]->pi;
            tp.delta = ga->insts[0]->delta;
            tp.n = ga->insts[0]->n;
            tp.stride = ga->insts[0]->stride;
        }
        PM_CUDA(pm_launch(k_ga_init_warp, groups, 1024, warp_init_smem, s, gps, K, one, X, improved, active,
                          static_cast<const uint32_t *>(ga->deme_best.ptr), ga->seed, st, co, tp));
    } else {
        PM_CUDA(pm_launch(k_ga_init, groups, 32, rows_in_smem ? init_smem : 0, s, gps, K, one, X, improved, active,
                          static_cast<const uint32_t *>(ga->deme_best.ptr), ga->seed, st, co, rows_in_smem));
    }
    pm_accept_args plain;
    plain.columns_ready = true;
    PM_TRY(ga_eval(ga, X, cost, plain, s));

    pm_accept_args acc;
    acc.mode = 1;
    acc.cur_cost = cost;
    acc.cur_masks = X;
    acc.cand_masks = Xc;
    acc.columns_ready = true;
    if (ga->gps[0].p / 2 > 0) {  // p = 1: no crossover (a batch has p >= 2 everywhere or p = 1 everywhere)
        for (int r = 0; r < ga->R; ++r) {
            PM_CUDA(pm_launch(k_ga_crossover, groups, 1024, rows_smem, s, gps, K, one, X, Xc, active, (uint32_t)r,
                              ga->seed, st, co, rows_smem ? 1 : 0));
            acc.improved = nullptr;
            PM_TRY(ga_eval(ga, Xc, nullptr, acc, s));
        }
    }
    if (ga->model) {
        // learned try: swap statistics -> candidate moves -> scores -> best swap -> exact evaluation
        const pm_instance *inst = ga->insts[0];
        int64_t *gain = static_cast<int64_t *>(ga->s_gain.ptr), *loss = static_cast<int64_t *>(ga->s_loss.ptr);
        int32_t *capc = static_cast<int32_t *>(ga->s_cap.ptr), *asg = static_cast<int32_t *>(ga->s_assign.ptr);
        int32_t *moves = static_cast<int32_t *>(ga->moves.ptr);
        const int64_t C = inst->p * ga->T;
        PM_TRY(pm_launch_learned_candidates(inst, X, ga->P, gain, capc, loss, asg, cost, ga->T, moves,
                                    static_cast<uint16_t *>(ga->xfeat.ptr), s));
        PM_TRY(pm_model_forward_dev(ga->model, ga->xfeat.ptr, ga->P * C, static_cast<float *>(ga->scores.ptr), s));
        PM_CUDA(pm_launch(k_ga_learned_pick, groups, 1024, 0, s, gps, K, one, X, Xc, active, improved,
                          static_cast<const float *>(ga->scores.ptr), moves, C, st, co));
        acc.improved = improved;
        PM_TRY(ga_eval(ga, Xc, nullptr, acc, s));
    }
    if (ga->spec) {
        // all Q tries at once: mutants -> one scan storing their costs -> first improving try per individual
        uint32_t *XQ = static_cast<uint32_t *>(ga->XQ.ptr);
        uint32_t *activeQ = static_cast<uint32_t *>(ga->activeQ.ptr);
        int64_t *costQ = static_cast<int64_t *>(ga->costQ.ptr);
        ColumnsOut coQ;
        coQ.colT = static_cast<uint32_t *>(ga->colQ.ptr);
        coQ.G = ga->spec_plan.groups;
        const ga_prob *gqs = static_cast<const ga_prob *>(ga->gqprobs.ptr);
        PM_CUDA(pm_launch(k_ga_mutate_all, (unsigned)ga->groupsQ_total, 1024, rows_smem, s, gps, gqs, K, one,
                          ga->gq, (int32_t)ga->Q, X, XQ, activeQ, improved, ga->seed, st, coQ, rows_smem ? 1 : 0));
        pm_scan_launch L;
        pm_scan_launch_from(ga->spec_plan, static_cast<const pm_prob *>(ga->probsQ.ptr), L);
        L.masks = XQ;
        L.colT = coQ.colT;
        L.active = activeQ;
        L.accum = static_cast<int64_t *>(ga->accumQ.ptr);
        L.tickets = static_cast<int *>(ga->ticketsQ.ptr);
        L.err = static_cast<int *>(ga->err.ptr);
        pm_accept_args store;
        store.columns_ready = true;
        PM_TRY(pm_launch_scan(L, store, costQ, ga->spec_plan.smem, s));
        PM_CUDA(pm_launch(k_ga_mutate_accept, (unsigned)pm_ceil_div(ga->plan.ind_total, 8), 256, 0, s, gps, gqs, K,
                          one, ga->gq, (int32_t)ga->Q, X, XQ, cost, costQ, improved, st));
    } else {
        for (int q = 0; q < ga->Q; ++q) {
            PM_CUDA(pm_launch(k_ga_mutate, groups, 1024, 0, s, gps, K, one, X, Xc, active, improved, (uint32_t)q,
                              ga->seed, st, co));
            acc.improved = improved;
            PM_TRY(ga_eval(ga, Xc, nullptr, acc, s));
        }
    }
    if (K == 1) {
        PM_CUDA(pm_launch(k_ga_generation_end_one, 1u, 1024u, 0, s, one, X, cost,
                          static_cast<uint32_t *>(ga->deme_best.ptr), static_cast<int64_t *>(ga->deme_cost.ptr),
                          static_cast<uint32_t *>(ga->best.ptr), st, static_cast<ga_glob *>(ga->glob.ptr), h,
                          in_graph));
        return PM_OK;
    }
    const int dthreads = (int)pm_round_up(std::min<int64_t>(ga->D, 1024), 32);
    PM_CUDA(pm_launch(k_ga_generation_end, (unsigned)ga->demes_total, (unsigned)dthreads, 0, s, gps, K, one, X,
                      cost, static_cast<uint32_t *>(ga->deme_best.ptr), static_cast<int64_t *>(ga->deme_cost.ptr),
                      static_cast<uint32_t *>(ga->best.ptr), st, static_cast<ga_glob *>(ga->glob.ptr), h, in_graph));
    return PM_OK;
}

// k_ga_begin's kernel-node parameters for a call of `gens` generations writing its trace to `tr` (nullptr:
// none); `args` holds the values the returned parameters point to.
struct BeginArgs {
    ga_glob *glob;
    ga_dev *st;
    int K;
    long long gens;
    long long *tr;
    unsigned *bar;
    void *ptrs[6];
};

static cudaKernelNodeParams begin_params(pm_ga *ga, long long gens, long long *tr, BeginArgs &a)
{
    a.glob = static_cast<ga_glob *>(ga->glob.ptr);
    a.st = static_cast<ga_dev *>(ga->st.ptr);
    a.K = ga->K;
    a.gens = gens;
    a.tr = tr;
    a.bar = static_cast<unsigned *>(ga->bar.ptr);
    a.ptrs[0] = &a.glob;
    a.ptrs[1] = &a.st;
    a.ptrs[2] = &a.K;
    a.ptrs[3] = &a.gens;
    a.ptrs[4] = &a.tr;
    a.ptrs[5] = &a.bar;
    cudaKernelNodeParams kp = {};
    kp.func = reinterpret_cast<void *>(k_ga_begin);
    kp.gridDim = dim3((unsigned)pm_ceil_div(ga->K, 256));
    kp.blockDim = dim3(256);
    kp.kernelParams = a.ptrs;
    return kp;
}

// The generation as a plain graph for calls of one generation: entering and leaving a conditional body costs
// about 6 us each way, a tenth of a graph900 generation.  Its root is k_ga_begin, so a call is one graph launch.
static pm_status build_graph_one(pm_ga *ga)
{
    PM_CUDA(cudaGraphCreate(&ga->graph1, 0));
    BeginArgs ba;
    const cudaKernelNodeParams kp = begin_params(ga, 1, nullptr, ba);
    PM_CUDA(cudaGraphAddKernelNode(&ga->begin_node1, ga->graph1, nullptr, 0, &kp));
    PM_CUDA(cudaStreamBeginCaptureToGraph(ga->cap, ga->graph1, &ga->begin_node1, nullptr, 1,
                                          cudaStreamCaptureModeThreadLocal));
    pm_status st_gen = enqueue_generation(ga, ga->cap, 0, 0);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(ga->cap, &captured);
    PM_TRY(st_gen);
    PM_CUDA(e);
    PM_CUDA(cudaGraphInstantiate(&ga->exec1, ga->graph1, 0));
    return PM_OK;
}

static pm_status build_graph(pm_ga *ga)
{
    if (!(ga->graphs & 1))
        return build_graph_one(ga);
    PM_CUDA(cudaGraphCreate(&ga->graph, 0));
    cudaGraphConditionalHandle h;
    PM_CUDA(cudaGraphConditionalHandleCreate(&h, ga->graph, 0, cudaGraphCondAssignDefault));
    // gate: sets the condition from the step's generation budget
    ga_glob *glob = static_cast<ga_glob *>(ga->glob.ptr);
    void *gate_args[] = {&glob, &h};
    cudaKernelNodeParams kp = {};
    kp.func = reinterpret_cast<void *>(k_ga_gate);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = gate_args;
    BeginArgs ba;
    const cudaKernelNodeParams bp = begin_params(ga, 1, nullptr, ba);
    PM_CUDA(cudaGraphAddKernelNode(&ga->begin_node, ga->graph, nullptr, 0, &bp));
    cudaGraphNode_t gate;
    PM_CUDA(cudaGraphAddKernelNode(&gate, ga->graph, &ga->begin_node, 1, &kp));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    PM_CUDA(cudaGraphAddNode(&loop, ga->graph, &gate, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    PM_CUDA(cudaStreamBeginCaptureToGraph(ga->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    pm_status st_gen = enqueue_generation(ga, ga->cap, h, 1);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(ga->cap, &captured);
    PM_TRY(st_gen);
    PM_CUDA(e);
    PM_CUDA(cudaGraphInstantiate(&ga->exec, ga->graph, 0));
    return (ga->graphs & 2) ? build_graph_one(ga) : PM_OK;
}

// Layout of the GA arrays over the instances, the scan plan and the buffers.
static void ga_layout(pm_ga *ga)
{
    const int K = ga->K;
    ga->gps.resize(K);
    int64_t grp = 0, deme = 0, dwords = 0, bestw = 0, Wmax = 0;
    for (int k = 0; k < K; ++k) {
        const pm_instance *in = ga->insts[k];
        const pm_prob &pr = ga->plan.probs[k];
        ga_prob &gp = ga->gps[k];
        gp = ga_prob{};
        gp.pop = ga->P;
        gp.D = ga->D;
        gp.NB = ga->NB;
        gp.W = (int32_t)in->W;
        gp.m = (int32_t)in->m;
        gp.p = (int32_t)in->p;
        gp.lgD = ga->lgD;
        gp.ind_base = pr.ind_base;
        gp.word_base = pr.word_base;
        gp.col_base = pr.col_base;
        gp.grp_base = grp;
        gp.deme_base = deme;
        gp.dword_base = dwords;
        gp.best_base = bestw;
        gp.sid = ga->sid + (uint32_t)k;
        gp.team = ga->team ? 1u : 0u;
        grp += pm_ceil_div(ga->P, 32);
        deme += ga->NB;
        dwords += ga->NB * in->W;
        bestw += in->W;
        Wmax = std::max<int64_t>(Wmax, in->W);
    }
    ga->groups_total = grp;
    ga->demes_total = deme;
    ga->dwords_total = dwords;
    ga->best_total = bestw;
    ga->Wmax = Wmax;
}

// Layout of the speculative mutation cycle's candidates: Q x pop candidate bitsets per instance, their
// facility-major copy, active bits, costs and the scan's accumulators, laid out by spec_plan; the candidates'
// per-instance layout (ga_prob) and scan table (pm_prob) on the device for batched GAs.
static void spec_layout(pm_ga *ga)
{
    const int K = ga->K;
    const int64_t QP = (int64_t)ga->Q * ga->P;
    ga->gqs.resize(K);
    int64_t grp = 0;
    for (int k = 0; k < K; ++k) {
        const pm_prob &pr = ga->spec_plan.probs[k];
        ga_prob &gq = ga->gqs[k];
        gq = ga->gps[k];
        gq.pop = QP;
        gq.ind_base = pr.ind_base;
        gq.word_base = pr.word_base;
        gq.col_base = pr.col_base;
        gq.grp_base = grp;
        grp += pm_ceil_div(QP, 32);
    }
    ga->gq = ga->gqs[0];
    ga->groupsQ_total = grp;
}

// The GA's device buffers, and those of the speculative cycle when `with_spec`, in one allocation: first the
// buffers zeroed at once (accumulators and tickets must start at zero; the rest is written before it is read),
// then the tables the host fills (st, glob, probs, gprobs and the candidates' gqprobs, probsQ), in one copy.
static pm_status ga_alloc(pm_ga *ga, cudaStream_t s, bool with_spec)
{
    const int K = ga->K;
    const size_t words = (size_t)ga->plan.words_total, inds = (size_t)ga->plan.ind_total;
    const size_t acc_bytes = ga->single_row ? pm_plan_partial_bytes(ga->single, ga->P) : inds * 8;
    const size_t tick_bytes = (size_t)pm_round_up(std::max<int64_t>(ga->plan.tiles_total, 1) * 4, 256);
    const pm_multi_plan &sp = ga->spec_plan;
    std::vector<pm_part> parts = {{&ga->X, words * 4},
                                  {&ga->Xc, words * 4},
                                  {&ga->cost, inds * 8},
                                  {&ga->active, inds / 8 + 4},
                                  {&ga->improved, inds},
                                  {&ga->deme_best, (size_t)ga->dwords_total * 4},
                                  {&ga->deme_cost, (size_t)ga->demes_total * 8},
                                  {&ga->best, (size_t)ga->best_total * 4},
                                  {&ga->trace, 8 * 1024},
                                  {&ga->accum, acc_bytes},
                                  {&ga->tickets, tick_bytes},
                                  {&ga->columns, (size_t)ga->plan.cols_total * 4},
                                  {&ga->err, 256}};
    if (with_spec) {
        const pm_part q[] = {{&ga->XQ, (size_t)sp.words_total * 4},
                             {&ga->costQ, (size_t)sp.ind_total * 8},
                             {&ga->activeQ, (size_t)pm_round_up(pm_ceil_div(sp.ind_total, 32) * 4, 256)},
                             {&ga->accumQ, (size_t)sp.ind_total * 8},
                             {&ga->ticketsQ, (size_t)pm_round_up(std::max<int64_t>(sp.tiles_total, 1) * 4, 256)},
                             {&ga->colQ, (size_t)sp.cols_total * 4}};
        parts.insert(parts.end(), q, q + 6);
    }
    const size_t n_zero = parts.size();
    parts.push_back({&ga->st, sizeof(ga_dev) * K});
    parts.push_back({&ga->glob, sizeof(ga_glob)});
    parts.push_back({&ga->probs, sizeof(pm_prob) * K});
    parts.push_back({&ga->gprobs, sizeof(ga_prob) * K});
    if (with_spec) {
        parts.push_back({&ga->gqprobs, sizeof(ga_prob) * K});
        parts.push_back({&ga->probsQ, sizeof(pm_prob) * K});
    }
    PM_TRY(pm_carve(ga->arena, parts.data(), (int)parts.size()));
    char *base = static_cast<char *>(ga->arena.ptr);
    const size_t host_off = static_cast<char *>(parts[n_zero].buf->ptr) - base;
    PM_CUDA(cudaMemsetAsync(base, 0, host_off, s));
    std::vector<char> host(ga->arena.bytes - host_off, 0);
    auto put = [&](const pm_dbuf &b, const void *src, size_t n) {
        std::memcpy(host.data() + (static_cast<char *>(b.ptr) - base - host_off), src, n);
    };
    std::vector<ga_dev> h(K);
    for (int k = 0; k < K; ++k) {
        h[k] = ga_dev{};
        h[k].best_cost = -1;
        h[k].saturation = ga->S;
    }
    ga_glob g = {};
    g.alive = K;
    put(ga->st, h.data(), sizeof(ga_dev) * K);
    put(ga->glob, &g, sizeof(g));
    put(ga->probs, ga->plan.probs.data(), sizeof(pm_prob) * K);
    put(ga->gprobs, ga->gps.data(), sizeof(ga_prob) * K);
    if (with_spec) {
        put(ga->gqprobs, ga->gqs.data(), sizeof(ga_prob) * K);
        put(ga->probsQ, sp.probs.data(), sizeof(pm_prob) * K);
    }
    PM_CUDA(cudaMemcpyAsync(base + host_off, host.data(), host.size(), cudaMemcpyHostToDevice, s));
    PM_CUDA(cudaStreamSynchronize(s));
    return PM_OK;
}

static pm_status ga_configure(pm_ga *ga, int64_t pop, uint64_t seed, const pm_ga_params *params)
{
    if (pop < 2)
        return PM_ERR_INVALID_ARG;
    pm_ga_params prm = {};
    prm.xover_rounds = -1;
    prm.mut_tries = -1;
    if (params)
        prm = *params;
    if ((prm.flags & ~(PM_GA_TUNE | PM_GA_MIGRATE_TEAM | PM_GA_INIT_COMBINADIC)) != 0 || prm.reserved != 0)
        return PM_ERR_INVALID_ARG;
    ga->model = prm.model;
    ga->T = prm.candidates > 0 ? prm.candidates : 4;
    if (ga->T > 8)
        return PM_ERR_INVALID_ARG;
    int64_t D = prm.deme ? prm.deme : std::min<int64_t>(pop, 256);
    if (D < 2 || D > 1024 || (D & (D - 1)) != 0 || pop % D != 0 || prm.saturation < 0)
        return PM_ERR_INVALID_ARG;
    if (pop > ((int64_t)1 << 31))
        return PM_ERR_INVALID_ARG;
    int lg = 0;
    while ((int64_t(1) << lg) < D)
        ++lg;
    ga->seed = seed;
    ga->P = pop;
    ga->D = D;
    ga->NB = pop / D;
    ga->lgD = lg;
    ga->R = prm.xover_rounds < 0 ? lg : prm.xover_rounds;
    ga->Q = prm.mut_tries < 0 ? lg : prm.mut_tries;
    if (ga->R > 255 || ga->Q > 255)
        return PM_ERR_INVALID_ARG;
    ga->S = prm.saturation;
    ga->sid = prm.stream_id;
    ga->team = (prm.flags & PM_GA_MIGRATE_TEAM) != 0;
    ga->comb = (prm.flags & PM_GA_INIT_COMBINADIC) != 0;
    if (ga->team && ga->NB > D)
        return PM_ERR_INVALID_ARG;  // deme 0 cannot hold every deme's best
    return PM_OK;
}

// PM_GA_FUSED=1 in the environment runs qualifying GAs in the persistent kernel; by default every GA uses the
// per-phase kernels and the graph, which measured faster on all but the largest scans (a grid barrier over
// the whole GPU costs about as much as the kernel boundary it replaces).
static bool fused_allowed()
{
    const char *v = std::getenv("PM_GA_FUSED");
    return v && v[0] == '1';
}

// Client splits of a persistent scan over `tiles` tiles on `grid` CTAs: the S (1 <= S <= smax) that minimises
// the items a CTA walks per split, ceil(tiles * S / grid) / S, the smallest S on ties (fewer, larger items).
static int64_t fused_splits(int64_t tiles, int64_t grid, int64_t smax)
{
    int64_t best = 1;
    double best_cost = 1e300;
    for (int64_t S = 1; S <= std::max<int64_t>(smax, 1); ++S) {
        const double c = (double)pm_ceil_div(tiles * S, grid) / (double)S;
        if (c < best_cost - 1e-12) {
            best_cost = c;
            best = S;
        }
    }
    return best;
}

template <int G>
static const void *fused_fn()
{
    return reinterpret_cast<const void *>(k_ga_fused<G>);
}

// Decide whether this GA runs its generations in the persistent kernel, and size it: one instance on the
// column path with the speculative mutation cycle, Floyd generation, no learned try, the packed split
// reduction, and a device that supports cooperative launches with one 1024-thread CTA per SM resident.
static pm_status fused_prepare(pm_ga *ga, cudaStream_t s)
{
    ga->fused = false;
    if (!fused_allowed() || ga->K != 1 || ga->single_row || !ga->spec || ga->model || ga->comb)
        return PM_OK;
    const pm_instance *inst = ga->insts[0];
    const int G = ga->plan.groups;
    if (G != 1 && G != 2 && G != 4)
        return PM_OK;
    int coop = 0;
    PM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, inst->device));
    if (!coop)
        return PM_OK;
    const int64_t W = inst->W, P = ga->P, QP = (int64_t)ga->Q * P;
    const size_t smem = (size_t)std::max<int64_t>(32 * W * G, 32 * (W + inst->p)) * 4;
    if (smem > 200 * 1024)
        return PM_OK;
    const void *fn = G == 4 ? fused_fn<4>() : (G == 2 ? fused_fn<2>() : fused_fn<1>());
    PM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFusedThreads, smem));
    if (per_sm < 1)
        return PM_OK;
    const int64_t grid = (int64_t)per_sm * inst->sm_count;
    const int64_t smax = std::max<int64_t>(1, inst->n / (kFusedThreads / 32));  // every warp gets a client
    ga->f_tiles = pm_ceil_div(P, 32 * G);
    ga->f_splits = fused_splits(ga->f_tiles, grid, smax);
    ga->f_cps = pm_ceil_div(inst->n, ga->f_splits);
    ga->f_tilesQ = pm_ceil_div(QP, 32 * G);
    ga->f_splitsQ = fused_splits(ga->f_tilesQ, grid, smax);
    ga->f_cpsQ = pm_ceil_div(inst->n, ga->f_splitsQ);
    if (!pm_packed_reduction_ok(inst, std::max(ga->f_splits, ga->f_splitsQ)))
        return PM_OK;
    // the candidates' facility-major copy in this G, the population's in the plan's G (the same G)
    PM_TRY(ga->colQ.reserve((size_t)ga->f_tilesQ * W * 32 * G * 4));
    PM_TRY(ga->bar.reserve(256));
    PM_CUDA(cudaMemsetAsync(ga->bar.ptr, 0, 256, s));
    PM_CUDA(cudaStreamSynchronize(s));
    ga->fused_G = G;
    ga->fused_grid = (unsigned)grid;
    ga->fused_smem = smem;
    ga->fused = true;
    return PM_OK;
}

static pm_status fused_launch(pm_ga *ga, cudaStream_t s)
{
    const pm_instance *inst = ga->insts[0];
    FusedArgs a{};
    a.gp = ga->gps[0];
    a.gq = ga->gq;
    a.pi = inst->pi;
    a.delta = inst->delta;
    a.n = inst->n;
    a.stride = inst->stride;
    a.L = (int32_t)inst->L;
    a.cum = inst->cum ? 1 : 0;
    a.tiles = ga->f_tiles;
    a.splits = ga->f_splits;
    a.cps = ga->f_cps;
    a.tilesQ = ga->f_tilesQ;
    a.splitsQ = ga->f_splitsQ;
    a.cpsQ = ga->f_cpsQ;
    a.R = ga->gps[0].p / 2 > 0 ? ga->R : 0;
    a.Q = ga->Q;
    a.seed = ga->seed;
    a.X = static_cast<uint32_t *>(ga->X.ptr);
    a.Xc = static_cast<uint32_t *>(ga->Xc.ptr);
    a.XQ = static_cast<uint32_t *>(ga->XQ.ptr);
    a.colT = static_cast<uint32_t *>(ga->columns.ptr);
    a.colQ = static_cast<uint32_t *>(ga->colQ.ptr);
    a.active = static_cast<uint32_t *>(ga->active.ptr);
    a.activeQ = static_cast<uint32_t *>(ga->activeQ.ptr);
    a.cost = static_cast<int64_t *>(ga->cost.ptr);
    a.costQ = static_cast<int64_t *>(ga->costQ.ptr);
    a.accum = static_cast<unsigned long long *>(ga->accum.ptr);
    a.accumQ = static_cast<unsigned long long *>(ga->accumQ.ptr);
    a.improved = static_cast<uint8_t *>(ga->improved.ptr);
    a.deme_best = static_cast<uint32_t *>(ga->deme_best.ptr);
    a.deme_cost = static_cast<int64_t *>(ga->deme_cost.ptr);
    a.best = static_cast<uint32_t *>(ga->best.ptr);
    a.st = static_cast<ga_dev *>(ga->st.ptr);
    a.glob = static_cast<ga_glob *>(ga->glob.ptr);
    a.bar = static_cast<unsigned *>(ga->bar.ptr);
    a.err = static_cast<int *>(ga->err.ptr);
    a.stall = pm_take_scan_stall() ? 1u : 0u;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ga->fused_grid);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = ga->fused_smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (ga->fused_G) {
    case 1:
        PM_CUDA(cudaLaunchKernelEx(&cfg, k_ga_fused<1>, a));
        break;
    case 2:
        PM_CUDA(cudaLaunchKernelEx(&cfg, k_ga_fused<2>, a));
        break;
    default:
        PM_CUDA(cudaLaunchKernelEx(&cfg, k_ga_fused<4>, a));
        break;
    }
    return PM_OK;
}

// The stream the generation graphs are captured on.
static pm_status ga_make_stream(pm_ga *ga)
{
    PM_CUDA(cudaStreamCreateWithFlags(&ga->cap, cudaStreamNonBlocking));
    return PM_OK;
}

static pm_status ga_create_common(pm_ga *ga, cudaStream_t s)
{
    // the warp-per-individual initialisation may use up to 200 KB of shared memory (set outside any capture)
    PM_CUDA(cudaFuncSetAttribute(k_ga_init_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    ga_layout(ga);
    if (ga->spec)
        spec_layout(ga);
    pm_status st = ga_alloc(ga, s, ga->spec);
    if (st != PM_OK && ga->spec) {
        // no room for the Q x pop candidates: run the mutation cycle try by try instead
        pm_dbuf *bufs[] = {&ga->XQ, &ga->costQ, &ga->activeQ, &ga->accumQ, &ga->ticketsQ, &ga->colQ,
                           &ga->gqprobs, &ga->probsQ};
        for (pm_dbuf *b : bufs)
            b->release();
        cudaGetLastError();
        ga->spec = false;
        st = ga_alloc(ga, s, false);
    }
    if (st == PM_OK)
        st = ga_make_stream(ga);
    if (st == PM_OK)
        st = fused_prepare(ga, s);
    if (st == PM_OK)
        st = build_graph(ga);
    return st;
}

// The binomial table of the combinadic generation (built once per GA on the
// stream).  K = the words of C(m, p) from a log-gamma estimate plus a spare
// word; the kernel reports an overflow if the estimate were ever short.
static pm_status comb_prepare(pm_ga *ga, const pm_instance *inst, cudaStream_t s)
{
    const double log2c = (std::lgamma((double)inst->m + 1.0) - std::lgamma((double)inst->p + 1.0) -
                          std::lgamma((double)(inst->m - inst->p) + 1.0)) / std::log(2.0);
    const int K = (int)(log2c / 32.0) + 2;
    int Q = 1;
    while (Q * 32 < K)
        Q *= 2;
    if (Q > 8)
        return PM_ERR_UNSUPPORTED;  // C(m, p) beyond 2^8192
    const size_t entries = (size_t)(inst->p + 1) * (size_t)(inst->m - inst->p + 1);
    const size_t bytes = comb_head_offset(entries, K) * 4 + entries * 8;  // the entries, then their heads
    if (bytes > ((size_t)4 << 30))
        return PM_ERR_UNSUPPORTED;  // table above 4 GiB
    ga->comb_K = K;
    ga->comb_Q = Q;
    ga->comb_entries = entries;
    PM_TRY(ga->comb_tab.reserve(bytes));
    int *flag = nullptr;
    PM_CUDA(pm_device_malloc_async(reinterpret_cast<void **>(&flag), sizeof(int), s));
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        uint32_t *T = static_cast<uint32_t *>(ga->comb_tab.ptr);
        k_comb_table<<<1, 1024, 0, s>>>(T, reinterpret_cast<uint64_t *>(T + comb_head_offset(entries, K)),
                                        (int32_t)inst->m, (int32_t)inst->p, K, flag);
        e = cudaGetLastError();
    }
    int overflow = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&overflow, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    cudaFreeAsync(flag, s);
    PM_CUDA(e);
    return overflow ? PM_ERR_UNSUPPORTED : PM_OK;
}

static pm_status ga_create_single(pm_instance *inst, uint64_t seed, int64_t pop, const pm_ga_params *params,
                                  void *stream, int graphs, pm_ga **out)
{
    if (!out || !inst)
        return PM_ERR_INVALID_ARG;
    *out = nullptr;
    pm_ga *ga = new (std::nothrow) pm_ga();
    if (!ga)
        return PM_ERR_OOM;
    ga->graphs = graphs;
    ga->insts.push_back(inst);
    ga->device = inst->device;
    ga->K = 1;
    pm_status st = ga_configure(ga, pop, seed, params);
    if (st == PM_OK && cudaSetDevice(inst->device) != cudaSuccess)
        st = PM_ERR_CUDA;
    if (st == PM_OK && params && (params->flags & PM_GA_TUNE))
        st = pm_tune_eval(inst, pop, stream, nullptr);
    if (st == PM_OK && ga->comb)
        st = comb_prepare(ga, inst, static_cast<cudaStream_t>(stream));
    if (st == PM_OK && ga->model) {
        const size_t Pm = (size_t)pop * inst->m, C = (size_t)inst->p * ga->T;
        st = pm_learn_prepare(inst, static_cast<cudaStream_t>(stream));
        if (st == PM_OK) st = ga->s_gain.reserve(Pm * 8);
        if (st == PM_OK) st = ga->s_loss.reserve(Pm * 8);
        if (st == PM_OK) st = ga->s_cap.reserve(Pm * 4);
        if (st == PM_OK) st = ga->s_assign.reserve(Pm * 4);
        if (st == PM_OK) st = ga->moves.reserve((size_t)pop * C * 8);
        if (st == PM_OK) st = ga->xfeat.reserve((size_t)pop * C * 32);
        if (st == PM_OK) st = ga->scores.reserve((size_t)pop * C * 4);
    }
    if (st == PM_OK) {
        ga->single = pm_plan_eval(inst, pop);
        ga->single_row = ga->single.groups == 0;
        ga->plan = pm_plan_from_single(inst, ga->single, pop);
        if (!ga->single_row && ga->Q >= 1 && spec_allowed()) {
            const int64_t QP = (int64_t)ga->Q * pop;
            if (params && (params->flags & PM_GA_TUNE))
                st = pm_tune_eval(inst, QP, stream, nullptr);
            if (st == PM_OK) {
                ga->spec_single = pm_plan_eval(inst, QP);
                ga->spec = ga->spec_single.groups > 0;
                if (ga->spec)
                    ga->spec_plan = pm_plan_from_single(inst, ga->spec_single, QP);
            }
        }
        if (st == PM_OK)
            st = ga_create_common(ga, static_cast<cudaStream_t>(stream));
    }
    if (st != PM_OK) {
        ga_free(ga);
        return st;
    }
    *out = ga;
    return PM_OK;
}

extern "C" pm_status pm_ga_create(pm_instance *inst, uint64_t seed, int64_t pop, const pm_ga_params *params,
                                  void *stream, pm_ga **out)
{
    return ga_create_single(inst, seed, pop, params, stream, 3, out);
}

extern "C" pm_status pm_batch_ga_create(pm_batch *b, uint64_t seed, int64_t pop, const pm_ga_params *params,
                                        void *stream, pm_ga **out)
{
    if (!out || !b)
        return PM_ERR_INVALID_ARG;
    *out = nullptr;
    const auto &insts = pm_batch_instances(b);
    pm_ga *ga = new (std::nothrow) pm_ga();
    if (!ga)
        return PM_ERR_OOM;
    for (const pm_instance *in : insts)
        ga->insts.push_back(const_cast<pm_instance *>(in));
    ga->device = insts.empty() ? 0 : insts[0]->device;
    ga->K = (int)insts.size();
    pm_status st = ga_configure(ga, pop, seed, params);
    if (st == PM_OK && (ga->model || ga->comb))
        st = PM_ERR_UNSUPPORTED;  // the learned try and the combinadic generation are for single-instance GAs
    // crossover runs for all instances or for none: p = 1 mixed with p >= 2 is not supported
    if (st == PM_OK) {
        const bool any1 = std::any_of(insts.begin(), insts.end(), [](const pm_instance *in) { return in->p < 2; });
        const bool all1 = std::all_of(insts.begin(), insts.end(), [](const pm_instance *in) { return in->p < 2; });
        if (any1 && !all1)
            st = PM_ERR_UNSUPPORTED;
    }
    if (st == PM_OK && cudaSetDevice(insts[0]->device) != cudaSuccess)
        st = PM_ERR_CUDA;
    if (st == PM_OK && params && (params->flags & PM_GA_TUNE)) {
        std::vector<int64_t> pops(insts.size(), pop);
        st = pm_batch_tune(b, pops.data(), stream, nullptr);
    }
    if (st == PM_OK)
        st = pm_batch_ga_plan(b, pop, ga->plan);
    // batched GAs evaluate their mutation tries one by one unless PM_GA_SPEC=1: their scans are long, and the
    // tries after an individual's first improvement, which the speculative cycle evaluates too, cost more than
    // the launches it saves (256 uneven instances: 20.4 ms per generation against 19.8 ms try by try)
    if (st == PM_OK && ga->Q >= 1 && spec_forced()) {
        st = pm_batch_ga_plan_candidates(b, pop, (int64_t)ga->Q * pop, ga->spec_plan);
        ga->spec = st == PM_OK;
    }
    if (st == PM_OK)
        st = ga_create_common(ga, static_cast<cudaStream_t>(stream));
    if (st != PM_OK) {
        ga_free(ga);
        return st;
    }
    *out = ga;
    return PM_OK;
}

// Report (and clear) a device-side failure recorded since the last check.  A scan CTA that gave up left its
// split's sums and tile tickets behind: they are zeroed so that later generations evaluate correctly.
static pm_status check_err(pm_ga *ga, cudaStream_t s)
{
    int e = 0;
    PM_CUDA(cudaMemcpyAsync(&e, ga->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaStreamSynchronize(s));
    if (!e)
        return PM_OK;
    pm_dbuf *bufs[] = {&ga->err, &ga->accum, &ga->tickets, &ga->accumQ, &ga->ticketsQ, &ga->bar};
    for (pm_dbuf *b : bufs)
        if (b->ptr)
            PM_CUDA(cudaMemsetAsync(b->ptr, 0, b->bytes, s));
    PM_CUDA(cudaStreamSynchronize(s));
    return (pm_status)e;
}

extern "C" pm_status pm_ga_step(pm_ga *ga, int64_t gens, int64_t *trace, void *stream)
{
    if (!ga || gens < 0)
        return PM_ERR_INVALID_ARG;
    if (gens == 0)
        return PM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pm_clear_stale_error();
    PM_CUDA(cudaSetDevice(ga->device));
    const bool trace_dev = trace && pm_is_device_ptr(trace);
    long long *tr = nullptr;
    const size_t tbytes = (size_t)gens * ga->K * 8;
    if (trace_dev) {
        tr = reinterpret_cast<long long *>(trace);
    } else if (trace) {
        PM_TRY(ga->trace.reserve(tbytes));
        tr = static_cast<long long *>(ga->trace.ptr);
    }
    const bool graph = !ga->fused && graph_mode();
    if (!graph) {
        k_ga_begin<<<(unsigned)pm_ceil_div(ga->K, 256), 256, 0, s>>>(static_cast<ga_glob *>(ga->glob.ptr),
                                                                    static_cast<ga_dev *>(ga->st.ptr), ga->K,
                                                                    (long long)gens, tr,
                                                                    static_cast<unsigned *>(ga->bar.ptr));
        PM_CUDA(cudaGetLastError());
    }
    if (ga->fused) {
        PM_TRY(fused_launch(ga, s));
    } else if (graph) {
        // the graph's root runs k_ga_begin with this call's budget and trace (the update applies to this and
        // later launches of the graph, not to launches already enqueued)
        const bool one = (gens == 1 && ga->exec1) || !ga->exec;
        BeginArgs ba;
        const cudaKernelNodeParams kp = begin_params(ga, (long long)gens, tr, ba);
        PM_CUDA(cudaGraphExecKernelNodeSetParams(one ? ga->exec1 : ga->exec, one ? ga->begin_node1 : ga->begin_node,
                                                 &kp));
        PM_CUDA(cudaGraphLaunch(one ? ga->exec1 : ga->exec, s));
    } else {
        // the same kernels, enqueued generation by generation (profilers cannot see
        // kernels inside conditional graphs); saturation needs the host to look
        for (int64_t g = 0; g < gens; ++g) {
            PM_TRY(enqueue_generation(ga, s, 0, 0));
            if (ga->S > 0) {
                ga_glob h;
                PM_CUDA(cudaMemcpyAsync(&h, ga->glob.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
                PM_CUDA(cudaStreamSynchronize(s));
                if (h.alive == 0)
                    break;
            }
        }
    }
    if (trace && !trace_dev) {
        // generations actually run may be fewer (saturation); copy all slots, the caller reads gens_run
        PM_CUDA(cudaMemcpyAsync(trace, tr, tbytes, cudaMemcpyDeviceToHost, s));
        return check_err(ga, s);
    }
    return PM_OK;
}

extern "C" pm_status pm_ga_instance_result(pm_ga *ga, int64_t k, int64_t *best_cost, uint32_t *best_mask,
                                           int64_t *gens_run, int64_t *evals, void *stream)
{
    if (!ga || k < 0 || k >= ga->K)
        return PM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_CUDA(cudaSetDevice(ga->insts[0]->device));
    ga_dev h;
    PM_CUDA(cudaMemcpyAsync(&h, static_cast<ga_dev *>(ga->st.ptr) + k, sizeof(h), cudaMemcpyDeviceToHost, s));
    if (best_mask)
        PM_CUDA(cudaMemcpyAsync(best_mask, static_cast<uint32_t *>(ga->best.ptr) + ga->gps[k].best_base,
                                (size_t)ga->gps[k].W * 4, cudaMemcpyDefault, s));
    PM_TRY(check_err(ga, s));
    if (best_cost)
        *best_cost = h.best_cost;
    if (gens_run)
        *gens_run = h.total_gens;
    if (evals)
        *evals = h.evals;
    return PM_OK;
}

extern "C" pm_status pm_ga_result(pm_ga *ga, int64_t *best_cost, uint32_t *best_mask, int64_t *gens_run,
                                  int64_t *evals, void *stream)
{
    return pm_ga_instance_result(ga, 0, best_cost, best_mask, gens_run, evals, stream);
}

extern "C" pm_status pm_ga_instance_population(pm_ga *ga, int64_t k, uint32_t *masks, int64_t *costs, void *stream)
{
    if (!ga || k < 0 || k >= ga->K)
        return PM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_CUDA(cudaSetDevice(ga->insts[0]->device));
    const ga_prob &gp = ga->gps[k];
    if (masks)
        PM_CUDA(cudaMemcpyAsync(masks, static_cast<uint32_t *>(ga->X.ptr) + gp.word_base, (size_t)ga->P * gp.W * 4,
                                cudaMemcpyDefault, s));
    if (costs)
        PM_CUDA(cudaMemcpyAsync(costs, static_cast<int64_t *>(ga->cost.ptr) + gp.ind_base, (size_t)ga->P * 8,
                                cudaMemcpyDefault, s));
    return check_err(ga, s);
}

extern "C" pm_status pm_ga_population(pm_ga *ga, uint32_t *masks, int64_t *costs, void *stream)
{
    return pm_ga_instance_population(ga, 0, masks, costs, stream);
}

// ------------------------------ checkpoints --------------------------------

namespace {
struct ga_header {
    char magic[8];
    uint32_t version;
    uint32_t sid;
    uint32_t flags;  // PM_GA_MIGRATE_TEAM, PM_GA_INIT_COMBINADIC
    uint32_t pad;
    int64_t n, m, p, P, D, R, Q, S;
    uint64_t seed;
    ga_dev state;
};
}  // namespace

static size_t ga_blob_size(const pm_ga *ga)
{
    const size_t W = (size_t)ga->insts[0]->W;
    return sizeof(ga_header) + (size_t)ga->NB * W * 4 + (size_t)ga->NB * 8 + W * 4 + (size_t)ga->P * W * 4 +
           (size_t)ga->P * 8;
}

extern "C" pm_status pm_ga_save(pm_ga *ga, void *buf, size_t *len, void *stream)
{
    if (!ga || !len || ga->K != 1 || ga->model)
        return PM_ERR_INVALID_ARG;
    const size_t need = ga_blob_size(ga);
    if (!buf) {
        *len = need;
        return PM_OK;
    }
    if (*len < need)
        return PM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const pm_instance *inst = ga->insts[0];
    PM_CUDA(cudaSetDevice(inst->device));
    ga_header h = {};
    std::memcpy(h.magic, "PMGASAV3", 8);
    h.version = 3;
    h.sid = ga->sid;
    h.flags = (ga->team ? PM_GA_MIGRATE_TEAM : 0u) | (ga->comb ? PM_GA_INIT_COMBINADIC : 0u);
    h.n = inst->n;
    h.m = inst->m;
    h.p = inst->p;
    h.P = ga->P;
    h.D = ga->D;
    h.R = ga->R;
    h.Q = ga->Q;
    h.S = ga->S;
    h.seed = ga->seed;
    const size_t W = (size_t)inst->W;
    char *b = static_cast<char *>(buf) + sizeof(ga_header);
    PM_CUDA(cudaMemcpyAsync(&h.state, ga->st.ptr, sizeof(ga_dev), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaMemcpyAsync(b, ga->deme_best.ptr, (size_t)ga->NB * W * 4, cudaMemcpyDeviceToHost, s));
    b += (size_t)ga->NB * W * 4;
    PM_CUDA(cudaMemcpyAsync(b, ga->deme_cost.ptr, (size_t)ga->NB * 8, cudaMemcpyDeviceToHost, s));
    b += (size_t)ga->NB * 8;
    PM_CUDA(cudaMemcpyAsync(b, ga->best.ptr, W * 4, cudaMemcpyDeviceToHost, s));
    b += W * 4;
    PM_CUDA(cudaMemcpyAsync(b, ga->X.ptr, (size_t)ga->P * W * 4, cudaMemcpyDeviceToHost, s));
    b += (size_t)ga->P * W * 4;
    PM_CUDA(cudaMemcpyAsync(b, ga->cost.ptr, (size_t)ga->P * 8, cudaMemcpyDeviceToHost, s));
    PM_TRY(check_err(ga, s));
    h.state.trace = nullptr;
    std::memcpy(buf, &h, sizeof(h));
    *len = need;
    return PM_OK;
}

extern "C" pm_status pm_ga_load(pm_instance *inst, const void *buf, size_t len, void *stream, pm_ga **out)
{
    if (!inst || !buf || !out || len < sizeof(ga_header))
        return PM_ERR_INVALID_ARG;
    *out = nullptr;
    ga_header h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "PMGASAV3", 8) != 0 || h.version != 3 || h.n != inst->n || h.m != inst->m ||
        h.p != inst->p)
        return PM_ERR_INVALID_ARG;
    pm_ga_params prm = {};
    prm.deme = h.D;
    prm.xover_rounds = (int32_t)h.R;
    prm.mut_tries = (int32_t)h.Q;
    prm.saturation = h.S;
    prm.stream_id = h.sid;
    prm.flags = h.flags & (PM_GA_MIGRATE_TEAM | PM_GA_INIT_COMBINADIC);
    pm_ga *ga = nullptr;
    PM_TRY(pm_ga_create(inst, h.seed, h.P, &prm, stream, &ga));
    if (len < ga_blob_size(ga)) {
        ga_free(ga);
        return PM_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t W = (size_t)inst->W;
    const char *b = static_cast<const char *>(buf) + sizeof(ga_header);
    ga_dev state = h.state;
    state.trace = nullptr;
    ga_glob g = {};
    g.alive = state.stop ? 0 : 1;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpyAsync(ga->st.ptr, &state, sizeof(ga_dev), cudaMemcpyHostToDevice, s);
    e = e ? e : cudaMemcpyAsync(ga->glob.ptr, &g, sizeof(g), cudaMemcpyHostToDevice, s);
    e = e ? e : cudaMemcpyAsync(ga->deme_best.ptr, b, (size_t)ga->NB * W * 4, cudaMemcpyHostToDevice, s);
    b += (size_t)ga->NB * W * 4;
    e = e ? e : cudaMemcpyAsync(ga->deme_cost.ptr, b, (size_t)ga->NB * 8, cudaMemcpyHostToDevice, s);
    b += (size_t)ga->NB * 8;
    e = e ? e : cudaMemcpyAsync(ga->best.ptr, b, W * 4, cudaMemcpyHostToDevice, s);
    b += W * 4;
    e = e ? e : cudaMemcpyAsync(ga->X.ptr, b, (size_t)ga->P * W * 4, cudaMemcpyHostToDevice, s);
    b += (size_t)ga->P * W * 4;
    e = e ? e : cudaMemcpyAsync(ga->cost.ptr, b, (size_t)ga->P * 8, cudaMemcpyHostToDevice, s);
    e = e ? e : cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ga_free(ga);
        return PM_ERR_CUDA;
    }
    *out = ga;
    return PM_OK;
}

extern "C" pm_status pm_ga_info(const pm_ga *ga, int64_t *pop, int64_t *deme, int32_t *xover_rounds,
                                int32_t *mut_tries, int64_t *kernels_per_generation, int64_t *kernels_per_step_call)
{
    if (!ga)
        return PM_ERR_INVALID_ARG;
    const int64_t per_eval = ga->single_row ? 2 : 1;  // column path: the operators write the columns themselves
    const int64_t rounds = ga->gps[0].p / 2 > 0 ? ga->R : 0;
    if (pop)
        *pop = ga->P;
    if (deme)
        *deme = ga->D;
    if (xover_rounds)
        *xover_rounds = ga->R;
    if (mut_tries)
        *mut_tries = ga->Q;
    if (ga->fused) {  // k_ga_begin and one persistent launch per call, whatever the number of generations
        if (kernels_per_generation)
            *kernels_per_generation = 0;
        if (kernels_per_step_call)
            *kernels_per_step_call = 2;
        return PM_OK;
    }
    if (kernels_per_generation)
        *kernels_per_generation = 1 + per_eval + rounds * (1 + per_eval) +
                                  (ga->spec ? 3 : ga->Q * (1 + per_eval)) + 1 + (ga->model ? 4 + per_eval : 0);
    if (kernels_per_step_call)
        *kernels_per_step_call = 1;  // k_ga_begin (a graph-mode call of several generations adds the loop's gate)
    return PM_OK;
}

extern "C" pm_status pm_ga_destroy(pm_ga *ga)
{
    ga_free(ga);
    return PM_OK;
}

extern "C" pm_status pm_ga_run(pm_instance *inst, uint64_t seed, int64_t pop, int64_t gens, const pm_ga_params *params,
                               int64_t *best_cost, uint32_t *best_mask, int64_t *gens_run, int64_t *evals,
                               int64_t *trace, void *stream)
{
    if (!inst || gens < 0)
        return PM_ERR_INVALID_ARG;
    pm_ga *ga = nullptr;
    // one job of `gens` generations: only the graph that runs them is built
    PM_TRY(ga_create_single(inst, seed, pop, params, stream, gens == 1 ? 2 : 1, &ga));
    pm_status st = pm_ga_step(ga, gens, trace, stream);
    if (st == PM_OK)
        st = pm_ga_result(ga, best_cost, best_mask, gens_run, evals, stream);
    ga_free(ga);
    return st;
}
