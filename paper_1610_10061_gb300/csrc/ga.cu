// The genetic algorithm of Sections 3.1, 3.2.2 and 4.3-4.5, run entirely on
// the device.
//
// One generation (the paper's Evolve call plus the host's population
// renewal and migration):
//   k_ga_init        fresh random population by Floyd sampling of a p-subset
//                    (the paper draws a random combinadic rank, Section 4.1;
//                    a 64-bit rank cannot index C(m,p) for the sizes used
//                    here); for generation g > 0 slot 0 of every deme gets that
//                    deme's best of generation g-1 (Section 4.5, variant (i)).
//   evaluate         the fitness kernels (Section 4.2).
//   crossover r      k_ga_crossover builds every child (butterfly partner
//                    t XOR (D >> (1 + r mod lg D)), Section 3.2.2 step 3), the
//                    children are evaluated, and the reduction kernel replaces
//                    a parent by its child iff strictly cheaper.  Children are
//                    built from the population as it was when the round
//                    started (the acceptance runs after all are built).
//   mutation q       k_ga_mutate rotates the whole bitset or a block of it
//                    (Section 4.4) for individuals not yet improved in this
//                    generation; the first strictly cheaper mutant replaces
//                    the individual (Section 3.2.2 step 5).
//   k_ga_deme_best   lowest (cost, index) per deme (Section 3.2.2 step 7).
//   k_ga_finish      global best (strict improvement), saturation counter,
//                    trace, generation counters, loop condition.
// The loop is one CUDA graph: a gate kernel and a conditional while-node
// whose body is one generation; the body's last kernel sets the condition.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), stateless, keyed by
// (seed) with counter (generation, unit, op * 2^16 + slot / 4, stream id);
// draw `slot` is word slot & 3.  U[0, N) = floor(u * N / 2^32).

#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pm_common.cuh"

namespace {

constexpr uint32_t OP_INIT = 0x001u;
constexpr uint32_t OP_XOVER = 0x100u;
constexpr uint32_t OP_MUT = 0x200u;

struct ga_dev {
    long long gen;         // index of the next generation
    long long remaining;   // generations left in the current step
    long long best_cost;   // -1 until the first generation finishes
    long long sat;         // generations since the best last improved
    long long evals;       // fitness evaluations so far
    long long step_gens;   // generations run in the current step
    long long total_gens;  // generations run since creation
    long long saturation;  // S (0 = off)
    long long *trace;      // device trace of the current step
    int stop;
    int pad;
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

// ------------------------------- kernels -----------------------------------

__global__ void k_ga_begin(ga_dev *st, long long gens, long long *trace)
{
    st->remaining = gens;
    st->step_gens = 0;
    st->trace = trace;
}

__global__ void k_ga_gate(ga_dev *st, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, (st->remaining > 0 && !st->stop) ? 1u : 0u);
}

// Where the operator kernels also write the facility-major copy the column
// fitness kernel reads: colT[tile][j][g] for tiles of 32*G individuals
// (colT == nullptr: the evaluation uses the row kernel and needs none).
struct ColumnsOut {
    uint32_t *colT;
    int32_t G;
};

// Transpose the 32 rows (individuals t0 .. t0+31, row r at rows + r*rs) into
// colT, one warp; rows of individuals >= P read as zero.
__device__ __forceinline__ void write_columns(const uint32_t *rows, int64_t rs, int64_t t0, int64_t P, int32_t W,
                                              ColumnsOut co, int lane, int w_begin, int w_step)
{
    if (co.colT == nullptr)
        return;
    const int64_t tile = t0 / (32 * co.G);
    const int32_t g = (int32_t)((t0 / 32) % co.G);
    for (int w = w_begin; w < W; w += w_step) {
        const uint32_t x = (t0 + lane < P) ? rows[(int64_t)lane * rs + w] : 0u;
        const uint32_t col = pm_transpose32(x, lane);
        co.colT[(tile * (int64_t)W * 32 + (int64_t)w * 32 + lane) * co.G + g] = col;
    }
}

// Floyd sampling + migration, one warp per 32 individuals (lane = individual,
// the bitsets in shared memory when they fit, else in place in X); also
// clears the per-generation improved flags and writes the columns.
__global__ void __launch_bounds__(32) k_ga_init(uint32_t *__restrict__ X, uint8_t *__restrict__ improved,
                                                const uint32_t *__restrict__ deme_best, int64_t P, int32_t W,
                                                int32_t m, int32_t p, int64_t D, uint64_t seed, uint32_t sid,
                                                const ga_dev *__restrict__ st, ColumnsOut co, int rows_in_smem)
{
    extern __shared__ uint32_t rows_s[];  // [32][Ws], Ws = W | 1 (odd stride: conflict-free transposes)
    const int lane = threadIdx.x;
    const int64_t t0 = (int64_t)blockIdx.x * 32;
    const int64_t t = t0 + lane;
    const int32_t Ws = W | 1;
    const uint32_t gen = (uint32_t)st->gen;
    uint32_t *row = rows_in_smem ? rows_s + (int64_t)lane * Ws : X + t * W;
    if (t < P) {
        improved[t] = 0;
        if (gen > 0 && (t % D) == 0) {
            const uint32_t *src = deme_best + (t / D) * W;
            for (int w = 0; w < W; ++w)
                row[w] = src[w];
        } else {
            for (int w = 0; w < W; ++w)
                row[w] = 0u;
            uint4 v = make_uint4(0, 0, 0, 0);
            for (int q = 0; q < p; ++q) {
                if ((q & 3) == 0)
                    v = draw_block(seed, gen, (uint32_t)t, OP_INIT, (uint32_t)q >> 2, sid);
                const uint32_t j = (uint32_t)(m - p + q);
                const uint32_t c = uniform_below(word_of(v, q & 3), j + 1);
                const uint32_t pick = ((row[c >> 5] >> (c & 31)) & 1u) ? j : c;
                row[pick >> 5] |= 1u << (pick & 31);
            }
        }
    }
    __syncwarp();
    if (rows_in_smem) {
        // copy the 32 rows out (rows of consecutive individuals are contiguous in X)
        const int64_t nrows = (P - t0) < 32 ? (P - t0) : 32;
        for (int64_t idx = lane; idx < nrows * W; idx += 32)
            X[t0 * W + idx] = rows_s[(idx / W) * Ws + (idx % W)];
        write_columns(rows_s, Ws, t0, P, W, co, lane, 0, 1);
    } else {
        write_columns(X + t0 * W, W, t0, P, W, co, lane, 0, 1);
    }
}

// One crossover round (Section 4.3).  CTA = 32 warps = 32 individuals; warp
// k builds the child of individual t0 + k.  The positions r1, r1+1, ...
// (circularly) are visited as W+1 segments: word w0 = r1/32 from bit r1%32
// up, the following words, and word w0 below bit r1%32.  A warp scan of the
// per-segment counts of 0->1 and 1->0 candidates (C != couple) tells each
// segment how many of its candidates to take; within a segment the lowest
// bits (earliest positions) come first.
__global__ void __launch_bounds__(1024) k_ga_crossover(const uint32_t *__restrict__ X, uint32_t *__restrict__ Xc,
                                                       uint32_t *__restrict__ active, int64_t P, int32_t W, int32_t m,
                                                       int32_t p, int64_t stride, uint32_t round, uint64_t seed,
                                                       uint32_t sid, ga_dev *__restrict__ st, ColumnsOut co)
{
    __shared__ uint32_t valid_s;
    const int lane = threadIdx.x & 31;
    const int k = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * 32;
    const int64_t t = t0 + k;
    if (threadIdx.x == 0)
        valid_s = 0u;
    __syncthreads();
    if (t < P) {
        const uint32_t gen = (uint32_t)st->gen;
        const int64_t partner = t ^ stride;
        const uint32_t pair = (uint32_t)(t < partner ? t : partner);
        const uint4 v = draw_block(seed, gen, pair, OP_XOVER + round, 0, sid);
        const uint32_t r1 = uniform_below(v.x, (uint32_t)m);
        const int i = 1 + (int)uniform_below(v.y, (uint32_t)(p / 2));
        const uint32_t *C = X + t * W;
        const uint32_t *K = X + partner * W;
        uint32_t *F = Xc + t * W;
        const int w0 = (int)(r1 >> 5);
        const uint32_t b0 = r1 & 31u;
        int c01 = 0, c10 = 0;      // candidates in the segments of earlier rounds
        uint32_t w0change = 0u;    // changes to word w0 (first and last segment)
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
                cw = C[w];
                const uint32_t kw = K[w];
                z = ~cw & kw & seg;
                o = cw & ~kw & seg;
            }
            // exclusive warp scan of the two counts packed in one word
            const uint32_t nz = __popc(z), no = __popc(o);
            uint32_t packed = nz | (no << 16);
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
            F[w0] = C[w0] ^ w0change;
        if (lane == 0 && p / 2 > 0 && c01 >= i && c10 >= i)
            atomicOr(&valid_s, 1u << k);
    }
    __syncthreads();
    if (threadIdx.x == 0 && t0 < P) {
        active[t0 >> 5] = valid_s;
        if (valid_s)
            atomicAdd(reinterpret_cast<unsigned long long *>(&st->evals), (unsigned long long)__popc(valid_s));
    }
    write_columns(Xc + t0 * W, W, t0, P, W, co, lane, k, 32);
}

// 32 bits of the bitset C starting at bit position s (s may be as low as
// -31; bits read from below position 0 are zero).
__device__ __forceinline__ uint32_t bits_from(const uint32_t *C, int32_t W, int64_t s)
{
    if (s < 0)
        return __ldg(C) << (uint32_t)(-s);
    const int64_t q = s >> 5;
    const uint32_t r = (uint32_t)(s & 31);
    const uint32_t lo = __ldg(C + q);
    const uint32_t hi = (q + 1 < W) ? __ldg(C + q + 1) : 0u;
    return __funnelshift_r(lo, hi, r);
}

__device__ __forceinline__ uint32_t range_mask(int64_t lo, int64_t hi)  // bits [lo, hi) of a word, 0 <= lo <= hi <= 32
{
    const uint32_t upto = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
    const uint32_t below = lo >= 32 ? 0xffffffffu : ((1u << lo) - 1u);
    return upto & ~below;
}

// One mutation try (Section 4.4).  CTA = 32 warps = 32 individuals; warp k
// rotates individual t0 + k's bits [a, a+len) left by kl: F[a+j] =
// C[a + (j+kl) mod len].  Each output word is at most three pieces, each a
// funnel-shifted 32-bit read of C.
__global__ void __launch_bounds__(1024) k_ga_mutate(const uint32_t *__restrict__ X, uint32_t *__restrict__ Xc,
                                                    uint32_t *__restrict__ active, const uint8_t *__restrict__ improved,
                                                    int64_t P, int32_t W, int32_t m, uint32_t q, uint64_t seed,
                                                    uint32_t sid, ga_dev *__restrict__ st, ColumnsOut co)
{
    __shared__ uint32_t on_s;
    const int lane = threadIdx.x & 31;
    const int k = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * 32;
    const int64_t t = t0 + k;
    if (threadIdx.x == 0)
        on_s = 0u;
    __syncthreads();
    if (t < P && improved[t] == 0) {
        if (lane == 0)
            atomicOr(&on_s, 1u << k);
        const uint32_t gen = (uint32_t)st->gen;
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
        const int64_t kl = right ? (len - kk) : kk;  // rotate left by kl, 1 <= kl < len
        const int64_t pwrap = a + len - kl;          // positions >= pwrap wrap to the start of the block
        const uint32_t *C = X + t * W;
        uint32_t *F = Xc + t * W;
        for (int w = lane; w < W; w += 32) {
            const int64_t pos0 = (int64_t)w * 32;
            const int64_t in_lo = a > pos0 ? a : pos0;
            const int64_t in_hi = (a + len) < (pos0 + 32) ? (a + len) : (pos0 + 32);
            const uint32_t cw = __ldg(C + w);
            if (in_lo >= in_hi) {
                F[w] = cw;
                continue;
            }
            uint32_t out = cw & ~range_mask(in_lo - pos0, in_hi - pos0);
            const int64_t e1 = in_hi < pwrap ? in_hi : pwrap;
            if (in_lo < e1)
                out |= bits_from(C, W, pos0 + kl) & range_mask(in_lo - pos0, e1 - pos0);
            const int64_t s2 = in_lo > pwrap ? in_lo : pwrap;
            if (s2 < in_hi)
                out |= bits_from(C, W, pos0 + kl - len) & range_mask(s2 - pos0, in_hi - pos0);
            F[w] = out;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && t0 < P) {
        active[t0 >> 5] = on_s;
        if (on_s)
            atomicAdd(reinterpret_cast<unsigned long long *>(&st->evals), (unsigned long long)__popc(on_s));
    }
    write_columns(Xc + t0 * W, W, t0, P, W, co, lane, k, 32);
}

// Lowest (cost, index) in each deme -> deme_best / deme_cost.  One CTA per deme.
__global__ void k_ga_deme_best(const uint32_t *__restrict__ X, const int64_t *__restrict__ cost, int64_t D, int32_t W,
                               uint32_t *__restrict__ deme_best, int64_t *__restrict__ deme_cost)
{
    __shared__ long long sc[32];
    __shared__ long long si[32];
    __shared__ long long win;
    const int64_t b = blockIdx.x;
    long long bc = 0x7fffffffffffffffLL, bi = 0x7fffffffffffffffLL;
    for (int64_t k = threadIdx.x; k < D; k += blockDim.x) {
        const int64_t t = b * D + k;
        const long long c = cost[t];
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
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
        deme_cost[b] = bc;
    }
    __syncthreads();
    const int64_t tw = win;
    for (int w = threadIdx.x; w < W; w += blockDim.x)
        deme_best[b * W + w] = X[tw * W + w];
}

// Global best, saturation, trace, counters and the loop condition.
__global__ void k_ga_finish(const uint32_t *__restrict__ deme_best, const int64_t *__restrict__ deme_cost, int64_t NB,
                            int32_t W, int64_t P, uint32_t *__restrict__ best, ga_dev *__restrict__ st,
                            cudaGraphConditionalHandle h, int in_graph)
{
    __shared__ long long sc[32];
    __shared__ long long si[32];
    __shared__ int improve;
    __shared__ long long winner;
    long long bc = 0x7fffffffffffffffLL, bi = 0x7fffffffffffffffLL;
    for (int64_t b = threadIdx.x; b < NB; b += blockDim.x) {
        const long long c = deme_cost[b];
        if (c < bc || (c == bc && b < bi)) {
            bc = c;
            bi = b;
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
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
        const bool better = st->best_cost < 0 || bc < st->best_cost;
        improve = better ? 1 : 0;
        winner = bi;
        if (better) {
            st->best_cost = bc;
            st->sat = 0;
        } else {
            st->sat += 1;
        }
    }
    __syncthreads();
    if (improve)
        for (int w = threadIdx.x; w < W; w += blockDim.x)
            best[w] = deme_best[winner * W + w];
    if (threadIdx.x == 0) {
        if (st->trace)
            st->trace[st->step_gens] = st->best_cost;
        st->evals += P;
        st->gen += 1;
        st->step_gens += 1;
        st->total_gens += 1;
        st->remaining -= 1;
        st->stop = (st->saturation > 0 && st->sat >= st->saturation) ? 1 : 0;
        if (in_graph)
            cudaGraphSetConditional(h, (st->remaining > 0 && !st->stop) ? 1u : 0u);
    }
}

}  // namespace

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
    pm_instance *inst = nullptr;
    uint64_t seed = 0;
    int64_t P = 0, D = 0, NB = 0;
    int lgD = 0, R = 0, Q = 0;
    int64_t S = 0;
    uint32_t sid = 0;
    pm_eval_plan plan;
    pm_dbuf X, Xc, cost, active, improved, deme_best, deme_cost, best, trace, partials, tickets, columns, st, err;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void ga_free(pm_ga *ga)
{
    if (!ga)
        return;
    cudaSetDevice(ga->inst->device);
    if (ga->exec)
        cudaGraphExecDestroy(ga->exec);
    if (ga->graph)
        cudaGraphDestroy(ga->graph);
    if (ga->cap)
        cudaStreamDestroy(ga->cap);
    pm_dbuf *bufs[] = {&ga->X,        &ga->Xc,        &ga->cost, &ga->active, &ga->improved,
                       &ga->deme_best, &ga->deme_cost, &ga->best, &ga->trace,  &ga->partials, &ga->tickets,
                       &ga->columns,  &ga->st,        &ga->err};
    for (pm_dbuf *b : bufs)
        b->release();
    delete ga;
}

// Enqueue one generation on `s`: under stream capture for the graph body
// (in_graph = 1), or directly on the stream (in_graph = 0).
static pm_status enqueue_generation(pm_ga *ga, cudaStream_t s, cudaGraphConditionalHandle h, int in_graph)
{
    pm_instance *inst = ga->inst;
    const int32_t W = (int32_t)inst->W, m = (int32_t)inst->m, p = (int32_t)inst->p;
    ga_dev *st = static_cast<ga_dev *>(ga->st.ptr);
    uint32_t *X = static_cast<uint32_t *>(ga->X.ptr);
    uint32_t *Xc = static_cast<uint32_t *>(ga->Xc.ptr);
    int64_t *cost = static_cast<int64_t *>(ga->cost.ptr);
    uint32_t *active = static_cast<uint32_t *>(ga->active.ptr);
    uint8_t *improved = static_cast<uint8_t *>(ga->improved.ptr);
    int64_t *partials = static_cast<int64_t *>(ga->partials.ptr);
    int *tickets = static_cast<int *>(ga->tickets.ptr);
    uint32_t *columns = static_cast<uint32_t *>(ga->columns.ptr);
    int *err = static_cast<int *>(ga->err.ptr);
    const int64_t P = ga->P;
    const unsigned groups32 = (unsigned)pm_ceil_div(P, 32);
    ColumnsOut co;
    co.colT = ga->plan.groups ? columns : nullptr;
    co.G = ga->plan.groups ? ga->plan.groups : 1;
    const int32_t Ws = W | 1;
    const size_t init_smem = (size_t)32 * Ws * 4;
    const int rows_in_smem = init_smem <= 48 * 1024 ? 1 : 0;

    k_ga_init<<<groups32, 32, rows_in_smem ? init_smem : 0, s>>>(
        X, improved, static_cast<const uint32_t *>(ga->deme_best.ptr), P, W, m, p, ga->D, ga->seed, ga->sid, st, co,
        rows_in_smem);
    PM_CUDA(cudaGetLastError());
    pm_accept_args plain;
    plain.columns_ready = true;
    PM_TRY(pm_launch_eval(inst, ga->plan, X, P, nullptr, cost, partials, tickets, columns, err, plain, s));

    pm_accept_args acc;
    acc.mode = 1;
    acc.cur_cost = cost;
    acc.cur_masks = X;
    acc.cand_masks = Xc;
    acc.columns_ready = true;
    if (p / 2 > 0) {
        for (int r = 0; r < ga->R; ++r) {
            const int64_t stride = ga->D >> (1 + (r % ga->lgD));
            k_ga_crossover<<<groups32, 1024, 0, s>>>(X, Xc, active, P, W, m, p, stride, (uint32_t)r, ga->seed, ga->sid,
                                                     st, co);
            PM_CUDA(cudaGetLastError());
            acc.improved = nullptr;
            PM_TRY(pm_launch_eval(inst, ga->plan, Xc, P, active, nullptr, partials, tickets, columns, err, acc, s));
        }
    }
    for (int q = 0; q < ga->Q; ++q) {
        k_ga_mutate<<<groups32, 1024, 0, s>>>(X, Xc, active, improved, P, W, m, (uint32_t)q, ga->seed, ga->sid, st,
                                              co);
        PM_CUDA(cudaGetLastError());
        acc.improved = improved;
        PM_TRY(pm_launch_eval(inst, ga->plan, Xc, P, active, nullptr, partials, tickets, columns, err, acc, s));
    }
    const int dthreads = (int)std::min<int64_t>(ga->D, 1024);
    k_ga_deme_best<<<(unsigned)ga->NB, (unsigned)pm_round_up(dthreads, 32), 0, s>>>(
        X, cost, ga->D, W, static_cast<uint32_t *>(ga->deme_best.ptr), static_cast<int64_t *>(ga->deme_cost.ptr));
    PM_CUDA(cudaGetLastError());
    k_ga_finish<<<1, 1024, 0, s>>>(static_cast<const uint32_t *>(ga->deme_best.ptr),
                                   static_cast<const int64_t *>(ga->deme_cost.ptr), ga->NB, W, P,
                                   static_cast<uint32_t *>(ga->best.ptr), st, h, in_graph);
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

static pm_status build_graph(pm_ga *ga)
{
    PM_CUDA(cudaGraphCreate(&ga->graph, 0));
    cudaGraphConditionalHandle h;
    PM_CUDA(cudaGraphConditionalHandleCreate(&h, ga->graph, 0, cudaGraphCondAssignDefault));
    // gate: sets the condition from the step's generation budget
    ga_dev *st = static_cast<ga_dev *>(ga->st.ptr);
    void *gate_args[] = {&st, &h};
    cudaKernelNodeParams kp = {};
    kp.func = reinterpret_cast<void *>(k_ga_gate);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = gate_args;
    cudaGraphNode_t gate;
    PM_CUDA(cudaGraphAddKernelNode(&gate, ga->graph, nullptr, 0, &kp));
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
    return PM_OK;
}

static pm_status ga_alloc(pm_ga *ga, cudaStream_t s)
{
    pm_instance *inst = ga->inst;
    const size_t W = (size_t)inst->W, P = (size_t)ga->P;
    PM_TRY(ga->X.reserve(P * W * 4));
    PM_TRY(ga->Xc.reserve(P * W * 4));
    PM_TRY(ga->cost.reserve(P * 8));
    PM_TRY(ga->active.reserve(pm_ceil_div((int64_t)P, 32) * 4));
    PM_TRY(ga->improved.reserve(P));
    PM_TRY(ga->deme_best.reserve((size_t)ga->NB * W * 4));
    PM_TRY(ga->deme_cost.reserve((size_t)ga->NB * 8));
    PM_TRY(ga->best.reserve(W * 4));
    PM_TRY(ga->trace.reserve(8 * 1024));
    ga->plan = pm_plan_eval(inst, ga->P);
    PM_TRY(ga->partials.reserve(pm_plan_partial_bytes(ga->plan, ga->P)));
    PM_TRY(ga->tickets.reserve(pm_plan_ticket_bytes(ga->plan)));
    PM_TRY(ga->columns.reserve(std::max<size_t>(pm_plan_column_bytes(inst, ga->plan), 256)));
    PM_TRY(ga->st.reserve(sizeof(ga_dev)));
    PM_TRY(ga->err.reserve(256));
    PM_CUDA(cudaMemsetAsync(ga->X.ptr, 0, P * W * 4, s));
    PM_CUDA(cudaMemsetAsync(ga->Xc.ptr, 0, P * W * 4, s));
    PM_CUDA(cudaMemsetAsync(ga->cost.ptr, 0, P * 8, s));
    PM_CUDA(cudaMemsetAsync(ga->active.ptr, 0, ga->active.bytes, s));
    PM_CUDA(cudaMemsetAsync(ga->improved.ptr, 0, P, s));
    PM_CUDA(cudaMemsetAsync(ga->deme_best.ptr, 0, ga->deme_best.bytes, s));
    PM_CUDA(cudaMemsetAsync(ga->deme_cost.ptr, 0, ga->deme_cost.bytes, s));
    PM_CUDA(cudaMemsetAsync(ga->best.ptr, 0, ga->best.bytes, s));
    PM_CUDA(cudaMemsetAsync(ga->err.ptr, 0, 256, s));
    PM_CUDA(cudaMemsetAsync(ga->tickets.ptr, 0, ga->tickets.bytes, s));    // tile tickets start at zero
    PM_CUDA(cudaMemsetAsync(ga->partials.ptr, 0, ga->partials.bytes, s));  // and so do the accumulators
    ga_dev h = {};
    h.best_cost = -1;
    h.saturation = ga->S;
    PM_CUDA(cudaMemcpyAsync(ga->st.ptr, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    PM_CUDA(cudaStreamSynchronize(s));
    PM_CUDA(cudaStreamCreateWithFlags(&ga->cap, cudaStreamNonBlocking));
    return PM_OK;
}

static pm_status ga_configure(pm_ga *ga, pm_instance *inst, uint64_t seed, int64_t pop, const pm_ga_params *params)
{
    if (!inst || pop < 2)
        return PM_ERR_INVALID_ARG;
    pm_ga_params prm = {};
    prm.xover_rounds = -1;
    prm.mut_tries = -1;
    if (params)
        prm = *params;
    if ((prm.flags & ~PM_GA_TUNE) != 0)
        return PM_ERR_INVALID_ARG;
    int64_t D = prm.deme ? prm.deme : std::min<int64_t>(pop, 256);
    if (D < 2 || D > 1024 || (D & (D - 1)) != 0 || pop % D != 0 || prm.saturation < 0)
        return PM_ERR_INVALID_ARG;
    if (pop > ((int64_t)1 << 31))
        return PM_ERR_INVALID_ARG;
    int lg = 0;
    while ((int64_t(1) << lg) < D)
        ++lg;
    ga->inst = inst;
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
    return PM_OK;
}

extern "C" pm_status pm_ga_create(pm_instance *inst, uint64_t seed, int64_t pop, const pm_ga_params *params,
                                  void *stream, pm_ga **out)
{
    if (!out)
        return PM_ERR_INVALID_ARG;
    *out = nullptr;
    pm_ga *ga = new (std::nothrow) pm_ga();
    if (!ga)
        return PM_ERR_OOM;
    pm_status st = ga_configure(ga, inst, seed, pop, params);
    if (st != PM_OK) {
        delete ga;
        return st;
    }
    cudaError_t e = cudaSetDevice(inst->device);
    if (e != cudaSuccess) {
        delete ga;
        return PM_ERR_CUDA;
    }
    if (params && (params->flags & PM_GA_TUNE))
        st = pm_tune_eval(inst, pop, stream, nullptr);
    if (st == PM_OK)
        st = ga_alloc(ga, static_cast<cudaStream_t>(stream));
    if (st == PM_OK)
        st = build_graph(ga);
    if (st != PM_OK) {
        ga_free(ga);
        return st;
    }
    *out = ga;
    return PM_OK;
}

// PM_GA_GRAPH=0 in the environment selects direct stream launches instead of
// the conditional-while graph (identical results; for profiling).
static bool graph_mode()
{
    const char *v = std::getenv("PM_GA_GRAPH");
    return !(v && v[0] == '0');
}

static pm_status check_err(pm_ga *ga, cudaStream_t s)
{
    int e = 0;
    PM_CUDA(cudaMemcpyAsync(&e, ga->err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaStreamSynchronize(s));
    return e ? (pm_status)e : PM_OK;
}

extern "C" pm_status pm_ga_step(pm_ga *ga, int64_t gens, int64_t *trace, void *stream)
{
    if (!ga || gens < 0)
        return PM_ERR_INVALID_ARG;
    if (gens == 0)
        return PM_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_CUDA(cudaSetDevice(ga->inst->device));
    const bool trace_dev = trace && pm_is_device_ptr(trace);
    long long *tr = nullptr;
    if (trace_dev) {
        tr = reinterpret_cast<long long *>(trace);
    } else if (trace) {
        PM_TRY(ga->trace.reserve((size_t)gens * 8));
        tr = static_cast<long long *>(ga->trace.ptr);
    }
    k_ga_begin<<<1, 1, 0, s>>>(static_cast<ga_dev *>(ga->st.ptr), (long long)gens, tr);
    PM_CUDA(cudaGetLastError());
    if (graph_mode()) {
        PM_CUDA(cudaGraphLaunch(ga->exec, s));
    } else {
        // the same kernels, enqueued generation by generation (profilers cannot see
        // kernels inside conditional graphs); saturation needs the host to look
        for (int64_t g = 0; g < gens; ++g) {
            PM_TRY(enqueue_generation(ga, s, 0, 0));
            if (ga->S > 0) {
                ga_dev h;
                PM_CUDA(cudaMemcpyAsync(&h, ga->st.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
                PM_CUDA(cudaStreamSynchronize(s));
                if (h.stop)
                    break;
            }
        }
    }
    if (trace && !trace_dev) {
        // generations actually run may be fewer (saturation); copy all `gens` slots, caller reads gens_run
        PM_CUDA(cudaMemcpyAsync(trace, tr, (size_t)gens * 8, cudaMemcpyDeviceToHost, s));
        return check_err(ga, s);
    }
    return PM_OK;
}

extern "C" pm_status pm_ga_result(pm_ga *ga, int64_t *best_cost, uint32_t *best_mask, int64_t *gens_run,
                                  int64_t *evals, void *stream)
{
    if (!ga)
        return PM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_CUDA(cudaSetDevice(ga->inst->device));
    ga_dev h;
    PM_CUDA(cudaMemcpyAsync(&h, ga->st.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
    if (best_mask)
        PM_CUDA(cudaMemcpyAsync(best_mask, ga->best.ptr, (size_t)ga->inst->W * 4, cudaMemcpyDefault, s));
    PM_TRY(check_err(ga, s));
    if (best_cost)
        *best_cost = h.best_cost;
    if (gens_run)
        *gens_run = h.total_gens;
    if (evals)
        *evals = h.evals;
    return PM_OK;
}

extern "C" pm_status pm_ga_population(pm_ga *ga, uint32_t *masks, int64_t *costs, void *stream)
{
    if (!ga)
        return PM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_CUDA(cudaSetDevice(ga->inst->device));
    if (masks)
        PM_CUDA(cudaMemcpyAsync(masks, ga->X.ptr, (size_t)ga->P * ga->inst->W * 4, cudaMemcpyDefault, s));
    if (costs)
        PM_CUDA(cudaMemcpyAsync(costs, ga->cost.ptr, (size_t)ga->P * 8, cudaMemcpyDefault, s));
    return check_err(ga, s);
}

// ------------------------------ checkpoints --------------------------------

namespace {
struct ga_header {
    char magic[8];
    uint32_t version;
    uint32_t sid;
    int64_t n, m, p, P, D, R, Q, S;
    uint64_t seed;
    ga_dev state;
};
}  // namespace

static size_t ga_blob_size(const pm_ga *ga)
{
    const size_t W = (size_t)ga->inst->W;
    return sizeof(ga_header) + (size_t)ga->NB * W * 4 + (size_t)ga->NB * 8 + W * 4 + (size_t)ga->P * W * 4 +
           (size_t)ga->P * 8;
}

extern "C" pm_status pm_ga_save(pm_ga *ga, void *buf, size_t *len, void *stream)
{
    if (!ga || !len)
        return PM_ERR_INVALID_ARG;
    const size_t need = ga_blob_size(ga);
    if (!buf) {
        *len = need;
        return PM_OK;
    }
    if (*len < need)
        return PM_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_CUDA(cudaSetDevice(ga->inst->device));
    ga_header h = {};
    std::memcpy(h.magic, "PMGASAV1", 8);
    h.version = 1;
    h.sid = ga->sid;
    h.n = ga->inst->n;
    h.m = ga->inst->m;
    h.p = ga->inst->p;
    h.P = ga->P;
    h.D = ga->D;
    h.R = ga->R;
    h.Q = ga->Q;
    h.S = ga->S;
    h.seed = ga->seed;
    const size_t W = (size_t)ga->inst->W;
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
    if (std::memcmp(h.magic, "PMGASAV1", 8) != 0 || h.version != 1 || h.n != inst->n || h.m != inst->m ||
        h.p != inst->p)
        return PM_ERR_INVALID_ARG;
    pm_ga_params prm = {};
    prm.deme = h.D;
    prm.xover_rounds = (int32_t)h.R;
    prm.mut_tries = (int32_t)h.Q;
    prm.saturation = h.S;
    prm.stream_id = h.sid;
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
    state.remaining = 0;
    state.step_gens = 0;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpyAsync(ga->st.ptr, &state, sizeof(ga_dev), cudaMemcpyHostToDevice, s);
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
    const int64_t per_eval = ga->plan.groups ? 1 : 2;  // the operators write the columns themselves
    const int64_t rounds = ga->inst->p / 2 > 0 ? ga->R : 0;
    if (pop)
        *pop = ga->P;
    if (deme)
        *deme = ga->D;
    if (xover_rounds)
        *xover_rounds = ga->R;
    if (mut_tries)
        *mut_tries = ga->Q;
    if (kernels_per_generation)
        *kernels_per_generation = 1 + per_eval + rounds * (1 + per_eval) + ga->Q * (1 + per_eval) + 2;
    if (kernels_per_step_call)
        *kernels_per_step_call = graph_mode() ? 2 : 1;  // k_ga_begin (and the gate in graph mode)
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
    PM_TRY(pm_ga_create(inst, seed, pop, params, stream, &ga));
    pm_status st = pm_ga_step(ga, gens, trace, stream);
    if (st == PM_OK)
        st = pm_ga_result(ga, best_cost, best_mask, gens_run, evals, stream);
    ga_free(ga);
    return st;
}
