// The Hammer-Beresnev polynomial of an instance, merged and evaluated on the
// device (Section 2.1, Eq. 6 and Example 1).
//
// Client i contributes Delta'_i[k] times the monomial prod_{s<k} z_{Pi'_i[s]}
// for k = 0 .. L-1 (k = 0 is the constant term); z_j = 1 - x_j, so a monomial
// is 1 exactly when none of its facilities is open.  Like monomials (equal
// facility sets, from different clients) are merged by adding their
// coefficients, and zero coefficients are dropped, which gives the reduced
// polynomial of Example 1.  The value at an open set is the cost (Eq. 4
// summed over clients), so this is a second, independent evaluator of the
// same integer the scan computes.
//
// Device construction:
//  * k_hbp_terms: a warp per client walks its row 32 ranks at a time; the
//    set of term (i, k) is the row's first k facilities, hashed by the XOR of
//    a 64-bit Philox key per facility (an exclusive XOR scan along the row),
//    so a set's hash does not depend on the order of its facilities.
//  * k_hbp_insert: a thread per term with a non-zero coefficient inserts it
//    into an open-addressing table keyed by (size, hash).  A slot is owned by
//    the first term that claims it (atomic compare-and-swap of its index);
//    a later term with the same size and hash is compared facility by
//    facility with the owner's set (both are prefixes of Pi' rows) and adds
//    its coefficient only if the sets are equal, else probes on, so the merge
//    is exact whatever the hash does.
//  * k_hbp_compact: the owned slots become the monomial list: a W-word bitset
//    of facilities and an int64 coefficient each, in table order.
//  * k_hbp_eval: a CTA per individual sums the coefficients of the monomials
//    disjoint from the individual's open set.
// The work is n * L terms to build and (terms x W) words per evaluation,
// against n * (m+1)/(p+1) steps of the scan: an evaluator for small
// instances and for checking, not for the GA.

#include <cstdint>
#include <new>

#include "pm_alloc.h"
#include "pm_common.cuh"

namespace {

constexpr int64_t kMaxTerms = int64_t(1) << 26;  // n * L limit of the dictionary
constexpr uint32_t kOpHbp = 0x400u;              // Philox operation id of the facility keys

__device__ __forceinline__ uint4 hbp_philox10(uint4 c, uint32_t k0, uint32_t k1)
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

// 64-bit key of facility j: two words of Philox4x32-10(counter (j, 0, 0x400 * 2^16, 0), key (0, 0)).
__device__ __forceinline__ unsigned long long facility_key(uint32_t j)
{
    const uint4 v = hbp_philox10(make_uint4(j, 0u, kOpHbp << 16, 0u), 0u, 0u);
    return ((unsigned long long)v.y << 32) | v.x;
}

// Term (i, k): hash of {Pi'_i[0..k-1]} and its coefficient Delta'_i[k] (from D' for cumulative tables).
__global__ void k_hbp_terms(const uint16_t *__restrict__ pi, const int32_t *__restrict__ delta, int64_t n,
                            int32_t L, int64_t stride, int cum, unsigned long long *__restrict__ hash,
                            int32_t *__restrict__ coef)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n)
        return;
    unsigned long long carry = 0ull;  // hash of the first `base` facilities
    int32_t prev_last = 0;            // D' of rank base - 1 (cumulative tables)
    for (int base = 0; base < L; base += 32) {
        const int k = base + lane;
        uint32_t j = 0;
        int32_t v = 0;
        if (k < L) {
            j = pi[i * stride + k];
            v = delta[i * stride + k];
        }
        // exclusive XOR scan of the keys: the set of term k holds ranks 0 .. k-1
        const unsigned long long key = (k < L) ? facility_key(j) : 0ull;
        unsigned long long x = key;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(PM_FULL_MASK, x, o);
            if (lane >= o)
                x ^= y;
        }
        const unsigned long long excl = carry ^ x ^ key;
        int32_t c = v;
        if (cum) {  // Delta' = consecutive differences of D'
            const int32_t left = __shfl_up_sync(PM_FULL_MASK, v, 1);
            c = v - (lane == 0 ? prev_last : left);
            prev_last = __shfl_sync(PM_FULL_MASK, v, 31);
        }
        if (k < L) {
            hash[i * L + k] = excl;
            coef[i * L + k] = c;
        }
        carry ^= __shfl_sync(PM_FULL_MASK, x, 31);
    }
}

// Are the first k facilities of rows a and b the same set?  Both are duplicate-free prefixes of Pi' rows, so
// the common leading run (equal rank by rank) is skipped and every later facility of a is looked up among the
// later facilities of b.
__device__ bool same_prefix_set(const uint16_t *__restrict__ pi, int64_t stride, int64_t a, int64_t b, int32_t k)
{
    const uint16_t *ra = pi + a * stride, *rb = pi + b * stride;
    int32_t s0 = 0;
    while (s0 < k && ra[s0] == rb[s0])
        ++s0;
    for (int32_t s = s0; s < k; ++s) {
        const uint16_t f = ra[s];
        bool found = false;
        for (int32_t q = s0; q < k && !found; ++q)
            found = rb[q] == f;
        if (!found)
            return false;
    }
    return true;
}

// Owned slots whose merged coefficient is not zero.
__global__ void k_hbp_count(const unsigned long long *__restrict__ owner, const unsigned long long *__restrict__ sum,
                            uint64_t slots, unsigned long long *__restrict__ count)
{
    const uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = slot < slots && owner[slot] != 0ull && sum[slot] != 0ull;
    const uint32_t b = __ballot_sync(PM_FULL_MASK, live);
    if ((threadIdx.x & 31) == 0 && b)
        atomicAdd(count, (unsigned long long)__popc(b));
}

__device__ __forceinline__ uint64_t slot_of(unsigned long long h, int32_t k, uint64_t mask)
{
    unsigned long long x = h ^ ((unsigned long long)(uint32_t)k * 0x9E3779B97F4A7C15ull);
    x ^= x >> 31;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 29;
    return x & mask;
}

// owner[slot]: 0 = empty, else 1 + the index (i * L + k) of the term that claimed it; sum[slot]: the merged
// coefficient.
__global__ void k_hbp_insert(const uint16_t *__restrict__ pi, int64_t stride, int64_t n, int32_t L,
                             const unsigned long long *__restrict__ hash, const int32_t *__restrict__ coef,
                             unsigned long long *__restrict__ owner, unsigned long long *__restrict__ sum,
                             uint64_t mask, int *__restrict__ err)
{
    const int64_t term = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (term >= n * L)
        return;
    const int32_t c = coef[term];
    if (c == 0)
        return;
    const int64_t i = term / L;
    const int32_t k = (int32_t)(term % L);
    const unsigned long long h = hash[term];
    uint64_t slot = slot_of(h, k, mask);
    for (uint64_t probe = 0; probe <= mask; ++probe, slot = (slot + 1) & mask) {
        unsigned long long o = atomicCAS(owner + slot, 0ull, (unsigned long long)term + 1ull);
        if (o != 0ull) {
            const int64_t ot = (int64_t)(o - 1ull);
            const int32_t ok = (int32_t)(ot % L);
            if (ok != k || hash[ot] != h || !same_prefix_set(pi, stride, i, ot / L, k))
                continue;  // another set in this slot
        }
        atomicAdd(sum + slot, (unsigned long long)(uint32_t)c);
        return;
    }
    atomicExch(err, (int)PM_ERR_OOM);  // table full (cannot happen at the sizes the host allocates)
}

// Owned slots with a non-zero sum -> monomial bitsets and coefficients.
__global__ void k_hbp_compact(const uint16_t *__restrict__ pi, int64_t stride, int32_t L, int32_t W,
                              const unsigned long long *__restrict__ owner, const unsigned long long *__restrict__ sum,
                              uint64_t slots, uint32_t *__restrict__ sets, long long *__restrict__ coeffs,
                              unsigned long long *__restrict__ count)
{
    const int lane = threadIdx.x & 31;
    const uint64_t slot = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (slot >= slots)
        return;
    const unsigned long long o = owner[slot];
    const unsigned long long c = sum[slot];
    if (o == 0ull || c == 0ull)
        return;
    unsigned long long idx = 0;
    if (lane == 0)
        idx = atomicAdd(count, 1ull);
    idx = __shfl_sync(PM_FULL_MASK, idx, 0);
    const int64_t term = (int64_t)(o - 1ull);
    const int64_t i = term / L;
    const int32_t k = (int32_t)(term % L);
    uint32_t *out = sets + idx * (uint64_t)W;
    for (int w = lane; w < W; w += 32)
        out[w] = 0u;
    __syncwarp();
    for (int32_t s = lane; s < k; s += 32) {
        const uint32_t f = pi[i * stride + s];
        atomicOr(out + (f >> 5), 1u << (f & 31));
    }
    if (lane == 0)
        coeffs[idx] = (long long)c;
}

// A CTA per individual: the sum of the coefficients of the monomials that share no facility with its open set.
__global__ void __launch_bounds__(256) k_hbp_eval(const uint32_t *__restrict__ sets,
                                                  const long long *__restrict__ coeffs, int64_t terms, int32_t W,
                                                  const uint32_t *__restrict__ masks, int64_t pop,
                                                  long long *__restrict__ costs)
{
    extern __shared__ uint32_t xs[];  // the individual's bitset
    __shared__ long long part[8];
    const int64_t t = blockIdx.x;
    for (int w = threadIdx.x; w < W; w += blockDim.x)
        xs[w] = masks[t * W + w];
    __syncthreads();
    long long acc = 0;
    for (int64_t q = threadIdx.x; q < terms; q += blockDim.x) {
        const uint32_t *s = sets + q * W;
        bool zero = true;  // z_j = 1 - x_j: the monomial is 1 iff none of its facilities is open
        for (int w = 0; w < W && zero; ++w)
            zero = (s[w] & xs[w]) == 0u;
        if (zero)
            acc += coeffs[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(PM_FULL_MASK, acc, o);
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long total = 0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi)
            total += part[wi];
        costs[t] = total;
    }
}

}  // namespace

struct pm_hbp {
    int device = 0;
    int64_t terms = 0, W = 0, m = 0;
    pm_dbuf sets, coeffs;
};

extern "C" pm_status pm_hbp_destroy(pm_hbp *h)
{
    if (!h)
        return PM_OK;
    pm_clear_error(cudaSetDevice(h->device));
    h->sets.release();
    h->coeffs.release();
    delete h;
    return PM_OK;
}

static pm_status hbp_build(pm_instance *inst, cudaStream_t s, pm_hbp *h)
{
    const int64_t n = inst->n, L = inst->L, T = n * L;
    uint64_t slots = 1024;
    while (slots < (uint64_t)(2 * T))
        slots <<= 1;
    pm_dbuf hash, coef, owner, sum, count, err;
    struct Release {  // scratch of the build, freed on every exit
        pm_dbuf *b[6];
        ~Release()
        {
            for (pm_dbuf *x : b)
                x->release();
        }
    } rel{{&hash, &coef, &owner, &sum, &count, &err}};
    PM_TRY(hash.reserve((size_t)T * 8));
    PM_TRY(coef.reserve((size_t)T * 4));
    PM_TRY(owner.reserve((size_t)slots * 8));
    PM_TRY(sum.reserve((size_t)slots * 8));
    PM_TRY(count.reserve(256));
    PM_TRY(err.reserve(256));
    PM_CUDA(cudaMemsetAsync(owner.ptr, 0, owner.bytes, s));
    PM_CUDA(cudaMemsetAsync(sum.ptr, 0, sum.bytes, s));
    PM_CUDA(cudaMemsetAsync(count.ptr, 0, count.bytes, s));
    PM_CUDA(cudaMemsetAsync(err.ptr, 0, err.bytes, s));
    const unsigned tblocks = (unsigned)pm_ceil_div(n * 32, 256);
    k_hbp_terms<<<tblocks, 256, 0, s>>>(inst->pi, inst->delta, n, (int32_t)L, inst->stride, inst->cum ? 1 : 0,
                                         static_cast<unsigned long long *>(hash.ptr), static_cast<int32_t *>(coef.ptr));
    PM_CUDA(cudaGetLastError());
    k_hbp_insert<<<(unsigned)pm_ceil_div(T, 256), 256, 0, s>>>(
        inst->pi, inst->stride, n, (int32_t)L, static_cast<const unsigned long long *>(hash.ptr),
        static_cast<const int32_t *>(coef.ptr), static_cast<unsigned long long *>(owner.ptr),
        static_cast<unsigned long long *>(sum.ptr), (uint64_t)(slots - 1), static_cast<int *>(err.ptr));
    PM_CUDA(cudaGetLastError());
    // count the merged monomials, then size the list
    k_hbp_count<<<(unsigned)pm_ceil_div((int64_t)slots, 256), 256, 0, s>>>(
        static_cast<const unsigned long long *>(owner.ptr), static_cast<const unsigned long long *>(sum.ptr), slots,
        static_cast<unsigned long long *>(count.ptr));
    PM_CUDA(cudaGetLastError());
    unsigned long long live = 0, claimed = 0;
    int e = 0;
    PM_CUDA(cudaMemcpyAsync(&e, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaMemcpyAsync(&live, count.ptr, sizeof(live), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaMemsetAsync(count.ptr, 0, count.bytes, s));
    PM_CUDA(cudaStreamSynchronize(s));
    if (e)
        return (pm_status)e;
    const size_t cap = (size_t)std::max<unsigned long long>(live, 1ull);
    if (cap * (size_t)inst->W * 4 > ((size_t)8 << 30))
        return PM_ERR_UNSUPPORTED;  // more than 8 GiB of monomial bitsets
    PM_TRY(h->sets.reserve(cap * (size_t)inst->W * 4));
    PM_TRY(h->coeffs.reserve(cap * 8));
    k_hbp_compact<<<(unsigned)pm_ceil_div((int64_t)slots * 32, 256), 256, 0, s>>>(
        inst->pi, inst->stride, (int32_t)L, (int32_t)inst->W, static_cast<const unsigned long long *>(owner.ptr),
        static_cast<const unsigned long long *>(sum.ptr), slots, static_cast<uint32_t *>(h->sets.ptr),
        static_cast<long long *>(h->coeffs.ptr), static_cast<unsigned long long *>(count.ptr));
    PM_CUDA(cudaGetLastError());
    PM_CUDA(cudaMemcpyAsync(&claimed, count.ptr, sizeof(claimed), cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaStreamSynchronize(s));
    h->terms = (int64_t)claimed;
    return PM_OK;
}

extern "C" pm_status pm_hbp_create(pm_instance *inst, void *stream, pm_hbp **out)
{
    if (!inst || !out)
        return PM_ERR_INVALID_ARG;
    *out = nullptr;
    if (inst->n * inst->L > kMaxTerms)
        return PM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(inst->lock);
    pm_clear_stale_error();
    PM_CUDA(cudaSetDevice(inst->device));
    pm_hbp *h = new (std::nothrow) pm_hbp();
    if (!h)
        return PM_ERR_OOM;
    h->device = inst->device;
    h->W = inst->W;
    h->m = inst->m;
    pm_status st = hbp_build(inst, static_cast<cudaStream_t>(stream), h);
    if (st != PM_OK) {
        pm_hbp_destroy(h);
        return st;
    }
    *out = h;
    return PM_OK;
}

extern "C" pm_status pm_hbp_info(const pm_hbp *h, int64_t *terms, int64_t *W)
{
    if (!h)
        return PM_ERR_INVALID_ARG;
    if (terms)
        *terms = h->terms;
    if (W)
        *W = h->W;
    return PM_OK;
}

extern "C" pm_status pm_hbp_terms(const pm_hbp *h, uint32_t *sets, int64_t *coeffs, void *stream)
{
    if (!h || (!sets && !coeffs))
        return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->terms > 0) {
        if (sets)
            PM_CUDA(cudaMemcpyAsync(sets, h->sets.ptr, (size_t)h->terms * h->W * 4, cudaMemcpyDefault, s));
        if (coeffs)
            PM_CUDA(cudaMemcpyAsync(coeffs, h->coeffs.ptr, (size_t)h->terms * 8, cudaMemcpyDefault, s));
    }
    PM_CUDA(cudaStreamSynchronize(s));
    return PM_OK;
}

extern "C" pm_status pm_hbp_eval(pm_hbp *h, const uint32_t *masks, int64_t pop, int64_t *costs, void *stream)
{
    if (!h || pop < 0)
        return PM_ERR_INVALID_ARG;
    if (pop == 0)
        return PM_OK;
    if (!masks || !costs || !pm_is_device_ptr(masks) || !pm_is_device_ptr(costs))
        return PM_ERR_INVALID_ARG;
    pm_clear_stale_error();
    PM_CUDA(cudaSetDevice(h->device));
    const size_t smem = (size_t)h->W * 4;
    k_hbp_eval<<<(unsigned)pop, 256, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint32_t *>(h->sets.ptr), static_cast<const long long *>(h->coeffs.ptr), h->terms,
        (int32_t)h->W, masks, pop, reinterpret_cast<long long *>(costs));
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}
