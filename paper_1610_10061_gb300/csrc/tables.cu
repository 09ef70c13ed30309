// Truncated ordering and increment tables (Section 2.1, Eq. 4 and the
// truncation argument after Eq. 6), built on the device.
//
// For client i, Pi'_i lists the facility ids in ascending order of d_ij
// (equal distances by ascending id) and Delta'_i holds the first distance
// followed by consecutive differences; only the first L = m - p + 1 ranks
// are kept.
//
// GB300 design: one CTA per row (grid-stride over rows), a stable LSD radix
// sort of the row's distances with 8-bit digits.  The row starts in facility
// order, so a stable sort on the distance alone yields the (distance, id)
// order; only ceil(bits(max d) / 8) passes are needed.  Each pass:
//   count   - every warp owns a contiguous segment of the row and walks it 32
//             keys at a time, one shared-memory atomic per key into the warp's
//             histogram (faster than grouping equal digits first, even when
//             every key of a row is equal);
//   offsets - per digit, the running count over warps, plus the exclusive
//             scan over digits;
//   scatter - the same walk; nine ballots give each lane the lanes holding
//             the same digit, a key's destination is its warp's offset for that
//             digit plus the number of those lanes below it, then the lowest of
//             them advances the offset.
// Keys (uint32) and ids (uint16) live in shared memory when the row fits
// (12 bytes per element), else in a per-CTA global scratch slice.  When every
// distance is below 2^16 (kPacked) a key and its id share one word,
// (distance << 16) | id, and the digits come from the upper half: 8 bytes per
// element, so two 10000-wide rows sort at once on an SM, and a scatter moves
// one word.  The epilogue writes Pi' and the differences Delta' into rows
// padded to a stride of round_up(L, 32) elements (padding = 0).

#include "pm_alloc.h"
#include "pm_common.cuh"

namespace {

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void k_minmax(const int32_t *__restrict__ d, int64_t count, int *__restrict__ out)
{
    int lo = 0x7fffffff, hi = (int)0x80000000;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = __ldg(d + i);
        lo = min(lo, v);
        hi = max(hi, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(PM_FULL_MASK, lo, o));
        hi = max(hi, __shfl_xor_sync(PM_FULL_MASK, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out + 0, lo);
        atomicMax(out + 1, hi);
    }
}

__global__ void k_minmax_init(int *out)
{
    out[0] = 0x7fffffff;
    out[1] = (int)0x80000000;
}

// The lanes whose 9-bit value equals this lane's (digits 0..255, 256 = no key): one ballot per bit.  Faster
// here than __match_any_sync, whose latency sits on every step of the scatter walk.
__device__ __forceinline__ unsigned equal_digit_lanes(uint32_t dig)
{
    unsigned peers = PM_FULL_MASK;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const unsigned bb = __ballot_sync(PM_FULL_MASK, (dig >> b) & 1u);
        peers &= ((dig >> b) & 1u) ? bb : ~bb;
    }
    return peers;
}

template <bool kPacked>
__global__ void __launch_bounds__(kSortThreads) k_tables(const int32_t *__restrict__ d, int64_t n, int32_t m,
                                                         int32_t L, int64_t stride, int passes, int cum,
                                                         uint16_t *__restrict__ pi, int32_t *__restrict__ delta,
                                                         unsigned char *__restrict__ gscratch)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ uint32_t whist[kSortWarps][256];
    __shared__ uint32_t digit_base[256];
    __shared__ uint32_t warp_tot[8];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    constexpr size_t kElemBytes = kPacked ? 8 : 12;
    constexpr uint32_t kKeyShift = kPacked ? 16 : 0;  // where the distance's digits start in a key word
    unsigned char *buf = gscratch ? gscratch + (size_t)blockIdx.x * (size_t)m * kElemBytes : sm_raw;
    uint32_t *keysA = reinterpret_cast<uint32_t *>(buf);
    uint32_t *keysB = keysA + m;
    uint16_t *valsA = reinterpret_cast<uint16_t *>(keysB + m);  // unused when kPacked
    uint16_t *valsB = valsA + m;
    const int seg = (((m + kSortWarps - 1) / kSortWarps) + 31) & ~31;
    const int s_begin = warp * seg;
    const int s_end = min(m, s_begin + seg);
    const unsigned lt_mask = (1u << lane) - 1u;

    for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
        const int32_t *drow = d + row * (int64_t)m;
        // the row into shared memory, eight independent loads in flight per thread before any is used
        for (int i0 = threadIdx.x; i0 < m; i0 += 8 * blockDim.x) {
            uint32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * (int)blockDim.x;
                v[u] = i < m ? (uint32_t)__ldg(drow + i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * (int)blockDim.x;
                if (i < m) {
                    if constexpr (kPacked) {
                        keysA[i] = (v[u] << 16) | (uint32_t)i;
                    } else {
                        keysA[i] = v[u];
                        valsA[i] = (uint16_t)i;
                    }
                }
            }
        }
        __syncthreads();
        uint32_t *kin = keysA, *kout = keysB;
        uint16_t *vin = valsA, *vout = valsB;
        for (int pass = 0; pass < passes; ++pass) {
            const int shift = kKeyShift + 8 * pass;
            for (int i = threadIdx.x; i < kSortWarps * 256; i += blockDim.x)
                (&whist[0][0])[i] = 0;
            __syncthreads();
            // count
            for (int base = s_begin; base < s_end; base += 32) {
                const int i = base + lane;
                const bool valid = i < s_end;
                if (valid)
                    atomicAdd(&whist[warp][(kin[i] >> shift) & 255u], 1u);
            }
            __syncthreads();
            // offsets: per digit over warps, then exclusive scan over digits
            if (threadIdx.x < 256) {
                const int dg = threadIdx.x;
                uint32_t run = 0;
                for (int w = 0; w < kSortWarps; ++w) {
                    const uint32_t c = whist[w][dg];
                    whist[w][dg] = run;
                    run += c;
                }
                // inclusive scan of run over the 256 digits: warp scan then warp totals
                uint32_t x = run;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(PM_FULL_MASK, x, o);
                    if (lane >= o)
                        x += y;
                }
                if (lane == 31)
                    warp_tot[warp] = x;
                digit_base[dg] = x - run;  // exclusive within the warp
            }
            __syncthreads();
            if (threadIdx.x < 256) {
                const int dg = threadIdx.x;
                uint32_t add = 0;
                for (int w = 0; w < (dg >> 5); ++w)
                    add += warp_tot[w];
                const uint32_t b = digit_base[dg] + add;
                for (int w = 0; w < kSortWarps; ++w)
                    whist[w][dg] += b;
            }
            __syncthreads();
            // scatter
            for (int base = s_begin; base < s_end; base += 32) {
                const int i = base + lane;
                const bool valid = i < s_end;
                uint32_t key = 0;
                uint16_t val = 0;
                if (valid) {
                    key = kin[i];
                    if constexpr (!kPacked)
                        val = vin[i];
                }
                const uint32_t dig = valid ? ((key >> shift) & 255u) : 256u;
                const unsigned peers = equal_digit_lanes(dig);
                if (valid) {
                    const uint32_t pos = whist[warp][dig] + __popc(peers & lt_mask);
                    kout[pos] = key;
                    if constexpr (!kPacked)
                        vout[pos] = val;
                }
                __syncwarp();
                if (valid && lane == __ffs(peers) - 1)
                    whist[warp][dig] += __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            uint32_t *tk = kin;
            kin = kout;
            kout = tk;
            uint16_t *tv = vin;
            vin = vout;
            vout = tv;
        }
        // epilogue: Pi' and Delta' (rank 0: the distance itself), or D' (the sorted distances, which are the
        // running sums of Delta') for cumulative tables
        uint16_t *prow = pi + row * stride;
        int32_t *qrow = delta + row * stride;
        for (int r = threadIdx.x; r < stride; r += blockDim.x) {
            if (r < L) {
                const uint32_t dist = kin[r] >> kKeyShift;
                const uint32_t prev = r > 0 ? kin[r - 1] >> kKeyShift : 0u;
                prow[r] = kPacked ? (uint16_t)(kin[r] & 0xffffu) : vin[r];
                qrow[r] = cum ? (int32_t)dist : (int32_t)(dist - prev);
            } else {
                prow[r] = 0;
                qrow[r] = 0;
            }
        }
        __syncthreads();
    }
}

// Delta' = consecutive differences of D' (rank 0: the value itself), n x L dense rows.
__global__ void k_increments(const int32_t *__restrict__ dcum, int64_t n, int32_t L, int64_t stride,
                             int32_t *__restrict__ out)
{
    const int64_t total = n * (int64_t)L;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / L;
        const int32_t r = (int32_t)(k - i * L);
        const int32_t v = dcum[i * stride + r];
        out[k] = r ? v - dcum[i * stride + r - 1] : v;
    }
}

}  // namespace

pm_status pm_launch_increments(const pm_instance *inst, int32_t *out, cudaStream_t stream)
{
    const int64_t total = inst->n * inst->L;
    const int64_t blocks = std::min<int64_t>(pm_ceil_div(total, 256), (int64_t)inst->sm_count * 16);
    k_increments<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, stream>>>(inst->delta, inst->n, (int32_t)inst->L,
                                                                             inst->stride, out);
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

static int bits_needed(uint32_t v)
{
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

pm_status pm_build_tables(pm_instance *inst, const int32_t *d_dev, cudaStream_t stream)
{
    const int64_t count = inst->n * inst->m;
    int *mm = nullptr;
    PM_TRY(inst->flag.reserve(64));
    mm = reinterpret_cast<int *>(inst->flag.ptr);
    k_minmax_init<<<1, 1, 0, stream>>>(mm);
    const int64_t blocks = std::min<int64_t>(pm_ceil_div(count, 256), (int64_t)inst->sm_count * 8);
    k_minmax<<<(unsigned)blocks, 256, 0, stream>>>(d_dev, count, mm);
    PM_CUDA(cudaGetLastError());
    int host_mm[2];
    PM_CUDA(cudaMemcpyAsync(host_mm, mm, sizeof(host_mm), cudaMemcpyDeviceToHost, stream));
    PM_CUDA(cudaStreamSynchronize(stream));
    if (host_mm[0] < 0)
        return PM_ERR_NEGATIVE_DIST;
    inst->max_d = host_mm[1];
    const int passes = (bits_needed((uint32_t)host_mm[1]) + 7) / 8;
    const bool packed = host_mm[1] < 65536;  // distance and facility id in one 32-bit word

    const size_t row_bytes = (size_t)inst->m * (packed ? 8 : 12);
    const size_t static_bytes = sizeof(uint32_t) * (kSortWarps * 256 + 256 + 8) + 1024;
    const bool in_smem = row_bytes + static_bytes <= inst->smem_optin;
    unsigned char *gscratch = nullptr;
    int64_t grid;
    size_t dyn = 0;
    if (in_smem) {
        dyn = row_bytes;
        PM_CUDA(cudaFuncSetAttribute(packed ? k_tables<true> : k_tables<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        const int64_t per_sm = std::max<int64_t>(1, std::min<int64_t>(4, (int64_t)(inst->smem_optin / (dyn + static_bytes))));
        grid = std::min<int64_t>(inst->n, (int64_t)inst->sm_count * per_sm);
    } else {
        grid = std::min<int64_t>(inst->n, (int64_t)inst->sm_count);
        PM_CUDA(pm_device_malloc_async(reinterpret_cast<void **>(&gscratch), (size_t)grid * row_bytes, stream));
    }
    if (packed)
        k_tables<true><<<(unsigned)grid, kSortThreads, dyn, stream>>>(d_dev, inst->n, (int32_t)inst->m,
                                                                     (int32_t)inst->L, inst->stride, passes,
                                                                     inst->cum ? 1 : 0, inst->pi, inst->delta,
                                                                     gscratch);
    else
        k_tables<false><<<(unsigned)grid, kSortThreads, dyn, stream>>>(d_dev, inst->n, (int32_t)inst->m,
                                                                      (int32_t)inst->L, inst->stride, passes,
                                                                      inst->cum ? 1 : 0, inst->pi, inst->delta,
                                                                      gscratch);
    cudaError_t le = cudaGetLastError();
    if (gscratch)
        cudaFreeAsync(gscratch, stream);
    PM_CUDA(le);
    return PM_OK;
}
