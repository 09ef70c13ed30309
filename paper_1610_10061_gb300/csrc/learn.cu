// The learned swap proposal (no counterpart in the paper): swap statistics
// from an extended scan, move features, a small perceptron on the tensor
// cores (BF16 weights and activations, FP32 accumulation) with hand-written
// forward, backward and Adam kernels, and the GA's learned mutation try.
//
// Swap statistics of an individual (per facility, m entries each): for
// client i with first open rank r1 (distance D1) and second open rank r2
// (distance D2; the last column's distance if none within the table):
//   gain[k]  += D1 - d(i, k)   for every facility k ranked before r1 by i
//   cap[k]   += 1              for the same facilities
//   loss[f1] += D2 - D1        (f1 = the facility at r1)
//   assign[f1] += 1
// gain[k] is exactly what opening k alone saves and loss[j] what closing j
// alone costs; the perceptron predicts the exact cost change of the swap
// (close j, open k) from these first-order quantities.  The statistics walk
// the rows of Pi' against the sorted distances D' (an instance with Delta'
// tables builds a D' copy once), so d(i, k) at a rank is a single load.
//
// Features of a move (8, zero-padded to 16 for one tensor-core k-step), Z =
// max(cost / p, 1):  loss_j/Z, gain_k/Z, assign_j/(n/p), cap_k/(n/p),
// (loss_j - gain_k)/Z, log1p(loss_j/Z), log1p(gain_k/Z), p/m.
//
// Perceptron: x(16) -> 128 (ReLU) -> 128 (ReLU) -> 1, y = prediction of the
// cost change / Z.  Parameters, flat FP32 masters: W1 [16][128], b1 [128],
// W2 [128][128], b2 [128], w3 [128], b3 [1] (row = input unit); BF16
// copies of W1, W2, w3 feed the tensor cores.  Hidden activations are
// rounded to BF16 after the ReLU; gradients of the hidden layers are rounded
// to BF16 before they enter a tensor-core product.  Inference runs on
// tcgen05 (k_mlp_fwd_tc), and so does training (k_mlp_train_tc: forward and
// the whole backward pass per 128-row tile, weight gradients accumulated in
// tensor memory and added into an FP32 gradient buffer); the mma.sync
// kernel k_mlp (64 rows per CTA) remains for comparison.  One Adam kernel
// updates the masters and refreshes the BF16 copies.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "pm_alloc.h"
#include "pm_common.cuh"

namespace {

constexpr int kIn = 16;       // padded input width
constexpr int kFeat = 8;      // real features
constexpr int kHid = 128;     // hidden width
constexpr int kRows = 64;     // rows per CTA
constexpr int kLdH = kHid + 8;   // padded row stride (bf16) of 128-wide tiles: conflict-free fragments
constexpr int kLdX = kIn + 8;    // padded row stride of 16-wide tiles
constexpr int kLdR = kRows + 8;  // padded stride of transposed (feature-major) 64-row tiles
constexpr int kParams = kIn * kHid + kHid + kHid * kHid + kHid + kHid + 1;
constexpr int kOffW1 = 0, kOffB1 = kIn * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t smem_u32_learn(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// A fragment (16 x 16, row-major source A[r][k], stride lda) at (r0, k0).
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16 *A, int lda, int r0, int k0, int lane)
{
    const int g = lane >> 2, c = lane & 3;
    a[0] = ld32(A + (r0 + g) * lda + k0 + 2 * c);
    a[1] = ld32(A + (r0 + g + 8) * lda + k0 + 2 * c);
    a[2] = ld32(A + (r0 + g) * lda + k0 + 8 + 2 * c);
    a[3] = ld32(A + (r0 + g + 8) * lda + k0 + 8 + 2 * c);
}

// B fragment (16 x 8) from a source stored n-major with k contiguous: B[n][k], stride ldb.
__device__ __forceinline__ void frag_b(uint32_t (&b)[2], const __nv_bfloat16 *B, int ldb, int n0, int k0, int lane)
{
    const int g = lane >> 2, c = lane & 3;
    b[0] = ld32(B + (n0 + g) * ldb + k0 + 2 * c);
    b[1] = ld32(B + (n0 + g) * ldb + k0 + 8 + 2 * c);
}

struct MlpSmem {
    __nv_bfloat16 X[kRows * kLdX];     // inputs [r][f]
    __nv_bfloat16 W1T[kHid * kLdX];    // W1 as [out][in]
    __nv_bfloat16 W2T[kHid * kLdH];    // W2 as [out][in] (forward B operand)
    __nv_bfloat16 H1[kRows * kLdH];    // [r][unit]
    float b1[kHid], b2[kHid], w3[kHid];
    float y[kRows];
    long long src[kRows];              // source row of each of the CTA's rows (its position through the shuffle)
};

struct MlpTrainSmem {
    __nv_bfloat16 W2[kHid * kLdH];      // W2 as [in][out] (backward B operand of dH1 = dH2 W2^T)
    __nv_bfloat16 H2[kRows * kLdH];     // [r][unit]
    __nv_bfloat16 XT[kIn * kLdR];       // [f][r]
    __nv_bfloat16 H1T[kHid * kLdR];     // [unit][r]
    __nv_bfloat16 dH2[kRows * kLdH];    // [r][unit]
    __nv_bfloat16 dH2T[kHid * kLdR];    // [unit][r]
    __nv_bfloat16 dH1T[kHid * kLdR];    // [unit][r]
    float dy[kRows];
};


// ---------------------------------------------------------------------------
// Inference forward on the 5th-generation tensor cores (tcgen05).  A
// persistent grid (three CTAs per SM, each holding 128 TMEM columns) walks
// 128-row tiles; each CTA stages W1 and W2 once.  Per tile both layers are
// tcgen05.mma.cta_group::1.kind::f16 (BF16 x BF16 -> FP32, M = N = 128)
// issued by one thread, operands in shared memory in the K-major no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix; k-chunks 128 B
// apart, 8-row groups K*16 B apart), accumulators in tensor memory (128
// columns, layer 1's, then layer 2's once layer 1's are read).  Eight warps read them back with
// tcgen05.ld (thread = row; warps w and w + 4 share TMEM lanes 32(w mod 4)
// and split the 128 columns): bias, then ReLU and BF16 rounding in one
// conversion per pair, written as 16-byte rows of the next layer's A tile;
// then the same for layer 2 and the dot product with w3.  Completion is signalled by
// tcgen05.commit on an mbarrier whose wait is bounded.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;
constexpr int kTcThreads = 256;
constexpr uint32_t kTmemCols = 128;  // both layers' accumulators, one after the other
constexpr uint32_t kTcSpinLimit = 1u << 22;
// instruction descriptor: D F32 (bits 4-5 = 1), A BF16 (7-9 = 1), B BF16 (10-12 = 1), both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint64_t umma_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = smem_u32_learn(p);
    uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for this architecture; base offset 0; no swizzle
    return d;
}

// element (row, k) of a K-major no-swizzle tile with K columns (in elements)
__device__ __forceinline__ int core_idx(int row, int k, int K)
{
    return ((row >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2) >> 1;
}

struct TcSmem {
    __nv_bfloat16 A1[kTcRows * kIn];  // X tile
    __nv_bfloat16 B1[kHid * kIn];     // W1 as (n = out, k = in)
    __nv_bfloat16 A2[kTcRows * kHid]; // H1 tile
    __nv_bfloat16 B2[kHid * kHid];    // W2 as (n = out, k = in)
    float b1[kHid], b2[kHid], w3[kHid];
    float part[kTcRows];              // second-half partial dot products
    uint64_t bar;
    uint32_t tmem;
};

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32_learn(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t spins = 0;
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32_learn(bar)), "r"(phase)
            : "memory");
        if (ok)
            return true;
        if (++spins > kTcSpinLimit)
            return false;
    }
}

// Two floats to a packed BF16 pair of their ReLUs (round to nearest even), lo in the low half.
__device__ __forceinline__ uint32_t pack_relu_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void tc_sync_for_mma()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // smem writes visible to the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads) k_mlp_fwd_tc(const __nv_bfloat16 *__restrict__ X, int64_t rows,
                                                           const __nv_bfloat16 *__restrict__ W1b,
                                                           const __nv_bfloat16 *__restrict__ W2b,
                                                           const __nv_bfloat16 *__restrict__ w3b,
                                                           const float *__restrict__ P, float *__restrict__ y_out,
                                                           int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(tc_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int quad = warp & 3, half = warp >> 2;  // TMEM lanes 32*quad..; columns [64*half, 64*half + 64)
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;

    // weights and biases, once per CTA
    for (int i = tid; i < kIn * kHid; i += blockDim.x) {  // W1 [in][out]
        const int in = i / kHid, out = i % kHid;
        S.B1[core_idx(out, in, kIn)] = W1b[i];
    }
    for (int i = tid; i < kHid * kHid; i += blockDim.x) {  // W2 [in][out]
        const int in = i / kHid, out = i % kHid;
        S.B2[core_idx(out, in, kHid)] = W2b[i];
    }
    for (int i = tid; i < kHid; i += blockDim.x) {
        S.b1[i] = P[kOffB1 + i];
        S.b2[i] = P[kOffB2 + i];
        S.w3[i] = __bfloat162float(w3b[i]);
    }
    const float b3 = P[kOffB3];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32_learn(&S.bar)), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32_learn(&S.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_sync_for_mma();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;  // this warp's TMEM lanes
    const int r = quad * 32 + lane;                         // this thread's row of the tile
    const int c0 = half * 64;                               // this thread's first column

    uint32_t phase = 0;  // parity of the next commit's completion
    bool ok = true;
    // thread tid moves 16 bytes of the X tile: row tid/2, features 8*(tid&1) .. +7; the next tile's chunk is
    // loaded into registers while the current tile is computed
    const int xr = tid >> 1, xh = tid & 1;
    auto load_x = [&](int64_t tile) {
        const int64_t row = tile * kTcRows + xr;
        return (tile < tiles && row < rows) ? __ldg(reinterpret_cast<const uint4 *>(X + row * kIn) + xh)
                                            : make_uint4(0u, 0u, 0u, 0u);
    };
    uint4 x_next = load_x(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int64_t row0 = tile * kTcRows;
        // X tile: 128 rows x two 16-byte halves (features 0-7, 8-15) into the core-matrix layout
        *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(S.A1) + (xr >> 3) * 256 + xh * 128 +
                                   (xr & 7) * 16) = x_next;
        tc_sync_for_mma();
        // layer 1: D[0,128) = X W1
        if (tid == 0) {
            tc_mma(tmem, umma_desc(S.A1, 128, (kIn / 8) * 128), umma_desc(S.B1, 128, (kIn / 8) * 128), kIdesc, 0u);
            tc_commit(&S.bar);
        }
        x_next = load_x(tile + gridDim.x);
        ok = tc_wait(&S.bar, phase);
        ok = __syncthreads_and(ok);
        if (!ok)
            break;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // H1 = bf16(relu(acc + b1)): 8 consecutive columns of a row are one 16-byte chunk of A2
        for (int cc = 0; cc < 64; cc += 32) {
            uint32_t v[32];
            tc_ld32(tmem + lane_off + (uint32_t)(c0 + cc), v);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int col = c0 + cc + 8 * g;
                const float4 ba = *reinterpret_cast<const float4 *>(&S.b1[col]);
                const float4 bb = *reinterpret_cast<const float4 *>(&S.b1[col + 4]);
                uint4 o;
                o.x = pack_relu_bf16x2(__uint_as_float(v[8 * g + 0]) + ba.x, __uint_as_float(v[8 * g + 1]) + ba.y);
                o.y = pack_relu_bf16x2(__uint_as_float(v[8 * g + 2]) + ba.z, __uint_as_float(v[8 * g + 3]) + ba.w);
                o.z = pack_relu_bf16x2(__uint_as_float(v[8 * g + 4]) + bb.x, __uint_as_float(v[8 * g + 5]) + bb.y);
                o.w = pack_relu_bf16x2(__uint_as_float(v[8 * g + 6]) + bb.z, __uint_as_float(v[8 * g + 7]) + bb.w);
                *reinterpret_cast<uint4 *>(S.A2 + core_idx(r, col, kHid)) = o;
            }
        }
        tc_sync_for_mma();
        // layer 2: D[0,128) = H1 W2 (layer 1's accumulators were read above), eight k-steps of 16
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < kHid / 16; ++s)
                tc_mma(tmem, umma_desc(S.A2 + s * 128, 128, (kHid / 8) * 128),
                       umma_desc(S.B2 + s * 128, 128, (kHid / 8) * 128), kIdesc, s > 0 ? 1u : 0u);
            tc_commit(&S.bar);
        }
        ok = tc_wait(&S.bar, phase);
        ok = __syncthreads_and(ok);
        if (!ok)
            break;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // y = w3 . bf16(relu(acc + b2)) + b3, the two column halves added through shared memory
        float ysum = 0.f;
        for (int cc = 0; cc < 64; cc += 32) {
            uint32_t v[32];
            tc_ld32(tmem + lane_off + (uint32_t)(c0 + cc), v);
#pragma unroll
            for (int q = 0; q < 32; q += 2) {
                const int col = c0 + cc + q;
                const float2 bv = *reinterpret_cast<const float2 *>(&S.b2[col]);
                const float2 wv = *reinterpret_cast<const float2 *>(&S.w3[col]);
                const uint32_t hb = pack_relu_bf16x2(__uint_as_float(v[q]) + bv.x, __uint_as_float(v[q + 1]) + bv.y);
                ysum = fmaf(__uint_as_float(hb << 16), wv.x, ysum);
                ysum = fmaf(__uint_as_float(hb & 0xffff0000u), wv.y, ysum);
            }
        }
        if (half == 1)
            S.part[r] = ysum;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // also: every warp is done with this tile's TMEM and A tiles
        if (half == 0 && row0 + r < rows)
            y_out[row0 + r] = ysum + S.part[r] + b3;
    }
    if (!ok) {
        if (tid == 0)
            atomicExch(err, (int)PM_ERR_TIMEOUT);
        (void)tc_wait(&S.bar, phase);  // let an MMA in flight finish (bounded) before its memory is released
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Epoch shuffle of the training rows: position i of an epoch holds row
// pi(i), pi a keyed permutation of [0, total): a four-round Feistel network on
// the `2 half` low bits (the smallest even bit count covering total), whose
// round function is MurmurHash3's 32-bit finaliser of (right half ^ round
// key), applied again while the result is >= total (cycle walking: the cycle
// through i returns below total, at the latest at i itself).  half == 0: the
// identity (position i holds row i).
struct RowMap {
    uint32_t key[4];
    int32_t half;
    int64_t total;
    int64_t pos0;  // position of the launch's first row
};

__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ int64_t shuffled_row(const RowMap &mp, int64_t i)
{
    if (mp.half == 0)
        return i;
    const uint32_t mask = (1u << mp.half) - 1u;
    uint32_t x = (uint32_t)i;
    do {
        uint32_t L = x >> mp.half, R = x & mask;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t nl = R;
            R = L ^ (fmix32(R ^ mp.key[r]) & mask);
            L = nl;
        }
        x = (L << mp.half) | R;
    } while ((int64_t)x >= mp.total);
    return (int64_t)x;
}

// Forward (and in TRAIN mode, backward) for rows [row0, row0 + 64).  4 warps.
//   X: rows x 16 bf16; Wb: bf16 copies (W1 [16][128], W2 [128][128], w3 [128]);
//   P: fp32 masters (biases read from here); y: rows fp32 predictions.
//   TRAIN: t targets, inv_batch = 1/B; grads fp32 (atomic adds), loss (atomic add of sum of squares).
template <bool TRAIN>
__global__ void __launch_bounds__(128) k_mlp(const __nv_bfloat16 *__restrict__ X, int64_t rows,
                                             const __nv_bfloat16 *__restrict__ W1b,
                                             const __nv_bfloat16 *__restrict__ W2b,
                                             const __nv_bfloat16 *__restrict__ w3b, const float *__restrict__ P,
                                             float *__restrict__ y_out, const float *__restrict__ t, float inv_batch,
                                             float *__restrict__ grads, float *__restrict__ loss, RowMap map)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
    MlpTrainSmem &T = *reinterpret_cast<MlpTrainSmem *>(smem_raw + ((sizeof(MlpSmem) + 15) & ~size_t(15)));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, c = lane & 3;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;

    // ---- stage weights and inputs ----
    for (int i = tid; i < kIn * kHid; i += blockDim.x) {  // W1 [in][out] -> W1T [out][in]
        const int in = i / kHid, out = i % kHid;
        S.W1T[out * kLdX + in] = W1b[i];
    }
    for (int i = tid; i < kHid * kHid; i += blockDim.x) {  // W2 [in][out]
        const int in = i / kHid, out = i % kHid;
        S.W2T[out * kLdH + in] = W2b[i];
        if (TRAIN)
            T.W2[in * kLdH + out] = W2b[i];
    }
    for (int i = tid; i < kHid; i += blockDim.x) {
        S.b1[i] = P[kOffB1 + i];
        S.b2[i] = P[kOffB2 + i];
        S.w3[i] = __bfloat162float(w3b[i]);
    }
    for (int r = tid; r < kRows; r += blockDim.x)
        S.src[r] = (row0 + r < rows) ? (long long)shuffled_row(map, map.pos0 + row0 + r) : -1ll;
    __syncthreads();
    for (int i = tid; i < kRows * kIn; i += blockDim.x) {
        const int r = i / kIn, f = i % kIn;
        const __nv_bfloat16 v = (row0 + r < rows) ? X[S.src[r] * kIn + f] : __float2bfloat16(0.0f);
        S.X[r * kLdX + f] = v;
        if (TRAIN)
            T.XT[f * kLdR + r] = v;
    }
    __syncthreads();

    const int r0 = warp * 16;  // this warp's 16 rows
    // ---- layer 1: H1 = relu(X W1 + b1) ----
    {
        uint32_t a[4];
        frag_a(a, S.X, kLdX, r0, 0, lane);
#pragma unroll
        for (int nt = 0; nt < kHid / 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t b[2];
            frag_b(b, S.W1T, kLdX, nt * 8, 0, lane);
            mma_bf16(d, a, b);
            const int col = nt * 8 + 2 * c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + g + 8 * h;
                const float v0 = fmaxf(d[2 * h] + S.b1[col], 0.f), v1 = fmaxf(d[2 * h + 1] + S.b1[col + 1], 0.f);
                const __nv_bfloat16 q0 = __float2bfloat16(v0), q1 = __float2bfloat16(v1);
                S.H1[r * kLdH + col] = q0;
                S.H1[r * kLdH + col + 1] = q1;
                if (TRAIN) {
                    T.H1T[col * kLdR + r] = q0;
                    T.H1T[(col + 1) * kLdR + r] = q1;
                }
            }
        }
    }
    __syncwarp();
    // ---- layer 2 + 3: H2 = relu(H1 W2 + b2), y = H2 w3 + b3 ----
    {
        float acc[kHid / 8][4];
#pragma unroll
        for (int nt = 0; nt < kHid / 8; ++nt)
            acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < kHid / 16; ++ks) {
            uint32_t a[4];
            frag_a(a, S.H1, kLdH, r0, ks * 16, lane);
#pragma unroll
            for (int nt = 0; nt < kHid / 8; ++nt) {
                uint32_t b[2];
                frag_b(b, S.W2T, kLdH, nt * 8, ks * 16, lane);
                mma_bf16(acc[nt], a, b);
            }
        }
        float ysum[2] = {0.f, 0.f};
#pragma unroll
        for (int nt = 0; nt < kHid / 8; ++nt) {
            const int col = nt * 8 + 2 * c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + g + 8 * h;
                const __nv_bfloat16 q0 = __float2bfloat16(fmaxf(acc[nt][2 * h] + S.b2[col], 0.f));
                const __nv_bfloat16 q1 = __float2bfloat16(fmaxf(acc[nt][2 * h + 1] + S.b2[col + 1], 0.f));
                ysum[h] += __bfloat162float(q0) * S.w3[col] + __bfloat162float(q1) * S.w3[col + 1];
                if (TRAIN) {
                    T.H2[r * kLdH + col] = q0;
                    T.H2[r * kLdH + col + 1] = q1;
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            ysum[h] += __shfl_xor_sync(PM_FULL_MASK, ysum[h], 1);
            ysum[h] += __shfl_xor_sync(PM_FULL_MASK, ysum[h], 2);
        }
        if (c == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + g + 8 * h;
                const float yv = ysum[h] + P[kOffB3];
                S.y[r] = yv;
                if (row0 + r < rows)
                    y_out[row0 + r] = yv;
            }
        }
    }
    if (!TRAIN)
        return;

    // ================= backward (mean squared error) =================
    __syncthreads();
    if (tid < kRows) {
        const int r = tid;
        float dy = 0.f, sq = 0.f;
        if (row0 + r < rows) {
            const float e = S.y[r] - t[S.src[r]];
            dy = 2.f * e * inv_batch;
            sq = e * e;
        }
        T.dy[r] = dy;
        // loss: sum of squares (the host divides by B)
        sq += __shfl_xor_sync(PM_FULL_MASK, sq, 16);
        sq += __shfl_xor_sync(PM_FULL_MASK, sq, 8);
        sq += __shfl_xor_sync(PM_FULL_MASK, sq, 4);
        sq += __shfl_xor_sync(PM_FULL_MASK, sq, 2);
        sq += __shfl_xor_sync(PM_FULL_MASK, sq, 1);
        if ((tid & 31) == 0)
            atomicAdd(loss, sq);
        float db3 = dy;
        db3 += __shfl_xor_sync(PM_FULL_MASK, db3, 16);
        db3 += __shfl_xor_sync(PM_FULL_MASK, db3, 8);
        db3 += __shfl_xor_sync(PM_FULL_MASK, db3, 4);
        db3 += __shfl_xor_sync(PM_FULL_MASK, db3, 2);
        db3 += __shfl_xor_sync(PM_FULL_MASK, db3, 1);
        if ((tid & 31) == 0)
            atomicAdd(grads + kOffB3, db3);
    }
    __syncthreads();
    // dw3[u] = sum_r h2[r][u] dy[r];  dH2[r][u] = bf16(dy[r] w3[u] [h2 > 0]);  db2[u] = sum_r dH2[r][u]
    for (int u = tid; u < kHid; u += blockDim.x) {
        float dw = 0.f, db = 0.f;
        for (int r = 0; r < kRows; ++r) {
            const float h2 = __bfloat162float(T.H2[r * kLdH + u]);
            const float dyr = T.dy[r];
            dw += h2 * dyr;
            const __nv_bfloat16 q = __float2bfloat16(h2 > 0.f ? dyr * S.w3[u] : 0.f);
            T.dH2[r * kLdH + u] = q;
            T.dH2T[u * kLdR + r] = q;
            db += __bfloat162float(q);
        }
        atomicAdd(grads + kOffW3 + u, dw);
        atomicAdd(grads + kOffB2 + u, db);
    }
    __syncthreads();
    // dH1 = bf16((dH2 W2^T) [h1 > 0]); warp w: rows r0..r0+15, all 128 units
    {
        float acc[kHid / 8][4];
#pragma unroll
        for (int nt = 0; nt < kHid / 8; ++nt)
            acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < kHid / 16; ++ks) {
            uint32_t a[4];
            frag_a(a, T.dH2, kLdH, r0, ks * 16, lane);
#pragma unroll
            for (int nt = 0; nt < kHid / 8; ++nt) {
                uint32_t b[2];
                frag_b(b, T.W2, kLdH, nt * 8, ks * 16, lane);  // B[k = out][n = in] = W2[in][out]
                mma_bf16(acc[nt], a, b);
            }
        }
#pragma unroll
        for (int nt = 0; nt < kHid / 8; ++nt) {
            const int col = nt * 8 + 2 * c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + g + 8 * h;
                const bool on0 = __bfloat162float(S.H1[r * kLdH + col]) > 0.f;
                const bool on1 = __bfloat162float(S.H1[r * kLdH + col + 1]) > 0.f;
                T.dH1T[col * kLdR + r] = __float2bfloat16(on0 ? acc[nt][2 * h] : 0.f);
                T.dH1T[(col + 1) * kLdR + r] = __float2bfloat16(on1 ? acc[nt][2 * h + 1] : 0.f);
            }
        }
    }
    __syncthreads();
    // db1[u] = sum_r dH1[r][u]
    for (int u = tid; u < kHid; u += blockDim.x) {
        float db = 0.f;
        for (int r = 0; r < kRows; ++r)
            db += __bfloat162float(T.dH1T[u * kLdR + r]);
        atomicAdd(grads + kOffB1 + u, db);
    }
    // dW2 = H1^T dH2 (128 x 128, k = the 64 rows); warp w: output rows 32w .. 32w+31, in two halves of 64 cols
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        float acc[2][8][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
                acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < kRows / 16; ++ks) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                uint32_t a[4];
                frag_a(a, T.H1T, kLdR, warp * 32 + mt * 16, ks * 16, lane);
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    uint32_t b[2];
                    frag_b(b, T.dH2T, kLdR, half * 64 + nt * 8, ks * 16, lane);
                    mma_bf16(acc[mt][nt], a, b);
                }
            }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int col = half * 64 + nt * 8 + 2 * c;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int in = warp * 32 + mt * 16 + g + 8 * h;
                    atomicAdd(grads + kOffW2 + in * kHid + col, acc[mt][nt][2 * h]);
                    atomicAdd(grads + kOffW2 + in * kHid + col + 1, acc[mt][nt][2 * h + 1]);
                }
            }
    }
    // dW1 = X^T dH1 (16 x 128, k = the 64 rows); warp w: units 32w .. 32w+31
    {
        float acc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
            acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < kRows / 16; ++ks) {
            uint32_t a[4];
            frag_a(a, T.XT, kLdR, 0, ks * 16, lane);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                uint32_t b[2];
                frag_b(b, T.dH1T, kLdR, warp * 32 + nt * 8, ks * 16, lane);
                mma_bf16(acc[nt], a, b);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int col = warp * 32 + nt * 8 + 2 * c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int in = g + 8 * h;
                atomicAdd(grads + kOffW1 + in * kHid + col, acc[nt][2 * h]);
                atomicAdd(grads + kOffW1 + in * kHid + col + 1, acc[nt][2 * h + 1]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Training (forward and backward) on the tcgen05 tensor cores.  A CTA takes
// `tpc` consecutive 128-row tiles of the batch (rows read through the epoch's
// permutation); per tile, with one thread issuing every MMA (BF16 operands
// in shared memory in the K-major no-swizzle core-matrix layout, FP32
// accumulators in tensor memory):
//   layer 1   C0 = X W1                       (M 128, N 128, K 16)
//   layer 2   C0 = H1 W2                      (K 128)
//   dH1       C0 = dH2 W2^T                   (A = dH2 rows, B = W2 rows)
//   dW2      C2 += H1^T dH2                   (A = H1^T, B = dH2^T; K = the tile's rows)
//   dW1^T    C3 += dH1^T X                    (N 16)
// where H1, H2 are the BF16 hidden activations after ReLU, dy = 2 (y - t) / B,
// dH2 = BF16(dy w3 [H2 > 0]) and dH1 = BF16((dH2 W2^T) [H1 > 0]) -- the
// arithmetic of the mma.sync kernel above and of the oracle with BF16
// rounding.  The weight gradients accumulate in tensor memory over the CTA's
// tiles and reach the global gradient with one atomic per parameter per CTA;
// the bias and w3 gradients are column sums in shared memory.  Eight warps
// read the accumulators (warps w and w + 4 share TMEM lanes 32 (w mod 4) and
// take half the columns each); every wait on an MMA is bounded.
// ---------------------------------------------------------------------------
constexpr int kTrThreads = 256;
constexpr uint32_t kTrTmemCols = 512;      // C0 [0,128), C2 [128,256), C3 [256,272)
constexpr int kLdT = 130;                  // row stride (elements) of the plain H2^T copy: odd in words
constexpr uint32_t kIdescN16 = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

struct TrSmem {
    __nv_bfloat16 AX[kTcRows * kIn];    // X tile as (m = row, k = feature)
    __nv_bfloat16 BXT[kIn * kTcRows];   // X^T as (n = feature, k = row)
    __nv_bfloat16 BW1[kHid * kIn];      // W1 as (n = out, k = in)
    __nv_bfloat16 BW2T[kHid * kHid];    // W2 as (n = out, k = in): layer 2
    __nv_bfloat16 BW2[kHid * kHid];     // W2 as (n = in, k = out): dH1 = dH2 W2^T
    __nv_bfloat16 R[kTcRows * kHid];    // H1 as (m = row, k = unit), then dH2
    __nv_bfloat16 T1[kHid * kTcRows];   // H1^T as (m = unit, k = row), then dH1^T
    __nv_bfloat16 T2[kHid * kTcRows];   // dH2^T as (n = unit, k = row)
    __nv_bfloat16 H2T[kHid * kLdT];     // H2 as [unit][row] (plain), for the w3 gradient
    float b1[kHid], b2[kHid], w3[kHid];
    float part[kTcRows], tgt[kTcRows], dy[kTcRows];
    float gb1[kHid], gb2[kHid], gw3[kHid];  // this CTA's bias and w3 gradients
    uint32_t mask1[kTcRows * 4];        // H1 > 0: row r, bit (unit & 31) of word 4 r + unit / 32
    float gb3, sq;
    uint64_t bar;
    uint32_t tmem;
};

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float bf16_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t p) { return __uint_as_float(p & 0xffff0000u); }
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__global__ void __launch_bounds__(kTrThreads, 1) k_mlp_train_tc(const __nv_bfloat16 *__restrict__ X, int64_t rows,
                                                                const __nv_bfloat16 *__restrict__ W1b,
                                                                const __nv_bfloat16 *__restrict__ W2b,
                                                                const __nv_bfloat16 *__restrict__ w3b,
                                                                const float *__restrict__ P,
                                                                const float *__restrict__ t, float inv_batch,
                                                                float *__restrict__ grads, float *__restrict__ loss,
                                                                RowMap map, int tpc, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char tr_raw[];
    TrSmem &S = *reinterpret_cast<TrSmem *>(tr_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int quad = warp & 3, half = warp >> 2;
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;

    for (int i = tid; i < kIn * kHid; i += blockDim.x) {  // W1 [in][out]
        const int in = i / kHid, out = i % kHid;
        S.BW1[core_idx(out, in, kIn)] = W1b[i];
    }
    for (int i = tid; i < kHid * kHid; i += blockDim.x) {  // W2 [in][out]
        const int in = i / kHid, out = i % kHid;
        S.BW2T[core_idx(out, in, kHid)] = W2b[i];
        S.BW2[core_idx(in, out, kHid)] = W2b[i];
    }
    for (int i = tid; i < kHid; i += blockDim.x) {
        S.b1[i] = P[kOffB1 + i];
        S.b2[i] = P[kOffB2 + i];
        S.w3[i] = __bfloat162float(w3b[i]);
        S.gb1[i] = 0.f;
        S.gb2[i] = 0.f;
        S.gw3[i] = 0.f;
    }
    const float b3 = P[kOffB3];
    if (tid == 0) {
        S.gb3 = 0.f;
        S.sq = 0.f;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32_learn(&S.bar)), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32_learn(&S.tmem)),
                     "r"(kTrTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_sync_for_mma();
    const uint32_t tmem = S.tmem, C0 = tmem, C2 = tmem + 128u, C3 = tmem + 256u;
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    const int r = quad * 32 + lane;  // this thread's row of the tile (its TMEM lane)
    const int c0 = half * 64;        // its first column
    constexpr uint32_t kSbo = (kHid / 8) * 128;

    uint32_t phase = 0;
    bool ok = true, any = false;
    auto wait_mma = [&]() {
        bool w = tc_wait(&S.bar, phase);
        w = __syncthreads_and(w);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return w;
    };
    const int64_t last = blockIdx.x * (int64_t)tpc + tpc;
    for (int64_t tile = blockIdx.x * (int64_t)tpc; tile < tiles && tile < last && ok; ++tile) {
        const int64_t pos0 = tile * kTcRows;
        // ---- the tile's rows: X (both layouts) and targets ----
        {
            const int xr = tid >> 1, xh = tid & 1;
            const bool valid = pos0 + xr < rows;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            int64_t src = 0;
            if (valid) {
                src = shuffled_row(map, map.pos0 + pos0 + xr);
                v = __ldg(reinterpret_cast<const uint4 *>(X + src * kIn) + xh);
            }
            *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(S.AX) + (xr >> 3) * 256 + xh * 128 +
                                       (xr & 7) * 16) = v;
            const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int f = 8 * xh + 2 * q;
                reinterpret_cast<uint16_t *>(S.BXT)[core_idx(f, xr, kTcRows)] = (uint16_t)(wv[q] & 0xffffu);
                reinterpret_cast<uint16_t *>(S.BXT)[core_idx(f + 1, xr, kTcRows)] = (uint16_t)(wv[q] >> 16);
            }
            if (xh == 0)
                S.tgt[xr] = valid ? t[src] : 0.f;
        }
        const int nvalid = (int)((rows - pos0) < kTcRows ? (rows - pos0) : kTcRows);
        tc_sync_for_mma();
        if (tid == 0) {  // layer 1
            tc_mma(C0, umma_desc(S.AX, 128, (kIn / 8) * 128), umma_desc(S.BW1, 128, (kIn / 8) * 128), kIdesc, 0u);
            tc_commit(&S.bar);
        }
        if (!(ok = wait_mma()))
            break;
        // ---- H1 = bf16(relu(C0 + b1)) into R (rows) and T1 (transposed); its sign bits ----
        for (int cc = 0; cc < 64; cc += 32) {
            uint32_t v[32];
            tc_ld32(C0 + lane_off + (uint32_t)(c0 + cc), v);
            uint32_t bits = 0u;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int col = c0 + cc + 8 * g;
                uint32_t pk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    pk[q] = pack_relu_bf16x2(__uint_as_float(v[8 * g + 2 * q]) + S.b1[col + 2 * q],
                                             __uint_as_float(v[8 * g + 2 * q + 1]) + S.b1[col + 2 * q + 1]);
                    const float lo = bf16_lo(pk[q]), hi = bf16_hi(pk[q]);
                    bits |= (lo > 0.f ? 1u : 0u) << (8 * g + 2 * q);
                    bits |= (hi > 0.f ? 1u : 0u) << (8 * g + 2 * q + 1);
                    reinterpret_cast<uint16_t *>(S.T1)[core_idx(col + 2 * q, r, kTcRows)] = (uint16_t)(pk[q] & 0xffffu);
                    reinterpret_cast<uint16_t *>(S.T1)[core_idx(col + 2 * q + 1, r, kTcRows)] = (uint16_t)(pk[q] >> 16);
                }
                *reinterpret_cast<uint4 *>(S.R + core_idx(r, col, kHid)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            S.mask1[4 * r + (c0 + cc) / 32] = bits;
        }
        tc_sync_for_mma();
        if (tid == 0) {  // layer 2
#pragma unroll
            for (int s = 0; s < kHid / 16; ++s)
                tc_mma(C0, umma_desc(S.R + s * 128, 128, kSbo), umma_desc(S.BW2T + s * 128, 128, kSbo), kIdesc,
                       s > 0 ? 1u : 0u);
            tc_commit(&S.bar);
        }
        if (!(ok = wait_mma()))
            break;
        // ---- H2 = bf16(relu(C0 + b2)) (kept packed), y, dy, then dH2 into R and T2 ----
        uint32_t h2[32];  // this thread's 64 columns of H2, packed pairs
        float ysum = 0.f;
        for (int cc = 0; cc < 64; cc += 32) {
            uint32_t v[32];
            tc_ld32(C0 + lane_off + (uint32_t)(c0 + cc), v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int col = c0 + cc + 2 * q;
                const uint32_t hb = pack_relu_bf16x2(__uint_as_float(v[2 * q]) + S.b2[col],
                                                     __uint_as_float(v[2 * q + 1]) + S.b2[col + 1]);
                h2[cc / 2 + q] = hb;
                ysum = fmaf(bf16_lo(hb), S.w3[col], ysum);
                ysum = fmaf(bf16_hi(hb), S.w3[col + 1], ysum);
                S.H2T[col * kLdT + r] = __ushort_as_bfloat16((unsigned short)(hb & 0xffffu));
                S.H2T[(col + 1) * kLdT + r] = __ushort_as_bfloat16((unsigned short)(hb >> 16));
            }
        }
        if (half == 1)
            S.part[r] = ysum;
        __syncthreads();
        if (half == 0) {
            const bool valid = r < nvalid;
            const float e = valid ? (ysum + S.part[r] + b3 - S.tgt[r]) : 0.f;
            const float dyv = valid ? 2.f * e * inv_batch : 0.f;
            S.dy[r] = dyv;
            float sq = e * e, d = dyv;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sq += __shfl_xor_sync(PM_FULL_MASK, sq, o);
                d += __shfl_xor_sync(PM_FULL_MASK, d, o);
            }
            if (lane == 0) {
                atomicAdd(&S.sq, sq);
                atomicAdd(&S.gb3, d);
            }
        }
        __syncthreads();
        {
            const float dyr = S.dy[r];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int col = c0 + 2 * q;
                const float g0 = bf16_lo(h2[q]) > 0.f ? dyr * S.w3[col] : 0.f;
                const float g1 = bf16_hi(h2[q]) > 0.f ? dyr * S.w3[col + 1] : 0.f;
                h2[q] = pack_bf16x2(g0, g1);  // dH2, packed
                reinterpret_cast<uint16_t *>(S.T2)[core_idx(col, r, kTcRows)] = (uint16_t)(h2[q] & 0xffffu);
                reinterpret_cast<uint16_t *>(S.T2)[core_idx(col + 1, r, kTcRows)] = (uint16_t)(h2[q] >> 16);
            }
#pragma unroll
            for (int g = 0; g < 8; ++g)
                *reinterpret_cast<uint4 *>(S.R + core_idx(r, c0 + 8 * g, kHid)) =
                    make_uint4(h2[4 * g], h2[4 * g + 1], h2[4 * g + 2], h2[4 * g + 3]);
        }
        tc_sync_for_mma();
        if (tid == 0) {  // dH1 pre-activation, and dW2 += H1^T dH2
#pragma unroll
            for (int s = 0; s < kHid / 16; ++s)
                tc_mma(C0, umma_desc(S.R + s * 128, 128, kSbo), umma_desc(S.BW2 + s * 128, 128, kSbo), kIdesc,
                       s > 0 ? 1u : 0u);
#pragma unroll
            for (int s = 0; s < kTcRows / 16; ++s)
                tc_mma(C2, umma_desc(S.T1 + s * 128, 128, kSbo), umma_desc(S.T2 + s * 128, 128, kSbo), kIdesc,
                       (any || s > 0) ? 1u : 0u);
            tc_commit(&S.bar);
        }
        // column sums of this tile while the tensor cores run: the w3 and layer-2 bias gradients
        if (tid < kHid) {
            float gw = 0.f, gb = 0.f;
            for (int rr = 0; rr < nvalid; ++rr) {
                gw = fmaf(__bfloat162float(S.H2T[tid * kLdT + rr]), S.dy[rr], gw);
                gb += __bfloat162float(S.T2[core_idx(tid, rr, kTcRows)]);
            }
            S.gw3[tid] += gw;
            S.gb2[tid] += gb;
        }
        if (!(ok = wait_mma()))
            break;
        // ---- dH1 = bf16(C0 [H1 > 0]) into T1 (transposed) ----
        for (int cc = 0; cc < 64; cc += 32) {
            uint32_t v[32];
            tc_ld32(C0 + lane_off + (uint32_t)(c0 + cc), v);
            const uint32_t bits = S.mask1[4 * r + (c0 + cc) / 32];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int col = c0 + cc + 2 * q;
                const float g0 = ((bits >> (2 * q)) & 1u) ? __uint_as_float(v[2 * q]) : 0.f;
                const float g1 = ((bits >> (2 * q + 1)) & 1u) ? __uint_as_float(v[2 * q + 1]) : 0.f;
                const uint32_t pk = pack_bf16x2(g0, g1);
                reinterpret_cast<uint16_t *>(S.T1)[core_idx(col, r, kTcRows)] = (uint16_t)(pk & 0xffffu);
                reinterpret_cast<uint16_t *>(S.T1)[core_idx(col + 1, r, kTcRows)] = (uint16_t)(pk >> 16);
            }
        }
        tc_sync_for_mma();
        if (tid == 0) {  // dW1^T += dH1^T X
#pragma unroll
            for (int s = 0; s < kTcRows / 16; ++s)
                tc_mma(C3, umma_desc(S.T1 + s * 128, 128, kSbo), umma_desc(S.BXT + s * 128, 128, kSbo), kIdescN16,
                       (any || s > 0) ? 1u : 0u);
            tc_commit(&S.bar);
        }
        if (tid < kHid) {  // the layer-1 bias gradient: row sums of dH1^T
            float gb = 0.f;
            for (int rr = 0; rr < nvalid; ++rr)
                gb += __bfloat162float(S.T1[core_idx(tid, rr, kTcRows)]);
            S.gb1[tid] += gb;
        }
        if (!(ok = wait_mma()))
            break;
        any = true;
    }
    if (ok && any) {
        // this CTA's weight gradients from tensor memory: dW2 (lane = in, column = out), dW1^T (lane = out,
        // column = in feature)
        for (int cc = 0; cc < 64; cc += 32) {
            uint32_t v[32];
            tc_ld32(C2 + lane_off + (uint32_t)(c0 + cc), v);
#pragma unroll
            for (int q = 0; q < 32; ++q)
                atomicAdd(grads + kOffW2 + r * kHid + c0 + cc + q, __uint_as_float(v[q]));
        }
        if (half == 0) {
            uint32_t v[16];
            tc_ld16(C3 + lane_off, v);
#pragma unroll
            for (int f = 0; f < 16; ++f)
                atomicAdd(grads + kOffW1 + f * kHid + r, __uint_as_float(v[f]));
        }
        if (tid < kHid) {
            atomicAdd(grads + kOffB1 + tid, S.gb1[tid]);
            atomicAdd(grads + kOffB2 + tid, S.gb2[tid]);
            atomicAdd(grads + kOffW3 + tid, S.gw3[tid]);
        }
        if (tid == 0) {
            atomicAdd(grads + kOffB3, S.gb3);
            atomicAdd(loss, S.sq);
        }
    }
    if (!ok) {
        if (tid == 0)
            atomicExch(err, (int)PM_ERR_TIMEOUT);
        (void)tc_wait(&S.bar, phase);  // let an MMA in flight finish (bounded) before its memory is released
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTrTmemCols) : "memory");
}

// Adam (Kingma & Ba 2015, Algorithm 1) on the FP32 masters; refreshes the BF16 copies.
// The gradient buffer is left zero for the next step.  loss_word (nullable): the step's sum of squares, which
// thread 0 moves (times inv_rows) into *loss_out and clears.
__global__ void k_adam(float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                       float *__restrict__ G, int n, float lr, float bc1, float bc2,
                       __nv_bfloat16 *__restrict__ W1b, __nv_bfloat16 *__restrict__ W2b,
                       __nv_bfloat16 *__restrict__ w3b, float *__restrict__ loss_word, float *__restrict__ loss_out,
                       float inv_rows)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && loss_word != nullptr) {
        *loss_out = *loss_word * inv_rows;
        *loss_word = 0.f;
    }
    if (i >= n)
        return;
    const float g = G[i];
    G[i] = 0.f;
    const float m = 0.9f * M[i] + 0.1f * g;
    const float v = 0.999f * V[i] + 0.001f * g * g;
    M[i] = m;
    V[i] = v;
    const float mhat = m / bc1, vhat = v / bc2;
    const float w = P[i] - lr * mhat / (sqrtf(vhat) + 1e-8f);
    P[i] = w;
    if (i < kOffB1)
        W1b[i - kOffW1] = __float2bfloat16(w);
    else if (i >= kOffW2 && i < kOffB2)
        W2b[i - kOffW2] = __float2bfloat16(w);
    else if (i >= kOffW3 && i < kOffB3)
        w3b[i - kOffW3] = __float2bfloat16(w);
}

__global__ void k_refresh_bf16(const float *__restrict__ P, __nv_bfloat16 *__restrict__ W1b,
                               __nv_bfloat16 *__restrict__ W2b, __nv_bfloat16 *__restrict__ w3b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kIn * kHid)
        W1b[i] = __float2bfloat16(P[kOffW1 + i]);
    if (i < kHid * kHid)
        W2b[i] = __float2bfloat16(P[kOffW2 + i]);
    if (i < kHid)
        w3b[i] = __float2bfloat16(P[kOffW3 + i]);
}

// ---------------------------------------------------------------------------
// D' from Delta': per row the running sums of the increments up to each rank
// (the row's sorted distances, Eq. 4 summed), zero in the padding past L.  One
// warp per row, 32 ranks per step with a carry.
// ---------------------------------------------------------------------------
__global__ void k_running_sums(const int32_t *__restrict__ delta, int64_t n, int32_t L, int64_t stride,
                               int32_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int32_t *row = delta + i * stride;
        int32_t *orow = out + i * stride;
        int32_t carry = 0;
        for (int64_t base = 0; base < stride; base += 32) {
            const int64_t r = base + lane;
            int32_t v = r < L ? __ldg(row + r) : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(PM_FULL_MASK, v, o);
                if (lane >= o)
                    v += y;
            }
            v += carry;
            if (r < stride)
                orow[r] = r < L ? v : 0;
            carry = __shfl_sync(PM_FULL_MASK, v, 31);
        }
    }
}

constexpr int kMaxCand = 8;  // closed candidates per individual in the learned try (pm_ga_params.candidates <= 8)

// (g, k) ahead of (h, j) in the candidates' order: gain descending, facility id ascending; an empty slot is
// (0, INT32_MAX), behind every facility.
__device__ __forceinline__ bool cand_before(unsigned long long g, int32_t k, unsigned long long h, int32_t j)
{
    return g > h || (g == h && k < j);
}

// The learned try's candidate moves straight from one individual's statistics
// in shared memory (the fused form of k_candidates, which reads them back from
// global memory): the open facilities in ascending order, the T closed
// facilities of largest gain (ties: lower id) by T block-wide arg-max passes,
// and the p * T feature rows (row a * T + b: the a-th open facility with the
// b-th candidate; the first open one stands in past the open count), each
// computed as k_candidates computes it.
struct CandOut {
    const int64_t *costs;  // the individuals' exact costs
    int32_t *moves;        // pop x p x T (j, k) pairs
    __nv_bfloat16 *X;      // pop x p x T feature rows of 16 BF16
    int32_t p;
    int32_t T;
    int64_t n;
};

template <typename Acc>
__device__ __forceinline__ void candidates_from_stats(const uint32_t *bits, const Acc *Gs, const Acc *Ls,
                                                      const int *Cs, const int *As, int32_t *open_s, int32_t W,
                                                      int32_t m, int64_t t, const CandOut &co)
{
    constexpr int32_t kNone = 0x7fffffff;
    __shared__ int32_t top_k[kMaxCand];
    __shared__ unsigned long long top_g[kMaxCand];
    __shared__ float top_f1[kMaxCand], top_f3[kMaxCand], top_f6[kMaxCand];
    __shared__ unsigned long long red_g[32];
    __shared__ int32_t red_k[32];
    __shared__ int32_t nopen;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int32_t p = co.p, T = co.T;
    for (int i = tid; i < p; i += blockDim.x)
        open_s[i] = 0;  // a bitset with fewer than p open facilities still yields valid ids
    __syncthreads();
    if (warp == 0) {
        int cnt = 0;
        for (int base = 0; base < W; base += 32) {
            const int w = base + lane;
            const uint32_t word = w < W ? bits[w] : 0u;
            const int pc = __popc(word);
            int incl = pc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(PM_FULL_MASK, incl, o);
                if (lane >= o)
                    incl += y;
            }
            int pos = cnt + incl - pc;
            uint32_t rest = word;
            while (rest) {
                const int b = __ffs(rest) - 1;
                rest &= rest - 1u;
                if (pos < p)
                    open_s[pos] = w * 32 + b;
                ++pos;
            }
            cnt += __shfl_sync(PM_FULL_MASK, incl, 31);
        }
        if (lane == 0)
            nopen = cnt < p ? cnt : p;
    }
    for (int b = 0; b < T; ++b) {
        unsigned long long bg = 0ull;
        int32_t bk = kNone;
        for (int k = tid; k < m; k += blockDim.x) {
            if ((bits[k >> 5] >> (k & 31)) & 1u)
                continue;
            bool taken = false;
            for (int q = 0; q < b; ++q)
                taken = taken || (top_k[q] == k);
            const unsigned long long gk = (unsigned long long)Gs[k];
            if (!taken && cand_before(gk, k, bg, bk)) {
                bg = gk;
                bk = k;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long og = __shfl_xor_sync(PM_FULL_MASK, bg, o);
            const int32_t ok = __shfl_xor_sync(PM_FULL_MASK, bk, o);
            if (cand_before(og, ok, bg, bk)) {
                bg = og;
                bk = ok;
            }
        }
        if (lane == 0) {
            red_g[warp] = bg;
            red_k[warp] = bk;
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long g0 = red_g[0];
            int32_t k0 = red_k[0];
            for (int w = 1; w < nwarps; ++w)
                if (cand_before(red_g[w], red_k[w], g0, k0)) {
                    g0 = red_g[w];
                    k0 = red_k[w];
                }
            if (k0 == kNone)  // fewer than T closed facilities: repeat the previous one
                k0 = b > 0 ? top_k[b - 1] : 0;
            top_k[b] = k0;
        }
        __syncthreads();
    }
    const float Z = fmaxf((float)co.costs[t] / (float)p, 1.f);
    const float per = (float)co.n / (float)p, ratio = (float)p / (float)m;
    if (tid < T) {
        const int32_t k = top_k[tid];
        const unsigned long long gk = (unsigned long long)Gs[k];
        top_g[tid] = gk;
        top_f1[tid] = (float)gk / Z;
        top_f3[tid] = (float)Cs[k] / per;
        top_f6[tid] = log1pf(top_f1[tid]);
    }
    __syncthreads();
    const uint32_t bf_ratio = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(ratio));
    for (int a = tid; a < p; a += blockDim.x) {
        const int32_t j = open_s[a < nopen ? a : 0];
        const unsigned long long lj = (unsigned long long)Ls[j];
        const float f0 = (float)lj / Z;
        const float f2 = (float)As[j] / per;
        const float f5 = log1pf(f0);
        const uint32_t bf0 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(f0));
        const uint32_t bf2 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(f2));
        const uint32_t bf5 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(f5));
        for (int b = 0; b < T; ++b) {
            const int64_t idx = t * (int64_t)p * T + (int64_t)a * T + b;
            const float f4 = (float)((long long)lj - (long long)top_g[b]) / Z;
            uint4 v;
            v.x = bf0 | ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(top_f1[b])) << 16);
            v.y = bf2 | ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(top_f3[b])) << 16);
            v.z = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(f4)) | (bf5 << 16);
            v.w = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(top_f6[b])) | (bf_ratio << 16);
            uint4 *out = reinterpret_cast<uint4 *>(co.X + idx * kIn);
            out[0] = v;
            out[1] = make_uint4(0u, 0u, 0u, 0u);
            reinterpret_cast<int2 *>(co.moves)[idx] = make_int2(j, top_k[b]);
        }
    }
}

// ---------------------------------------------------------------------------
// Swap statistics: one CTA per individual over the rows of Pi' and of the
// sorted distances D' (the instance's table when it is cumulative, else the
// running sums of Delta' built once per instance), so that a rank's distance
// is one load and needs no scan; accumulators in shared memory when they fit
// (else in the output arrays, zeroed by the caller).
// ---------------------------------------------------------------------------
template <typename Acc, bool kSmem, bool kCand>
__global__ void __launch_bounds__(1024, 2) k_swap_stats(const uint16_t *__restrict__ pi,
                                                     const int32_t *__restrict__ dist, int64_t n, int32_t L,
                                                     int64_t stride, int32_t W, int32_t m,
                                                     const uint32_t *__restrict__ masks, int64_t pop,
                                                     unsigned long long *__restrict__ gain, int *__restrict__ cap,
                                                     unsigned long long *__restrict__ loss, int *__restrict__ assign,
                                                     CandOut co)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int64_t t = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *bits = reinterpret_cast<uint32_t *>(sm);
    const size_t off = ((size_t)W * 4 + 15) & ~size_t(15);
    // accumulators: in shared memory (kSmem; Acc of 32 or 64 bits, chosen by the host so sums cannot overflow)
    // or directly in the outputs (64 bits, zeroed by the caller)
    Acc *Gs = reinterpret_cast<Acc *>(sm + off);
    Acc *Ls = Gs + m;
    int *Cs = reinterpret_cast<int *>(Ls + m);
    int *As = Cs + m;
    const int64_t tm = t * m;
    auto add_stat = [&](bool first, uint32_t k, int32_t v) {  // add_loss if first, else add_gain
        if constexpr (kSmem) {
            atomicAdd((first ? Ls : Gs) + k, (Acc)(uint32_t)v);
            atomicAdd((first ? As : Cs) + k, 1);
        } else {
            atomicAdd((first ? loss : gain) + tm + k, (unsigned long long)(uint32_t)v);
            atomicAdd((first ? assign : cap) + tm + k, 1);
        }
    };
    auto add_gain = [&](uint32_t k, int32_t v) { add_stat(false, k, v); };  // closed k, ranked before the first open
    auto add_loss = [&](uint32_t j, int32_t v) { add_stat(true, j, v); };   // the first open facility j
    if constexpr (kSmem) {
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            Gs[j] = 0;
            Ls[j] = 0;
            Cs[j] = 0;
            As[j] = 0;
        }
    }
    for (int w = threadIdx.x; w < W; w += blockDim.x)
        bits[w] = masks[t * W + w];
    // the first 32 ranks of this warp's first client (constant tables: no dependence on the zeroing above)
    const int nc = (int)n;        // clients (the tables of one GPU hold far fewer than 2^31 rows)
    const int st = (int)stride;   // row stride of Pi'/D' (at most 65536)
    uint32_t j_nx = 0;
    int32_t d_nx = 0;
    if (warp < nc && lane < L) {
        j_nx = __ldg(pi + (size_t)warp * st + lane);
        d_nx = __ldg(dist + (size_t)warp * st + lane);
    }
    __syncthreads();
    for (int i = warp; i < nc; i += nwarps) {
        const uint16_t *prow = pi + (size_t)i * st;
        const int32_t *drow = dist + (size_t)i * st;
        // first 32 ranks (loaded a client ahead).  When the first open rank r1 is among them -- the usual case
        // unless p/m is tiny -- every gain comes from this step: the ranks before r1 gain d1 - d(i, k) and the
        // facility at r1 loses d2 - d1, with d2 at the second open rank (later steps are read only for it).
        {
            const uint32_t j0 = j_nx;
            const int32_t d0 = d_nx;
            const int inext = i + nwarps;  // the next client's first step, loaded while this one runs
            j_nx = 0;
            d_nx = 0;
            if (inext < nc && lane < L) {
                j_nx = __ldg(pi + (size_t)inext * st + lane);
                d_nx = __ldg(dist + (size_t)inext * st + lane);
            }
            const bool open0 = (lane < L) && ((bits[j0 >> 5] >> (j0 & 31)) & 1u);
            const uint32_t bal0 = __ballot_sync(PM_FULL_MASK, open0);
            if (bal0 != 0u) {
                const int f1 = __ffs(bal0) - 1;
                const int32_t d1 = __shfl_sync(PM_FULL_MASK, d0, f1);
                const uint32_t rest = bal0 & (bal0 - 1u);
                int32_t d2;
                if (rest != 0u) {
                    d2 = __shfl_sync(PM_FULL_MASK, d0, __ffs(rest) - 1);
                } else {  // the second open rank lies beyond this step, or the row holds no second one
                    bool got = false;
                    d2 = 0;
                    for (int base = 32; base < L; base += 32) {
                        const int r = base + lane;
                        uint32_t j = 0;
                        int32_t dl = 0;
                        if (r < L) {
                            j = __ldg(prow + r);
                            dl = __ldg(drow + r);
                        }
                        const uint32_t bal = __ballot_sync(PM_FULL_MASK, (r < L) && ((bits[j >> 5] >> (j & 31)) & 1u));
                        if (bal != 0u) {
                            d2 = __shfl_sync(PM_FULL_MASK, dl, __ffs(bal) - 1);
                            got = true;
                            break;
                        }
                    }
                    if (!got)  // the last distance of the truncated row
                        d2 = __ldg(drow + L - 1);
                }
                if (lane <= f1) {  // one pair of atomics per lane: lane f1 holds the first open facility itself
                    const bool first = lane == f1;
                    add_stat(first, j0, first ? d2 - d1 : d1 - d0);
                }
                continue;
            }
        }
        // general path (no open facility among the first 32 ranks) -- pass 1: first and second open ranks
        int32_t d1 = 0, d2 = 0;
        int r1 = -1, found = 0;
        uint32_t f1 = 0;
        uint32_t j_nx1 = 0;  // the next step's ranks, loaded one step ahead
        int32_t d_nx1 = 0;
        if (32 + lane < L) {
            j_nx1 = __ldg(prow + 32 + lane);
            d_nx1 = __ldg(drow + 32 + lane);
        }
        for (int base = 32; base < L && found < 2; base += 32) {
            const int r = base + lane;
            const uint32_t j = j_nx1;
            const int32_t dl = d_nx1;
            j_nx1 = 0;
            d_nx1 = 0;
            if (r + 32 < L) {
                j_nx1 = __ldg(prow + r + 32);
                d_nx1 = __ldg(drow + r + 32);
            }
            uint32_t bal = __ballot_sync(PM_FULL_MASK, (r < L) && ((bits[j >> 5] >> (j & 31)) & 1u));
            if (bal == 0u)
                continue;
            if (found == 0) {
                const int f = __ffs(bal) - 1;
                d1 = __shfl_sync(PM_FULL_MASK, dl, f);
                f1 = __shfl_sync(PM_FULL_MASK, j, f);
                r1 = base + f;
                found = 1;
                bal &= bal - 1u;
                // the ranks of this step before r1 gain d1 - d(i, k) now; earlier steps are revisited below
                if (lane < f)
                    add_gain(j, d1 - dl);
            }
            if (found == 1 && bal) {
                d2 = __shfl_sync(PM_FULL_MASK, dl, __ffs(bal) - 1);
                found = 2;
            }
        }
        if (found == 0)
            continue;  // fewer than p open facilities: no statistics for this client
        if (found == 1)
            d2 = __ldg(drow + L - 1);  // no second open facility within the table: its last distance
        if (lane == 0)
            add_loss(f1, d2 - d1);
        // pass 2: the facilities of the steps before r1's step (no open one among them) gain d1 - d(i, k)
        const int r1_step = r1 & ~31;
        for (int base = 0; base < r1_step; base += 32) {
            const int r = base + lane;
            add_gain(__ldg(prow + r), d1 - __ldg(drow + r));
        }
    }
    if constexpr (kSmem) {
        __syncthreads();
        if constexpr (kCand) {  // the learned try's candidates from the statistics in place (kept off global memory)
            const size_t open_off = ((size_t)(reinterpret_cast<unsigned char *>(As + m) - sm) + 15) & ~size_t(15);
            candidates_from_stats<Acc>(bits, Gs, Ls, Cs, As, reinterpret_cast<int32_t *>(sm + open_off), W, m, t,
                                       co);
        } else {
            for (int j = threadIdx.x; j < m; j += blockDim.x) {
                gain[tm + j] = (unsigned long long)Gs[j];
                loss[tm + j] = (unsigned long long)Ls[j];
                cap[tm + j] = Cs[j];
                assign[tm + j] = As[j];
            }
        }
    }
}

__device__ __forceinline__ void move_feature_row(__nv_bfloat16 *out, float lj, float gk, float aj, float ck, float Z,
                                                 float per, float pm_ratio, float ldiff)
{
    float f[kFeat];
    f[0] = lj / Z;
    f[1] = gk / Z;
    f[2] = aj / per;
    f[3] = ck / per;
    f[4] = ldiff / Z;
    f[5] = log1pf(f[0]);
    f[6] = log1pf(f[1]);
    f[7] = pm_ratio;
#pragma unroll
    for (int q = 0; q < kFeat; ++q)
        out[q] = __float2bfloat16(f[q]);
#pragma unroll
    for (int q = kFeat; q < kIn; ++q)
        out[q] = __float2bfloat16(0.f);
}

// Features of given moves: moves[(t*C + c)*2 + {0,1}] = (j closed, k opened).
__global__ void k_move_features(const unsigned long long *__restrict__ gain, const int *__restrict__ cap,
                                const unsigned long long *__restrict__ loss, const int *__restrict__ assign,
                                const int64_t *__restrict__ costs, const int32_t *__restrict__ moves, int64_t pop,
                                int64_t C, int32_t m, int64_t n, int32_t p, __nv_bfloat16 *__restrict__ X)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= pop * C)
        return;
    const int64_t t = idx / C;
    const int32_t j = min(max(moves[idx * 2], 0), m - 1), k = min(max(moves[idx * 2 + 1], 0), m - 1);
    const float Z = fmaxf((float)costs[t] / (float)p, 1.f);
    const unsigned long long lj = loss[t * m + j], gk = gain[t * m + k];
    move_feature_row(X + idx * kIn, (float)lj, (float)gk, (float)assign[t * m + j], (float)cap[t * m + k], Z,
                     (float)n / (float)p, (float)p / (float)m, (float)((long long)lj - (long long)gk));
}

// Candidate moves of the learned try, one CTA per individual: the T closed
// facilities with the largest gain (ties: lower id), each paired with every
// open facility: C = p * T rows (j = the a-th open facility, k = the b-th
// best, row a * T + b).
__global__ void __launch_bounds__(256) k_candidates(const uint32_t *__restrict__ masks, int32_t W, int32_t m,
                                                    int32_t p, int64_t n, const unsigned long long *__restrict__ gain,
                                                    const int *__restrict__ cap,
                                                    const unsigned long long *__restrict__ loss,
                                                    const int *__restrict__ assign, const int64_t *__restrict__ costs,
                                                    int T, int32_t *__restrict__ moves, __nv_bfloat16 *__restrict__ X)
{
    constexpr int32_t kNone = 0x7fffffff;
    extern __shared__ __align__(16) unsigned char sm[];
    int32_t *open_s = reinterpret_cast<int32_t *>(sm);  // p entries
    for (int i = threadIdx.x; i < p; i += blockDim.x)
        open_s[i] = 0;  // a bitset with fewer than p open facilities still yields valid ids
    __syncthreads();
    __shared__ int32_t top_k[kMaxCand];
    __shared__ unsigned long long top_g[kMaxCand];
    __shared__ float top_f1[kMaxCand], top_f3[kMaxCand], top_f6[kMaxCand];
    __shared__ int32_t nopen;
    const int64_t t = blockIdx.x;
    const uint32_t *x = masks + t * W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // open facilities in ascending order (warp 0)
    if (warp == 0) {
        int cnt = 0;
        for (int base = 0; base < W; base += 32) {
            const int w = base + lane;
            const uint32_t word = w < W ? x[w] : 0u;
            const int pc = __popc(word);
            int incl = pc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(PM_FULL_MASK, incl, o);
                if (lane >= o)
                    incl += y;
            }
            int pos = cnt + incl - pc;
            uint32_t rest = word;
            while (rest) {
                const int b = __ffs(rest) - 1;
                rest &= rest - 1u;
                if (pos < p)
                    open_s[pos] = w * 32 + b;
                ++pos;
            }
            cnt += __shfl_sync(PM_FULL_MASK, incl, 31);
        }
        if (lane == 0)
            nopen = cnt < p ? cnt : p;
    }
    // top-T closed facilities by gain, in one pass over the gains: each thread keeps its own best T (in the
    // candidates' order) of the facilities it reads, then T rounds of a block-wide arg-max over the threads'
    // heads, the winner's owner dropping it -- the same T facilities, in the same order, as T arg-max passes
    unsigned long long lg[kMaxCand];
    int32_t lk[kMaxCand];
#pragma unroll
    for (int i = 0; i < kMaxCand; ++i) {
        lg[i] = 0ull;
        lk[i] = kNone;
    }
    for (int k = tid; k < m; k += blockDim.x) {
        if ((x[k >> 5] >> (k & 31)) & 1u)
            continue;
        unsigned long long cg = gain[t * m + k];
        int32_t ck = k;
#pragma unroll
        for (int i = 0; i < kMaxCand; ++i) {  // insertion: the displaced entry moves down
            if (i < T && cand_before(cg, ck, lg[i], lk[i])) {
                const unsigned long long tg = lg[i];
                const int32_t tk = lk[i];
                lg[i] = cg;
                lk[i] = ck;
                cg = tg;
                ck = tk;
            }
        }
    }
    __shared__ unsigned long long red_g[8];
    __shared__ int32_t red_k[8];
    for (int b = 0; b < T; ++b) {
        unsigned long long bg = lg[0];
        int32_t bk = lk[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long og = __shfl_xor_sync(PM_FULL_MASK, bg, o);
            const int32_t ok = __shfl_xor_sync(PM_FULL_MASK, bk, o);
            if (cand_before(og, ok, bg, bk)) {
                bg = og;
                bk = ok;
            }
        }
        if (lane == 0) {
            red_g[warp] = bg;
            red_k[warp] = bk;
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long g0 = red_g[0];
            int32_t k0 = red_k[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (cand_before(red_g[w], red_k[w], g0, k0)) {
                    g0 = red_g[w];
                    k0 = red_k[w];
                }
            if (k0 == kNone)  // fewer than T closed facilities: repeat the previous one
                k0 = b > 0 ? top_k[b - 1] : 0;
            top_k[b] = k0;
        }
        __syncthreads();
        if (lk[0] != kNone && lk[0] == top_k[b]) {  // the owner drops the winner
#pragma unroll
            for (int i = 0; i + 1 < kMaxCand; ++i) {
                lg[i] = lg[i + 1];
                lk[i] = lk[i + 1];
            }
            lg[kMaxCand - 1] = 0ull;
            lk[kMaxCand - 1] = kNone;
        }
    }
    const float Z = fmaxf((float)costs[t] / (float)p, 1.f);
    const float per = (float)n / (float)p, ratio = (float)p / (float)m;
    // the features that depend on the candidate k alone, once per k
    if (tid < T) {
        const int32_t k = top_k[tid];
        const unsigned long long gk = gain[t * m + k];
        top_g[tid] = gk;
        top_f1[tid] = (float)gk / Z;
        top_f3[tid] = (float)cap[t * m + k] / per;
        top_f6[tid] = log1pf(top_f1[tid]);
    }
    __syncthreads();
    // rows a*T .. a*T + T-1: open facility a (the first open one stands in past nopen) with each candidate; the
    // features of j once per a; a row is 16 BF16 (8 features, 8 zeros) written as two 16-byte stores
    const uint32_t bf_ratio = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(ratio));
    for (int a = tid; a < p; a += blockDim.x) {
        const int32_t j = open_s[a < nopen ? a : 0];
        const unsigned long long lj = loss[t * m + j];
        const float f0 = (float)lj / Z;
        const float f2 = (float)assign[t * m + j] / per;
        const float f5 = log1pf(f0);
        const uint32_t bf0 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(f0));
        const uint32_t bf2 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(f2));
        const uint32_t bf5 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(f5));
        for (int b = 0; b < T; ++b) {
            const int64_t idx = t * (int64_t)p * T + (int64_t)a * T + b;
            const float f4 = (float)((long long)lj - (long long)top_g[b]) / Z;
            uint4 v;
            v.x = bf0 | ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(top_f1[b])) << 16);
            v.y = bf2 | ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(top_f3[b])) << 16);
            v.z = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(f4)) | (bf5 << 16);
            v.w = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(top_f6[b])) | (bf_ratio << 16);
            uint4 *out = reinterpret_cast<uint4 *>(X + idx * kIn);
            out[0] = v;
            out[1] = make_uint4(0u, 0u, 0u, 0u);
            reinterpret_cast<int2 *>(moves)[idx] = make_int2(j, top_k[b]);
        }
    }
}

// Philox4x32-10 (Salmon et al., SC'11) for sampling training moves.
__device__ __forceinline__ uint4 philox_draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c)
{
    uint4 x = make_uint4(a, b, c, 0x4C45524Eu);
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * x.x, hi0 = __umulhi(0xD2511F53u, x.x);
        const uint32_t lo1 = 0xCD9E8D57u * x.z, hi1 = __umulhi(0xCD9E8D57u, x.z);
        x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
    }
    return x;
}

__device__ __forceinline__ uint32_t below(uint32_t u, uint32_t N) { return (uint32_t)(((unsigned long long)u * N) >> 32); }

// Training moves, one CTA per individual: j uniform among the open
// facilities; k among the 4 largest-gain closed facilities with probability
// 3/4 (the learned try's candidates), else uniform among the closed ones.
__global__ void __launch_bounds__(256) k_sample_moves(const uint32_t *__restrict__ masks, int32_t W, int32_t m,
                                                      int32_t p, const unsigned long long *__restrict__ gain,
                                                      int64_t per, uint64_t seed, int32_t *__restrict__ moves)
{
    extern __shared__ __align__(16) unsigned char sm[];
    int32_t *open_s = reinterpret_cast<int32_t *>(sm);
    for (int i = threadIdx.x; i < p; i += blockDim.x)
        open_s[i] = 0;  // a bitset with fewer than p open facilities still yields valid ids
    __syncthreads();
    __shared__ int32_t top_k[4];
    __shared__ unsigned long long red_g[8];
    __shared__ int32_t red_k[8];
    const int64_t t = blockIdx.x;
    const uint32_t *x = masks + t * W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {
        int cnt = 0;
        for (int base = 0; base < W; base += 32) {
            const int w = base + lane;
            const uint32_t word = w < W ? x[w] : 0u;
            const int pc = __popc(word);
            int incl = pc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(PM_FULL_MASK, incl, o);
                if (lane >= o)
                    incl += y;
            }
            int pos = cnt + incl - pc;
            uint32_t rest = word;
            while (rest) {
                const int b = __ffs(rest) - 1;
                rest &= rest - 1u;
                if (pos < p)
                    open_s[pos] = w * 32 + b;
                ++pos;
            }
            cnt += __shfl_sync(PM_FULL_MASK, incl, 31);
        }
    }
    for (int b = 0; b < 4; ++b) {
        unsigned long long bg = 0ull;
        int32_t bk = 0x7fffffff;
        for (int k = tid; k < m; k += blockDim.x) {
            if ((x[k >> 5] >> (k & 31)) & 1u)
                continue;
            bool taken = false;
            for (int q = 0; q < b; ++q)
                taken = taken || (top_k[q] == k);
            if (taken)
                continue;
            const unsigned long long gk = gain[t * m + k];
            if (bk == 0x7fffffff || gk > bg || (gk == bg && k < bk)) {
                bg = gk;
                bk = k;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long og = __shfl_xor_sync(PM_FULL_MASK, bg, o);
            const int32_t ok = __shfl_xor_sync(PM_FULL_MASK, bk, o);
            if (ok != 0x7fffffff && (bk == 0x7fffffff || og > bg || (og == bg && ok < bk))) {
                bg = og;
                bk = ok;
            }
        }
        if (lane == 0) {
            red_g[warp] = bg;
            red_k[warp] = bk;
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long g0 = red_g[0];
            int32_t k0 = red_k[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (red_k[w] != 0x7fffffff && (k0 == 0x7fffffff || red_g[w] > g0 || (red_g[w] == g0 && red_k[w] < k0))) {
                    g0 = red_g[w];
                    k0 = red_k[w];
                }
            top_k[b] = k0 == 0x7fffffff ? (b > 0 ? top_k[b - 1] : 0) : k0;
        }
        __syncthreads();
    }
    for (int64_t q = tid; q < per; q += blockDim.x) {
        const uint4 v = philox_draw(seed, (uint32_t)t, (uint32_t)q, 0u);
        const int32_t j = open_s[below(v.x, (uint32_t)p)];
        int32_t k = top_k[below(v.y, 4u)];
        if (below(v.z, 4u) == 3u) {  // uniform closed facility (bounded rejection)
            uint32_t u = v.w;
            for (int tries = 0; tries < 64; ++tries) {
                const int32_t c = (int32_t)below(u, (uint32_t)m);
                if (!((x[c >> 5] >> (c & 31)) & 1u)) {
                    k = c;
                    break;
                }
                u = philox_draw(seed, (uint32_t)t, (uint32_t)q, (uint32_t)(tries + 1)).x;
            }
        }
        moves[(t * per + q) * 2] = j;
        moves[(t * per + q) * 2 + 1] = k;
    }
}

// Swapped bitsets: row (t * per + q) = individual t with moves[..][0] closed and moves[..][1] opened.
__global__ void k_apply_moves(const uint32_t *__restrict__ masks, int32_t W, int64_t pop, int64_t per,
                              const int32_t *__restrict__ moves, uint32_t *__restrict__ out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= pop * per * W)
        return;
    const int64_t row = idx / W;
    const int32_t w = (int32_t)(idx % W);
    const int64_t t = row / per;
    uint32_t v = masks[t * W + w];
    const int32_t j = moves[row * 2], k = moves[row * 2 + 1];
    if ((j >> 5) == w)
        v &= ~(1u << (j & 31));
    if ((k >> 5) == w)
        v |= 1u << (k & 31);
    out[idx] = v;
}

__global__ void k_targets(const int64_t *__restrict__ before, const int64_t *__restrict__ after, int64_t pop,
                          int64_t per, int32_t p, float *__restrict__ t_out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= pop * per)
        return;
    const int64_t t = idx / per;
    const float Z = fmaxf((float)before[t] / (float)p, 1.f);
    t_out[idx] = (float)(after[idx] - before[t]) / Z;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: the model object
// ---------------------------------------------------------------------------

pm_status pm_learn_prepare(const pm_instance *inst, cudaStream_t s);

struct pm_model {
    int device = 0;
    int sm_count = 1;
    pm_dbuf P, M, V, G, W1b, W2b, w3b, loss, err;
    int64_t step = 0;
    std::mutex lock;
};

static size_t mlp_smem(bool train)
{
    size_t s = (sizeof(MlpSmem) + 15) & ~size_t(15);
    if (train)
        s += sizeof(MlpTrainSmem);
    return s;
}

// dynamic shared memory of the tcgen05 forward (about 74 KB: three CTAs share an SM, and even four would hold
// only 4 x 128 TMEM columns, the SM's 512)
static size_t tc_smem() { return sizeof(TcSmem); }

// PM_TRAIN_TC=0 in the environment trains with the mma.sync kernel instead of the tcgen05 one (for comparison).
static bool train_tc()
{
    static const bool on = [] {
        const char *e = std::getenv("PM_TRAIN_TC");
        return !(e && e[0] == '0');
    }();
    return on;
}

static pm_status mlp_init_attrs()
{
    PM_CUDA(cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem()));
    PM_CUDA(cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrSmem)));
    PM_CUDA(cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem(false)));
    PM_CUDA(cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem(true)));
    return PM_OK;
}

static pm_status model_refresh(pm_model *md, cudaStream_t s)
{
    k_refresh_bf16<<<(kHid * kHid + 255) / 256, 256, 0, s>>>(
        static_cast<const float *>(md->P.ptr), static_cast<__nv_bfloat16 *>(md->W1b.ptr),
        static_cast<__nv_bfloat16 *>(md->W2b.ptr), static_cast<__nv_bfloat16 *>(md->w3b.ptr));
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_model_create(int device, uint64_t seed, pm_model **out)
{
    if (!out || device < 0)
        return PM_ERR_INVALID_ARG;
    *out = nullptr;
    PM_CUDA(cudaSetDevice(device));
    pm_model *md = new (std::nothrow) pm_model();
    if (!md)
        return PM_ERR_OOM;
    md->device = device;
    if (cudaDeviceGetAttribute(&md->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete md;
        return PM_ERR_CUDA;
    }
    pm_status st = PM_OK;
    pm_dbuf *bufs[] = {&md->P, &md->M, &md->V, &md->G};
    for (pm_dbuf *b : bufs)
        if (st == PM_OK)
            st = b->reserve(kParams * sizeof(float));
    if (st == PM_OK)
        st = md->W1b.reserve(kIn * kHid * 2);
    if (st == PM_OK)
        st = md->W2b.reserve(kHid * kHid * 2);
    if (st == PM_OK)
        st = md->w3b.reserve(kHid * 2);
    if (st == PM_OK)
        st = md->loss.reserve(256);
    if (st == PM_OK)
        st = md->err.reserve(256);
    if (st == PM_OK && cudaMemset(md->err.ptr, 0, 256) != cudaSuccess)
        st = PM_ERR_CUDA;
    if (st == PM_OK)
        st = mlp_init_attrs();
    if (st != PM_OK) {
        pm_model_destroy(md);
        return st;
    }
    // He-style initialisation from a seeded host generator (splitmix64 + Box-Muller)
    std::vector<float> h(kParams, 0.f);
    uint64_t z = seed ^ 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t r = z;
        r = (r ^ (r >> 30)) * 0xBF58476D1CE4E5B9ull;
        r = (r ^ (r >> 27)) * 0x94D049BB133111EBull;
        return r ^ (r >> 31);
    };
    auto normal = [&]() {
        const double u1 = ((next() >> 11) + 1.0) / 9007199254740993.0, u2 = (next() >> 11) / 9007199254740992.0;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int i = 0; i < kFeat; ++i)  // rows of the padded inputs stay zero
        for (int o = 0; o < kHid; ++o)
            h[kOffW1 + i * kHid + o] = (float)(normal() * std::sqrt(2.0 / kFeat));
    for (int i = 0; i < kHid * kHid; ++i)
        h[kOffW2 + i] = (float)(normal() * std::sqrt(2.0 / kHid));
    for (int i = 0; i < kHid; ++i)
        h[kOffW3 + i] = (float)(normal() * std::sqrt(1.0 / kHid));
    st = pm_model_set_params(md, h.data(), nullptr);
    if (st != PM_OK) {
        pm_model_destroy(md);
        return st;
    }
    *out = md;
    return PM_OK;
}

extern "C" pm_status pm_model_destroy(pm_model *md)
{
    if (!md)
        return PM_OK;
    pm_clear_error(cudaSetDevice(md->device));
    pm_dbuf *bufs[] = {&md->P, &md->M, &md->V, &md->G, &md->W1b, &md->W2b, &md->w3b, &md->loss, &md->err};
    for (pm_dbuf *b : bufs)
        b->release();
    delete md;
    return PM_OK;
}

extern "C" int64_t pm_model_num_params(void) { return kParams; }

extern "C" pm_status pm_model_set_params(pm_model *md, const float *params, void *stream)
{
    if (!md || !params)
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(md->lock);
    PM_CUDA(cudaSetDevice(md->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_CUDA(cudaMemcpyAsync(md->P.ptr, params, kParams * sizeof(float), cudaMemcpyDefault, s));
    PM_CUDA(cudaMemsetAsync(md->M.ptr, 0, kParams * sizeof(float), s));
    PM_CUDA(cudaMemsetAsync(md->V.ptr, 0, kParams * sizeof(float), s));
    md->step = 0;
    PM_TRY(model_refresh(md, s));
    PM_CUDA(cudaStreamSynchronize(s));
    return PM_OK;
}

extern "C" pm_status pm_model_get_params(pm_model *md, float *params, void *stream)
{
    if (!md || !params)
        return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(md->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_CUDA(cudaMemcpyAsync(params, md->P.ptr, kParams * sizeof(float), cudaMemcpyDefault, s));
    PM_CUDA(cudaStreamSynchronize(s));
    return PM_OK;
}

static pm_status mlp_launch(pm_model *md, bool train, const void *x, int64_t rows, float *y, const float *t,
                            float inv_batch, cudaStream_t s, RowMap map = RowMap{})
{
    const unsigned grid = (unsigned)pm_ceil_div(rows, kRows);
    const __nv_bfloat16 *X = static_cast<const __nv_bfloat16 *>(x);
    const __nv_bfloat16 *W1b = static_cast<const __nv_bfloat16 *>(md->W1b.ptr);
    const __nv_bfloat16 *W2b = static_cast<const __nv_bfloat16 *>(md->W2b.ptr);
    const __nv_bfloat16 *w3b = static_cast<const __nv_bfloat16 *>(md->w3b.ptr);
    const float *P = static_cast<const float *>(md->P.ptr);
    if (train && train_tc()) {
        // one tile per CTA while the batch fits the GPU (a training step's latency), more per CTA beyond it (fewer
        // gradient atomics: the weight gradients accumulate in tensor memory)
        const int64_t tiles = pm_ceil_div(rows, kTcRows);
        const int tpc = (int)std::max<int64_t>(1, pm_ceil_div(tiles, (int64_t)md->sm_count));
        k_mlp_train_tc<<<(unsigned)pm_ceil_div(tiles, tpc), kTrThreads, sizeof(TrSmem), s>>>(
            X, rows, W1b, W2b, w3b, P, t, inv_batch, static_cast<float *>(md->G.ptr),
            static_cast<float *>(md->loss.ptr), map, tpc, static_cast<int *>(md->err.ptr));
    }
    else if (train)
        k_mlp<true><<<grid, 128, mlp_smem(true), s>>>(X, rows, W1b, W2b, w3b, P, y, t, inv_batch,
                                                      static_cast<float *>(md->G.ptr),
                                                      static_cast<float *>(md->loss.ptr), map);
    else
        k_mlp_fwd_tc<<<(unsigned)std::min<int64_t>(pm_ceil_div(rows, kTcRows), 3 * (int64_t)md->sm_count),
                       kTcThreads, tc_smem(), s>>>(X, rows, W1b, W2b, w3b, P, y, static_cast<int *>(md->err.ptr));
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

pm_status pm_model_forward_dev(pm_model *md, const void *x_dev, int64_t rows, float *y_dev, cudaStream_t s)
{
    if (rows <= 0)
        return PM_OK;
    return mlp_launch(md, false, x_dev, rows, y_dev, nullptr, 0.f, s);
}

extern "C" pm_status pm_model_forward(pm_model *md, const uint16_t *x, int64_t rows, float *y, void *stream)
{
    if (!md || !x || !y || rows < 0)
        return PM_ERR_INVALID_ARG;
    if (!pm_is_device_ptr(x) || !pm_is_device_ptr(y))
        return PM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0)
        return PM_ERR_INVALID_ARG;  // input rows are read as 16-byte vectors
    PM_CUDA(cudaSetDevice(md->device));
    return pm_model_forward_dev(md, x, rows, y, static_cast<cudaStream_t>(stream));
}

// Gradients of the mean squared error (into md->G) and the loss; returns the
// mean squared error in *loss_out (synchronises).
static pm_status model_grad(pm_model *md, const uint16_t *x, const float *t, int64_t rows, float *loss_out,
                            cudaStream_t s)
{
    PM_TRY(md->loss.reserve(256));
    PM_CUDA(cudaMemsetAsync(md->G.ptr, 0, kParams * sizeof(float), s));
    PM_CUDA(cudaMemsetAsync(md->loss.ptr, 0, sizeof(float), s));
    // predictions go to a scratch area behind the loss word
    pm_dbuf &yb = md->loss;
    PM_TRY(yb.reserve(256 + (size_t)rows * 4));
    PM_CUDA(cudaMemsetAsync(yb.ptr, 0, sizeof(float), s));
    float *y = reinterpret_cast<float *>(static_cast<char *>(yb.ptr) + 256);
    PM_TRY(mlp_launch(md, true, x, rows, y, t, 1.0f / (float)rows, s));
    if (loss_out) {
        float sq = 0.f;
        PM_CUDA(cudaMemcpyAsync(&sq, yb.ptr, sizeof(float), cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaStreamSynchronize(s));
        *loss_out = sq / (float)rows;
    }
    return PM_OK;
}

extern "C" pm_status pm_model_grad(pm_model *md, const uint16_t *x, const float *t, int64_t rows, float *grads,
                                   float *loss, void *stream)
{
    if (!md || !x || !t || rows < 1 || (reinterpret_cast<uintptr_t>(x) & 15u) != 0)
        return PM_ERR_INVALID_ARG;
    if (!pm_is_device_ptr(x) || !pm_is_device_ptr(t))
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(md->lock);
    PM_CUDA(cudaSetDevice(md->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_TRY(model_grad(md, x, t, rows, loss, s));
    if (grads)
        PM_CUDA(cudaMemcpyAsync(grads, md->G.ptr, kParams * sizeof(float), cudaMemcpyDefault, s));
    PM_CUDA(cudaStreamSynchronize(s));
    return PM_OK;
}

extern "C" pm_status pm_model_train_step(pm_model *md, const uint16_t *x, const float *t, int64_t rows, float lr,
                                         float *loss, void *stream)
{
    if (!md || !x || !t || rows < 1 || !(lr > 0.f) || (reinterpret_cast<uintptr_t>(x) & 15u) != 0)
        return PM_ERR_INVALID_ARG;
    if (!pm_is_device_ptr(x) || !pm_is_device_ptr(t))
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(md->lock);
    PM_CUDA(cudaSetDevice(md->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_TRY(model_grad(md, x, t, rows, loss, s));
    md->step += 1;
    const float bc1 = 1.f - std::pow(0.9f, (float)md->step), bc2 = 1.f - std::pow(0.999f, (float)md->step);
    k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(
        static_cast<float *>(md->P.ptr), static_cast<float *>(md->M.ptr), static_cast<float *>(md->V.ptr),
        static_cast<float *>(md->G.ptr), kParams, lr, bc1, bc2, static_cast<__nv_bfloat16 *>(md->W1b.ptr),
        static_cast<__nv_bfloat16 *>(md->W2b.ptr), static_cast<__nv_bfloat16 *>(md->w3b.ptr), nullptr, nullptr,
        0.f);
    PM_CUDA(cudaGetLastError());
    if (loss)
        PM_CUDA(cudaStreamSynchronize(s));
    return PM_OK;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) on the host: the round keys of the epoch shuffle.
static void philox10_host(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

constexpr uint32_t kOpShuffle = 0x300u;  // operation id of the epoch shuffle's draws

extern "C" pm_status pm_model_train(pm_model *md, const uint16_t *x, const float *t, int64_t rows, int32_t epochs,
                                    int64_t batch, float lr, uint64_t seed, float *losses, void *stream)
{
    if (!md || !x || !t || rows < 1 || rows >= ((int64_t)1 << 31) || epochs < 0 || batch < 1 || !(lr > 0.f) ||
        (reinterpret_cast<uintptr_t>(x) & 15u) != 0)
        return PM_ERR_INVALID_ARG;
    if (!pm_is_device_ptr(x) || !pm_is_device_ptr(t))
        return PM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(md->lock);
    PM_CUDA(cudaSetDevice(md->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t per_epoch = pm_ceil_div(rows, batch);
    const int64_t steps = per_epoch * (int64_t)epochs;
    if (steps == 0)
        return PM_OK;
    const bool losses_dev = losses && pm_is_device_ptr(losses);
    // the step losses (device), then the predictions of the training kernel (scratch)
    const size_t loss_bytes = (size_t)pm_round_up(steps * 4, 256);
    const int64_t bmax = std::min(batch, rows);
    PM_TRY(md->loss.reserve(256 + loss_bytes + (size_t)bmax * 4));
    char *lb = static_cast<char *>(md->loss.ptr);
    float *loss_word = reinterpret_cast<float *>(lb);
    float *step_loss = losses_dev ? losses : reinterpret_cast<float *>(lb + 256);
    float *y = reinterpret_cast<float *>(lb + 256 + loss_bytes);
    PM_CUDA(cudaMemsetAsync(md->G.ptr, 0, kParams * sizeof(float), s));
    PM_CUDA(cudaMemsetAsync(loss_word, 0, sizeof(float), s));
    int bits = 2;
    while (bits < 62 && ((int64_t)1 << bits) < rows)
        bits += 2;
    int64_t k = 0;
    for (int32_t e = 0; e < epochs; ++e) {
        RowMap map{};
        uint32_t c[4] = {(uint32_t)e, 0u, kOpShuffle << 16, 0u};
        philox10_host(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        for (int r = 0; r < 4; ++r)
            map.key[r] = c[r];
        map.half = bits / 2;
        map.total = rows;
        for (int64_t b0 = 0; b0 < rows; b0 += batch, ++k) {
            const int64_t nrow = std::min(batch, rows - b0);
            map.pos0 = b0;
            PM_TRY(mlp_launch(md, true, x, nrow, y, t, 1.0f / (float)nrow, s, map));
            md->step += 1;
            const float bc1 = 1.f - std::pow(0.9f, (float)md->step);
            const float bc2 = 1.f - std::pow(0.999f, (float)md->step);
            k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(
                static_cast<float *>(md->P.ptr), static_cast<float *>(md->M.ptr), static_cast<float *>(md->V.ptr),
                static_cast<float *>(md->G.ptr), kParams, lr, bc1, bc2, static_cast<__nv_bfloat16 *>(md->W1b.ptr),
                static_cast<__nv_bfloat16 *>(md->W2b.ptr), static_cast<__nv_bfloat16 *>(md->w3b.ptr), loss_word,
                step_loss + k, 1.0f / (float)nrow);
            PM_CUDA(cudaGetLastError());
        }
    }
    if (losses && !losses_dev) {
        PM_CUDA(cudaMemcpyAsync(losses, step_loss, (size_t)steps * 4, cudaMemcpyDeviceToHost, s));
        PM_CUDA(cudaStreamSynchronize(s));
    }
    return PM_OK;
}

// ---------------------------------------------------------------------------
// Swap statistics, move features, logging of training tuples
// ---------------------------------------------------------------------------

pm_status pm_launch_swap_stats(const pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *gain,
                               int32_t *cap, int64_t *loss, int32_t *assign, cudaStream_t s)
{
    if (pop <= 0)
        return PM_OK;
    const size_t bits = (size_t)pm_round_up(inst->W * 4, 16);
    // 32-bit shared accumulators suffice when no sum can reach 2^32: every gain and loss is at most n * max d
    const bool narrow = (double)inst->n * (double)std::max(inst->max_d, 1) < 4294967295.0;
    const size_t acc = (size_t)inst->m * (narrow ? 16 : 24);
    const bool in_smem = bits + acc + 1024 <= inst->smem_optin;
    const size_t smem = in_smem ? bits + acc : bits;
    if (!in_smem) {
        PM_CUDA(cudaMemsetAsync(gain, 0, (size_t)pop * inst->m * 8, s));
        PM_CUDA(cudaMemsetAsync(loss, 0, (size_t)pop * inst->m * 8, s));
        PM_CUDA(cudaMemsetAsync(cap, 0, (size_t)pop * inst->m * 4, s));
        PM_CUDA(cudaMemsetAsync(assign, 0, (size_t)pop * inst->m * 4, s));
    }
    // the sorted distances: the instance's own table when cumulative, else the running sums that
    // pm_learn_prepare builds (every caller prepares the instance first)
    const int32_t *dist = inst->cum ? inst->delta : static_cast<const int32_t *>(inst->dsorted.ptr);
    if (!dist)
        return PM_ERR_INVALID_ARG;
    const CandOut none{nullptr, nullptr, nullptr, 0, 0, 0};
#define PM_STATS_ARGS                                                                                              \
    inst->pi, dist, inst->n, (int32_t)inst->L, inst->stride, (int32_t)inst->W, (int32_t)inst->m, masks, pop,       \
        reinterpret_cast<unsigned long long *>(gain), cap, reinterpret_cast<unsigned long long *>(loss), assign, none
    if (narrow && in_smem)
        k_swap_stats<unsigned int, true, false><<<(unsigned)pop, 1024, smem, s>>>(PM_STATS_ARGS);
    else if (in_smem)
        k_swap_stats<unsigned long long, true, false><<<(unsigned)pop, 1024, smem, s>>>(PM_STATS_ARGS);
    else
        k_swap_stats<unsigned long long, false, false><<<(unsigned)pop, 1024, smem, s>>>(PM_STATS_ARGS);
#undef PM_STATS_ARGS
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_swap_stats(pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *gain, int32_t *cap,
                                   int64_t *loss, int32_t *assign, void *stream)
{
    if (!inst || pop < 0 || !masks || !gain || !cap || !loss || !assign)
        return PM_ERR_INVALID_ARG;
    const void *ptrs[] = {masks, gain, cap, loss, assign};
    for (const void *p : ptrs)
        if (!pm_is_device_ptr(p))
            return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(inst->device));
    PM_TRY(pm_learn_prepare(inst, static_cast<cudaStream_t>(stream)));
    return pm_launch_swap_stats(inst, masks, pop, gain, cap, loss, assign, static_cast<cudaStream_t>(stream));
}

pm_status pm_launch_move_features(const pm_instance *inst, const int64_t *gain, const int32_t *cap, const int64_t *loss,
                                  const int32_t *assign, const int64_t *costs, const int32_t *moves, int64_t pop,
                                  int64_t C, uint16_t *x, cudaStream_t s)
{
    const int64_t rows = pop * C;
    if (rows <= 0)
        return PM_OK;
    k_move_features<<<(unsigned)pm_ceil_div(rows, 256), 256, 0, s>>>(
        reinterpret_cast<const unsigned long long *>(gain), cap, reinterpret_cast<const unsigned long long *>(loss),
        assign, costs, moves, pop, C, (int32_t)inst->m, inst->n, (int32_t)inst->p,
        reinterpret_cast<__nv_bfloat16 *>(x));
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_move_features(pm_instance *inst, const int64_t *gain, const int32_t *cap, const int64_t *loss,
                                      const int32_t *assign, const int64_t *costs, const int32_t *moves, int64_t pop,
                                      int64_t C, uint16_t *x, void *stream)
{
    if (!inst || pop < 0 || C < 0)
        return PM_ERR_INVALID_ARG;
    const void *ptrs[] = {gain, cap, loss, assign, costs, moves, x};
    for (const void *p : ptrs)
        if (!pm_is_device_ptr(p))
            return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(inst->device));
    return pm_launch_move_features(inst, gain, cap, loss, assign, costs, moves, pop, C, x,
                                   static_cast<cudaStream_t>(stream));
}

pm_status pm_launch_candidates(const pm_instance *inst, const uint32_t *masks, int64_t pop, const int64_t *gain,
                               const int32_t *cap, const int64_t *loss, const int32_t *assign, const int64_t *costs,
                               int T, int32_t *moves, uint16_t *x, cudaStream_t s)
{
    if (pop <= 0)
        return PM_OK;
    const size_t smem = (size_t)pm_round_up(inst->p * 4, 16);
    k_candidates<<<(unsigned)pop, 256, smem, s>>>(masks, (int32_t)inst->W, (int32_t)inst->m, (int32_t)inst->p, inst->n,
                                                  reinterpret_cast<const unsigned long long *>(gain), cap,
                                                  reinterpret_cast<const unsigned long long *>(loss), assign, costs, T,
                                                  moves, reinterpret_cast<__nv_bfloat16 *>(x));
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

pm_status pm_launch_learned_candidates(const pm_instance *inst, const uint32_t *masks, int64_t pop, int64_t *gain,
                                       int32_t *cap, int64_t *loss, int32_t *assign, const int64_t *costs, int T,
                                       int32_t *moves, uint16_t *x, cudaStream_t s)
{
    if (pop <= 0)
        return PM_OK;
    const size_t bits = (size_t)pm_round_up(inst->W * 4, 16);
    const bool narrow = (double)inst->n * (double)std::max(inst->max_d, 1) < 4294967295.0;
    const size_t acc = (size_t)inst->m * (narrow ? 16 : 24);
    const size_t smem = (size_t)pm_round_up(bits + acc, 16) + (size_t)pm_round_up(inst->p * 4, 16);
    const int32_t *dist = inst->cum ? inst->delta : static_cast<const int32_t *>(inst->dsorted.ptr);
    const char *env = std::getenv("PM_LEARN_FUSED");  // PM_LEARN_FUSED=0: always the two kernels (for comparison)
    if (!dist || smem + 1024 > inst->smem_optin || (env && env[0] == '0')) {
        // the two kernels, the statistics through global memory
        PM_TRY(pm_launch_swap_stats(inst, masks, pop, gain, cap, loss, assign, s));
        return pm_launch_candidates(inst, masks, pop, gain, cap, loss, assign, costs, T, moves, x, s);
    }
    const CandOut co{costs, moves, reinterpret_cast<__nv_bfloat16 *>(x), (int32_t)inst->p, T, inst->n};
#define PM_STATS_ARGS                                                                                              \
    inst->pi, dist, inst->n, (int32_t)inst->L, inst->stride, (int32_t)inst->W, (int32_t)inst->m, masks, pop,       \
        nullptr, nullptr, nullptr, nullptr, co
    if (narrow)
        k_swap_stats<unsigned int, true, true><<<(unsigned)pop, 1024, smem, s>>>(PM_STATS_ARGS);
    else
        k_swap_stats<unsigned long long, true, true><<<(unsigned)pop, 1024, smem, s>>>(PM_STATS_ARGS);
#undef PM_STATS_ARGS
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

int pm_mlp_in_width() { return kIn; }

// Kernel attributes of the learned path for this instance (call outside stream capture).
pm_status pm_learn_prepare(const pm_instance *inst, cudaStream_t s)
{
    if (!inst->cum) {
        // the running sums D' of a Delta' instance, once (on s, waited for: later launches may use any stream)
        std::lock_guard<std::mutex> g(inst->dsorted_mu);
        if (!inst->dsorted.ptr) {
            const size_t bytes = (size_t)inst->n * (size_t)inst->stride * sizeof(int32_t);
            PM_TRY(inst->dsorted.reserve(bytes));
            const int64_t blocks = std::min<int64_t>(pm_ceil_div(inst->n, 8), (int64_t)inst->sm_count * 8);
            k_running_sums<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(
                inst->delta, inst->n, (int32_t)inst->L, inst->stride, static_cast<int32_t *>(inst->dsorted.ptr));
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                inst->dsorted.release();
                PM_CUDA(e);
            }
        }
    }
    const int cap = (int)(inst->smem_optin > 1024 ? inst->smem_optin - 1024 : inst->smem_optin);
    // the shared-memory accumulator variants (the global one holds only the bitset: at most 8 KB)
    PM_CUDA(cudaFuncSetAttribute(k_swap_stats<unsigned int, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 cap));
    PM_CUDA(cudaFuncSetAttribute(k_swap_stats<unsigned long long, true, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    PM_CUDA(cudaFuncSetAttribute(k_swap_stats<unsigned int, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 cap));
    PM_CUDA(cudaFuncSetAttribute(k_swap_stats<unsigned long long, true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    PM_CUDA(cudaFuncSetAttribute(k_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    return mlp_init_attrs();
}

extern "C" pm_status pm_log_moves(pm_instance *inst, const uint32_t *masks, const int64_t *costs, int64_t pop,
                                  int64_t per, uint64_t seed, uint16_t *x, float *t, int32_t *moves, void *stream)
{
    if (!inst || pop < 1 || per < 1 || !masks || !costs || !x || !t || !moves)
        return PM_ERR_INVALID_ARG;
    const void *ptrs[] = {masks, costs, x, t, moves};
    for (const void *ptr : ptrs)
        if (!pm_is_device_ptr(ptr))
            return PM_ERR_INVALID_ARG;
    PM_CUDA(cudaSetDevice(inst->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PM_TRY(pm_learn_prepare(inst, s));
    const size_t Pm = (size_t)pop * inst->m, rows = (size_t)pop * per;
    char *buf = nullptr;
    const size_t bytes = Pm * 24 + rows * inst->W * 4 + rows * 8 + 1024;
    PM_CUDA(pm_device_malloc_async(reinterpret_cast<void **>(&buf), bytes, s));
    int64_t *gain = reinterpret_cast<int64_t *>(buf);
    int64_t *loss = gain + Pm;
    int32_t *cap = reinterpret_cast<int32_t *>(loss + Pm);
    int32_t *asg = cap + Pm;
    uint32_t *swapped = reinterpret_cast<uint32_t *>(asg + Pm);
    int64_t *after = reinterpret_cast<int64_t *>(swapped + rows * inst->W + (rows * inst->W & 1));
    pm_status st = pm_launch_swap_stats(inst, masks, pop, gain, cap, loss, asg, s);
    if (st == PM_OK) {
        const size_t smem = (size_t)pm_round_up(inst->p * 4, 16);
        cudaFuncSetAttribute(k_sample_moves, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_sample_moves<<<(unsigned)pop, 256, smem, s>>>(masks, (int32_t)inst->W, (int32_t)inst->m, (int32_t)inst->p,
                                                        reinterpret_cast<const unsigned long long *>(gain), per, seed,
                                                        moves);
        st = cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
    }
    if (st == PM_OK)
        st = pm_launch_move_features(inst, gain, cap, loss, asg, costs, moves, pop, per, x, s);
    if (st == PM_OK) {
        const int64_t n = (int64_t)rows * inst->W;
        k_apply_moves<<<(unsigned)pm_ceil_div(n, 256), 256, 0, s>>>(masks, (int32_t)inst->W, pop, per, moves, swapped);
        st = cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
    }
    if (st == PM_OK)
        st = pm_eval_population(inst, swapped, (int64_t)rows, after, 0, stream);
    if (st == PM_OK) {
        k_targets<<<(unsigned)pm_ceil_div((int64_t)rows, 256), 256, 0, s>>>(costs, after, pop, per, (int32_t)inst->p, t);
        st = cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
    }
    cudaFreeAsync(buf, s);
    return st;
}
