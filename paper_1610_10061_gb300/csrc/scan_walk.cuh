// The client walk of the fitness scan (Section 4.2, Fitness; Eq. 6), shared by
// the evaluation kernels (fitness.cu) and the GA's persistent generation
// kernel (ga.cu): a warp walks one client's row of Pi'/Delta' 32 ranks per
// step against a tile of 32 G individuals held facility-major in shared
// memory (word (j, g) = the individuals of group g with facility j open), and
// adds each individual's term at its first open rank.
#pragma once

#include <cstdint>

#include "pm_common.cuh"

constexpr int kWalkSparseLanes = 3;  // resolve by walking hit lanes up to this many

// The G words of facility j (groups 0..G-1) with one shared-memory load.
template <int G>
__device__ __forceinline__ void load_cols(const uint32_t *cb, uint32_t j, uint32_t (&w)[G])
{
    if constexpr (G == 4) {
        const uint4 v = reinterpret_cast<const uint4 *>(cb)[j];
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    } else if constexpr (G == 2) {
        const uint2 v = reinterpret_cast<const uint2 *>(cb)[j];
        w[0] = v.x;
        w[1] = v.y;
    } else {
        w[0] = cb[j];
    }
}

// One warp's walk over the clients c, c + step, ... (< c_end) of one tile:
// the tile's facility-major bits are in colbits, a0[g] marks its active
// individuals; every resolved individual's distance is added to acc[g] at
// the lane of the individual.  load(cc, base, j, dl) yields rank base + lane
// of client cc (Pi' and Delta', zeros past the row or past c_end); the
// caller passes the first two steps of clients c and c + step already loaded.
//
// With cumulative tables (cum) the row holds D' -- the running sums of Delta',
// i.e. the sorted distances -- so a step needs neither the carry nor the warp
// scan: the value at the first open rank is the term itself (Eq. 4 summed).
template <int G, typename Ld>
__device__ __forceinline__ void scan_clients(const uint32_t *__restrict__ colbits, const uint32_t (&a0)[G], int64_t c,
                                             int64_t c_end, int step, int32_t L, int lane, bool cum, Ld &load,
                                             uint32_t j_cur, int32_t d_cur, uint32_t j_nxt, int32_t d_nxt,
                                             uint32_t j_nc, int32_t d_nc, uint32_t j_nc1, int32_t d_nc1,
                                             unsigned long long (&acc)[G])
{
    uint32_t a[G];
#pragma unroll
    for (int g = 0; g < G; ++g)
        a[g] = a0[g];
    int32_t carry = 0;
    int base = 0;
    for (;;) {
        uint32_t w[G];
        if (base + lane < L) {
            load_cols<G>(colbits, j_cur, w);
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g)
                w[g] = 0u;
        }
        uint32_t hit = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            w[g] &= a[g];
            hit |= w[g];
        }
        if (!__any_sync(PM_FULL_MASK, hit != 0u)) {
            if (!cum)
                carry += __reduce_add_sync(PM_FULL_MASK, d_cur);
        } else {
            // running sum of Delta' up to this lane's rank = the sorted distance at that rank
            int32_t cs = d_cur;
            if (!cum) {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(PM_FULL_MASK, cs, o);
                    if (lane >= o)
                        cs += y;
                }
                cs += carry;
                carry = __shfl_sync(PM_FULL_MASK, cs, 31);
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                uint32_t hl = __ballot_sync(PM_FULL_MASK, w[g] != 0u);
                if (hl == 0u)
                    continue;
                if (__popc(hl) <= kWalkSparseLanes) {
                    uint32_t ag = a[g];
                    do {
                        const int r = __ffs(hl) - 1;
                        hl &= hl - 1u;
                        const uint32_t hb = __shfl_sync(PM_FULL_MASK, w[g], r) & ag;
                        const int32_t v = __shfl_sync(PM_FULL_MASK, cs, r);
                        if ((hb >> lane) & 1u)
                            acc[g] += (unsigned long long)(uint32_t)v;
                        ag &= ~hb;
                    } while (hl);
                    a[g] = ag;
                } else {
                    const uint32_t T = pm_transpose32(w[g], lane);
                    const int f = __ffs(T) - 1;
                    const int32_t v = __shfl_sync(PM_FULL_MASK, cs, f & 31);
                    if (T)
                        acc[g] += (unsigned long long)(uint32_t)v;
                    a[g] &= ~__ballot_sync(PM_FULL_MASK, T != 0u);
                }
            }
        }
        uint32_t left = 0;
#pragma unroll
        for (int g = 0; g < G; ++g)
            left |= a[g];
        base += 32;
        if (left != 0u && base < L) {
            j_cur = j_nxt;
            d_cur = d_nxt;
            load(c, base + 32, j_nxt, d_nxt);
            continue;
        }
        // next client of this warp: its first two steps were loaded a client ago; load the next one's
        c += step;
        if (c >= c_end)
            break;
        j_cur = j_nc;
        d_cur = d_nc;
        j_nxt = j_nc1;
        d_nxt = d_nc1;
        load(c + step, 0, j_nc, d_nc);
        load(c + step, 32, j_nc1, d_nc1);
        base = 0;
        carry = 0;
#pragma unroll
        for (int g = 0; g < G; ++g)
            a[g] = a0[g];
    }
}

