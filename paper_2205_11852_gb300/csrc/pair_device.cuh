// Device helpers shared by the pair-count kernels (Sect. 2.1 counts, Sect.
// 4.3 bins): the exact integer bin of a pair, the hardware reciprocal
// square root, a warp prefix sum and 32-bit shared-memory addresses.
#pragma once

#include "plan.h"

namespace tpcf {
namespace {

typedef unsigned __int128 u128;
typedef __int128 i128;

// Exact bin of the pair (ia, ib) from integer grid coordinates; -1 if unbinned.
__device__ __noinline__ int exact_bin(const CountParams &prm, const unsigned long long *T,
                                      const uint32_t *__restrict__ us, uint32_t N, uint32_t ia, uint32_t ib)
{
    long long d[3];
    uint32_t ua[3], ub[3];
    unsigned long long D2 = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        ua[c] = us[(size_t)c * N + ia];
        ub[c] = us[(size_t)c * N + ib];
        d[c] = (prm.geometry == TPCF_PERIODIC) ? (long long)(int)(ua[c] - ub[c])
                                               : (long long)ua[c] - (long long)ub[c];
        D2 += (unsigned long long)(d[c] * d[c]);
    }
    const int n_s = prm.n_s;
    if (D2 < T[0] || D2 >= T[n_s]) return -1;
    int lo = 0, hi = n_s - 1;        // largest k with T[k] <= D2
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T[mid] <= D2) lo = mid; else hi = mid - 1;
    }
    const int k = lo;
    const int n_mu = prm.n_mu;
    int j = 0;
    if (n_mu > 1) {
        u128 num, den;
        if (prm.los == TPCF_LOS_X) {
            num = (u128)(unsigned long long)(d[0] * d[0]);
            den = (u128)D2;
        } else {
            i128 dot = 0;
            u128 l2 = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const i128 l = (i128)ua[c] + (i128)ub[c] - 2 * (i128)prm.obs[c];
                dot += (i128)d[c] * l;
                l2 += (u128)(l * l);
            }
            const u128 ad = (u128)(dot < 0 ? -dot : dot);
            num = ad * ad;
            den = (u128)D2 * l2;
        }
        if (den != 0) {
            const u128 lhs = (u128)(unsigned)(n_mu * n_mu) * num;
            j = n_mu - 1;
            while (j > 0 && lhs < (u128)(unsigned)(j * j) * den) j--;
        }
    }
    return k * n_mu + j;
}

__device__ __forceinline__ uint32_t warp_exclusive_sum(uint32_t v, int lane, uint32_t &total)
{
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// MUFU reciprocal square root without denormal handling (relative error
// within 2 ulp); every use carries that error in its ambiguity band
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 32-bit shared-memory accesses (addresses from __cvta_generic_to_shared)
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

}  // namespace
// Global nanosecond timer.
__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Lane 0 of each warp at the end of a pair-count launch: stats[4] = max of
// ~start (so ~stats[4] is the earliest start), stats[5] = latest end,
// stats[6] = sum of the warps' spans, stats[7] = warps.  The launch's idle
// fraction 1 - stats[6] / (stats[7] (stats[5] - ~stats[4])) is the share of
// warp time spent finished while others still worked (the last-wave tail).
__device__ __forceinline__ void record_warp_span(unsigned long long *stats, unsigned long long t0)
{
    const unsigned long long t1 = gtimer();
    atomicMax(&stats[4], ~t0);
    atomicMax(&stats[5], t1);
    atomicAdd(&stats[6], t1 - t0);
    atomicAdd(&stats[7], 1ull);
}

}  // namespace tpcf
