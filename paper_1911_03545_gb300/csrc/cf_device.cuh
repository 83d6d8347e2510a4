// cf_device.cuh -- device helpers shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cf_internal.h"

#define CF_FULL 0xFFFFFFFFu

typedef unsigned long long u64;

// ---- packed FP32 pairs (PTX f32x2, sm_100+): lane h of a u64 is float h ----
__device__ __forceinline__ u64 f2_add(u64 a, u64 b)
{
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 f2_mul(u64 a, u64 b)
{
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 f2_fma(u64 a, u64 b, u64 c)
{
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ u64 f2_pack(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(u64 v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(u64 v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint32_t f2_lo_bits(u64 v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t f2_hi_bits(u64 v) { return (uint32_t)(v >> 32); }

// ---- asynchronous global -> shared copies (16 or 4 bytes per lane), grouped and awaited by group ----
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// sqrt.approx.f32: relative error within a few ulp; used only for ravg sums (1e-6 tolerance)
__device__ __forceinline__ float f_sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- cell origin: precomputed on the host (cfp_origin in cf_plan.cpp) ----
__device__ __forceinline__ double cf_origin(const CfDevPlan *plan, int a, int i) { return plan->origin[plan->ooff[a] + i]; }
// origin of cell c on axis a: the 3-D grid's per-axis table (index ia), or the angular grid's per-cell one
__device__ __forceinline__ double cf_cell_origin(const CfDevPlan *plan, int a, int c, int ia)
{
    return plan->ang ? plan->origin[3 * c + a] : plan->origin[plan->ooff[a] + ia];
}
// band of a cell of the angular grid (binary search over the band bases)
__device__ __forceinline__ int cf_band_of(const CfDevPlan *plan, int c)
{
    int lo = 0, hi = plan->nband - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (plan->band[m].base <= c) lo = m;
        else hi = m - 1;
    }
    return lo;
}

__device__ __forceinline__ int cf_cell_axis(const CfGrid &g, int a, double x)
{
    double t = (x - g.lo[a]) * g.inv[a];
    int i = (int)floor(t);
    if (i < 0) i = 0;
    if (i > g.n[a] - 1) i = g.n[a] - 1;
    return i;
}

__device__ __forceinline__ double cf_load(const void *p, int dtype, int64_t i)
{
    return dtype ? ((const double *)p)[i] : (double)((const float *)p)[i];
}

// order-preserving map of a double to an unsigned 64-bit key (for atomic min / max)
__device__ __forceinline__ unsigned long long cf_dkey(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
