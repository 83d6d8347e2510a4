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
__device__ __forceinline__ u64 f2_sub(u64 a, u64 b)
{
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
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
// the same origin as float32 (exact)
__device__ __forceinline__ float cf_cell_origin32(const CfDevPlan *plan, int a, int c, int ia)
{
    return plan->ang ? plan->origin32[3 * c + a] : plan->origin32[plan->ooff[a] + ia];
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

// DD(rp, pi) of observed positions in FP64, as the result definition states it (Appendix A.2.1,
// the line of sight of Fisher et al.): s = a - b, l = 0.5 (a + b) per axis; s.l, l.l and s.s as
// ((x + y) + z) sums of products; pi^2 = (s.l)^2 / l.l (0 when l.l = 0); rp^2 = s.s - pi^2,
// clamped at 0.  Explicit round-to-nearest operations, no fused multiply-add.
__device__ __forceinline__ void cf_mocks64(double ax, double ay, double az, double bx, double by, double bz,
                                           double &rp2, double &pi2)
{
    const double sx = __dsub_rn(ax, bx), sy = __dsub_rn(ay, by), sz = __dsub_rn(az, bz);
    const double lx = __dmul_rn(0.5, __dadd_rn(ax, bx));
    const double ly = __dmul_rn(0.5, __dadd_rn(ay, by));
    const double lz = __dmul_rn(0.5, __dadd_rn(az, bz));
    const double sl = __dadd_rn(__dadd_rn(__dmul_rn(sx, lx), __dmul_rn(sy, ly)), __dmul_rn(sz, lz));
    const double ll = __dadd_rn(__dadd_rn(__dmul_rn(lx, lx), __dmul_rn(ly, ly)), __dmul_rn(lz, lz));
    const double ss = __dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)), __dmul_rn(sz, sz));
    pi2 = ll > 0.0 ? __ddiv_rn(__dmul_rn(sl, sl), ll) : 0.0;
    rp2 = __dsub_rn(ss, pi2);
    if (rp2 < 0.0) rp2 = 0.0;
}
