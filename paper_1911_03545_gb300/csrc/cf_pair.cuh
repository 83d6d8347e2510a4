// cf_pair.cuh -- the persistent pair kernel (template; instantiated per kind in cf_pair_*.cu).
//
// Sec. 4.3-4.7 on a GPU: every warp repeatedly takes one work item -- an i tile of one cell
// (<= 128 points, two per lane per pack) against a j range of a neighbour cell -- from a global
// atomic cursor.  The i points sit in registers already translated by the cell-pair shift
// (Sec. 4.4, Code corrfunc_pbc: the shift is added once per i, not per pair).  Each j point is
// a broadcast load; the three separations and the squared distance of two pairs are formed by
// packed FP32x2 add / mul / fma on cell-relative coordinates.  The bin is found on the bit
// pattern of the FP32 squared separation with a coarse table (Sec. 4.7: squared space, no
// sqrt); cells of the table that hold an edge resolve through a fine entry of <= 2 thresholds.
// A value within the proven FP32 error band of an edge is not binned here: the pair goes to a
// queue and is re-evaluated in FP64 by the recheck kernel, so counts equal the FP64 result.
// Histograms live in shared memory per warp (Sec. 4.8: private histograms, merged once): for
// r / theta / wp one private copy per lane (no conflicts, no atomics contention; weighted sums
// are Kahan-compensated FP32), for rp-pi one copy per warp with shared atomics.  They are
// merged into the global FP64/u64 histogram when a warp moves to another job and at exit.
#pragma once
#include "cf_build.h"
#include "cf_device.cuh"

namespace cfpair {

constexpr int KIND_R = 0, KIND_RPPI = 1, KIND_WP = 2, KIND_THETA = 3;

__device__ __forceinline__ uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

template <int KIND, bool W, bool R>
__host__ __device__ __forceinline__ uint32_t warp_hist_bytes(int nslot)
{
    if (KIND == KIND_RPPI) {
        uint32_t b = ((uint32_t)nslot * 4u + 7u) & ~7u;
        if (W) b += nslot * 8u;
        if (R) b += nslot * 8u;
        return (b + 15u) & ~15u;
    }
    uint32_t b = nslot * 32u * 4u;
    if (W) b += nslot * 32u * 8u;
    if (R) b += nslot * 32u * 8u;
    return b;
}

__device__ __forceinline__ void kahan_add(float2 *p, float v)
{
    float2 sc = *p;
    float y = v - sc.y;
    float t = sc.x + y;
    sc.y = (t - sc.x) - y;
    sc.x = t;
    *p = sc;
}

struct Lut {
    uint32_t base, shift, last;
    const uint32_t *words;   // shared
};

__device__ __forceinline__ uint32_t lut_class(const Lut &L, const CfFine *__restrict__ fine, uint32_t vb)
{
    int t = (int)(vb - L.base);
    t = t > 0 ? t : 0;
    uint32_t idx = min((uint32_t)t >> L.shift, L.last);
    uint32_t c = L.words[idx];
    if (c >= CFI_FINE_FLAG) {
        const CfFine f = fine[c - CFI_FINE_FLAG];
        uint32_t seg = (vb >= f.t1 ? 1u : 0u) + (vb >= f.t2 ? 1u : 0u);
        c = (f.code >> (8u * seg)) & 0xFFu;
    }
    return c;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ u64 wrap2(u64 d, float L, float invL)
{
    float a = f2_lo(d), b = f2_hi(d);
    a = fmaf(-L, rintf(a * invL), a);
    b = fmaf(-L, rintf(b * invL), b);
    return f2_pack(a, b);
}

template <int KIND, bool W, bool R, bool WRAP, bool LO>
struct Warp {
    // per-kernel constants
    const CfPairArgs &a;
    Lut lr, lp;
    const CfFine *fine;
    uint32_t *h_cnt;        // lane-private [nslot][32] or per-warp [nslot]
    float2 *h_w, *h_r;      // lane-private Kahan pairs
    double *h_wd, *h_rd;    // per-warp FP64 (rp-pi)
    int lane, nb, npi, nslot;
    uint32_t icnt;          // points of the current i tile (wrap mode masks empty slots with it)
    float Lx, Ly, Lz, iLx, iLy, iLz;

    __device__ Warp(const CfPairArgs &args) : a(args) {}

    __device__ __forceinline__ void push(uint32_t ip, uint32_t jp, uint32_t job)
    {
        uint32_t k = atomicAdd(a.qcount, 1u);
        if (k < a.qcap) a.queue[k] = make_uint4(a.orig[ip], a.orig[jp], job, 0u);
    }

    __device__ __forceinline__ void acc_lp(uint32_t c, float d2, float wp)
    {
        uint32_t idx = c * 32u + lane;
        atomicAdd(h_cnt + idx, 1u);
        if (W) kahan_add(h_w + idx, wp);
        if (R) {
            float r = f_sqrt_approx(d2);
            if (KIND == KIND_THETA) r = 2.0f * asinf(0.5f * r) * 57.29577951308232f;
            kahan_add(h_r + idx, W ? wp * r : r);
        }
    }

    __device__ __forceinline__ void acc_sh(uint32_t slot, float rp2, float wp)
    {
        atomicAdd(h_cnt + slot, 1u);
        if (W) atomicAdd(h_wd + slot, (double)wp);
        if (R) {
            float r = f_sqrt_approx(rp2);
            atomicAdd(h_rd + slot, (double)(W ? wp * r : r));
        }
    }

    // one pair (one half of a packed result)
    template <bool DIAG>
    __device__ __forceinline__ void bin3(uint32_t vb, float wp, uint32_t il, uint32_t j, uint32_t ibeg,
                                         uint32_t jbeg, uint32_t job)
    {
        uint32_t c = lut_class(lr, fine, vb);
        bool live = (!DIAG || j > il) && (!WRAP || il < icnt);
        if (c < (uint32_t)nb) {
            if (live) acc_lp(c, __uint_as_float(vb), wp);
        } else if (c == CFI_CLS_AMB) {
            if (live) push(ibeg + il, jbeg + j, job);
        }
    }

    template <bool DIAG>
    __device__ __forceinline__ void bin2(uint32_t rb, uint32_t zb, float wp, uint32_t il, uint32_t j,
                                         uint32_t ibeg, uint32_t jbeg, uint32_t job)
    {
        uint32_t cz = lut_class(lp, fine, zb);
        if (cz == CFI_CLS_OUT) return;
        uint32_t cr = lut_class(lr, fine, rb);
        bool live = (!DIAG || j > il) && (!WRAP || il < icnt);
        if (cr < (uint32_t)nb && cz < CFI_CLS_OUT) {
            if (live) {
                if (KIND == KIND_RPPI) acc_sh(cr * npi + cz, __uint_as_float(rb), wp);
                else acc_lp(cr, __uint_as_float(rb), wp);
            }
        } else if (cr != CFI_CLS_OUT) {
            if (live) push(ibeg + il, jbeg + j, job);
        }
    }

    template <int P, bool DIAG>
    __device__ __forceinline__ void run(const CfItem &it)
    {
        const uint32_t icnt = it.cnt & 0xFFFFu, jcnt = it.cnt >> 16;
        const uint32_t job = it.meta & CFI_ITEM_JOBMASK;
        this->icnt = icnt;
        u64 sx[P], sy[P], sz[P], ex[P], ey[P], ez[P], wi[P];
#pragma unroll
        for (int p = 0; p < P; p++) {
            float vs[3][2], ve[3][2], vw[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                uint32_t il = lane + 32u * (2 * p + h);
                if (il < icnt) {
                    const ulonglong2 A = a.pa[it.ibeg + il], B = a.pb[it.ibeg + il];
                    float X[3] = {-f2_lo(A.x), -f2_lo(A.y), -f2_lo(B.x)};
                    vw[h] = f2_lo(B.y);
                    float XL[3] = {0.f, 0.f, 0.f};
                    if (LO) {
                        const ulonglong2 C = a.plo[2 * (size_t)(it.ibeg + il)], D = a.plo[2 * (size_t)(it.ibeg + il) + 1];
                        XL[0] = -f2_lo(C.x);
                        XL[1] = -f2_lo(C.y);
                        XL[2] = -f2_lo(D.x);
                    }
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        if (R) {
                            float s, e;
                            two_sum(X[d], it.s[d], s, e);
                            vs[d][h] = s;
                            ve[d][h] = (e + it.slo[d]) + XL[d];
                        } else {
                            vs[d][h] = X[d] + it.s[d];
                            ve[d][h] = 0.f;
                        }
                    }
                } else {
                    // empty slot: far outside every bin (1e18^2 < FLT_MAX); in wrap mode the
                    // minimum image would fold it back, so there the slot is also masked by icnt
#pragma unroll
                    for (int d = 0; d < 3; d++) { vs[d][h] = 1e18f; ve[d][h] = 0.f; }
                    vw[h] = 0.f;
                }
            }
            sx[p] = f2_pack(vs[0][0], vs[0][1]);
            sy[p] = f2_pack(vs[1][0], vs[1][1]);
            sz[p] = f2_pack(vs[2][0], vs[2][1]);
            ex[p] = f2_pack(ve[0][0], ve[0][1]);
            ey[p] = f2_pack(ve[1][0], ve[1][1]);
            ez[p] = f2_pack(ve[2][0], ve[2][1]);
            wi[p] = f2_pack(vw[0], vw[1]);
        }
        const ulonglong2 *__restrict__ pa = a.pa + it.jbeg;
        const ulonglong2 *__restrict__ pb = a.pb + it.jbeg;
#pragma unroll 2
        for (uint32_t j = 0; j < jcnt; j++) {
            const ulonglong2 A = __ldg(pa + j), B = __ldg(pb + j);
            u64 lx = 0, ly = 0, lz = 0;
            if (LO) {
                const ulonglong2 C = __ldg(a.plo + 2 * (size_t)(it.jbeg + j));
                const ulonglong2 D = __ldg(a.plo + 2 * (size_t)(it.jbeg + j) + 1);
                lx = C.x;
                ly = C.y;
                lz = D.x;
            }
#pragma unroll
            for (int p = 0; p < P; p++) {
                u64 dx = f2_add(sx[p], A.x), dy = f2_add(sy[p], A.y), dz = f2_add(sz[p], B.x);
                if (R) {
                    dx = f2_add(dx, LO ? f2_add(ex[p], lx) : ex[p]);
                    dy = f2_add(dy, LO ? f2_add(ey[p], ly) : ey[p]);
                    dz = f2_add(dz, LO ? f2_add(ez[p], lz) : ez[p]);
                }
                if (WRAP) {
                    if (Lx > 0.f) dx = wrap2(dx, Lx, iLx);
                    if (Ly > 0.f) dy = wrap2(dy, Ly, iLy);
                    if (Lz > 0.f) dz = wrap2(dz, Lz, iLz);
                }
                u64 wp = 0;
                if (W) wp = f2_mul(wi[p], B.y);
                const uint32_t il0 = lane + 64u * p, il1 = il0 + 32u;
                if (KIND == KIND_R || KIND == KIND_THETA) {
                    u64 d2 = f2_mul(dx, dx);
                    d2 = f2_fma(dy, dy, d2);
                    d2 = f2_fma(dz, dz, d2);
                    bin3<DIAG>(f2_lo_bits(d2), f2_lo(wp), il0, j, it.ibeg, it.jbeg, job);
                    bin3<DIAG>(f2_hi_bits(d2), f2_hi(wp), il1, j, it.ibeg, it.jbeg, job);
                } else {
                    u64 rp2 = f2_mul(dx, dx);
                    rp2 = f2_fma(dy, dy, rp2);
                    u64 adz = dz & 0x7FFFFFFF7FFFFFFFull;
                    bin2<DIAG>(f2_lo_bits(rp2), f2_lo_bits(adz), f2_lo(wp), il0, j, it.ibeg, it.jbeg, job);
                    bin2<DIAG>(f2_hi_bits(rp2), f2_hi_bits(adz), f2_hi(wp), il1, j, it.ibeg, it.jbeg, job);
                }
            }
        }
    }

    __device__ void flush(uint32_t job)
    {
        __syncwarp();
        const size_t g0 = (size_t)job * nslot;
        for (int sl = lane; sl < nslot; sl += 32) {
            unsigned long long c = 0;
            double ws = 0.0, rs = 0.0;
            if (KIND == KIND_RPPI) {
                c = h_cnt[sl];
                h_cnt[sl] = 0;
                if (W) { ws = h_wd[sl]; h_wd[sl] = 0.0; }
                if (R) { rs = h_rd[sl]; h_rd[sl] = 0.0; }
            } else {
                for (int l = 0; l < 32; l++) {
                    int idx = sl * 32 + ((l + lane) & 31);
                    c += h_cnt[idx];
                    h_cnt[idx] = 0;
                    if (W) {
                        float2 v = h_w[idx];
                        ws += (double)v.x - (double)v.y;
                        h_w[idx] = make_float2(0.f, 0.f);
                    }
                    if (R) {
                        float2 v = h_r[idx];
                        rs += (double)v.x - (double)v.y;
                        h_r[idx] = make_float2(0.f, 0.f);
                    }
                }
            }
            if (c) atomicAdd(a.hcnt + g0 + sl, c);
            if (W && ws != 0.0) atomicAdd(a.hw + g0 + sl, ws);
            if (R && rs != 0.0) atomicAdd(a.hr + g0 + sl, rs);
        }
        __syncwarp();
    }
};

template <int KIND, bool W, bool R, bool WRAP, bool LO>
__global__ void __launch_bounds__(256) pair_kernel(const CfPairArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const CfDevPlan *__restrict__ P = a.plan;
    const int nlw = P->nlut_words, nf = P->nfine;
    uint32_t *s_lut = (uint32_t *)smem;
    CfFine *s_fine = (CfFine *)(smem + align16(4u * nlw));
    unsigned char *hist = (unsigned char *)(s_fine + nf);
    for (int i = threadIdx.x; i < nlw; i += blockDim.x) s_lut[i] = a.lut[i];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) s_fine[i] = a.fine[i];
    const uint32_t wb = warp_hist_bytes<KIND, W, R>(a.nslot);
    {
        uint32_t *h = (uint32_t *)hist;
        const uint32_t words = wb * (blockDim.x >> 5) / 4u;
        for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) h[i] = 0u;
    }
    __syncthreads();

    Warp<KIND, W, R, WRAP, LO> w(a);
    w.lane = threadIdx.x & 31;
    w.nb = a.nb;
    w.npi = a.npi;
    w.nslot = a.nslot;
    w.fine = s_fine;
    w.lr = {P->lr.base, P->lr.shift, P->lr.last, s_lut + P->lr.coff};
    w.lp = {P->lp.base, P->lp.shift, P->lp.last, s_lut + P->lp.coff};
    w.Lx = a.L[0]; w.Ly = a.L[1]; w.Lz = a.L[2];
    w.iLx = a.L[0] > 0.f ? 1.0f / a.L[0] : 0.f;
    w.iLy = a.L[1] > 0.f ? 1.0f / a.L[1] : 0.f;
    w.iLz = a.L[2] > 0.f ? 1.0f / a.L[2] : 0.f;
    unsigned char *my = hist + (size_t)(threadIdx.x >> 5) * wb;
    w.h_cnt = (uint32_t *)my;
    if (KIND == KIND_RPPI) {
        uint32_t o = ((uint32_t)a.nslot * 4u + 7u) & ~7u;
        w.h_wd = (double *)(my + o);
        w.h_rd = (double *)(my + o + (W ? a.nslot * 8u : 0u));
        w.h_w = w.h_r = nullptr;
    } else {
        uint32_t o = a.nslot * 32u * 4u;
        w.h_w = (float2 *)(my + o);
        w.h_r = (float2 *)(my + o + (W ? a.nslot * 32u * 8u : 0u));
        w.h_wd = w.h_rd = nullptr;
    }

    const uint32_t nitems = min(*a.nitems_dev, a.items_cap);
    int cur = -1;
    for (;;) {
        uint32_t t = 0;
        if (w.lane == 0) t = atomicAdd(a.cursor, 1u);
        t = __shfl_sync(CF_FULL, t, 0);
        if (t >= nitems) break;
        const CfItem it = a.items[t];
        const int job = (int)(it.meta & CFI_ITEM_JOBMASK);
        if (job != cur) {
            if (cur >= 0) w.flush((uint32_t)cur);
            cur = job;
        }
        const bool diag = (it.meta & CFI_ITEM_DIAG) != 0;
        if (it.meta & CFI_ITEM_P2) {
            if (diag) w.template run<2, true>(it);
            else w.template run<2, false>(it);
        } else {
            if (diag) w.template run<1, true>(it);
            else w.template run<1, false>(it);
        }
    }
    if (cur >= 0) w.flush((uint32_t)cur);
}

template <int KIND, bool W, bool R, bool WRAP, bool LO>
cudaError_t launch_one(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                       int *warps_out)
{
    auto k = pair_kernel<KIND, W, R, WRAP, LO>;
    int dev;
    cudaGetDevice(&dev);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int warps = c.warps > 0 ? (c.warps > 8 ? 8 : c.warps) : 8;
    size_t smem = 0;
    for (; warps >= 1; warps--) {
        smem = cfp_pair_smem(c, warps);
        if (smem <= (size_t)maxsm) break;
    }
    if (warps < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = c.ctas_per_sm;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, warps * 32, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    int grid = per_sm * num_sms;
    k<<<grid, warps * 32, smem, st>>>(a);
    if (grid_out) *grid_out = grid;
    if (warps_out) *warps_out = warps;
    return cudaGetLastError();
}

}  // namespace cfpair
