// cf_pair.cuh -- the persistent pair kernel (template; instantiated per kind in cf_pair_*.cu).
//
// Sec. 4.3-4.7 on a GPU.  Every warp repeatedly takes one work item -- an i tile of one cell
// (<= 128 points, four per lane as two packed pairs) against a j range (<= 512 points) of a
// neighbour cell -- from a global atomic cursor.  The i points sit in registers already
// translated by the cell-pair shift (Sec. 4.4, Code corrfunc_pbc: the shift is added once per
// i, not per pair).  Each j point is a broadcast load.
//
// Phase A (every pair): the separations and squared distance of two pairs at a time are formed
// by packed FP32x2 add / mul / fma on cell-relative coordinates -- with the shift's low part and
// the TwoSum residual of the i translation when ravg needs relative accuracy -- and each pair is
// tested against one cut: the FP32 value above which every value lies outside all bins (Sec.
// 4.7: squared space, no sqrt).  A lane keeps the values of a block of 16 pairs (4 j points x 4
// i points) in a lane-private buffer and their outcome in a bit mask.
// Compaction: the warp scans the mask counts and appends each candidate -- its FP32 value (and
// |dz| for rp-pi / wp) and a 16-bit code (i slot, j) -- to a per-warp ring in shared memory.
// Phase B (candidates only, 32 or 64 per pass, all lanes busy): the bin of the stored value is
// looked up on its FP32 bit pattern through a coarse table (cells holding an edge resolve
// through a fine entry of <= 2 thresholds).  A value within the proven FP32 error band of an
// edge is not binned: the pair goes to a global queue and is re-evaluated in FP64 by the
// recheck kernel, so counts equal the FP64 result.
//
// Histograms live in shared memory per warp (Sec. 4.8: private histograms, merged once): for
// r / theta / wp one private copy per lane (no bank conflicts, no contention; weighted sums
// Kahan-compensated in FP32), for rp-pi one copy per warp updated by shared atomics (FP64 for
// weighted sums).  They are merged into the global histogram when a warp moves to another job
// and at exit.
#pragma once
#include "cf_build.h"
#include "cf_device.cuh"

namespace cfpair {

constexpr int KIND_R = 0, KIND_RPPI = 1, KIND_WP = 2, KIND_THETA = 3;
constexpr uint32_t QM = CFI_QN - 1;

__host__ __device__ __forceinline__ uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// per-warp shared memory: block buffer | candidate ring | i weights | histogram
//   block buffer: the FP32 values phase A formed for one block of 16 pair slots per lane,
//                 [j][lane][slot] (and the same for |dz| in rp-pi and wp)
//   ring:         CFI_QN candidates: value bits (u32) [, |dz| bits (u32)], code (u16)
constexpr uint32_t SLOTS_PER_BLOCK = 16;
__host__ __device__ __forceinline__ uint32_t warp_hist_bytes(int kind, bool W, bool R, int nslot)
{
    if (kind == KIND_RPPI) {
        uint32_t b = ((uint32_t)nslot * 4u + 7u) & ~7u;
        if (W) b += nslot * 8u;
        if (R) b += nslot * 8u;
        return align16(b);
    }
    uint32_t b = nslot * 32u * 4u;
    if (W) b += nslot * 32u * 8u;
    if (R) b += nslot * 32u * 8u;
    return b;
}
__host__ __device__ __forceinline__ bool has_z(int kind) { return kind == KIND_RPPI || kind == KIND_WP; }
__host__ __device__ __forceinline__ uint32_t warp_buf_bytes(int kind) { return SLOTS_PER_BLOCK * 32u * 4u * (has_z(kind) ? 2u : 1u); }
__host__ __device__ __forceinline__ uint32_t warp_ring_bytes(int kind) { return CFI_QN * (has_z(kind) ? 10u : 6u); }
__host__ __device__ __forceinline__ uint32_t warp_stage_bytes(bool W) { return W ? 128u * 4u : 0u; }
constexpr uint32_t JSTAGE = 32;    // j points per staged chunk of the direct variant
__host__ __device__ __forceinline__ uint32_t warp_jbuf_bytes() { return 2u * JSTAGE * 32u; }   // 2 chunks x (pa, pb)
__host__ __device__ __forceinline__ uint32_t warp_bytes(int kind, bool W, bool R, int nslot, bool direct)
{
    if (direct) return warp_jbuf_bytes() + warp_hist_bytes(kind, W, R, nslot);
    return warp_buf_bytes(kind) + warp_ring_bytes(kind) + warp_stage_bytes(W) + warp_hist_bytes(kind, W, R, nslot);
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

// lookup for a value known to lie below the table's tail (the start of its final "outside
// every bin" segment): the index then never passes the last cell, so no upper clamp is needed
__device__ __forceinline__ uint32_t lut_class_in(const Lut &L, const CfFine *__restrict__ fine, uint32_t vb)
{
    const uint32_t t = max(vb, L.base) - L.base;
    uint32_t c = L.words[t >> L.shift];
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

__device__ __forceinline__ float wrap1(float d, float L, float invL) { return fmaf(-L, rintf(d * invL), d); }

__device__ __forceinline__ u64 wrap2(u64 d, float L, float invL)
{
    return f2_pack(wrap1(f2_lo(d), L, invL), wrap1(f2_hi(d), L, invL));
}

template <int KIND, bool W, bool R, bool WRAP, bool LO>
struct Warp {
    const CfPairArgs &a;
    Lut lr, lp;
    const CfFine *fine;
    uint32_t *h_cnt;        // lane-private [nslot][32] or per-warp [nslot]
    float2 *h_w, *h_r;      // lane-private Kahan pairs
    double *h_wd, *h_rd;    // per-warp FP64 (rp-pi)
    float *buf, *bufz;      // block buffer: [j][lane][slot]
    uint32_t *ring_d, *ring_z;
    uint16_t *ring_c;       // candidate code: (i slot << 9) | j
    float *stage_w;         // weights of the i tile
    ulonglong2 *jbuf;       // direct variant: 2 chunks of JSTAGE j points, pa then pb per chunk
    int lane, nb, npi, nslot;
    uint32_t icnt, ibeg, jbeg, job, head, tail;
    float cut_r, cut_p;
    float Lx, Ly, Lz, iLx, iLy, iLz;

    __device__ Warp(const CfPairArgs &args) : a(args) {}

    __device__ __forceinline__ void push(uint32_t ip, uint32_t jp)
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

    __device__ __forceinline__ float weight(uint32_t il, uint32_t j) const
    {
        return stage_w[il] * __ldg(reinterpret_cast<const float *>(a.pb + jbeg + j) + 2);
    }

    // Phase B for one candidate (valid == false: the lane only takes part in the warp's flow)
    __device__ __forceinline__ void finish(uint32_t vb, uint32_t zb, uint32_t code, bool valid)
    {
        const uint32_t il = code >> 9, j = code & (CFI_JMAX - 1);
        if (KIND == KIND_R || KIND == KIND_THETA) {
            const uint32_t c = lut_class(lr, fine, vb);
            if (valid && c < (uint32_t)nb) acc_lp(c, __uint_as_float(vb), W ? weight(il, j) : 0.f);
            else if (valid && c == CFI_CLS_AMB) push(ibeg + il, jbeg + j);
        } else {
            const uint32_t cz = lut_class(lp, fine, zb);
            const uint32_t cr = lut_class(lr, fine, vb);
            if (valid && cz != CFI_CLS_OUT && cr != CFI_CLS_OUT) {
                if (cr < (uint32_t)nb && cz < CFI_CLS_OUT) {
                    const float wp = W ? weight(il, j) : 0.f;
                    if (KIND == KIND_RPPI) acc_sh(cr * npi + cz, __uint_as_float(vb), wp);
                    else acc_lp(cr, __uint_as_float(vb), wp);
                } else {
                    push(ibeg + il, jbeg + j);
                }
            }
        }
    }

    // drain K*32 candidates (or the `count` left at the end) from the ring
    template <int K>
    __device__ __forceinline__ void drain(uint32_t count)
    {
        uint32_t vb[K], zb[K], code[K];
        bool v[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint32_t idx = lane + 32u * k;
            const uint32_t e = (head + idx) & QM;
            v[k] = idx < count;
            vb[k] = ring_d[e];
            zb[k] = has_z(KIND) ? ring_z[e] : 0u;
            code[k] = ring_c[e];
        }
#pragma unroll
        for (int k = 0; k < K; k++) finish(vb[k], zb[k], code[k], v[k]);
        head += count;
        __syncwarp();
    }

    template <int P, bool DIAG>
    __device__ __forceinline__ void run(const CfItem &it)
    {
        constexpr int SL = 2 * P;                           // pair slots per j per lane
        constexpr int JB = SLOTS_PER_BLOCK / SL;            // j points per block
        icnt = it.cnt & 0xFFFFu;
        const uint32_t jcnt = it.cnt >> 16;
        ibeg = it.ibeg;
        jbeg = it.jbeg;
        job = it.meta & CFI_ITEM_JOBMASK;
        // ---- i tile: translate by the shift; with ravg keep the TwoSum residual too ----
        u64 sx[P], sy[P], sz[P], ex[P], ey[P], ez[P];
#pragma unroll
        for (int p = 0; p < P; p++) {
            float vs[3][2], ve[3][2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t il = lane + 32u * (2 * p + h);
                float w = 0.f;
#pragma unroll
                for (int d = 0; d < 3; d++) { vs[d][h] = 1e18f; ve[d][h] = 0.f; }
                // empty slots sit far outside every bin (1e18^2 < FLT_MAX); in wrap mode the
                // minimum image would fold them back, so there they are also masked by icnt
                if (il < icnt) {
                    const ulonglong2 A = a.pa[ibeg + il], B = a.pb[ibeg + il];
                    const float X[3] = {-f2_lo(A.x), -f2_lo(A.y), -f2_lo(B.x)};
                    float XL[3] = {0.f, 0.f, 0.f};
                    if (LO) {
                        const ulonglong2 C = a.plo[2 * (size_t)(ibeg + il)], D = a.plo[2 * (size_t)(ibeg + il) + 1];
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
                        }
                    }
                    w = f2_lo(B.y);
                }
                if (W) stage_w[il] = w;
            }
            sx[p] = f2_pack(vs[0][0], vs[0][1]);
            sy[p] = f2_pack(vs[1][0], vs[1][1]);
            sz[p] = f2_pack(vs[2][0], vs[2][1]);
            ex[p] = f2_pack(ve[0][0], ve[0][1]);
            ey[p] = f2_pack(ve[1][0], ve[1][1]);
            ez[p] = f2_pack(ve[2][0], ve[2][1]);
        }
        __syncwarp();
        head = tail = 0;
        const ulonglong2 *__restrict__ pa = a.pa + jbeg;
        const ulonglong2 *__restrict__ pb = a.pb + jbeg;
        for (uint32_t j0 = 0; j0 < jcnt; j0 += JB) {
            // ---- phase A: the exact FP32 value phase B will bin, one cut per pair ----
            uint32_t mask = 0;
#pragma unroll
            for (int jj = 0; jj < JB; jj++) {
                const uint32_t j = j0 + jj;
                if (j < jcnt) {
                    const ulonglong2 A = __ldg(pa + j), B = __ldg(pb + j);
                    u64 lx = 0, ly = 0, lz = 0;
                    if (LO) {
                        const ulonglong2 C = __ldg(a.plo + 2 * (size_t)(jbeg + j));
                        const ulonglong2 D = __ldg(a.plo + 2 * (size_t)(jbeg + j) + 1);
                        lx = C.x;
                        ly = C.y;
                        lz = D.x;
                    }
                    float dv[SL], zv[SL];
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
                        bool c0, c1;
                        if (KIND == KIND_R || KIND == KIND_THETA) {
                            u64 d2 = f2_mul(dx, dx);
                            d2 = f2_fma(dy, dy, d2);
                            d2 = f2_fma(dz, dz, d2);
                            dv[2 * p] = f2_lo(d2);
                            dv[2 * p + 1] = f2_hi(d2);
                            c0 = dv[2 * p] < cut_r;
                            c1 = dv[2 * p + 1] < cut_r;
                        } else {
                            u64 rp2 = f2_mul(dx, dx);
                            rp2 = f2_fma(dy, dy, rp2);
                            const u64 adz = dz & 0x7FFFFFFF7FFFFFFFull;
                            dv[2 * p] = f2_lo(rp2);
                            dv[2 * p + 1] = f2_hi(rp2);
                            zv[2 * p] = f2_lo(adz);
                            zv[2 * p + 1] = f2_hi(adz);
                            c0 = dv[2 * p] < cut_r && zv[2 * p] < cut_p;
                            c1 = dv[2 * p + 1] < cut_r && zv[2 * p + 1] < cut_p;
                        }
                        const uint32_t il0 = lane + 64u * p, il1 = il0 + 32u;
                        if (DIAG) {
                            c0 = c0 && j > il0;
                            c1 = c1 && j > il1;
                        }
                        if (WRAP) {
                            c0 = c0 && il0 < icnt;
                            c1 = c1 && il1 < icnt;
                        }
                        const int bit = jj * SL + 2 * p;
                        mask |= (c0 ? 1u : 0u) << bit;
                        mask |= (c1 ? 1u : 0u) << (bit + 1);
                    }
                    float *bp = buf + ((uint32_t)jj * 32u + lane) * SL;
                    if (P == 2) *reinterpret_cast<float4 *>(bp) = make_float4(dv[0], dv[1], dv[2], dv[3]);
                    else *reinterpret_cast<float2 *>(bp) = make_float2(dv[0], dv[1]);
                    if (has_z(KIND)) {
                        float *zp = bufz + ((uint32_t)jj * 32u + lane) * SL;
                        if (P == 2) *reinterpret_cast<float4 *>(zp) = make_float4(zv[0], zv[1], zv[2], zv[3]);
                        else *reinterpret_cast<float2 *>(zp) = make_float2(zv[0], zv[1]);
                    }
                }
            }
            // ---- compaction into the warp's ring ----
            const uint32_t n = __popc(mask);
            uint32_t pre = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(CF_FULL, pre, o);
                if (lane >= o) pre += t;
            }
            const uint32_t tot = __shfl_sync(CF_FULL, pre, 31);
            uint32_t pos = tail + pre - n;
            while (mask) {
                const uint32_t b = (uint32_t)(__ffs(mask) - 1);
                mask &= mask - 1;
                const uint32_t q = b % SL, jj = b / SL;
                const uint32_t e = pos & QM;
                const uint32_t o = (jj * 32u + lane) * SL + q;
                ring_d[e] = __float_as_uint(buf[o]);
                if (has_z(KIND)) ring_z[e] = __float_as_uint(bufz[o]);
                ring_c[e] = (uint16_t)(((lane + 32u * q) << 9) | (j0 + jj));
                pos++;
            }
            tail += tot;
            __syncwarp();
            // ---- phase B ----
            while (tail - head >= 64) drain<2>(64);
        }
        while (tail - head >= 32) drain<1>(32);
        if (tail != head) drain<1>(tail - head);
    }

    // ---- direct variant: every pair is binned where it is formed (no compaction) ----
    // Bin one pair that passed the FP32 cut (squared separation below cut_r and, for rp-pi and
    // wp, |dz| below cut_p): both tables are then read without the upper clamp.
    __device__ __forceinline__ void bin_in(uint32_t vb, uint32_t zb, float wp, uint32_t il, uint32_t j)
    {
        if (KIND == KIND_R || KIND == KIND_THETA) {
            const uint32_t c = lut_class_in(lr, fine, vb);
            if (c < (uint32_t)nb) acc_lp(c, __uint_as_float(vb), wp);
            else if (c == CFI_CLS_AMB) push(ibeg + il, jbeg + j);
        } else {
            // the pi table starts at 0 with bin 0, so below cut_p it yields a bin or AMB
            const uint32_t cr = lut_class_in(lr, fine, vb);
            const uint32_t cz = lut_class_in(lp, fine, zb);
            if (max(cr, cz) < CFI_CLS_OUT) {
                if (KIND == KIND_RPPI) acc_sh(cr * npi + cz, __uint_as_float(vb), wp);
                else acc_lp(cr, __uint_as_float(vb), wp);
            } else if (cr != CFI_CLS_OUT) {
                push(ibeg + il, jbeg + j);
            }
        }
    }

    template <int P, bool DIAG>
    __device__ __forceinline__ void run_direct(const CfItem &it)
    {
        icnt = it.cnt & 0xFFFFu;
        const uint32_t jcnt = it.cnt >> 16;
        ibeg = it.ibeg;
        jbeg = it.jbeg;
        job = it.meta & CFI_ITEM_JOBMASK;
        u64 sx[P], sy[P], sz[P], ex[P], ey[P], ez[P], wi[P];
#pragma unroll
        for (int p = 0; p < P; p++) {
            float vs[3][2], ve[3][2], vw[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t il = lane + 32u * (2 * p + h);
                vw[h] = 0.f;
#pragma unroll
                for (int d = 0; d < 3; d++) { vs[d][h] = 1e18f; ve[d][h] = 0.f; }
                // empty slots sit far outside every bin (1e18^2 < FLT_MAX); in wrap mode the
                // minimum image would fold them back, so there they are also masked by icnt
                if (il < icnt) {
                    const ulonglong2 A = a.pa[ibeg + il], B = a.pb[ibeg + il];
                    const float X[3] = {-f2_lo(A.x), -f2_lo(A.y), -f2_lo(B.x)};
                    float XL[3] = {0.f, 0.f, 0.f};
                    if (LO) {
                        const ulonglong2 C = a.plo[2 * (size_t)(ibeg + il)], D = a.plo[2 * (size_t)(ibeg + il) + 1];
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
                        }
                    }
                    vw[h] = f2_lo(B.y);
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
        // j points stream through a double-buffered shared-memory stage: chunk c+1 is copied
        // asynchronously while chunk c is evaluated from broadcast shared loads
        const ulonglong2 *__restrict__ pa = a.pa + jbeg;
        const ulonglong2 *__restrict__ pb = a.pb + jbeg;
        const uint32_t nchunk = (jcnt + JSTAGE - 1) / JSTAGE;
        if (lane < jcnt) {
            cp_async16(jbuf + lane, pa + lane);
            cp_async16(jbuf + JSTAGE + lane, pb + lane);
        }
        cp_async_commit();
        for (uint32_t c = 0; c < nchunk; c++) {
            const uint32_t j0 = c * JSTAGE;
            if (c + 1 < nchunk) {
                ulonglong2 *nb2 = jbuf + ((c + 1) & 1) * 2 * JSTAGE;
                const uint32_t jn = j0 + JSTAGE + lane;
                if (jn < jcnt) {
                    cp_async16(nb2 + lane, pa + jn);
                    cp_async16(nb2 + JSTAGE + lane, pb + jn);
                }
            }
            cp_async_commit();
            cp_async_wait<1>();
            __syncwarp();
            const ulonglong2 *ca = jbuf + (c & 1) * 2 * JSTAGE;
            const uint32_t n = min(JSTAGE, jcnt - j0);
#pragma unroll 2
            for (uint32_t jj = 0; jj < n; jj++) {
                const uint32_t j = j0 + jj;
                const ulonglong2 A = ca[jj], B = ca[JSTAGE + jj];
                u64 lx = 0, ly = 0, lz = 0;
                if (LO) {
                    const ulonglong2 C = __ldg(a.plo + 2 * (size_t)(jbeg + j));
                    const ulonglong2 D = __ldg(a.plo + 2 * (size_t)(jbeg + j) + 1);
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
                    const uint32_t il0 = lane + 64u * p, il1 = il0 + 32u;
                    u64 v2, az = 0ull;
                    bool in0, in1;
                    if (KIND == KIND_R || KIND == KIND_THETA) {
                        v2 = f2_mul(dx, dx);
                        v2 = f2_fma(dy, dy, v2);
                        v2 = f2_fma(dz, dz, v2);
                        in0 = f2_lo(v2) < cut_r;
                        in1 = f2_hi(v2) < cut_r;
                    } else {
                        v2 = f2_mul(dx, dx);
                        v2 = f2_fma(dy, dy, v2);
                        az = dz & 0x7FFFFFFF7FFFFFFFull;
                        in0 = f2_lo(v2) < cut_r && f2_lo(az) < cut_p;
                        in1 = f2_hi(v2) < cut_r && f2_hi(az) < cut_p;
                    }
                    // within a cell paired with itself only j > i counts; in wrap mode the
                    // minimum image folds the far-away empty slots back, so mask them here
                    if (DIAG) {
                        in0 = in0 && j > il0;
                        in1 = in1 && j > il1;
                    }
                    if (WRAP) {
                        in0 = in0 && il0 < icnt;
                        in1 = in1 && il1 < icnt;
                    }
                    if (in0 || in1) {
                        const u64 wp = W ? f2_mul(wi[p], B.y) : 0ull;
                        if (in0) bin_in(f2_lo_bits(v2), f2_lo_bits(az), f2_lo(wp), il0, j);
                        if (in1) bin_in(f2_hi_bits(v2), f2_hi_bits(az), f2_hi(wp), il1, j);
                    }
                }
            }
            __syncwarp();       // the chunk buffer is refilled two chunks later
        }
        cp_async_wait<0>();
        __syncwarp();
    }

    __device__ void flush(uint32_t jb)
    {
        __syncwarp();
        const size_t g0 = (size_t)jb * nslot;
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

// resident CTAs (of 256 threads) the register budget is sized for: the compacting form is held
// to one CTA per SM by its shared memory; the direct form keeps 2 (weights / ravg) or 3 CTAs
__host__ __device__ constexpr int pair_min_blocks(bool W, bool R, bool DIRECT) { return !DIRECT ? 1 : ((W || R) ? 2 : 3); }

template <int KIND, bool W, bool R, bool WRAP, bool LO, bool DIRECT>
__global__ void __launch_bounds__(256, pair_min_blocks(W, R, DIRECT)) pair_kernel(const CfPairArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const CfDevPlan *__restrict__ P = a.plan;
    const int nlw = P->nlut_words, nf = P->nfine;
    uint32_t *s_lut = (uint32_t *)smem;
    CfFine *s_fine = (CfFine *)(smem + align16(4u * nlw));
    unsigned char *wbase = (unsigned char *)(s_fine + nf);
    for (int i = threadIdx.x; i < nlw; i += blockDim.x) s_lut[i] = a.lut[i];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) s_fine[i] = a.fine[i];
    const uint32_t wb = warp_bytes(KIND, W, R, a.nslot, DIRECT);
    const uint32_t hoff = DIRECT ? warp_jbuf_bytes() : warp_buf_bytes(KIND) + warp_ring_bytes(KIND) + warp_stage_bytes(W);
    unsigned char *my = wbase + (size_t)(threadIdx.x >> 5) * wb;
    {
        // zero this warp's histogram (the buffers need no initial value)
        uint32_t *h = (uint32_t *)(my + hoff);
        const uint32_t words = warp_hist_bytes(KIND, W, R, a.nslot) / 4u;
        for (uint32_t i = threadIdx.x & 31; i < words; i += 32) h[i] = 0u;
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
    w.cut_r = P->cut_r;
    w.cut_p = P->cut_p;
    w.Lx = a.L[0]; w.Ly = a.L[1]; w.Lz = a.L[2];
    w.iLx = a.L[0] > 0.f ? 1.0f / a.L[0] : 0.f;
    w.iLy = a.L[1] > 0.f ? 1.0f / a.L[1] : 0.f;
    w.iLz = a.L[2] > 0.f ? 1.0f / a.L[2] : 0.f;
    {
        const bool z = has_z(KIND);
        unsigned char *q = my;
        w.buf = (float *)q;
        w.bufz = (float *)(q + SLOTS_PER_BLOCK * 32u * 4u);
        q += warp_buf_bytes(KIND);
        w.ring_d = (uint32_t *)q;
        w.ring_z = (uint32_t *)(q + CFI_QN * 4u);
        w.ring_c = (uint16_t *)(q + CFI_QN * (z ? 8u : 4u));
        q += warp_ring_bytes(KIND);
        w.stage_w = (float *)q;
        w.jbuf = (ulonglong2 *)my;
    }
    w.h_cnt = (uint32_t *)(my + hoff);
    if (KIND == KIND_RPPI) {
        uint32_t o = ((uint32_t)a.nslot * 4u + 7u) & ~7u;
        w.h_wd = (double *)(my + hoff + o);
        w.h_rd = (double *)(my + hoff + o + (W ? a.nslot * 8u : 0u));
        w.h_w = w.h_r = nullptr;
    } else {
        uint32_t o = a.nslot * 32u * 4u;
        w.h_w = (float2 *)(my + hoff + o);
        w.h_r = (float2 *)(my + hoff + o + (W ? a.nslot * 32u * 8u : 0u));
        w.h_wd = w.h_rd = nullptr;
    }

    const uint32_t nitems = min(*a.nitems_dev, a.items_cap);
    int cur = -1;
    // the next item's index and descriptor are fetched before the current item is processed
    uint32_t t = 0;
    if (w.lane == 0) t = atomicAdd(a.cursor, 1u);
    t = __shfl_sync(CF_FULL, t, 0);
    CfItem it;
    if (t < nitems) it = a.items[t];
    for (;;) {
        if (t >= nitems) break;
        uint32_t tn = 0;
        if (w.lane == 0) tn = atomicAdd(a.cursor, 1u);
        tn = __shfl_sync(CF_FULL, tn, 0);
        CfItem nx;
        if (tn < nitems) nx = a.items[tn];
        const int job = (int)(it.meta & CFI_ITEM_JOBMASK);
        if (job != cur) {
            if (cur >= 0) w.flush((uint32_t)cur);
            cur = job;
        }
        const bool diag = (it.meta & CFI_ITEM_DIAG) != 0;
        if (DIRECT) {
            if (it.meta & CFI_ITEM_P2) {
                if (diag) w.template run_direct<2, true>(it);
                else w.template run_direct<2, false>(it);
            } else {
                if (diag) w.template run_direct<1, true>(it);
                else w.template run_direct<1, false>(it);
            }
        } else if (it.meta & CFI_ITEM_P2) {
            if (diag) w.template run<2, true>(it);
            else w.template run<2, false>(it);
        } else {
            if (diag) w.template run<1, true>(it);
            else w.template run<1, false>(it);
        }
        t = tn;
        it = nx;
    }
    if (cur >= 0) w.flush((uint32_t)cur);
}

template <int KIND, bool W, bool R, bool WRAP, bool LO, bool DIRECT>
cudaError_t launch_variant(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                           int *warps_out)
{
    auto k = pair_kernel<KIND, W, R, WRAP, LO, DIRECT>;
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

// variant 1 = direct, 2 = compacting (0 picks one per kind: see cfp_default_variant)
template <int KIND, bool W, bool R, bool WRAP, bool LO>
cudaError_t launch_one(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                       int *warps_out)
{
    if (c.variant == 2) return launch_variant<KIND, W, R, WRAP, LO, false>(c, a, num_sms, st, grid_out, warps_out);
    return launch_variant<KIND, W, R, WRAP, LO, true>(c, a, num_sms, st, grid_out, warps_out);
}

}  // namespace cfpair
