// cf_pair.cuh -- the persistent pair kernel (template; instantiated per kind in cf_pair_*.cu).
//
// Sec. 4.3-4.7 on a GPU.  Every warp repeatedly takes one work item -- an i tile of one cell
// (<= 128 points) against a j range (<= 512 points) of a neighbour cell -- from a global atomic
// cursor (in the order of cfb_order: items of one instance together).  Lane l holds the i points
// l + 32 q (q < Q; Q = 1 to 4 by the tile's size, mocks 1, 2 or 4) in
// registers, already translated by the cell-pair shift (Sec. 4.4, Code corrfunc_pbc: the shift
// is added once per i, not per pair), each duplicated into both halves of a packed FP32 pair.
// The j points stream through a double-buffered shared-memory stage (cp.async) as float arrays
// and are read two at a time by broadcast 8-byte loads: one packed add forms the separations of
// an i point from two j points.
//
// Per pair: the separation and squared distance by packed FP32x2 add / mul / fma on
// cell-relative coordinates -- with the shift's low part and the TwoSum residual of the i
// translation when ravg needs relative accuracy -- and one cut: the FP32 value from which on
// every value lies outside all bins (Sec. 4.7: squared space, no sqrt; rp-pi and wp also cut
// |dz|).  A pair below the cut is binned on its FP32 bit pattern through a coarse table (cells
// holding an edge resolve through a fine entry of <= 2 thresholds).  A value within the proven
// FP32 error band of an edge is not binned: the pair goes to a global queue and is re-evaluated
// in FP64 by the recheck kernel, so counts equal the FP64 result.
//
// Two forms of that binning step, with identical results:
//   direct     (variant 1): each lane bins its own pairs below the cut where they are formed;
//   compacting (variant 2): the warp appends its pairs below the cut (value bits, |dz| bits,
//              i/j code, weight product) to a per-warp ring in shared memory at offsets from a
//              ballot prefix sum, and bins them 32 at a time with every lane busy.
//
// Histograms live in shared memory per warp (Sec. 4.8: private histograms, merged once): for
// r / theta / wp one private copy per lane (no bank conflicts, no contention; weighted sums
// Kahan-compensated in FP32), for rp-pi one copy per warp updated by shared atomics (weight and
// ravg sums in fixed point where the host found scales for the terms' range, else FP64).  They are
// merged into the global histogram when a warp moves to another job, after every 2^28 evaluated
// pairs (2^18 with fixed-point sums), and at exit.
//
// The fixed-point sums use 32-bit shared atomics only (64-bit shared atomics are several times
// slower): a term t adds m = round(t * S) (S a power of two the host chose so that every term of
// the sum lies in [2^21, 2^26) units, so that rounding moves a term by at most 2^-22 of itself) to
// two 32-bit words of its slot, m modulo 2^32 and m >> 12.  A warp flushes before its slots can
// hold 2^18 terms: the second word then stays below 2^32 and places the true sum within 2^30 below
// its value times 2^12, and the first word gives the sum exactly (fx_sum).
#pragma once
#include "cf_build.h"
#include "cf_device.cuh"

namespace cfpair {

constexpr int KIND_R = 0, KIND_RPPI = 1, KIND_WP = 2, KIND_THETA = 3, KIND_MOCKS = 4;

// rp-pi kinds keep one histogram per warp updated by shared atomics (nb * npi slots)
__host__ __device__ constexpr bool warp_hist(int kind) { return kind == KIND_RPPI || kind == KIND_MOCKS; }

__host__ __device__ __forceinline__ uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// per-warp shared memory: j stage | candidate ring (compacting form) | histogram
//   j stage: 2 chunks x 3-7 float arrays (x, y, z[, w][, lo parts of x, y, z]) of JSTAGE points
//   ring:    RING candidates as arrays: value bits, |dz| bits (rp-pi, wp), weight product (W),
//            code (u16: i slot | j << 7)
// a warp flushes its histograms once it has evaluated more than this many pairs of one job;
// with the item in hand that keeps every flushed batch at <= 2^28 pairs (an item: <= 2^16)
constexpr uint32_t CF_FLUSH_PAIRS = (1u << 28) - (1u << 16);
// with fixed-point sums: fewer than 2^18 terms per slot between flushes
constexpr uint32_t FX_FLUSH_PAIRS = (1u << 18) - (1u << 16);
constexpr uint32_t FX_HI_SHIFT = 12;

// True sum of the fixed-point terms of a slot from its two words: lo = the sum modulo 2^32, hi = the
// sum of (m >> 12).  For fewer than 2^18 terms below 2^26, hi * 2^12 lies in (T - 2^30, T].
__device__ __forceinline__ unsigned long long fx_sum(uint32_t lo, uint32_t hi)
{
    const unsigned long long c = (unsigned long long)hi << FX_HI_SHIFT;
    return c + (uint32_t)(lo - (uint32_t)c);
}
constexpr uint32_t JSTAGE = 32;
constexpr uint32_t RING = 512;
constexpr uint32_t RM = RING - 1;
static_assert(CFI_JMAX <= 512, "a ring code holds a 7-bit i slot and a 9-bit j");
__host__ __device__ __forceinline__ uint32_t warp_hist_bytes(int kind, bool W, bool R, int nslot)
{
    if (warp_hist(kind)) {
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
__host__ __device__ constexpr bool has_z(int kind) { return kind == KIND_RPPI || kind == KIND_WP; }
__host__ __device__ constexpr uint32_t stage_arrays(bool W, bool LO) { return LO ? 7u : (W ? 4u : 3u); }
__host__ __device__ constexpr uint32_t warp_jbuf_bytes(bool W, bool LO) { return 2u * stage_arrays(W, LO) * JSTAGE * 4u; }
__host__ __device__ __forceinline__ uint32_t warp_ring_bytes(int kind, bool W)
{
    return RING * (4u + (has_z(kind) ? 4u : 0u) + (W ? 4u : 0u) + 2u);
}
__host__ __device__ __forceinline__ uint32_t warp_bytes(int kind, bool W, bool R, bool LO, int nslot, bool compact)
{
    return warp_jbuf_bytes(W, LO) + (compact ? warp_ring_bytes(kind, W) : 0u) + warp_hist_bytes(kind, W, R, nslot);
}

// Kahan-compensated FP32 sum: s holds the sum, c the negated lost low part
__device__ __forceinline__ void kahan_step(float &s, float &c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}
__device__ __forceinline__ void kahan_add(float2 *p, float v)
{
    float2 sc = *p;
    kahan_step(sc.x, sc.y, v);
    *p = sc;
}

struct Lut {
    uint32_t base, shift, last;
    const uint16_t *words;   // shared
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

// Lookup for a value known to lie below the table's tail (the start of its final "outside
// every bin" segment): the index then never passes the last cell, so no upper clamp is needed.
// Split in two so that several lookups can issue their table reads before any fine resolution.
__device__ __forceinline__ uint32_t lut_raw_in(const Lut &L, uint32_t vb)
{
    return L.words[(max(vb, L.base) - L.base) >> L.shift];
}
__device__ __forceinline__ uint32_t lut_fine(const CfFine *__restrict__ fine, uint32_t c, uint32_t vb)
{
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

// queue one pair for the FP64 recheck (rare: kept out of line so the pair loops stay small)
static __device__ __noinline__ void push_recheck(const CfPairArgs &a, uint32_t ip, uint32_t jp, uint32_t job)
{
    const unsigned long long k = atomicAdd(a.qcount, 1ull);
    if (k < a.qcap) a.queue[k] = make_uint4(a.orig[ip], a.orig[jp], job, 0u);
}

// rp of a counted pair of the mocks kind, for ravg (Appendix A.2.1).  rp^2 = |s x l|^2 / |l|^2,
// and s x l = s x v_i because l = v_i - s / 2: the cancellation that makes s.s - pi^2 inaccurate
// for rp << pi moves into one cross product of exactly known numbers (s as a hi + lo pair from
// the cell-relative coordinates, v_i as float32 plus its lo part), taken by Kahan's difference of
// products (error <= 2u of each component).  ip: the i point; bs, jl: the stage buffer and the j
// point's index in it; sh / sl: the item's shift, hi and lo.  Rare (counted pairs with ravg
// only), so kept out of line.
template <bool LO>
static __device__ __noinline__ float mocks_rp(const CfPairArgs &a, uint32_t ip, const float *bs, uint32_t jl,
                                              float shx, float shy, float shz, float slx, float sly, float slz)
{
    const float4 A = reinterpret_cast<const float4 *>(a.pa)[ip];
    const float4 B = reinterpret_cast<const float4 *>(a.pb)[ip];
    const float X[3] = {-A.x, -A.z, -B.x}, Ah[3] = {A.y, A.w, B.y};
    const float ish[3] = {shx, shy, shz}, isl[3] = {slx, sly, slz};
    float XL[3] = {0.f, 0.f, 0.f}, AL[3] = {0.f, 0.f, 0.f}, XJL[3] = {0.f, 0.f, 0.f};
    if (LO) {
        const float4 C = reinterpret_cast<const float4 *>(a.plo)[2 * (size_t)ip];
        const float4 D = reinterpret_cast<const float4 *>(a.plo)[2 * (size_t)ip + 1];
        XL[0] = -C.x; XL[1] = -C.z; XL[2] = -D.x;
        AL[0] = C.y; AL[1] = C.w; AL[2] = D.y;
        XJL[0] = bs[4 * JSTAGE + jl]; XJL[1] = bs[5 * JSTAGE + jl]; XJL[2] = bs[6 * JSTAGE + jl];
    }
    const float XJ[3] = {bs[jl], bs[JSTAGE + jl], bs[2 * JSTAGE + jl]};   // -X_j
    float sh[3], sl[3], l[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        float h, e, h2, e2;
        two_sum(X[d], ish[d], h, e);          // X_i + shift hi, exactly h + e
        two_sum(h, XJ[d], h2, e2);            // - X_j, exactly h2 + e2
        sh[d] = h2;
        sl[d] = ((e + e2) + isl[d]) + (XL[d] + XJL[d]);
        l[d] = fmaf(-0.5f, sh[d], Ah[d]) + (AL[d] - 0.5f * sl[d]);
    }
    float c2 = 0.f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int p = (d + 1) % 3, q = (d + 2) % 3;
        // component d of s x A: s_p A_q - s_q A_p
        const float w = sh[q] * Ah[p];
        const float err = fmaf(sh[q], Ah[p], -w);
        const float f = fmaf(sh[p], Ah[q], -w);
        const float corr = (sh[p] * AL[q] - sh[q] * AL[p]) + (sl[p] * Ah[q] - sl[q] * Ah[p]);
        const float c = (f - err) + corr;
        c2 = fmaf(c, c, c2);
    }
    const float ll = fmaf(l[2], l[2], fmaf(l[1], l[1], l[0] * l[0]));
    return sqrtf(__fdiv_rn(c2, ll));
}

// GH (rp-pi and mocks only): no per-warp histogram; every pair adds straight into the job's global
// histogram (CfPairArgs::ghist).  FX (rp-pi and mocks, per-warp histogram): the weight and ravg sums
// are fixed point (two 32-bit words per slot) at the scales CfPairArgs::fxw / fxr_bin, else FP64.
template <int KIND, bool W, bool R, bool WRAP, bool LO, bool GH, bool FX>
struct Warp {
    const CfPairArgs &a;
    Lut lr, lp;
    const CfFine *fine;
    uint32_t *h_cnt;        // lane-private [nslot][32] or per-warp [nslot]
    float2 *h_w, *h_r;      // lane-private Kahan pairs (interleaved when both are kept)
    double *h_wd, *h_rd;    // per-warp sums (rp-pi, mocks): FP64, or with FX two 32-bit words per slot
                            // (nslot low words, then nslot high words)
    const float *fxr_bin;   // with FX and ravg: the scale of each rp bin's ravg terms (shared memory)
    float *jst;             // j stage
    uint32_t *rv, *rz;      // ring: value bits, |dz| bits
    float *rw;              // ring: weight product
    uint16_t *rc;           // ring: code, i slot | j << 7
    int lane, nb, npi, nslot;
    uint32_t icnt, ibeg, jbeg, job, head, tail, ltmask;
    float cut_r, cut_p;
    float Lx, Ly, Lz, iLx, iLy, iLz;
    float near2, cut_su;    // mocks: the near-observer test (near2 = 0: off)
    float ish[3], isl[3];   // mocks with ravg: the item's shift, hi and lo

    __device__ Warp(const CfPairArgs &args) : a(args) {}

    __device__ __forceinline__ void push(uint32_t ip, uint32_t jp) { push_recheck(a, ip, jp, job); }

    __device__ __forceinline__ void acc_lp(uint32_t c, float d2, float wp)
    {
        uint32_t idx = c * 32u + lane;
        atomicAdd(h_cnt + idx, 1u);
        float r = 0.f;
        if (R) {
            r = f_sqrt_approx(d2);
            if (KIND == KIND_THETA) r = 2.0f * asinf(0.5f * r) * 57.29577951308232f;
        }
        if (W && R) {
            // both sums of a lane's bin sit in one float4: one 16-byte load and store
            float4 *p = reinterpret_cast<float4 *>(h_w) + idx;
            float4 v = *p;
            kahan_step(v.x, v.y, wp);
            kahan_step(v.z, v.w, wp * r);
            *p = v;
        } else {
            if (W) kahan_add(h_w + idx, wp);
            if (R) kahan_add(h_r + idx, r);
        }
    }

    __device__ __forceinline__ void acc_sh(uint32_t slot, uint32_t rbin, float rp2, float wp)
    {
        if (GH) {
            // no per-warp histogram: straight into the job's global one
            const size_t g = (size_t)job * (uint32_t)nslot + slot;
            atomicAdd(a.hcnt + g, 1ull);
            if (W) atomicAdd(a.hw + g, (double)wp);
            if (R) {
                const float r = f_sqrt_approx(rp2);
                atomicAdd(a.hr + g, (double)(W ? wp * r : r));
            }
            return;
        }
        atomicAdd(h_cnt + slot, 1u);
        if (W) add_sum(h_wd, slot, wp, a.fxw);
        if (R) {
            float r = f_sqrt_approx(rp2);
            add_sum(h_rd, slot, W ? wp * r : r, FX ? fxr_bin[rbin] : 0.f);
        }
    }

    // One term of a per-warp sum: with FX m = round(t * scale) into the slot's two 32-bit words (m
    // and m >> 12; the scale is a power of two, so t * scale is exact), else an FP64 add.
    __device__ __forceinline__ void add_sum(double *h, uint32_t slot, float t, float scale) const
    {
        if (FX) {
            uint32_t *w = reinterpret_cast<uint32_t *>(h);
            const uint32_t m = __float2uint_rn(t * scale);
            atomicAdd(w + slot, m);
            atomicAdd(w + nslot + slot, m >> FX_HI_SHIFT);
        } else {
            atomicAdd(h + slot, (double)t);
        }
    }

    // Histogram slot of N pairs that passed the FP32 cut (squared separation below cut_r and,
    // for rp-pi and wp, |dz| below cut_p), or K_AMB (re-evaluate in FP64) or K_OUT (outside
    // every bin).  The table reads of all N are issued before any fine resolution.
    static constexpr uint32_t K_AMB = 0xFFFFFFFFu, K_OUT = 0xFFFFFFFEu;
    template <int N>
    __device__ __forceinline__ void classify(const uint32_t (&vb)[N], const uint32_t (&zb)[N], uint32_t (&k)[N],
                                             uint32_t (&kr)[N]) const
    {
        uint32_t cr[N], cz[N];
#pragma unroll
        for (int n = 0; n < N; n++) {
            cr[n] = lut_raw_in(lr, vb[n]);
            cz[n] = has_z(KIND) ? lut_raw_in(lp, zb[n]) : 0u;
        }
#pragma unroll
        for (int n = 0; n < N; n++) {
            cr[n] = lut_fine(fine, cr[n], vb[n]);
            if (has_z(KIND)) cz[n] = lut_fine(fine, cz[n], zb[n]);
            if (KIND == KIND_R || KIND == KIND_THETA) {
                k[n] = cr[n] < (uint32_t)nb ? cr[n] : (cr[n] == CFI_CLS_AMB ? K_AMB : K_OUT);
            } else {
                // the pi table starts at 0 with bin 0, so below cut_p it yields a bin or AMB
                if (max(cr[n], cz[n]) < CFI_CLS_OUT) k[n] = KIND == KIND_RPPI ? cr[n] * npi + cz[n] : cr[n];
                else k[n] = cr[n] != CFI_CLS_OUT ? K_AMB : K_OUT;
            }
            kr[n] = cr[n];
        }
    }

    __device__ __forceinline__ void finish(uint32_t k, uint32_t kr, uint32_t vb, float wp, uint32_t il, uint32_t j)
    {
        if (k < K_OUT) {
            if (warp_hist(KIND)) acc_sh(k, kr, __uint_as_float(vb), wp);
            else acc_lp(k, __uint_as_float(vb), wp);
        } else if (k == K_AMB) {
            push(ibeg + il, jbeg + j);
        }
    }

    __device__ __forceinline__ void bin_in(uint32_t vb, uint32_t zb, float wp, uint32_t il, uint32_t j)
    {
        const uint32_t v[1] = {vb}, z[1] = {zb};
        uint32_t k[1], kr[1];
        classify<1>(v, z, k, kr);
        finish(k[0], kr[0], vb, wp, il, j);
    }

    // bin the ring's candidates with every lane busy: two per lane while 64 are queued, then
    // 32 at a time; with all = true also the last, partial pass
    __device__ __forceinline__ void drain(bool all)
    {
        __syncwarp();
        while (tail - head >= 64u) {
            const uint32_t e0 = (head + lane) & RM, e1 = (head + 32u + lane) & RM;
            const uint32_t v[2] = {rv[e0], rv[e1]};
            const uint32_t z[2] = {has_z(KIND) ? rz[e0] : 0u, has_z(KIND) ? rz[e1] : 0u};
            const uint32_t c0 = rc[e0], c1 = rc[e1];
            const float w0 = W ? rw[e0] : 0.f, w1 = W ? rw[e1] : 0.f;
            uint32_t k[2], kr[2];
            classify<2>(v, z, k, kr);
            finish(k[0], kr[0], v[0], w0, c0 & 0x7Fu, c0 >> 7);
            finish(k[1], kr[1], v[1], w1, c1 & 0x7Fu, c1 >> 7);
            head += 64u;
        }
        for (;;) {
            const uint32_t left = tail - head;
            if (left == 0u || (!all && left < 32u)) break;
            const uint32_t n = min(left, 32u);
            if ((uint32_t)lane < n) {
                const uint32_t e = (head + lane) & RM;
                const uint32_t c = rc[e];
                bin_in(rv[e], has_z(KIND) ? rz[e] : 0u, W ? rw[e] : 0.f, c & 0x7Fu, c >> 7);
            }
            head += n;
        }
        __syncwarp();
    }

    // Stage chunk c of the j range into its buffer: arrays 0 x, 1 y, 2 z, 3 w, 4-6 lo parts of
    // x, y, z (all negated as stored); a j past the end of the range reads the far-away sentinel
    __device__ __forceinline__ void stage(uint32_t c, uint32_t jcnt)
    {
        constexpr uint32_t NA = stage_arrays(W, LO);
        float *bs = jst + (c & 1u) * NA * JSTAGE;
        const uint32_t j = c * JSTAGE + lane;
        if (j < jcnt) {
            const float *fa = reinterpret_cast<const float *>(a.pa + jbeg + j);
            const float *fb = reinterpret_cast<const float *>(a.pb + jbeg + j);
            cp_async4(bs + lane, fa);
            cp_async4(bs + JSTAGE + lane, fa + 2);
            cp_async4(bs + 2 * JSTAGE + lane, fb);
            if (W) cp_async4(bs + 3 * JSTAGE + lane, fb + 2);
            if (LO) {
                const float *fl = reinterpret_cast<const float *>(a.plo + 2 * (size_t)(jbeg + j));
                cp_async4(bs + 4 * JSTAGE + lane, fl);
                cp_async4(bs + 5 * JSTAGE + lane, fl + 2);
                cp_async4(bs + 6 * JSTAGE + lane, fl + 4);
            }
        } else {
            bs[lane] = 1e18f;
            bs[JSTAGE + lane] = 1e18f;
            bs[2 * JSTAGE + lane] = 1e18f;
            if (W) bs[3 * JSTAGE + lane] = 0.f;
            if (LO) bs[4 * JSTAGE + lane] = bs[5 * JSTAGE + lane] = bs[6 * JSTAGE + lane] = 0.f;
        }
    }

    // One work item.  Q = i slots per lane; DIAG: the i tile and the j range are the same cell
    // (only j > i counts; one instance with Q = 4 serves every tile size, the slots past the
    // tile skipped at run time); COMPACT selects the binning form.
    template <int Q, bool DIAG, bool COMPACT>
    __device__ __forceinline__ void run(const CfItem &it)
    {
        // direct form: r and theta issue the distances of all slots before binning any (more
        // independent chains); rp-pi and wp, whose binning is larger, bin each slot right away
        constexpr bool SPLIT = !has_z(KIND);
        icnt = it.cnt & 0xFFFFu;
        const uint32_t jcnt = it.cnt >> 16;
        ibeg = it.ibeg;
        jbeg = it.jbeg;
        job = it.meta & CFI_ITEM_JOBMASK;
        u64 sx[Q], sy[Q], sz[Q], ex[Q], ey[Q], ez[Q], wi[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) {
            const uint32_t il = lane + 32u * q;
            float vs[3], ve[3], vw = 0.f;
#pragma unroll
            for (int d = 0; d < 3; d++) { vs[d] = 1e18f; ve[d] = 0.f; }
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
                        vs[d] = s;
                        ve[d] = (e + it.slo[d]) + XL[d];
                    } else {
                        vs[d] = X[d] + it.s[d];
                    }
                }
                vw = f2_lo(B.y);
            }
            sx[q] = f2_pack(vs[0], vs[0]);
            sy[q] = f2_pack(vs[1], vs[1]);
            sz[q] = f2_pack(vs[2], vs[2]);
            ex[q] = f2_pack(ve[0], ve[0]);
            ey[q] = f2_pack(ve[1], ve[1]);
            ez[q] = f2_pack(ve[2], ve[2]);
            wi[q] = f2_pack(vw, vw);
        }
        constexpr uint32_t NA = stage_arrays(W, LO);
        const uint32_t nchunk = (jcnt + JSTAGE - 1) / JSTAGE;
        stage(0, jcnt);
        cp_async_commit();
        for (uint32_t c = 0; c < nchunk; c++) {
            if (c + 1 < nchunk) stage(c + 1, jcnt);
            cp_async_commit();
            cp_async_wait<1>();
            __syncwarp();
            const float *bs = jst + (c & 1u) * NA * JSTAGE;
            const uint32_t j0 = c * JSTAGE;
            const uint32_t n = min(JSTAGE, jcnt - j0);
            // within a cell paired with itself, slot q (i >= 32 q) has a live pair in this
            // chunk (j <= 32 c + 31) only if q <= c, and none past the tile
            const int nq = DIAG ? min((int)((icnt + 31u) >> 5), (int)c + 1) : Q;
#pragma unroll 1
            for (uint32_t jj = 0; jj < n; jj += 2) {
                const uint32_t j = j0 + jj;
                const u64 xj = *reinterpret_cast<const u64 *>(bs + jj);
                const u64 yj = *reinterpret_cast<const u64 *>(bs + JSTAGE + jj);
                const u64 zj = *reinterpret_cast<const u64 *>(bs + 2 * JSTAGE + jj);
                // the j weights, read once for all slots (rp-pi / wp bin where formed)
                const u64 wjd = (W && !SPLIT && !COMPACT) ? *reinterpret_cast<const u64 *>(bs + 3 * JSTAGE + jj) : 0ull;
                u64 lx = 0, ly = 0, lz = 0;
                if (LO) {
                    lx = *reinterpret_cast<const u64 *>(bs + 4 * JSTAGE + jj);
                    ly = *reinterpret_cast<const u64 *>(bs + 5 * JSTAGE + jj);
                    lz = *reinterpret_cast<const u64 *>(bs + 6 * JSTAGE + jj);
                }
                // the distances and cuts of every slot first (independent chains), then the
                // binning; in the compacting form bits 2q and 2q + 1 of m: slot q's pair with j
                // and with j + 1 is below the cut
                u64 v2[Q], az[Q];
                bool p0[Q], p1[Q];
                uint32_t m = 0;
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    v2[q] = az[q] = 0ull;
                    p0[q] = p1[q] = false;
                    if (DIAG && q >= nq) continue;
                    u64 dx = f2_add(sx[q], xj), dy = f2_add(sy[q], yj), dz = f2_add(sz[q], zj);
                    if (R) {
                        dx = f2_add(dx, LO ? f2_add(ex[q], lx) : ex[q]);
                        dy = f2_add(dy, LO ? f2_add(ey[q], ly) : ey[q]);
                        dz = f2_add(dz, LO ? f2_add(ez[q], lz) : ez[q]);
                    }
                    if (WRAP) {
                        if (Lx > 0.f) dx = wrap2(dx, Lx, iLx);
                        if (Ly > 0.f) dy = wrap2(dy, Ly, iLy);
                        if (Lz > 0.f) dz = wrap2(dz, Lz, iLz);
                    }
                    const uint32_t il = lane + 32u * q;
                    bool in0, in1;
                    v2[q] = f2_mul(dx, dx);
                    v2[q] = f2_fma(dy, dy, v2[q]);
                    if (KIND == KIND_R || KIND == KIND_THETA) {
                        v2[q] = f2_fma(dz, dz, v2[q]);
                        in0 = f2_lo(v2[q]) < cut_r;
                        in1 = f2_hi(v2[q]) < cut_r;
                    } else {
                        az[q] = dz & 0x7FFFFFFF7FFFFFFFull;
                        in0 = f2_lo(v2[q]) < cut_r && f2_lo(az[q]) < cut_p;
                        in1 = f2_hi(v2[q]) < cut_r && f2_hi(az[q]) < cut_p;
                    }
                    // within a cell paired with itself only j > i counts; in wrap mode the
                    // minimum image folds the far-away sentinels back, so mask them here
                    if (DIAG) {
                        in0 = in0 && j > il;
                        in1 = in1 && j + 1 > il;
                    }
                    if (WRAP) {
                        const bool li = il < icnt;
                        in0 = in0 && li;
                        in1 = in1 && li && j + 1 < jcnt;
                    }
                    p0[q] = in0;
                    p1[q] = in1;
                    if (COMPACT) {
                        m |= (in0 ? 1u : 0u) << (2 * q);
                        m |= (in1 ? 2u : 0u) << (2 * q);
                    } else if (!SPLIT && (in0 || in1)) {
                        // direct form, rp-pi / wp: bin where formed
                        const u64 wp = W ? f2_mul(wi[q], wjd) : 0ull;
                        if (in0) bin_in(f2_lo_bits(v2[q]), f2_lo_bits(az[q]), f2_lo(wp), il, j);
                        if (in1) bin_in(f2_hi_bits(v2[q]), f2_hi_bits(az[q]), f2_hi(wp), il, j + 1);
                    }
                }
                if (!COMPACT && SPLIT) {
                    // direct form, r / theta: bin after every slot's distances are issued (the j
                    // weights read once for all slots)
                    const u64 wj = W ? *reinterpret_cast<const u64 *>(bs + 3 * JSTAGE + jj) : 0ull;
#pragma unroll
                    for (int q = 0; q < Q; q++) {
                        if (p0[q] || p1[q]) {
                            const uint32_t il = lane + 32u * q;
                            const u64 wp = W ? f2_mul(wi[q], wj) : 0ull;
                            if (p0[q]) bin_in(f2_lo_bits(v2[q]), f2_lo_bits(az[q]), f2_lo(wp), il, j);
                            if (p1[q]) bin_in(f2_hi_bits(v2[q]), f2_hi_bits(az[q]), f2_hi(wp), il, j + 1);
                        }
                    }
                }
                if (COMPACT && __any_sync(CF_FULL, m != 0u)) {
                    // offsets of this lane's candidates: a prefix sum of the per-lane counts
                    // (<= 2Q) from one ballot per bit of the count
                    const u64 wj = W ? *reinterpret_cast<const u64 *>(bs + 3 * JSTAGE + jj) : 0ull;
                    const uint32_t cnt = __popc(m);
                    constexpr int CB = Q == 1 ? 2 : (Q == 2 ? 3 : 4);
                    uint32_t pre = 0, tot = 0;
#pragma unroll
                    for (int b = 0; b < CB; b++) {
                        const uint32_t bal = __ballot_sync(CF_FULL, (cnt >> b) & 1u);
                        pre += (uint32_t)__popc(bal & ltmask) << b;
                        tot += (uint32_t)__popc(bal) << b;
                    }
                    uint32_t pos = tail + pre;
#pragma unroll
                    for (int q = 0; q < Q; q++) {
                        const uint32_t mq = (m >> (2 * q)) & 3u;
                        if (!mq) continue;
                        const u64 wp = W ? f2_mul(wi[q], wj) : 0ull;
                        const uint32_t code = (lane + 32u * q) | (j << 7);
                        if (mq & 1u) {
                            const uint32_t e = pos & RM;
                            rv[e] = f2_lo_bits(v2[q]);
                            if (has_z(KIND)) rz[e] = f2_lo_bits(az[q]);
                            rc[e] = (uint16_t)code;
                            if (W) rw[e] = f2_lo(wp);
                            pos++;
                        }
                        if (mq & 2u) {
                            const uint32_t e = pos & RM;
                            rv[e] = f2_hi_bits(v2[q]);
                            if (has_z(KIND)) rz[e] = f2_hi_bits(az[q]);
                            rc[e] = (uint16_t)(code + 128u);    // j + 1
                            if (W) rw[e] = f2_hi(wp);
                            pos++;
                        }
                    }
                    // the ring held < 32 candidates and took <= 64 Q: at most 287 of RING
                    tail += tot;
                    if (tail - head >= 32u) drain(false);
                }
            }
            __syncwarp();       // the chunk buffer is refilled two chunks later
        }
        cp_async_wait<0>();
        __syncwarp();
        if (COMPACT) drain(true);
    }

    // ---- DD(rp, pi) of observed positions (Appendix A.2.1) ----
    // Bin one mocks candidate from its FP32 |s x A_i|^2, (s.l)^2 and l.l: pi^2 = (s.l)^2 / l.l and
    // rp^2 = |s x A_i|^2 / l.l (s x A_i = s x l), whose error scales with rp where s.s - pi^2 would
    // lose everything below the rounding of s.s when rp << pi.  il, j: the pair within the item
    // (j's chunk is the one staged now).
    __device__ __forceinline__ void bin_mocks(float c2, float sl2, float ll, float wp, uint32_t il, uint32_t j)
    {
        if (near2 > 0.f && ll < near2) {
            push(ibeg + il, jbeg + j);        // midpoint near the observer: FP64
            return;
        }
        const float r = __fdividef(1.0f, ll);
        const float pi2 = sl2 * r;
        const float rp2 = c2 * r;
        const uint32_t cr = lut_class(lr, fine, __float_as_uint(rp2));
        const uint32_t cz = lut_class(lp, fine, __float_as_uint(pi2));
        if (cr == CFI_CLS_OUT || cz == CFI_CLS_OUT) return;
        if (max(cr, cz) == CFI_CLS_AMB) {
            push(ibeg + il, jbeg + j);
            return;
        }
        const uint32_t slot = cr * (uint32_t)npi + cz;
        if (GH) {
            const size_t g = (size_t)job * (uint32_t)nslot + slot;
            atomicAdd(a.hcnt + g, 1ull);
            if (W) atomicAdd(a.hw + g, (double)wp);
            if (R) {
                constexpr uint32_t NA = stage_arrays(W, LO);
                const float *bs = jst + ((j / JSTAGE) & 1u) * NA * JSTAGE;
                const float rr = mocks_rp<LO>(a, ibeg + il, bs, j % JSTAGE, ish[0], ish[1], ish[2], isl[0], isl[1],
                                              isl[2]);
                atomicAdd(a.hr + g, (double)(W ? wp * rr : rr));
            }
            return;
        }
        atomicAdd(h_cnt + slot, 1u);
        if (W) add_sum(h_wd, slot, wp, a.fxw);
        if (R) {
            // the j point is in the stage buffer of its chunk
            constexpr uint32_t NA = stage_arrays(W, LO);
            const float *bs = jst + ((j / JSTAGE) & 1u) * NA * JSTAGE;
            const float rr = mocks_rp<LO>(a, ibeg + il, bs, j % JSTAGE, ish[0], ish[1], ish[2], isl[0], isl[1],
                                          isl[2]);
            add_sum(h_rd, slot, W ? wp * rr : rr, FX ? fxr_bin[cr] : 0.f);
        }
    }

    // One work item of the mocks kind (the direct form; Q and DIAG as in run).  Per pair, packed
    // FP32x2: s = v_i - v_j (cell-relative), l = A_i - s / 2, u = s.s - cut_r, s.l, l.l; the
    // candidate cut needs no division: rp^2 = s.s - pi^2 < cut_r and pi^2 < cut_p become
    // u l.l < (s.l)^2 < cut_p l.l (cut_r lies above the last edge by twice this form's error).
    // When either pair of a slot passes, |s x A_i|^2 of both is formed packed and each passing
    // pair is binned by bin_mocks where it was formed.  (A compacting form -- candidates to a
    // per-warp ring by ballot prefix, binned 32 at a time -- was measured slower: 4.69 against
    // 4.32 ms on the 200k x 2M survey cone, more warp instructions and full-width shared
    // atomics on few slots.)
    template <int Q, bool DIAG>
    __device__ __forceinline__ void run_mocks(const CfItem &it)
    {
        icnt = it.cnt & 0xFFFFu;
        const uint32_t jcnt = it.cnt >> 16;
        ibeg = it.ibeg;
        jbeg = it.jbeg;
        job = it.meta & CFI_ITEM_JOBMASK;
        if (R) {
#pragma unroll
            for (int d = 0; d < 3; d++) { ish[d] = it.s[d]; isl[d] = it.slo[d]; }
        }
        u64 sx[Q], sy[Q], sz[Q], ex[Q], ey[Q], ez[Q], ax[Q], ay[Q], az[Q], wi[Q];
#pragma unroll
        for (int q = 0; q < Q; q++) {
            const uint32_t il = lane + 32u * q;
            float vs[3], ve[3], va[3], vw = 0.f;
#pragma unroll
            for (int d = 0; d < 3; d++) { vs[d] = 1e18f; ve[d] = 0.f; va[d] = 0.f; }
            if (il < icnt) {
                const ulonglong2 A = a.pa[ibeg + il], B = a.pb[ibeg + il];
                const float X[3] = {-f2_lo(A.x), -f2_lo(A.y), -f2_lo(B.x)};
                va[0] = f2_hi(A.x);
                va[1] = f2_hi(A.y);
                va[2] = f2_hi(B.x);
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
                        float t, e;
                        two_sum(X[d], it.s[d], t, e);
                        vs[d] = t;
                        ve[d] = (e + it.slo[d]) + XL[d];
                    } else {
                        vs[d] = X[d] + it.s[d];
                    }
                }
                vw = f2_lo(B.y);
            }
            sx[q] = f2_pack(vs[0], vs[0]);
            sy[q] = f2_pack(vs[1], vs[1]);
            sz[q] = f2_pack(vs[2], vs[2]);
            ex[q] = f2_pack(ve[0], ve[0]);
            ey[q] = f2_pack(ve[1], ve[1]);
            ez[q] = f2_pack(ve[2], ve[2]);
            ax[q] = f2_pack(va[0], va[0]);
            ay[q] = f2_pack(va[1], va[1]);
            az[q] = f2_pack(va[2], va[2]);
            wi[q] = f2_pack(vw, vw);
        }
        const u64 NH = f2_pack(-0.5f, -0.5f), NCR = f2_pack(-cut_r, -cut_r), CP = f2_pack(cut_p, cut_p);
        constexpr uint32_t NA = stage_arrays(W, LO);
        const uint32_t nchunk = (jcnt + JSTAGE - 1) / JSTAGE;
        stage(0, jcnt);
        cp_async_commit();
        for (uint32_t c = 0; c < nchunk; c++) {
            if (c + 1 < nchunk) stage(c + 1, jcnt);
            cp_async_commit();
            cp_async_wait<1>();
            __syncwarp();
            const float *bs = jst + (c & 1u) * NA * JSTAGE;
            const uint32_t j0 = c * JSTAGE;
            const uint32_t n = min(JSTAGE, jcnt - j0);
            const int nq = DIAG ? min((int)((icnt + 31u) >> 5), (int)c + 1) : Q;
#pragma unroll 1
            for (uint32_t jj = 0; jj < n; jj += 2) {
                const uint32_t j = j0 + jj;
                const u64 xj = *reinterpret_cast<const u64 *>(bs + jj);
                const u64 yj = *reinterpret_cast<const u64 *>(bs + JSTAGE + jj);
                const u64 zj = *reinterpret_cast<const u64 *>(bs + 2 * JSTAGE + jj);
                u64 lxj = 0, lyj = 0, lzj = 0;
                if (LO) {
                    lxj = *reinterpret_cast<const u64 *>(bs + 4 * JSTAGE + jj);
                    lyj = *reinterpret_cast<const u64 *>(bs + 5 * JSTAGE + jj);
                    lzj = *reinterpret_cast<const u64 *>(bs + 6 * JSTAGE + jj);
                }
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    if (DIAG && q >= nq) continue;
                    u64 dx = f2_add(sx[q], xj), dy = f2_add(sy[q], yj), dz = f2_add(sz[q], zj);
                    if (R) {
                        dx = f2_add(dx, LO ? f2_add(ex[q], lxj) : ex[q]);
                        dy = f2_add(dy, LO ? f2_add(ey[q], lyj) : ey[q]);
                        dz = f2_add(dz, LO ? f2_add(ez[q], lzj) : ez[q]);
                    }
                    const u64 lx = f2_fma(dx, NH, ax[q]), ly = f2_fma(dy, NH, ay[q]), lz = f2_fma(dz, NH, az[q]);
                    u64 uu = f2_fma(dx, dx, NCR);
                    uu = f2_fma(dy, dy, uu);
                    uu = f2_fma(dz, dz, uu);
                    u64 sl = f2_mul(dx, lx);
                    sl = f2_fma(dy, ly, sl);
                    sl = f2_fma(dz, lz, sl);
                    u64 ll = f2_mul(lx, lx);
                    ll = f2_fma(ly, ly, ll);
                    ll = f2_fma(lz, lz, ll);
                    const u64 sl2 = f2_mul(sl, sl);
                    const u64 m = f2_mul(uu, ll);
                    const u64 cpl = f2_mul(CP, ll);
                    bool in0 = f2_lo(m) < f2_lo(sl2) && f2_lo(sl2) < f2_lo(cpl);
                    bool in1 = f2_hi(m) < f2_hi(sl2) && f2_hi(sl2) < f2_hi(cpl);
                    if (near2 > 0.f) {
                        // a midpoint near the observer makes the multiplied cut meaningless:
                        // there only s.s decides, and the pair goes to FP64
                        if (f2_lo(ll) < near2) in0 = f2_lo(uu) < cut_su;
                        if (f2_hi(ll) < near2) in1 = f2_hi(uu) < cut_su;
                    }
                    const uint32_t il = lane + 32u * q;
                    // empty slots and j past the range hold far-away sentinels whose products
                    // overflow; mask them by index rather than rely on those comparisons
                    in0 = in0 && il < icnt;
                    in1 = in1 && il < icnt && j + 1 < jcnt;
                    if (DIAG) {
                        in0 = in0 && j > il;
                        in1 = in1 && j + 1 > il;
                    }
                    if (in0 || in1) {
                        // |s x A_i|^2 of both pairs at once
                        const u64 cx = f2_sub(f2_mul(dy, az[q]), f2_mul(dz, ay[q]));
                        const u64 cy = f2_sub(f2_mul(dz, ax[q]), f2_mul(dx, az[q]));
                        const u64 cz = f2_sub(f2_mul(dx, ay[q]), f2_mul(dy, ax[q]));
                        const u64 c2 = f2_fma(cz, cz, f2_fma(cy, cy, f2_mul(cx, cx)));
                        const u64 wj = W ? *reinterpret_cast<const u64 *>(bs + 3 * JSTAGE + jj) : 0ull;
                        const u64 wp = W ? f2_mul(wi[q], wj) : 0ull;
                        if (in0) bin_mocks(f2_lo(c2), f2_lo(sl2), f2_lo(ll), f2_lo(wp), il, j);
                        if (in1) bin_mocks(f2_hi(c2), f2_hi(sl2), f2_hi(ll), f2_hi(wp), il, j + 1);
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
        if (GH) return;         // nothing held per warp
        __syncwarp();
        const size_t g0 = (size_t)jb * nslot;
        for (int sl = lane; sl < nslot; sl += 32) {
            unsigned long long c = 0;
            double ws = 0.0, rs = 0.0;
            if (warp_hist(KIND)) {
                c = h_cnt[sl];
                h_cnt[sl] = 0;
                if (W) {
                    if (FX) {
                        uint32_t *w = reinterpret_cast<uint32_t *>(h_wd);
                        ws = (double)fx_sum(w[sl], w[nslot + sl]) * a.ifxw;
                        w[sl] = w[nslot + sl] = 0u;
                    } else {
                        ws = h_wd[sl];
                        h_wd[sl] = 0.0;
                    }
                }
                if (R) {
                    if (FX) {
                        uint32_t *w = reinterpret_cast<uint32_t *>(h_rd);
                        rs = (double)fx_sum(w[sl], w[nslot + sl]) / (double)fxr_bin[sl / npi];
                        w[sl] = w[nslot + sl] = 0u;
                    } else {
                        rs = h_rd[sl];
                        h_rd[sl] = 0.0;
                    }
                }
            } else {
                constexpr int ST = (W && R) ? 2 : 1;     // float2 stride of the Kahan sums
                for (int l = 0; l < 32; l++) {
                    int idx = sl * 32 + ((l + lane) & 31);
                    c += h_cnt[idx];
                    h_cnt[idx] = 0;
                    if (W) {
                        float2 v = h_w[ST * idx];
                        ws += (double)v.x - (double)v.y;
                        h_w[ST * idx] = make_float2(0.f, 0.f);
                    }
                    if (R) {
                        float2 v = h_r[ST * idx];
                        rs += (double)v.x - (double)v.y;
                        h_r[ST * idx] = make_float2(0.f, 0.f);
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

// CTA shape the register budget is sized for.  With weights or ravg the lane-private histograms
// (about 13 KB per warp for 20 bins) hold an SM to one CTA, so it may take up to 16 warps (the
// launcher takes as many as fit); count-only CTAs are small, and a budget for 4 of 256 threads per
// SM (64 registers, no spills in the rp-pi instances) keeps more of them resident than one for 3.
__host__ __device__ constexpr int pair_max_threads(bool W, bool R) { return (W || R) ? 512 : 256; }
__host__ __device__ constexpr int pair_min_blocks(bool W, bool R) { return (!W && !R) ? 4 : 1; }

template <int KIND, bool W, bool R, bool WRAP, bool LO, bool COMPACT, bool GH, bool FX>
__global__ void __launch_bounds__(pair_max_threads(W, R), pair_min_blocks(W, R))
    pair_kernel(const CfPairArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const CfDevPlan *__restrict__ P = a.plan;
    const int nlw = P->nlut_words, nf = P->nfine;
    uint16_t *s_lut = (uint16_t *)smem;
    CfFine *s_fine = (CfFine *)(smem + align16(2u * nlw));
    float *s_fxr = (float *)(s_fine + nf);      // rp-pi / mocks: per rp bin scale of the ravg terms
    unsigned char *wbase = (unsigned char *)s_fxr + (warp_hist(KIND) ? align16(4u * (uint32_t)a.nb) : 0u);
    for (int i = threadIdx.x; i < nlw; i += blockDim.x) s_lut[i] = a.lut[i];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) s_fine[i] = a.fine[i];
    if (FX && R)
        for (int i = threadIdx.x; i < a.nb; i += blockDim.x) s_fxr[i] = a.fxr_bin[i];
    const int hslots = GH ? 0 : a.nslot;        // slots of the per-warp histogram
    const uint32_t wb = warp_bytes(KIND, W, R, LO, hslots, COMPACT);
    const uint32_t hoff = warp_jbuf_bytes(W, LO) + (COMPACT ? warp_ring_bytes(KIND, W) : 0u);
    unsigned char *my = wbase + (size_t)(threadIdx.x >> 5) * wb;
    {
        // zero this warp's histogram (the buffers need no initial value)
        uint32_t *h = (uint32_t *)(my + hoff);
        const uint32_t words = warp_hist_bytes(KIND, W, R, hslots) / 4u;
        for (uint32_t i = threadIdx.x & 31; i < words; i += 32) h[i] = 0u;
    }
    __syncthreads();

    Warp<KIND, W, R, WRAP, LO, GH, FX> w(a);
    w.lane = threadIdx.x & 31;
    w.nb = a.nb;
    w.npi = a.npi;
    w.nslot = a.nslot;
    w.fine = s_fine;
    w.fxr_bin = s_fxr;
    w.lr = {P->lr.base, P->lr.shift, P->lr.last, s_lut + P->lr.coff};
    w.lp = {P->lp.base, P->lp.shift, P->lp.last, s_lut + P->lp.coff};
    w.cut_r = P->cut_r;
    w.cut_p = P->cut_p;
    w.near2 = P->near2;
    w.cut_su = P->cut_su;
    w.Lx = a.L[0]; w.Ly = a.L[1]; w.Lz = a.L[2];
    w.iLx = a.L[0] > 0.f ? 1.0f / a.L[0] : 0.f;
    w.iLy = a.L[1] > 0.f ? 1.0f / a.L[1] : 0.f;
    w.iLz = a.L[2] > 0.f ? 1.0f / a.L[2] : 0.f;
    w.ltmask = (1u << w.lane) - 1u;
    w.head = w.tail = 0u;
    w.jst = (float *)my;
    {
        unsigned char *q = my + warp_jbuf_bytes(W, LO);
        w.rv = (uint32_t *)q;
        q += RING * 4u;
        w.rz = has_z(KIND) ? (uint32_t *)q : nullptr;
        q += has_z(KIND) ? RING * 4u : 0u;
        w.rw = W ? (float *)q : nullptr;
        q += W ? RING * 4u : 0u;
        w.rc = (uint16_t *)q;
    }
    w.h_cnt = (uint32_t *)(my + hoff);
    if (warp_hist(KIND)) {
        uint32_t o = ((uint32_t)hslots * 4u + 7u) & ~7u;
        w.h_wd = (double *)(my + hoff + o);
        w.h_rd = (double *)(my + hoff + o + (W ? hslots * 8u : 0u));
        w.h_w = w.h_r = nullptr;
    } else {
        uint32_t o = a.nslot * 32u * 4u;
        // with both sums they interleave (float4 per lane and bin: w, w-comp, r, r-comp)
        w.h_w = (float2 *)(my + hoff + o);
        w.h_r = (W && R) ? w.h_w + 1 : (float2 *)(my + hoff + o + (W ? a.nslot * 32u * 8u : 0u));
        w.h_wd = w.h_rd = nullptr;
    }

    const uint32_t nitems = min(*a.nitems_dev, a.items_cap);
    int cur = -1;
    // pairs evaluated since the last flush: a warp flushes at the latest every 2^28 (an item holds
    // at most 128 x 512 = 2^16), so no 32-bit count and no fixed-point sum it holds can overflow
    uint32_t pend = 0;
    // the next item's index and descriptor are fetched before the current item is processed
    uint32_t t = 0;
    if (w.lane == 0) t = atomicAdd(a.cursor, 1u);
    t = __shfl_sync(CF_FULL, t, 0);
    CfItem it;
    if (t < nitems) it = a.items[a.order ? a.order[t] : t];
    for (;;) {
        if (t >= nitems) break;
        uint32_t tn = 0;
        if (w.lane == 0) tn = atomicAdd(a.cursor, 1u);
        tn = __shfl_sync(CF_FULL, tn, 0);
        CfItem nx;
        if (tn < nitems) nx = a.items[a.order ? a.order[tn] : tn];
        const int job = (int)(it.meta & CFI_ITEM_JOBMASK);
        if (job != cur || pend > (FX ? FX_FLUSH_PAIRS : CF_FLUSH_PAIRS)) {
            if (cur >= 0) w.flush((uint32_t)cur);
            cur = job;
            pend = 0;
        }
        const bool diag = (it.meta & CFI_ITEM_DIAG) != 0;
        const uint32_t ic = it.cnt & 0xFFFFu;
        pend += ic * (it.cnt >> 16);
        // the instances below are the classes of cf_item_class; the work list comes ordered by
        // class, so the warps of an SM mostly run one instance (its code stays in the
        // instruction cache)
        if (KIND == KIND_MOCKS) {
            if (diag) w.template run_mocks<4, true>(it);
            else if (ic <= 32u) w.template run_mocks<1, false>(it);
            else if (ic <= 64u) w.template run_mocks<2, false>(it);
            else w.template run_mocks<4, false>(it);
        } else {
            if (diag) w.template run<4, true, COMPACT>(it);
            else if (ic <= 32u) w.template run<1, false, COMPACT>(it);
            else if (ic <= 64u) w.template run<2, false, COMPACT>(it);
            else if (ic <= 96u) w.template run<3, false, COMPACT>(it);
            else w.template run<4, false, COMPACT>(it);
        }
        t = tn;
        it = nx;
    }
    if (cur >= 0) w.flush((uint32_t)cur);
}

template <int KIND, bool W, bool R, bool WRAP, bool LO, bool COMPACT, bool GH = false, bool FX = false>
cudaError_t launch_variant(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                           int *warps_out)
{
    auto k = pair_kernel<KIND, W, R, WRAP, LO, COMPACT, GH, FX>;
    int dev;
    cudaGetDevice(&dev);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int maxw = pair_max_threads(W, R) / 32;
    int warps = c.warps > 0 ? (c.warps > maxw ? maxw : c.warps) : maxw;
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
    // global histograms (rp-pi tables too large for shared memory): the direct form only
    if constexpr (warp_hist(KIND))
        if (c.ghist) return launch_variant<KIND, W, R, WRAP, LO, false, true>(c, a, num_sms, st, grid_out, warps_out);
    // fixed-point per-warp sums: the direct form only
    if constexpr (warp_hist(KIND) && (W || R))
        if (a.fxw != 0.f || a.fxr != 0.f)
            return launch_variant<KIND, W, R, WRAP, LO, false, false, true>(c, a, num_sms, st, grid_out, warps_out);
    if (c.variant == 2) return launch_variant<KIND, W, R, WRAP, LO, true>(c, a, num_sms, st, grid_out, warps_out);
    return launch_variant<KIND, W, R, WRAP, LO, false>(c, a, num_sms, st, grid_out, warps_out);
}

}  // namespace cfpair
