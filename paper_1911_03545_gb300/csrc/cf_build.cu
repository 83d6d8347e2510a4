// cf_build.cu -- cell build (Sec. 4.1 grid, Sec. 4.3 contiguous per-cell storage) and the work
// list of cell pairs (Sec. 4.2-4.3), as a counting sort: count -> exclusive scan -> scatter.
#include "cf_build.h"
#include "cf_device.cuh"

// ---------------------------------------------------------------------------------------------
// Bounding box and validity of every point set: min / max per axis, count of non-finite values.
// grid = (blocks, nsets); out[s*W + 0..5] = key(min x,y,z), key(max x,y,z); out[s*W+6] = bad;
// out[s*W+7] = bits of the largest | |v|^2 - 1 |; out[s*W+8] = bits of the smallest |v|^2;
// out[s*W+9], [10] = bits of the smallest nonzero and the largest |w|; out[s*W+11] = negative
// weights (W = CFB_BBOX_WORDS; a non-negative double's bits order like its value).
// ---------------------------------------------------------------------------------------------
__global__ void cf_bbox_kernel(const CfSetDesc *__restrict__ sets, unsigned long long *__restrict__ out)
{
    const CfSetDesc S = sets[blockIdx.y];
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0}, bad = 0, nrm = 0, rmin = ~0ull;
    unsigned long long wmn = ~0ull, wmx = 0, wng = 0;    // |w| range (nonzero minimum), negatives
    const void *P[3] = {S.x, S.y, S.z};
    bool warp_reduced = false;
    if (S.dtype == CF_F32) {
        // float32 inputs: minima, maxima, |v|^2 and its deviation from 1 in float32 (the FP64 pipe
        // runs at a small fraction of the FP32 rate), four points per thread and step through
        // 16-byte loads when the arrays allow it, reduced across the warp in float32; keys once per
        // warp.  |v|^2 carries <= 3 roundings here, which its users allow for.
        const float *X = (const float *)S.x, *Y = (const float *)S.y, *Z = (const float *)S.z;
        const float *Wt = (const float *)S.w;
        float fmn[3] = {INFINITY, INFINITY, INFINITY}, fmx[3] = {-INFINITY, -INFINITY, -INFINITY};
        float fnrm = 0.f, frmin = INFINITY, fwmn = INFINITY, fwmx = 0.f;
        uint32_t nbad = 0, nneg = 0;
        auto visit = [&](float x, float y, float z) {
            const float v[3] = {x, y, z};
            bool ok = true;
            for (int a = 0; a < 3; a++) {
                if (!isfinite(v[a])) {
                    nbad++;
                    ok = false;
                    continue;
                }
                fmn[a] = fminf(fmn[a], v[a]);
                fmx[a] = fmaxf(fmx[a], v[a]);
            }
            if (ok) {
                const float r2 = fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0]));
                fnrm = fmaxf(fnrm, fabsf(r2 - 1.0f));
                frmin = fminf(frmin, r2);
            }
        };
        auto visit_w = [&](float w) {
            if (!isfinite(w)) {
                nbad++;
            } else {
                const float aw = fabsf(w);
                if (w < 0.f) nneg++;
                if (aw > 0.f) fwmn = fminf(fwmn, aw);
                fwmx = fmaxf(fwmx, aw);
            }
        };
        const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
        const bool vec = (((uintptr_t)X | (uintptr_t)Y | (uintptr_t)Z | (uintptr_t)Wt) & 15u) == 0;
        const int64_t n4 = vec ? S.n / 4 : 0;
        for (int64_t q = tid; q < n4; q += nthr) {
            const float4 x = ((const float4 *)X)[q], y = ((const float4 *)Y)[q], z = ((const float4 *)Z)[q];
            visit(x.x, y.x, z.x);
            visit(x.y, y.y, z.y);
            visit(x.z, y.z, z.z);
            visit(x.w, y.w, z.w);
            if (Wt) {
                const float4 w = ((const float4 *)Wt)[q];
                visit_w(w.x);
                visit_w(w.y);
                visit_w(w.z);
                visit_w(w.w);
            }
        }
        for (int64_t i = 4 * n4 + tid; i < S.n; i += nthr) {
            visit(X[i], Y[i], Z[i]);
            if (Wt) visit_w(Wt[i]);
        }
        for (int o = 16; o; o >>= 1) {
            for (int a = 0; a < 3; a++) {
                fmn[a] = fminf(fmn[a], __shfl_xor_sync(CF_FULL, fmn[a], o));
                fmx[a] = fmaxf(fmx[a], __shfl_xor_sync(CF_FULL, fmx[a], o));
            }
            fnrm = fmaxf(fnrm, __shfl_xor_sync(CF_FULL, fnrm, o));
            frmin = fminf(frmin, __shfl_xor_sync(CF_FULL, frmin, o));
            fwmn = fminf(fwmn, __shfl_xor_sync(CF_FULL, fwmn, o));
            fwmx = fmaxf(fwmx, __shfl_xor_sync(CF_FULL, fwmx, o));
            nbad += __shfl_xor_sync(CF_FULL, nbad, o);
            nneg += __shfl_xor_sync(CF_FULL, nneg, o);
        }
        for (int a = 0; a < 3; a++)
            if (fmn[a] <= fmx[a]) {
                mn[a] = cf_dkey((double)fmn[a]);
                mx[a] = cf_dkey((double)fmx[a]);
            }
        bad = nbad;
        wng = nneg;
        nrm = (unsigned long long)__double_as_longlong((double)fnrm);
        if (frmin < INFINITY) rmin = (unsigned long long)__double_as_longlong((double)frmin);
        if (fwmn < INFINITY) wmn = (unsigned long long)__double_as_longlong((double)fwmn);
        wmx = (unsigned long long)__double_as_longlong((double)fwmx);
        warp_reduced = true;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; S.dtype != CF_F32 && i < S.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double r2 = 0.0;
        for (int a = 0; a < 3; a++) {
            double v = cf_load(P[a], S.dtype, i);
            if (!isfinite(v)) { bad++; continue; }
            r2 += v * v;
            unsigned long long k = cf_dkey(v);
            mn[a] = k < mn[a] ? k : mn[a];
            mx[a] = k > mx[a] ? k : mx[a];
        }
        // largest | |v|^2 - 1 | (unit vectors for the angular grid of DD(theta)); a non-negative
        // double's bits order like the value
        const unsigned long long d = (unsigned long long)__double_as_longlong(fabs(r2 - 1.0));
        nrm = d > nrm ? d : nrm;
        // smallest |v|^2 (distance from the observer at the origin, for mocks)
        const unsigned long long r2b = (unsigned long long)__double_as_longlong(r2);
        rmin = r2b < rmin ? r2b : rmin;
        if (S.w) {
            double w = cf_load(S.w, S.dtype, i);
            if (!isfinite(w)) {
                bad++;
            } else {
                const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(w));
                if (w < 0.0) wng++;
                if (b) wmn = b < wmn ? b : wmn;
                wmx = b > wmx ? b : wmx;
            }
        }
    }
    for (int o = 16; !warp_reduced && o; o >>= 1) {
        for (int a = 0; a < 3; a++) {
            unsigned long long t = __shfl_xor_sync(CF_FULL, mn[a], o);
            mn[a] = t < mn[a] ? t : mn[a];
            t = __shfl_xor_sync(CF_FULL, mx[a], o);
            mx[a] = t > mx[a] ? t : mx[a];
        }
        bad += __shfl_xor_sync(CF_FULL, bad, o);
        const unsigned long long t = __shfl_xor_sync(CF_FULL, nrm, o);
        nrm = t > nrm ? t : nrm;
        const unsigned long long t2 = __shfl_xor_sync(CF_FULL, rmin, o);
        rmin = t2 < rmin ? t2 : rmin;
        const unsigned long long t3 = __shfl_xor_sync(CF_FULL, wmn, o);
        wmn = t3 < wmn ? t3 : wmn;
        const unsigned long long t4 = __shfl_xor_sync(CF_FULL, wmx, o);
        wmx = t4 > wmx ? t4 : wmx;
        wng += __shfl_xor_sync(CF_FULL, wng, o);
    }
    // block reduction through shared memory, then one atomic per block and value
    __shared__ unsigned long long red[CFB_BBOX_WORDS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        for (int a = 0; a < 3; a++) {
            red[a][w] = mn[a];
            red[3 + a][w] = mx[a];
        }
        red[6][w] = bad;
        red[7][w] = nrm;
        red[8][w] = rmin;
        red[9][w] = wmn;
        red[10][w] = wmx;
        red[11][w] = wng;
    }
    __syncthreads();
    if (w == 0) {
        unsigned long long v[CFB_BBOX_WORDS];
        for (int a = 0; a < 3; a++) {
            v[a] = lane < nw ? red[a][lane] : ~0ull;
            v[3 + a] = lane < nw ? red[3 + a][lane] : 0ull;
        }
        v[6] = lane < nw ? red[6][lane] : 0ull;
        v[7] = lane < nw ? red[7][lane] : 0ull;
        v[8] = lane < nw ? red[8][lane] : ~0ull;
        v[9] = lane < nw ? red[9][lane] : ~0ull;
        v[10] = lane < nw ? red[10][lane] : 0ull;
        v[11] = lane < nw ? red[11][lane] : 0ull;
        for (int o = 16; o; o >>= 1) {
            for (int a = 0; a < 3; a++) {
                unsigned long long t = __shfl_xor_sync(CF_FULL, v[a], o);
                v[a] = t < v[a] ? t : v[a];
                t = __shfl_xor_sync(CF_FULL, v[3 + a], o);
                v[3 + a] = t > v[3 + a] ? t : v[3 + a];
            }
            v[6] += __shfl_xor_sync(CF_FULL, v[6], o);
            const unsigned long long t = __shfl_xor_sync(CF_FULL, v[7], o);
            v[7] = t > v[7] ? t : v[7];
            const unsigned long long t2 = __shfl_xor_sync(CF_FULL, v[8], o);
            v[8] = t2 < v[8] ? t2 : v[8];
            const unsigned long long t3 = __shfl_xor_sync(CF_FULL, v[9], o);
            v[9] = t3 < v[9] ? t3 : v[9];
            const unsigned long long t4 = __shfl_xor_sync(CF_FULL, v[10], o);
            v[10] = t4 > v[10] ? t4 : v[10];
            v[11] += __shfl_xor_sync(CF_FULL, v[11], o);
        }
        if (lane == 0) {
            unsigned long long *o = out + blockIdx.y * CFB_BBOX_WORDS;
            for (int a = 0; a < 3; a++) {
                atomicMin(o + a, v[a]);
                atomicMax(o + 3 + a, v[3 + a]);
            }
            if (v[6]) atomicAdd(o + 6, v[6]);
            atomicMax(o + 7, v[7]);
            atomicMin(o + 8, v[8]);
            atomicMin(o + 9, v[9]);
            atomicMax(o + 10, v[10]);
            if (v[11]) atomicAdd(o + 11, v[11]);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Cell assignment (Sec. 4.1, Eq. 3): cell = (ix*ny + iy)*nz + iz.  Inside its cell a point also
// gets one of sub^3 sub-cells (sub = 1, 2 or 4 per axis) in Morton order, and the counting sort
// runs on the key cell * sub^3 + sub-cell: every cell stays contiguous and its points come out in
// spatial order, so 32 consecutive points of a cell are spatially compact.  The rank within the
// key comes from an atomic counter.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cf_morton3(uint32_t x, uint32_t y, uint32_t z, int sub)
{
    if (sub == 2) return (x << 2) | (y << 1) | z;
    // sub == 4: interleave two bits per axis, high bits first
    return (((x >> 1) & 1u) << 5) | (((y >> 1) & 1u) << 4) | (((z >> 1) & 1u) << 3) | ((x & 1u) << 2) |
           ((y & 1u) << 1) | (z & 1u);
}

__global__ void __launch_bounds__(256, 6) cf_assign_kernel(const CfDevPlan *__restrict__ plan, const CfSetDesc *__restrict__ sets, int sub,
                                 uint32_t *__restrict__ count, uint32_t *__restrict__ key,
                                 uint32_t *__restrict__ slot)
{
    const CfSetDesc S = sets[blockIdx.y];
    const CfGrid &g = plan->g;
    const uint32_t ns = (uint32_t)(sub * sub * sub);
    const bool f32 = S.dtype == CF_F32;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x) {
        // float32 inputs stay float32 here (the FP64 pipe runs at a small fraction of the FP32 rate)
        float xf[3];
        double xd[3] = {0.0, 0.0, 0.0};
        if (f32) {
            xf[0] = ((const float *)S.x)[i];
            xf[1] = ((const float *)S.y)[i];
            xf[2] = ((const float *)S.z)[i];
        } else {
            xd[0] = ((const double *)S.x)[i];
            xd[1] = ((const double *)S.y)[i];
            xd[2] = ((const double *)S.z)[i];
            for (int a = 0; a < 3; a++) xf[a] = (float)xd[a];
        }
        uint32_t sa[3] = {0u, 0u, 0u};
        uint32_t c;
        if (plan->ang) {
            // angular grid: declination band of the vector's direction (atan2 of z over the projected
            // length: independent of |v| and well conditioned at the poles), then right-ascension
            // cell in [0, 2 pi).  Float32 is enough: any cell choice is correct as long as the point
            // lies in the cell's box, whose margin (2e-6) is far above these ~1e-7 errors.
            const double dec = (double)atan2f(xf[2], sqrtf(xf[0] * xf[0] + xf[1] * xf[1]));
            double ra = (double)atan2f(xf[1], xf[0]);
            if (ra < 0.0) ra += 2.0 * M_PI;
            int b = (int)floor((dec - plan->adlo) / plan->ah);
            b = b < 0 ? 0 : (b > plan->nband - 1 ? plan->nband - 1 : b);
            const CfBand &B = plan->band[b];
            const double tr = ra * B.inv_w;
            int r = (int)floor(tr);
            r = r < 0 ? 0 : (r > B.nra - 1 ? B.nra - 1 : r);
            c = (uint32_t)(B.base + r);
            const double fr[2] = {(dec - B.dlo) / (B.dhi - B.dlo), tr - (double)r};
            for (int a = 0; a < 2; a++) {
                const int s = (int)(fr[a] * sub);
                sa[a] = (uint32_t)(s < 0 ? 0 : (s > sub - 1 ? sub - 1 : s));
            }
        } else {
            int ia[3];
            for (int a = 0; a < 3; a++) {
                // the cell coordinate in float32 decides the cell as the FP64 one would, unless it
                // lies within the plan's guard of a cell boundary: then (and for float64 inputs) FP64
                float fr;
                int cc;
                const float t32 = (xf[a] - plan->lo32[a]) * plan->inv32[a];
                const float f32c = floorf(t32), r32 = t32 - f32c;
                if (f32 && r32 >= plan->cguard[a] && r32 <= 1.0f - plan->cguard[a]) {
                    cc = (int)f32c;
                    fr = r32;
                } else {
                    const double x = f32 ? (double)xf[a] : xd[a];
                    const double t = (x - g.lo[a]) * g.inv[a];
                    const double ft = floor(t);
                    cc = (int)ft;
                    fr = (float)(t - ft);
                }
                cc = cc < 0 ? 0 : (cc > g.n[a] - 1 ? g.n[a] - 1 : cc);
                ia[a] = cc;
                // the sub-cell orders points inside the cell; it does not change any result
                const int s = (int)(fr * (float)sub);
                sa[a] = (uint32_t)(s < 0 ? 0 : (s > sub - 1 ? sub - 1 : s));
            }
            c = (uint32_t)((ia[0] * g.n[1] + ia[1]) * g.n[2] + ia[2]);
        }
        const uint32_t k = ((uint32_t)S.cbeg + c) * ns + (sub > 1 ? cf_morton3(sa[0], sa[1], sa[2], sub) : 0u);
        int64_t p = S.pbeg + i;
        key[p] = k;
        slot[p] = atomicAdd(count + k, 1u);
    }
}

// ---------------------------------------------------------------------------------------------
// Origins of the angular grid's cells (Sec. 4.1.2 cells on the unit sphere).  The box of a cell's
// (RA, DEC) patch bounds x = cos(dec) cos(ra), y = cos(dec) sin(ra), z = sin(dec); widened by 0.1 %
// + 2e-6 for float32 vectors up to 1e-3 off unit length.  Per axis the origin is 0 when the box
// holds 0, else the multiple of the float32 spacing at the box's largest magnitude nearest to 0 that
// still lies between 0 and every value: x - origin is then exact in float32 for every float32 x of
// the cell (the 3-D grid's rule, cfp_origin).
// ---------------------------------------------------------------------------------------------
__device__ void cf_trig_range(double a0, double a1, int c, double &mn, double &mx)
{
    mn = c ? fmin(cos(a0), cos(a1)) : fmin(sin(a0), sin(a1));
    mx = c ? fmax(cos(a0), cos(a1)) : fmax(sin(a0), sin(a1));
    const double q = 0.5 * M_PI;
    for (double k = ceil(a0 / q); k * q <= a1; k += 1.0) {
        const int m = ((int)k % 4 + 4) % 4;   // multiples of pi / 2: cos 1, 0, -1, 0; sin 0, 1, 0, -1
        const double v = c ? (m == 0 ? 1.0 : (m == 2 ? -1.0 : 0.0)) : (m == 1 ? 1.0 : (m == 3 ? -1.0 : 0.0));
        mn = fmin(mn, v);
        mx = fmax(mx, v);
    }
}

__device__ double cf_origin_of_interval(double lo, double hi)
{
    if (lo <= 0.0 && hi >= 0.0) return 0.0;
    int e;
    frexp(fmax(fabs(lo), fabs(hi)) * (1.0 + 1.0 / 1048576.0), &e);
    const double sp = ldexp(1.0, e - 24);
    return lo > 0.0 ? floor(lo / sp) * sp : ceil(hi / sp) * sp;
}

__global__ void cf_ang_origin_kernel(const CfDevPlan *__restrict__ plan, int ncell, double *__restrict__ origin,
                                     float *__restrict__ origin32)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const int b = cf_band_of(plan, c);
        const CfBand &B = plan->band[b];
        const int r = c - B.base;
        double cmin, cmax, zmn, zmx, ca0, ca1, sa0, sa1;
        cf_trig_range(B.dlo, B.dhi, 1, cmin, cmax);
        cf_trig_range(B.dlo, B.dhi, 0, zmn, zmx);
        cmin = fmax(cmin, 0.0);
        cf_trig_range(r * B.w, (r + 1) * B.w, 1, ca0, ca1);
        cf_trig_range(r * B.w, (r + 1) * B.w, 0, sa0, sa1);
        const double lo[3] = {ca0 >= 0 ? cmin * ca0 : cmax * ca0, sa0 >= 0 ? cmin * sa0 : cmax * sa0, zmn};
        const double hi[3] = {ca1 >= 0 ? cmax * ca1 : cmin * ca1, sa1 >= 0 ? cmax * sa1 : cmin * sa1, zmx};
        for (int a = 0; a < 3; a++) {
            const double o = cf_origin_of_interval(lo[a] - 1e-3 * fabs(lo[a]) - 2e-6, hi[a] + 1e-3 * fabs(hi[a]) + 2e-6);
            origin[3 * c + a] = o;
            origin32[3 * c + a] = (float)o;     // exact: a multiple of the float32 spacing
        }
    }
}

// cell start of every cell from the start of its first sub-cell (and the total at the end)
// ---------------------------------------------------------------------------------------------
// Exclusive scan of u32 counts into u32 offsets (+ total at out[n]) in two passes over tiles of
// 4096 values: tile totals (the last block to finish scans them), then each tile's own scan plus
// its offset.  The input is read twice and the output written once.
// ---------------------------------------------------------------------------------------------
#define SCAN_T 256
#define SCAN_V 16
#define SCAN_TILE (SCAN_T * SCAN_V)

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(CF_FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < (SCAN_T / 32) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(CF_FULL, s, o);
            if (lane >= o) s += t;
        }
        if (lane < (SCAN_T / 32)) sh[lane] = s;
    }
    __syncthreads();
    uint32_t pre = (w ? sh[w - 1] : 0) + x - v;
    if (total) *total = sh[SCAN_T / 32 - 1];
    __syncthreads();
    return pre;
}

// this thread's SCAN_V consecutive values (0 past n), through 16-byte loads where they can be used
__device__ __forceinline__ void scan_load(const uint32_t *__restrict__ in, int64_t n, int64_t base, uint32_t *v)
{
    if (base + SCAN_V <= n && ((uintptr_t)in & 15u) == 0) {
        const uint4 *q = (const uint4 *)(in + base);
#pragma unroll
        for (int k = 0; k < SCAN_V / 4; k++) {
            const uint4 t = q[k];
            v[4 * k] = t.x;
            v[4 * k + 1] = t.y;
            v[4 * k + 2] = t.z;
            v[4 * k + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_V; k++) v[k] = (base + k < n) ? in[base + k] : 0u;
    }
}

// pass 1: tile totals into tile_tot[]; the block that finishes last (one ticket per block on
// *done, zeroed by the caller) turns them into exclusive tile offsets and writes the grand total
// at tile_tot[ntiles]
__global__ void cf_scan_reduce(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ tile_tot,
                               uint32_t *__restrict__ done)
{
    __shared__ uint32_t sh[SCAN_T / 32];
    __shared__ bool last;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_V;
    uint32_t v[SCAN_V], s = 0;
    scan_load(in, n, base, v);
#pragma unroll
    for (int k = 0; k < SCAN_V; k++) s += v[k];
    uint32_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) {
        tile_tot[blockIdx.x] = tot;
        __threadfence();                              // the total is visible before the ticket
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int ntiles = (int)gridDim.x;
    uint32_t carry = 0;
    for (int base0 = 0; base0 < ntiles; base0 += SCAN_TILE) {
        const int b = base0 + threadIdx.x * SCAN_V;
        uint32_t t[SCAN_V], ts = 0;
#pragma unroll
        for (int k = 0; k < SCAN_V; k++) {
            t[k] = (b + k < ntiles) ? __ldcg(tile_tot + b + k) : 0u;    // from L2: other blocks wrote them
            ts += t[k];
        }
        uint32_t ttot;
        uint32_t pre = block_excl_scan(ts, sh, &ttot) + carry;
#pragma unroll
        for (int k = 0; k < SCAN_V; k++) {
            if (b + k < ntiles) tile_tot[b + k] = pre;
            pre += t[k];
        }
        carry += ttot;
    }
    if (threadIdx.x == 0) tile_tot[ntiles] = carry;
}

// pass 2: each tile's scan plus its offset.  every (optional) receives out[i] at each multiple i of
// 2^every_shift, i.e. every[i >> every_shift] (the start of each cell among its sub-cell starts);
// n is a multiple of that stride.
__global__ void cf_scan_apply(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
                              const uint32_t *__restrict__ tile_off, uint32_t *__restrict__ total_copy,
                              uint32_t *__restrict__ every, int every_shift)
{
    __shared__ uint32_t sh[SCAN_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_V;
    uint32_t v[SCAN_V], s = 0;
    scan_load(in, n, base, v);
#pragma unroll
    for (int k = 0; k < SCAN_V; k++) s += v[k];
    uint32_t pre = block_excl_scan(s, sh, nullptr) + tile_off[blockIdx.x];
    uint32_t o[SCAN_V];
#pragma unroll
    for (int k = 0; k < SCAN_V; k++) {
        o[k] = pre;
        pre += v[k];
    }
    if (base + SCAN_V <= n && ((uintptr_t)out & 15u) == 0) {
        uint4 *q = (uint4 *)(out + base);
#pragma unroll
        for (int k = 0; k < SCAN_V / 4; k++) q[k] = make_uint4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_V; k++)
            if (base + k < n) out[base + k] = o[k];
    }
    if (every) {
        const int64_t mask = ((int64_t)1 << every_shift) - 1;
#pragma unroll
        for (int k = 0; k < SCAN_V; k++)
            if (base + k < n && ((base + k) & mask) == 0) every[(base + k) >> every_shift] = o[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        const uint32_t grand = tile_off[gridDim.x];
        out[n] = grand;
        if (total_copy) *total_copy = grand;
        if (every) every[n >> every_shift] = grand;
    }
}

// ---------------------------------------------------------------------------------------------
// Scatter into cell order (Sec. 4.3).  Writes the packed j-side layout pa/pb (cell-relative,
// negated, duplicated), the FP64 residual plo when requested, and the original index.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 6) cf_scatter_kernel(const CfDevPlan *__restrict__ plan, const CfSetDesc *__restrict__ sets,
                                  uint32_t ns, const uint32_t *__restrict__ fstart, const uint32_t *__restrict__ key,
                                  const uint32_t *__restrict__ slot, float4 *__restrict__ pa,
                                  float4 *__restrict__ pb, float4 *__restrict__ plo,
                                  uint32_t *__restrict__ orig)
{
    const CfSetDesc S = sets[blockIdx.y];
    const CfGrid &g = plan->g;
    const int lo = plan->f64lo;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = S.pbeg + i;
        const uint32_t k = key[p];
        const uint32_t c = k / ns - (uint32_t)S.cbeg;
        int iz = c % g.n[2];
        int iy = (c / g.n[2]) % g.n[1];
        int ix = c / (g.n[2] * g.n[1]);
        int64_t dst = fstart[k] + slot[p];
        const bool mocks = plan->kind == CF_DD_RPPI_MOCKS;
        if (S.dtype == CF_F32 && !lo) {
            // float32 inputs: x - o is exact in float32 (o is a multiple of the float32 spacing at
            // the cell's magnitude and lies between 0 and x), the same value the FP64 form rounds to
            const float vx = ((const float *)S.x)[i], vy = ((const float *)S.y)[i], vz = ((const float *)S.z)[i];
            const float xf = vx - cf_cell_origin32(plan, 0, (int)c, ix);
            const float yf = vy - cf_cell_origin32(plan, 1, (int)c, iy);
            const float zf = vz - cf_cell_origin32(plan, 2, (int)c, iz);
            const float w = S.w ? ((const float *)S.w)[i] : 1.0f;
            const float ax = mocks ? vx : -xf, ay = mocks ? vy : -yf, az = mocks ? vz : -zf;
            pa[dst] = make_float4(-xf, ax, -yf, ay);
            pb[dst] = make_float4(-zf, az, w, w);
            orig[dst] = (uint32_t)i;
            continue;
        }
        const double vx = cf_load(S.x, S.dtype, i), vy = cf_load(S.y, S.dtype, i), vz = cf_load(S.z, S.dtype, i);
        double X = vx - cf_cell_origin(plan, 0, (int)c, ix);
        double Y = vy - cf_cell_origin(plan, 1, (int)c, iy);
        double Z = vz - cf_cell_origin(plan, 2, (int)c, iz);
        float xf = (float)X, yf = (float)Y, zf = (float)Z;
        float w = S.w ? (float)cf_load(S.w, S.dtype, i) : 1.0f;
        // second copies: X again, or for mocks the absolute position (its line of sight)
        const float ax = mocks ? (float)vx : -xf, ay = mocks ? (float)vy : -yf, az = mocks ? (float)vz : -zf;
        pa[dst] = make_float4(-xf, ax, -yf, ay);
        pb[dst] = make_float4(-zf, az, w, w);
        if (lo) {
            float xl = (float)(X - (double)xf), yl = (float)(Y - (double)yf), zl = (float)(Z - (double)zf);
            const float axl = mocks ? (float)(vx - (double)ax) : -xl;
            const float ayl = mocks ? (float)(vy - (double)ay) : -yl;
            const float azl = mocks ? (float)(vz - (double)az) : -zl;
            plo[2 * dst] = make_float4(-xl, axl, -yl, ayl);
            plo[2 * dst + 1] = make_float4(-zl, azl, 0.f, 0.f);
        }
        orig[dst] = (uint32_t)i;
    }
}

// ---------------------------------------------------------------------------------------------
// Tight bounding box of each cell's points in the cell-relative float32 coordinates of the pair
// kernel (x - origin; lo then hi per axis, 6 floats per cell of every point set).  One warp per
// cell; an empty cell keeps (+inf, -inf).  The work list uses it to skip cell pairs whose points
// are all farther apart than the largest edge: the paper's late entry / early exit (Sec. 4.5) at
// the granularity of cells.  With gbox, also the box of every group of 32 consecutive points of a
// cell (counted from the cell's first point), at gbox[6 p] for the group's first point p; the work
// list prunes at that granularity.
// ---------------------------------------------------------------------------------------------
__global__ void cf_cellbox_kernel(const uint32_t *__restrict__ cell_start, int64_t ncell_all,
                                  const float4 *__restrict__ pa, const float4 *__restrict__ pb, float *__restrict__ box,
                                  float *__restrict__ gbox)
{
    const uint32_t lane = threadIdx.x & 31u;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < ncell_all; c += wstride) {
        const uint32_t b = cell_start[c], e = cell_start[c + 1];
        if (b == e) {
            // most cells of a fine grid are empty: no reduction for them (b, e are warp-uniform)
            if (lane < 6u) box[6 * c + lane] = lane < 3u ? INFINITY : -INFINITY;
            continue;
        }
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (uint32_t p0 = b; p0 < e; p0 += 32u) {
            float glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY};
            const uint32_t p = p0 + lane;
            if (p < e) {
                const float4 A = pa[p], B = pb[p];
                const float v[3] = {-A.x, -A.z, -B.x};
                for (int a = 0; a < 3; a++) glo[a] = ghi[a] = v[a];
            }
            if (gbox) {
                for (int o = 16; o; o >>= 1)
                    for (int a = 0; a < 3; a++) {
                        glo[a] = fminf(glo[a], __shfl_xor_sync(CF_FULL, glo[a], o));
                        ghi[a] = fmaxf(ghi[a], __shfl_xor_sync(CF_FULL, ghi[a], o));
                    }
                if (lane < 6u) gbox[6 * (size_t)p0 + lane] = lane < 3u ? glo[lane] : ghi[lane - 3u];
            }
            for (int a = 0; a < 3; a++) {
                lo[a] = fminf(lo[a], glo[a]);
                hi[a] = fmaxf(hi[a], ghi[a]);
            }
        }
        for (int o = 16; o; o >>= 1)
            for (int a = 0; a < 3; a++) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(CF_FULL, lo[a], o));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(CF_FULL, hi[a], o));
            }
        if (lane < 6u) box[6 * c + lane] = lane < 3u ? lo[lane] : hi[lane - 3u];
    }
}

// The units (job, i cell) whose i cell holds points, in any order, and their number in *nlive
// (zeroed by the caller): on a grid with far more cells than points the work-list pass then skips
// the empty ones without a warp iteration each.  One thread per unit, one atomic per warp.
__global__ void cf_live_units_kernel(const CfDevPlan *__restrict__ plan, const CfSetDesc *__restrict__ sets,
                                     const CfJobDesc *__restrict__ jobs, const uint32_t *__restrict__ cell_start,
                                     uint32_t *__restrict__ live, uint32_t *__restrict__ nlive)
{
    const CfGrid &g = plan->g;
    const int64_t nunit = (int64_t)g.ncell * plan->njobs;
    const uint32_t lane = threadIdx.x & 31u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;      // a multiple of 32: warp-uniform loop
    for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; b < nunit; b += stride) {
        const int64_t u = b + lane;
        bool has = false;
        if (u < nunit) {
            const int job = (int)(u / g.ncell);
            const int64_t c = sets[jobs[job].a].cbeg + (u - (int64_t)job * g.ncell);
            has = cell_start[c + 1] > cell_start[c];
        }
        const uint32_t m = __ballot_sync(CF_FULL, has);
        uint32_t base = 0;
        if (lane == 0 && m) base = atomicAdd(nlive, (uint32_t)__popc(m));
        base = __shfl_sync(CF_FULL, base, 0);
        if (has) live[base + (uint32_t)__popc(m & ((1u << lane) - 1u))] = (uint32_t)u;
    }
}

// Work items, one warp per (job, i cell).  The lanes walk the cell's stencil (Sec. 4.3: neighbours
// +-k per axis, periodic shift per cell pair, auto keeps cj >= ci), a warp prefix sum orders the
// items of the cell, and an empty i cell costs one load.  i tiles are full (tile points) plus one
// remainder tile, so a tile wastes at most 31 pair-kernel slots; j ranges split evenly (<= jchunk).
// With group boxes (gbox), each i tile is tested against every 32-point group of the j cell with
// the cell-pair test's margins, and only runs of groups that may hold a pair within the largest
// edge become j ranges (<= jchunk): the late entry / early exit of Sec. 4.5 at group granularity.
// mode 0 writes the item count of each (job, cell) and adds the number of items, counted in 64 bits,
// to *evaluated (the 32-bit scan of the counts would wrap silently past 2^32 items); mode 1 writes
// the items at the scanned offsets and adds the pairs they hold to *evaluated.  Mode 2 needs no
// count pass: a block stages the items of its warps' cells in shared memory (each warp reserves
// the items of 32 stencil entries there with a shared atomic), then reserves them in the global
// list with one atomic on counts[0] (the list's length when the kernel ends) and copies them out
// with 16-byte stores.  Entries that do not fit the stage reserve and write globally.  Their
// number is added in 64 bits to *total64.  The list's order then follows the blocks' arrival
// instead of (job, cell).
// GP: the instance with group pruning (its group code holds registers the other need not pay for)
template <bool GP>
__global__ void __launch_bounds__(256, GP ? 3 : 4)
    cf_items_kernel(const CfDevPlan *__restrict__ plan, const CfSetDesc *__restrict__ sets,
                                const CfJobDesc *__restrict__ jobs, const CfStencil *__restrict__ stencil,
                                const uint32_t *__restrict__ cell_start, const float *__restrict__ cbox,
                                const float *__restrict__ gbox, const uint32_t *__restrict__ live,
                                const uint32_t *__restrict__ nlive, int mode,
                                uint32_t *__restrict__ counts, const uint32_t *__restrict__ offsets,
                                CfItem *__restrict__ items, uint32_t items_cap,
                                unsigned long long *__restrict__ evaluated, unsigned long long *__restrict__ total64)
{
    const CfGrid &g = plan->g;
    const int nst = g.nstencil;
    // box pruning needs the cell pair's own shift, which wrap axes (explicit minimum image) lack
    const bool prune = cbox != nullptr && !g.wrap[0] && !g.wrap[1] && !g.wrap[2];
    const bool gp = GP && prune && gbox != nullptr && (plan->tile & 31u) == 0u && plan->jchunk >= 32u;
    const bool zsep = plan->kind == CF_DD_RPPI || plan->kind == CF_WP;
    // (the plan's e2max32 bounds a counted pair's squared separation: for mocks, whose line of sight
    // varies, |s|^2 < rmax^2 + pimax^2; zmax32 bounds |dz| for rp-pi and wp)
    const int64_t nunit = (int64_t)g.ncell * plan->njobs;
    const uint32_t tile = plan->tile, jchunk = plan->jchunk;
    const uint32_t lane = threadIdx.x & 31u;
    unsigned long long ev = 0, nres = 0;
    __shared__ uint32_t s_n, s_base;
    __shared__ __align__(16) CfItem s_items[CFB_ITEM_STAGE];
    // every warp of a block runs the same number of iterations (block-wide barriers in mode 2)
    const int64_t wpb = blockDim.x >> 5, warp = threadIdx.x >> 5;
    // with a list of the units whose i cell holds points, only those (the same count in every thread)
    const int64_t nloop = live ? (int64_t)min(*nlive, (uint32_t)nunit) : nunit;
    for (int64_t ub = blockIdx.x * wpb; ub < nloop; ub += (int64_t)gridDim.x * wpb) {
        if (mode == 2) {
            if (threadIdx.x == 0) s_n = 0;
            __syncthreads();
        }
        if (ub + warp < nloop) {
            const int64_t u = live ? (int64_t)live[ub + warp] : ub + warp;
            const int job = (int)(u / g.ncell);
            const int c = (int)(u - (int64_t)job * g.ncell);
            const CfJobDesc J = jobs[job];
            const CfSetDesc &A = sets[J.a];
            const CfSetDesc &B = sets[J.b];
            const uint32_t ia = cell_start[A.cbeg + c], na = cell_start[A.cbeg + c + 1] - ia;
            uint32_t total = 0;
            if (na) {
                const int ci[3] = {c / (g.n[2] * g.n[1]), (c / g.n[2]) % g.n[1], c % g.n[2]};
                const uint32_t nti = (na + tile - 1) / tile;
                const uint32_t base = mode == 1 ? offsets[u] : 0u;
                // the items of one cell pair under group pruning, in a fixed order (the count and
                // the write enumerate the same ones): for each i tile its box from the groups it
                // holds, then the tile with itself (a cell with itself), then the runs of j groups
                // within reach, each cut into ranges of at most jchunk points.  cache 1 keeps the
                // masks of tiles 0 and 1 when each fits one word, cache 2 takes them from there.
                auto group_items = [&](bool dg, uint32_t jb0, uint32_t nbj, const float (&shv)[3], uint32_t (&mc)[2],
                                       int cache, auto &&emit) {
                    const uint32_t gpt = tile >> 5, gpc = jchunk >> 5;
                    const uint32_t ngi = (na + 31u) >> 5, ngj = (nbj + 31u) >> 5;
                    for (uint32_t a0 = 0; a0 < nti; a0++) {
                        const uint32_t i0 = a0 * tile, ic = min(tile, na - i0);
                        // the runs of set bits of m (groups kb + t) give the j ranges
                        auto runs = [&](uint32_t m, uint32_t kb) {
                            while (m) {
                                const uint32_t t0 = __ffs(m) - 1u;
                                const uint32_t rest = ~(m >> t0);          // zero bits past the run
                                const uint32_t len = min(rest ? __ffs(rest) - 1u : 32u - t0, gpc);
                                const uint32_t k = kb + t0, k1 = k + len;
                                emit(i0, ic, 32u * k, min(32u * k1, nbj) - 32u * k, false);
                                m &= len + t0 >= 32u ? 0u : ~((1u << (t0 + len)) - 1u);
                            }
                        };
                        if (dg) emit(i0, ic, i0, ic, true);
                        const uint32_t kb0 = dg ? (a0 + 1u) * gpt : 0u;
                        const bool one = a0 < 2u && ngj <= kb0 + 32u;
                        if (cache == 2 && one) {
                            runs(a0 == 0u ? mc[0] : mc[1], kb0);
                            continue;
                        }
                        float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
                        for (uint32_t k = a0 * gpt; k < min((a0 + 1u) * gpt, ngi); k++) {
                            const float *q = gbox + 6 * (size_t)(ia + 32u * k);
                            for (int a = 0; a < 3; a++) {
                                blo[a] = fminf(blo[a], q[a]);
                                bhi[a] = fmaxf(bhi[a], q[3 + a]);
                            }
                        }
                        auto within = [&](uint32_t k) {
                            const float *q = gbox + 6 * (size_t)(jb0 + 32u * k);
                            float s2 = 0.f, gz = 0.f;
                            for (int a = 0; a < 3; a++) {
                                const float lo = (blo[a] + shv[a]) - q[3 + a];
                                const float hi = (bhi[a] + shv[a]) - q[a];
                                float gap = lo > 0.f ? lo : (hi < 0.f ? -hi : 0.f);
                                gap = fmaxf(0.f, gap - plan->pmargin[a]);
                                if (zsep && a == 2) gz = gap;
                                else s2 = fmaf(gap, gap, s2);
                            }
                            return !(s2 >= plan->e2max32 || (zsep && gz >= plan->zmax32));
                        };
                        if (cache == 1 && one) {
                            if (a0 == 0u) mc[0] = 0u;
                            else mc[1] = 0u;
                        }
                        // the tests of up to 32 groups are independent (their loads overlap)
                        for (uint32_t kb = kb0; kb < ngj; kb += 32u) {
                            const uint32_t kn = min(32u, ngj - kb);
                            uint32_t m = 0;
#pragma unroll 4
                            for (uint32_t t = 0; t < kn; t++) m |= (within(kb + t) ? 1u : 0u) << t;
                            if (cache == 1 && one) {
                                if (a0 == 0u) mc[0] = m;
                                else mc[1] = m;
                            }
                            runs(m, kb);
                        }
                    }
                };
                // target cells: the 3-D stencil, or for the angular grid the RA cells of the bands
                // within k of this one whose RA range comes within the search angle: two points at
                // declinations up to dm apart by an angle <= t differ in RA by at most
                // 2 asin(sin(t / 2) / cos dm) (from the haversine formula)
                int ncand = nst, nbs = 0;
                int bsel[2 * CFI_MAX_ANG_K + 1], blo[2 * CFI_MAX_ANG_K + 1], bn[2 * CFI_MAX_ANG_K + 1];
                if (plan->ang) {
                    const int ab = cf_band_of(plan, c);
                    const CfBand &Bi = plan->band[ab];
                    const int ar = c - Bi.base, k = g.k[0];
                    ncand = 0;
                    for (int b2 = max(0, ab - k); b2 <= min(plan->nband - 1, ab + k); b2++) {
                        const CfBand &Bj = plan->band[b2];
                        const double da = Bi.da[b2 - ab + k];
                        int lo = 0, n = Bj.nra;
                        if (da >= 0.0) {
                            lo = (int)floor((ar * Bi.w - da) * Bj.inv_w);
                            n = (int)floor(((ar + 1) * Bi.w + da) * Bj.inv_w) - lo + 1;
                            if (n >= Bj.nra) { lo = 0; n = Bj.nra; }
                        }
                        bsel[nbs] = b2;
                        blo[nbs] = lo;
                        bn[nbs] = n;
                        nbs++;
                        ncand += n;
                    }
                }
                for (int s0 = 0; s0 < ncand; s0 += 32) {
                    const int s = s0 + (int)lane;
                    uint32_t cnt = 0, jb = 0, nb = 0, ntj = 0, tsj = 0;
                    bool diag = false;
                    int ct = 0, tj[3] = {0, 0, 0};
                    double delta[3] = {0.0, 0.0, 0.0};      // image of the j point: x_j + delta
                    float sh32[3] = {0.f, 0.f, 0.f};        // the cell pair's shift in float32 (pruning)
                    uint32_t mc[2] = {0u, 0u};              // group masks of the first two i tiles
                    if (s < ncand) {
                        bool ok = true;
                        if (plan->ang) {
                            int q = 0, off = s;
                            while (off >= bn[q]) { off -= bn[q]; q++; }
                            const CfBand &Bj = plan->band[bsel[q]];
                            int rr = (blo[q] + off) % Bj.nra;
                            if (rr < 0) rr += Bj.nra;
                            ct = Bj.base + rr;
                        } else {
                            for (int a = 0; a < 3; a++) {
                                int v = ci[a] + stencil[s].d[a];
                                if (g.wrap[a]) {
                                    v %= g.n[a];
                                } else if (g.periodic) {
                                    if (v < 0) { v += g.n[a]; delta[a] = -g.L[a]; }
                                    else if (v >= g.n[a]) { v -= g.n[a]; delta[a] = g.L[a]; }
                                } else if (v < 0 || v >= g.n[a]) {
                                    ok = false;
                                }
                                tj[a] = v;
                            }
                            ct = (tj[0] * g.n[1] + tj[1]) * g.n[2] + tj[2];
                        }
                        if (ok) {
                            if (!(J.autoc && ct < c)) {
                                jb = cell_start[B.cbeg + ct];
                                nb = cell_start[B.cbeg + ct + 1] - jb;
                                if (nb && prune) {
                                    // separation range of the two boxes per axis under this shift, in
                                    // float32; each gap is shrunk by a margin above this arithmetic's
                                    // rounding and that of the cell-relative coordinates, so a skipped
                                    // pair is out of every bin in FP64 as well
                                    const float *bi = cbox + 6 * (A.cbeg + c), *bj = cbox + 6 * (B.cbeg + ct);
                                    float s2 = 0.f, gz = 0.f;
                                    for (int a = 0; a < 3; a++) {
                                        const float sh =
                                            plan->ang ? plan->origin32[3 * c + a] - plan->origin32[3 * ct + a]
                                                      : (cf_cell_origin32(plan, a, c, ci[a]) -
                                                         cf_cell_origin32(plan, a, ct, tj[a])) - (float)delta[a];
                                        sh32[a] = sh;
                                        const float lo = (bi[a] + sh) - bj[3 + a];
                                        const float hi = (bi[3 + a] + sh) - bj[a];
                                        float gap = lo > 0.f ? lo : (hi < 0.f ? -hi : 0.f);
                                        gap = fmaxf(0.f, gap - plan->pmargin[a]);
                                        if (zsep && a == 2) gz = gap;
                                        else s2 = fmaf(gap, gap, s2);
                                    }
                                    if (s2 >= plan->e2max32 || (zsep && gz >= plan->zmax32)) nb = 0;
                                }
                                if (nb) {
                                    diag = J.autoc && ct == c;
                                    if (diag) {
                                        ntj = nti;
                                        tsj = tile;
                                    } else {
                                        ntj = (nb + jchunk - 1) / jchunk;
                                        tsj = (nb + ntj - 1) / ntj;
                                    }
                                    cnt = diag ? nti * (nti + 1) / 2 : nti * ntj;
                                    if (GP && gp) {
                                        cnt = 0;
                                        group_items(diag, jb, nb, sh32, mc, 1,
                                                    [&](uint32_t, uint32_t, uint32_t, uint32_t, bool) { cnt++; });
                                    }
                                    if (mode == 0) ev += cnt;
                                }
                            }
                        }
                    }
                    uint32_t incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t v = __shfl_up_sync(CF_FULL, incl, o);
                        if ((int)lane >= o) incl += v;
                    }
                    uint32_t cbase = base + total;
                    bool staged = false;
                    if (mode == 2) {
                        const uint32_t ctot = __shfl_sync(CF_FULL, incl, 31);
                        uint32_t r = 0, st = 0;
                        if (lane == 0 && ctot) {
                            // a place in the stage when the entries fit (the CAS only fails when another
                            // warp of the block reserved; bounded, then global), else in the list
                            uint32_t old = *(volatile uint32_t *)&s_n;
                            for (int t = 0; t < 64 && old + ctot <= CFB_ITEM_STAGE; t++) {
                                const uint32_t seen = atomicCAS(&s_n, old, old + ctot);
                                if (seen == old) {
                                    r = old;
                                    st = 1;
                                    break;
                                }
                                old = seen;
                            }
                            if (!st) r = atomicAdd(counts, ctot);
                        }
                        cbase = __shfl_sync(CF_FULL, r, 0);
                        staged = __shfl_sync(CF_FULL, st, 0) != 0;
                        nres += ctot;
                    }
                    if (mode != 0 && cnt) {
                        uint32_t o = cbase + (incl - cnt);
                        // the item's shift in FP64, split into float32 hi + lo (Sec. 4.4 applied per cell)
                        float sh[3], sl[3];
                        for (int a = 0; a < 3; a++) {
                            const double shift =
                                plan->ang ? plan->origin[3 * c + a] - plan->origin[3 * ct + a]
                                          : cf_origin(plan, a, ci[a]) - cf_origin(plan, a, tj[a]) - delta[a];
                            sh[a] = (float)shift;
                            sl[a] = (float)(shift - (double)sh[a]);
                        }
                        auto put = [&](uint32_t i0, uint32_t ic, uint32_t j0, uint32_t jc, bool dflag) {
                            CfItem it;
                            it.ibeg = ia + i0;
                            it.jbeg = jb + j0;
                            it.cnt = ic | (jc << 16);
                            it.meta = (uint32_t)job | (dflag ? CFI_ITEM_DIAG : 0u);
                            it.s[0] = sh[0]; it.s[1] = sh[1]; it.s[2] = sh[2]; it.pad0 = 0.f;
                            it.slo[0] = sl[0]; it.slo[1] = sl[1]; it.slo[2] = sl[2]; it.pad1 = 0.f;
                            if (staged) s_items[o] = it;
                            else if (o < items_cap) items[o] = it;
                            o++;
                            ev += (unsigned long long)ic * jc;
                        };
                        if (GP && gp) {
                            group_items(diag, jb, nb, sh32, mc, 2, put);
                        } else {
                            for (uint32_t a0 = 0; a0 < nti; a0++) {
                                const uint32_t i0 = a0 * tile, ic = min(tile, na - i0);
                                for (uint32_t b = diag ? a0 : 0; b < ntj; b++) {
                                    const uint32_t j0 = b * tsj, jc = min(tsj, nb - j0);
                                    put(i0, ic, j0, jc, diag && b == a0);
                                }
                            }
                        }
                    }
                    total += __shfl_sync(CF_FULL, incl, 31);
                }
            }
            if (mode == 0 && lane == 0) counts[u] = total;
        }
        if (mode == 2) {
            // the block's staged items: one reservation, then 16-byte stores (48-byte items)
            __syncthreads();
            const uint32_t n = s_n;
            if (threadIdx.x == 0 && n) s_base = atomicAdd(counts, n);
            __syncthreads();
            const uint32_t b0 = s_base;
            const uint4 *src = (const uint4 *)s_items;
            uint4 *dst = (uint4 *)(items + b0);
            for (uint32_t k = threadIdx.x; k < 3u * n; k += blockDim.x)
                if (b0 + k / 3u < items_cap) dst[k] = src[k];
            __syncthreads();
        }
    }
    if (evaluated) {
        for (int o = 16; o; o >>= 1) ev += __shfl_xor_sync(CF_FULL, ev, o);
        if ((threadIdx.x & 31) == 0 && ev) atomicAdd(evaluated, ev);
    }
    if (mode == 2 && lane == 0 && nres) atomicAdd(total64, nres);     // nres is the same in every lane
}

// ---------------------------------------------------------------------------------------------
// Order of the work list: the pair kernel dispatches each item to one of four instances of its
// loop (cf_item_class).  Taken in list order, neighbouring warps of an SM would run all four at
// once, and their code together does not stay in the instruction cache; taken class by class, an
// SM runs one at a time (largest tiles first, so the small ones fill the end of the launch).
// A counting sort by class without atomics: block b owns the items [b C, (b + 1) C) with
// C = ceil(n / blocks); the first pass writes each block's class sizes to part[b][k], the second
// finds its offsets from them (the classes before k, the blocks before b) and writes each item's
// index in list order.  The order is the same on every call.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void order_chunk(uint32_t n, uint32_t &beg, uint32_t &end)
{
    const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
    beg = min(n, blockIdx.x * per);
    end = min(n, beg + per);
}

__device__ __forceinline__ uint32_t order_class(const CfItem *__restrict__ items, uint32_t i, uint32_t end)
{
    if (i >= end) return CFI_ITEM_CLASSES;
    const uint2 cm = *reinterpret_cast<const uint2 *>(&items[i].cnt);       // cnt, meta
    return cf_item_class(cm.x, cm.y);
}

__global__ void __launch_bounds__(256) cf_order_count_kernel(const CfItem *__restrict__ items,
                                                             const uint32_t *__restrict__ nitems_dev,
                                                             uint32_t items_cap, uint32_t *__restrict__ part)
{
    __shared__ uint32_t s_c[8][CFI_ITEM_CLASSES];
    uint32_t beg, end;
    order_chunk(min(*nitems_dev, items_cap), beg, end);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t cnt[CFI_ITEM_CLASSES] = {};
    for (uint32_t t = beg; t < end; t += 256u) {
        const uint32_t c = order_class(items, t + threadIdx.x, end);
#pragma unroll
        for (uint32_t k = 0; k < CFI_ITEM_CLASSES; k++) cnt[k] += (uint32_t)__popc(__ballot_sync(CF_FULL, c == k));
    }
    if (lane == 0)
        for (uint32_t k = 0; k < CFI_ITEM_CLASSES; k++) s_c[warp][k] = cnt[k];
    __syncthreads();
    if (threadIdx.x < CFI_ITEM_CLASSES) {
        uint32_t s = 0;
        for (uint32_t w = 0; w < (blockDim.x >> 5); w++) s += s_c[w][threadIdx.x];
        part[blockIdx.x * CFI_ITEM_CLASSES + threadIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) cf_order_scatter_kernel(const CfItem *__restrict__ items,
                                                               const uint32_t *__restrict__ nitems_dev,
                                                               uint32_t items_cap, const uint32_t *__restrict__ part,
                                                               uint32_t *__restrict__ order)
{
    __shared__ uint32_t s_w[8][CFI_ITEM_CLASSES];      // per warp: before this block, then per tile
    __shared__ uint32_t s_base[CFI_ITEM_CLASSES];      // where this block's next item of class k goes
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    {
        // the classes' sizes over all blocks, and over the blocks before this one
        uint32_t tot[CFI_ITEM_CLASSES] = {}, pre[CFI_ITEM_CLASSES] = {};
        for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            for (uint32_t k = 0; k < CFI_ITEM_CLASSES; k++) {
                const uint32_t v = part[b * CFI_ITEM_CLASSES + k];
                tot[k] += v;
                pre[k] += b < blockIdx.x ? v : 0u;
            }
        for (uint32_t k = 0; k < CFI_ITEM_CLASSES; k++)
            for (int o = 16; o; o >>= 1) {
                tot[k] += __shfl_xor_sync(CF_FULL, tot[k], o);
                pre[k] += __shfl_xor_sync(CF_FULL, pre[k], o);
            }
        __shared__ uint32_t s_tot[8][CFI_ITEM_CLASSES];
        if (lane == 0)
            for (uint32_t k = 0; k < CFI_ITEM_CLASSES; k++) {
                s_tot[warp][k] = tot[k];
                s_w[warp][k] = pre[k];
            }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t off = 0;
            for (uint32_t k = 0; k < CFI_ITEM_CLASSES; k++) {
                uint32_t t = 0, p = 0;
                for (uint32_t w = 0; w < nw; w++) {
                    t += s_tot[w][k];
                    p += s_w[w][k];
                }
                s_base[k] = off + p;
                off += t;
            }
        }
        __syncthreads();
    }
    uint32_t beg, end;
    order_chunk(min(*nitems_dev, items_cap), beg, end);
    const uint32_t below = (1u << lane) - 1u;
    for (uint32_t t = beg; t < end; t += 256u) {
        const uint32_t i = t + threadIdx.x;
        const uint32_t c = order_class(items, i, end);
        uint32_t mine = 0;      // the ballot of this thread's class
#pragma unroll
        for (uint32_t k = 0; k < CFI_ITEM_CLASSES; k++) {
            const uint32_t m = __ballot_sync(CF_FULL, c == k);
            if (c == k) mine = m;
            if (lane == 0) s_w[warp][k] = (uint32_t)__popc(m);
        }
        __syncthreads();
        if (c < CFI_ITEM_CLASSES) {
            uint32_t r = s_base[c] + (uint32_t)__popc(mine & below);
            for (uint32_t w = 0; w < warp; w++) r += s_w[w][c];
            order[r] = i;       // r < n: the class's place plus its rank among the class's n_k items
        }
        __syncthreads();
        if (threadIdx.x < CFI_ITEM_CLASSES) {
            uint32_t s = 0;
            for (uint32_t w = 0; w < nw; w++) s += s_w[w][threadIdx.x];
            s_base[threadIdx.x] += s;
        }
        __syncthreads();
    }
}

// sum of w^2 per set (self pairs of a weighted auto-correlation whose first edge is 0)
__global__ void cf_wsq_kernel(const CfSetDesc *__restrict__ sets, double *__restrict__ out)
{
    const CfSetDesc S = sets[blockIdx.y];
    double s = 0;
    if (S.w)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.n; i += (int64_t)gridDim.x * blockDim.x) {
            double w = cf_load(S.w, S.dtype, i);
            s += w * w;
        }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(CF_FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0) atomicAdd(out + blockIdx.y, s);
}

// ---------------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------------
static int blocks_for(int64_t n, int threads, int cap)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// the starting values of cf_bbox_kernel's reductions (minima at ~0, maxima and counters at 0)
__global__ void cf_bbox_init_kernel(unsigned long long *__restrict__ out, int nsets)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsets * CFB_BBOX_WORDS; i += gridDim.x * blockDim.x) {
        const int a = i % CFB_BBOX_WORDS;
        out[i] = (a < 3 || a == 8 || a == 9) ? ~0ull : 0ull;
    }
}

cudaError_t cfb_bbox_init(unsigned long long *out, int nsets, cudaStream_t st)
{
    cf_bbox_init_kernel<<<blocks_for((int64_t)nsets * CFB_BBOX_WORDS, 256, 64), 256, 0, st>>>(out, nsets);
    return cudaGetLastError();
}

cudaError_t cfb_bbox(const CfSetDesc *sets, int nsets, int64_t nmax, unsigned long long *out, cudaStream_t st)
{
    dim3 grid(blocks_for((nmax + 3) / 4, 256, 1024), nsets);     // four float32 points per thread and step
    cf_bbox_kernel<<<grid, 256, 0, st>>>(sets, out);
    return cudaGetLastError();
}

cudaError_t cfb_assign(const CfDevPlan *plan, const CfSetDesc *sets, int nsets, int64_t nmax, int sub,
                       uint32_t *count, uint32_t *key, uint32_t *slot, cudaStream_t st)
{
    dim3 grid(blocks_for(nmax, 256, 4096), nsets);
    cf_assign_kernel<<<grid, 256, 0, st>>>(plan, sets, sub, count, key, slot);
    return cudaGetLastError();
}

cudaError_t cfb_ang_origins(const CfDevPlan *plan, int ncell, double *origin, float *origin32, cudaStream_t st)
{
    cf_ang_origin_kernel<<<blocks_for(ncell, 256, 4096), 256, 0, st>>>(plan, ncell, origin, origin32);
    return cudaGetLastError();
}

int64_t cfb_scan_tmp_words(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 8; }

cudaError_t cfb_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, uint32_t *done, cudaStream_t st,
                     uint32_t *total_copy, uint32_t *every, int every_shift)
{
    int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles < 1) ntiles = 1;
    cf_scan_reduce<<<(unsigned)ntiles, SCAN_T, 0, st>>>(in, n, tmp, done);
    cf_scan_apply<<<(unsigned)ntiles, SCAN_T, 0, st>>>(in, out, n, tmp, total_copy, every, every_shift);
    return cudaGetLastError();
}

cudaError_t cfb_scatter(const CfDevPlan *plan, const CfSetDesc *sets, int nsets, int64_t nmax, int sub,
                        const uint32_t *fstart, const uint32_t *key, const uint32_t *slot, float4 *pa,
                        float4 *pb, float4 *plo, uint32_t *orig, cudaStream_t st)
{
    dim3 grid(blocks_for(nmax, 256, 4096), nsets);
    cf_scatter_kernel<<<grid, 256, 0, st>>>(plan, sets, (uint32_t)(sub * sub * sub), fstart, key, slot, pa, pb, plo,
                                            orig);
    return cudaGetLastError();
}

cudaError_t cfb_cellbox(const uint32_t *cell_start, int64_t ncell_all, const float4 *pa, const float4 *pb, float *box,
                        float *gbox, cudaStream_t st)
{
    cf_cellbox_kernel<<<blocks_for(ncell_all * 32, 256, 8192), 256, 0, st>>>(cell_start, ncell_all, pa, pb, box, gbox);
    return cudaGetLastError();
}

cudaError_t cfb_live_units(const CfDevPlan *plan, const CfSetDesc *sets, const CfJobDesc *jobs,
                           const uint32_t *cell_start, int64_t nunits, uint32_t *live, uint32_t *nlive,
                           cudaStream_t st)
{
    cf_live_units_kernel<<<blocks_for(nunits, 256, 4096), 256, 0, st>>>(plan, sets, jobs, cell_start, live, nlive);
    return cudaGetLastError();
}

cudaError_t cfb_items(const CfDevPlan *plan, const CfSetDesc *sets, const CfJobDesc *jobs, const CfStencil *stencil,
                      const uint32_t *cell_start, const float *cbox, const float *gbox, const uint32_t *live,
                      const uint32_t *nlive, int64_t nunits, int mode, uint32_t *counts, const uint32_t *offsets,
                      CfItem *items, uint32_t items_cap, unsigned long long *evaluated, unsigned long long *total64,
                      cudaStream_t st)
{
    const int nb = blocks_for(nunits * 32, 256, 8192);
    if (gbox)
        cf_items_kernel<true><<<nb, 256, 0, st>>>(plan, sets, jobs, stencil, cell_start, cbox, gbox, live, nlive,
                                                  mode, counts, offsets, items, items_cap, evaluated, total64);
    else
        cf_items_kernel<false><<<nb, 256, 0, st>>>(plan, sets, jobs, stencil, cell_start, cbox, nullptr, live, nlive,
                                                   mode, counts, offsets, items, items_cap, evaluated, total64);
    return cudaGetLastError();
}

cudaError_t cfb_order(const CfItem *items, const uint32_t *nitems_dev, uint32_t items_cap, uint32_t *order,
                      uint32_t *part, int num_sms, cudaStream_t st)
{
    const int nb = cfb_order_blocks(items_cap, num_sms);
    cf_order_count_kernel<<<nb, 256, 0, st>>>(items, nitems_dev, items_cap, part);
    cf_order_scatter_kernel<<<nb, 256, 0, st>>>(items, nitems_dev, items_cap, part, order);
    return cudaGetLastError();
}

cudaError_t cfb_wsq(const CfSetDesc *sets, int nsets, int64_t nmax, double *out, cudaStream_t st)
{
    dim3 grid(blocks_for(nmax, 256, 1024), nsets);
    cf_wsq_kernel<<<grid, 256, 0, st>>>(sets, out);
    return cudaGetLastError();
}
