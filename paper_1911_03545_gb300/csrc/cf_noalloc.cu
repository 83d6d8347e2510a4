// cf_noalloc.cu -- a pair count that allocates no memory, for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's memory pool
// (every device byte must come from that pool, and a stray allocation breaks its accounting or
// fragments it), plugins that run where allocation is forbidden or may block, and programs
// that must not allocate after start-up because an allocation can synchronise the device.
// cf_count_noalloc serves them: the caller passes device inputs and device outputs, and the
// only scratch this function uses is the fixed array below, part of the library's image.
//
// The kernel is a variant of the FP64 recheck kernel (cf_recheck.cu) applied to every pair of
// the inputs without a cell list: the exact FP64 separation and bin of each pair, accumulated
// in a block-private shared-memory histogram and added into the scratch histogram.  It is
// meant for small inputs; its cost grows with N1 * N2.
//
// Scratch: `g_noalloc_scratch`, CF_NOALLOC_SCRATCH_BYTES bytes in every device that loads the
// library, held until the process exits.  In host code the symbol is only a host-side stand-in
// for the device array, so its device address is obtained once per device with
// cudaGetSymbolAddress (the first call on a device does this, with that device current; make
// that first call before any stream capture).  All calls share the array and it keeps the last
// call's contents: each call clears its histogram first, and calls whose work overlaps on the
// GPU (different streams, or the same stream from several host threads without ordering) race
// on it and must not be issued.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "cf_device.cuh"
#include "cf_plan.h"

namespace {

struct NaParams {
    int kind, nb, npi, nslot;
    int autoc, weighted, ravg, self_pairs;
    double L[3];
    double pimax;
    double e2[CF_MAX_BINS + 1];
    double pe[CF_MAX_PIBINS + 1];
};

// layout of the scratch array: [ count u64 | wsum f64 | rsum f64 ] x CF_NOALLOC_MAX_SLOTS, then
// the sum of w^2 (self pairs of a weighted auto-correlation)
constexpr size_t kHistBytes = (size_t)CF_NOALLOC_MAX_SLOTS * 24;
static_assert(kHistBytes + 64 <= CF_NOALLOC_SCRATCH_BYTES, "scratch too small");

__device__ __align__(256) unsigned char g_noalloc_scratch[CF_NOALLOC_SCRATCH_BYTES];

__device__ __forceinline__ double na_sep(double a, double b, double L)
{
    double d = __dsub_rn(a, b);
    if (L > 0.0) {
        double h = 0.5 * L;
        if (d > h) d = __dsub_rn(d, L);
        if (d <= -h) d = __dadd_rn(d, L);
    }
    return d;
}

__device__ __forceinline__ int na_find(const double *e, int n, double s)
{
    int k = n - 1;
    while (k > 0 && s < e[k]) k--;
    return k;
}

// clear the three per-slot arrays (each CF_NOALLOC_MAX_SLOTS long) and the w^2 sum
__global__ void na_clear(unsigned char *scratch, int nslot)
{
    unsigned long long *h = (unsigned long long *)scratch;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nslot; i += gridDim.x * blockDim.x) {
        h[i] = 0ull;
        h[CF_NOALLOC_MAX_SLOTS + i] = 0ull;
        h[2 * CF_NOALLOC_MAX_SLOTS + i] = 0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *(double *)(scratch + kHistBytes) = 0.0;
}

// every pair (i, j): j > i for an auto-correlation, all j for a cross-correlation
__global__ void na_pairs(const NaParams P, CfSetDesc A, CfSetDesc B, unsigned char *scratch)
{
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long *sc = (unsigned long long *)sm;
    double *sw = (double *)(sm + 8 * (size_t)P.nslot);
    double *sr = sw + P.nslot;
    for (int i = threadIdx.x; i < P.nslot; i += blockDim.x) {
        sc[i] = 0ull;
        sw[i] = 0.0;
        sr[i] = 0.0;
    }
    __syncthreads();
    double wsq = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double xi = cf_load(A.x, A.dtype, i), yi = cf_load(A.y, A.dtype, i), zi = cf_load(A.z, A.dtype, i);
        const double wi = P.weighted ? cf_load(A.w, A.dtype, i) : 1.0;
        if (P.self_pairs) wsq += __dmul_rn(wi, wi);
        for (int64_t j = P.autoc ? i + 1 : 0; j < B.n; j++) {
            if (P.kind == 4) {
                // mocks (Appendix A.2.1): squared pi edges in pe
                double rp2, pi2;
                cf_mocks64(xi, yi, zi, cf_load(B.x, B.dtype, j), cf_load(B.y, B.dtype, j), cf_load(B.z, B.dtype, j),
                           rp2, pi2);
                if (!(pi2 < P.pe[P.npi]) || rp2 < P.e2[0] || rp2 >= P.e2[P.nb]) continue;
                const int slot = na_find(P.e2, P.nb, rp2) * P.npi + na_find(P.pe, P.npi, pi2);
                const double ww = P.weighted ? __dmul_rn(wi, cf_load(B.w, B.dtype, j)) : 1.0;
                atomicAdd(sc + slot, 1ull);
                if (P.weighted) atomicAdd(sw + slot, ww);
                if (P.ravg) atomicAdd(sr + slot, __dmul_rn(ww, sqrt(rp2)));
                continue;
            }
            const double dx = na_sep(xi, cf_load(B.x, B.dtype, j), P.L[0]);
            const double dy = na_sep(yi, cf_load(B.y, B.dtype, j), P.L[1]);
            const double dz = na_sep(zi, cf_load(B.z, B.dtype, j), P.L[2]);
            int slot;
            double sep = 0.0;
            if (P.kind == 0 || P.kind == 3) {
                double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                s = __dadd_rn(s, __dmul_rn(dz, dz));
                if (s < P.e2[0] || s >= P.e2[P.nb]) continue;
                slot = na_find(P.e2, P.nb, s);
                if (P.ravg) {
                    double c = sqrt(s);
                    sep = P.kind == 3 ? 2.0 * asin(0.5 * c) * (180.0 / 3.141592653589793) : c;
                }
            } else {
                double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                double pi = fabs(dz);
                if (s < P.e2[0] || s >= P.e2[P.nb] || !(pi < P.pimax)) continue;
                slot = na_find(P.e2, P.nb, s);
                if (P.ravg) sep = sqrt(s);
                if (P.kind == 1) slot = slot * P.npi + na_find(P.pe, P.npi, pi);
            }
            const double ww = P.weighted ? __dmul_rn(wi, cf_load(B.w, B.dtype, j)) : 1.0;
            atomicAdd(sc + slot, 1ull);
            if (P.weighted) atomicAdd(sw + slot, ww);
            if (P.ravg) atomicAdd(sr + slot, __dmul_rn(ww, sep));
        }
    }
    __syncthreads();
    unsigned long long *gc = (unsigned long long *)scratch;
    double *gw = (double *)(scratch + 8 * (size_t)CF_NOALLOC_MAX_SLOTS);
    double *gr = gw + CF_NOALLOC_MAX_SLOTS;
    for (int k = threadIdx.x; k < P.nslot; k += blockDim.x) {
        if (sc[k]) atomicAdd(gc + k, sc[k]);
        if (sw[k] != 0.0) atomicAdd(gw + k, sw[k]);
        if (sr[k] != 0.0) atomicAdd(gr + k, sr[k]);
    }
    if (P.self_pairs && P.weighted) {
        for (int o = 16; o; o >>= 1) wsq += __shfl_xor_sync(CF_FULL, wsq, o);
        if ((threadIdx.x & 31) == 0 && wsq != 0.0) atomicAdd((double *)(scratch + kHistBytes), wsq);
    }
}

// outputs: doubling and self pairs of an auto-correlation (Sec. 4.3, Appendix B), ravg
__global__ void na_finish(const NaParams P, int64_t n1, const unsigned char *scratch, uint64_t *npairs,
                          double *wsum, double *ravg)
{
    const unsigned long long *gc = (const unsigned long long *)scratch;
    const double *gw = (const double *)(scratch + 8 * (size_t)CF_NOALLOC_MAX_SLOTS);
    const double *gr = gw + CF_NOALLOC_MAX_SLOTS;
    const double wsq = *(const double *)(scratch + kHistBytes);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.nslot; k += gridDim.x * blockDim.x) {
        const unsigned long long m = P.autoc ? 2ull : 1ull;
        unsigned long long c = gc[k] * m;
        double w = P.weighted ? gw[k] * (double)m : 0.0;
        const double r = gr[k] * (double)m;
        if (k == 0 && P.autoc && P.self_pairs) {
            c += (unsigned long long)n1;
            w += wsq;
        }
        if (!P.weighted) w = (double)c;
        if (npairs) npairs[k] = c;
        if (wsum) wsum[k] = w;
        if (ravg) {
            const double den = P.weighted ? w : (double)c;
            ravg[k] = (P.ravg && den > 0) ? r / den : 0.0;
        }
    }
}

std::mutex g_mu;
void *g_addr[64] = {nullptr};
thread_local std::string g_err;   // detail of the last failure (for debugging)

}  // namespace

extern "C" cf_status cf_count_noalloc(const cf_params *params, const cf_points *d1, const cf_points *d2,
                                      uint64_t *npairs, double *wsum, double *ravg, void *cuda_stream)
{
    g_err.clear();
    std::string err;
    if (cfp_check_params(params, err) != CF_OK) {
        g_err = err;
        return CF_ERR_ARG;
    }
    if (!d1 || (params->autocorr ? d2 != nullptr : d2 == nullptr)) {
        g_err = "d2 must be NULL for an auto-correlation and given for a cross-correlation";
        return CF_ERR_ARG;
    }
    const cf_points *sets[2] = {d1, params->autocorr ? d1 : d2};
    for (const cf_points *d : sets) {
        if (!d->on_device && d->n > 0) {
            g_err = "inputs must be device arrays";
            return CF_ERR_ARG;
        }
        if (d->n < 0 || d->n >= ((int64_t)1 << 31) || (d->dtype != CF_F32 && d->dtype != CF_F64) ||
            (d->n > 0 && (!d->x || !d->y || !d->z)) || (params->weight == CF_W_PAIR_PRODUCT && d->n > 0 && !d->w)) {
            g_err = "invalid point set";
            return CF_ERR_ARG;
        }
    }
    NaParams P;
    std::memset(&P, 0, sizeof(P));
    P.kind = params->kind;
    P.nb = params->nbins;
    P.npi = (params->kind == CF_DD_RPPI || params->kind == CF_DD_RPPI_MOCKS) ? params->npibins : 1;
    P.nslot = P.nb * P.npi;
    if (P.nslot > CF_NOALLOC_MAX_SLOTS) {
        g_err = "more than " + std::to_string(CF_NOALLOC_MAX_SLOTS) + " histogram slots (the scratch limit)";
        return CF_ERR_ARG;
    }
    P.autoc = params->autocorr ? 1 : 0;
    P.weighted = params->weight == CF_W_PAIR_PRODUCT;
    P.ravg = params->output_ravg ? 1 : 0;
    P.self_pairs = (P.autoc && params->edges[0] == 0.0) ? 1 : 0;
    for (int a = 0; a < 3; a++) P.L[a] = params->periodic ? params->box[a] : 0.0;
    P.pimax = params->pimax;
    cfp_edges(params, P.e2, P.pe);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        g_err = "no current CUDA device";
        return CF_ERR_CUDA;
    }
    void *scratch;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return CF_ERR_CUDA;
            }
            g_addr[dev] = p;
        }
        scratch = g_addr[dev];
    }
    CfSetDesc A, B;
    std::memset(&A, 0, sizeof(A));
    std::memset(&B, 0, sizeof(B));
    const cf_points *s2 = sets[1];
    A.x = d1->x; A.y = d1->y; A.z = d1->z; A.w = P.weighted ? d1->w : nullptr; A.n = d1->n; A.dtype = d1->dtype;
    B.x = s2->x; B.y = s2->y; B.z = s2->z; B.w = P.weighted ? s2->w : nullptr; B.n = s2->n; B.dtype = s2->dtype;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    na_clear<<<8, 256, 0, st>>>((unsigned char *)scratch, P.nslot);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = 24 * (size_t)P.nslot;
    int64_t blocks = (A.n + 127) / 128;
    if (blocks > 4 * sms) blocks = 4 * sms;
    if (blocks < 1) blocks = 1;
    if (A.n > 0 && B.n > 0) na_pairs<<<(unsigned)blocks, 128, smem, st>>>(P, A, B, (unsigned char *)scratch);
    na_finish<<<(P.nslot + 255) / 256, 256, 0, st>>>(P, d1->n, (const unsigned char *)scratch, npairs, wsum, ravg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_err = std::string("launch: ") + cudaGetErrorString(e);
        return CF_ERR_CUDA;
    }
    return CF_OK;
}
