// cf_recheck.cu -- FP64 re-evaluation of pairs whose FP32 squared separation fell within the
// error band of a bin edge, and the pair-kernel dispatcher.
//
// The arithmetic is the result definition itself (Sec. 2.1 Code naivecorr; Appendix A.1 Eq. sep;
// Sec. 4.4 Code normal_pbc), evaluated on the original coordinates in FP64 with explicit
// round-to-nearest operations and no fused multiply-add: d = a - b, wrapped once each way for a
// periodic axis, s = (dx*dx + dy*dy) + dz*dz, bins half-open against the FP64 squared edges.
// Mocks (Appendix A.2.1) take cf_mocks64: pi^2 and rp^2 from the pair's line of sight.
#include "cf_build.h"
#include "cf_device.cuh"
#include "cf_pair.cuh"

__device__ __forceinline__ double cf_sep64(double a, double b, double L)
{
    double d = __dsub_rn(a, b);
    if (L > 0.0) {
        double h = 0.5 * L;
        if (d > h) d = __dsub_rn(d, L);
        if (d <= -h) d = __dadd_rn(d, L);
    }
    return d;
}

__device__ __forceinline__ int cf_find64(const double *e, int n, double s)
{
    int k = n - 1;
    while (k > 0 && s < e[k]) k--;
    return k;
}

__global__ void cf_recheck_kernel(const CfDevPlan *__restrict__ P, const CfSetDesc *__restrict__ sets,
                                  const CfJobDesc *__restrict__ jobs, const uint4 *__restrict__ queue,
                                  const unsigned long long *__restrict__ qcount, uint32_t qcap,
                                  unsigned long long *__restrict__ hcnt, double *__restrict__ hw,
                                  double *__restrict__ hr)
{
    const uint32_t n = (uint32_t)min(*qcount, (unsigned long long)qcap);
    const int kind = P->kind, nb = P->nb, npi = P->npi, nslot = P->nslot;
    const double L0 = P->g.periodic ? P->g.L[0] : 0.0;
    const double L1 = P->g.periodic ? P->g.L[1] : 0.0;
    const double L2 = P->g.periodic ? P->g.L[2] : 0.0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint4 e = queue[k];
        const CfJobDesc J = jobs[e.z];
        const CfSetDesc &A = sets[J.a];
        const CfSetDesc &B = sets[J.b];
        int slot;
        double sep = 0.0;
        if (kind == 4) {
            // mocks (Appendix A.2.1): squared pi edges in pe, pimax^2 = pe[npi]
            double rp2, pi2;
            cf_mocks64(cf_load(A.x, A.dtype, e.x), cf_load(A.y, A.dtype, e.x), cf_load(A.z, A.dtype, e.x),
                       cf_load(B.x, B.dtype, e.y), cf_load(B.y, B.dtype, e.y), cf_load(B.z, B.dtype, e.y), rp2, pi2);
            if (!(pi2 < P->pe[npi])) continue;
            if (rp2 < P->e2[0] || rp2 >= P->e2[nb]) continue;
            slot = cf_find64(P->e2, nb, rp2) * npi + cf_find64(P->pe, npi, pi2);
            if (P->ravg) sep = sqrt(rp2);
            const size_t g = (size_t)e.z * nslot + slot;
            atomicAdd(hcnt + g, 1ull);
            double ww = 1.0;
            if (P->weighted) ww = __dmul_rn(cf_load(A.w, A.dtype, e.x), cf_load(B.w, B.dtype, e.y));
            if (P->weighted) atomicAdd(hw + g, ww);
            if (P->ravg) atomicAdd(hr + g, __dmul_rn(ww, sep));
            continue;
        }
        double dx = cf_sep64(cf_load(A.x, A.dtype, e.x), cf_load(B.x, B.dtype, e.y), L0);
        double dy = cf_sep64(cf_load(A.y, A.dtype, e.x), cf_load(B.y, B.dtype, e.y), L1);
        double dz = cf_sep64(cf_load(A.z, A.dtype, e.x), cf_load(B.z, B.dtype, e.y), L2);
        if (kind == 0 || kind == 3) {
            double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            s = __dadd_rn(s, __dmul_rn(dz, dz));
            if (s < P->e2[0] || s >= P->e2[nb]) continue;
            slot = cf_find64(P->e2, nb, s);
            if (P->ravg) {
                double c = sqrt(s);
                sep = kind == 3 ? 2.0 * asin(0.5 * c) * (180.0 / 3.141592653589793) : c;
            }
        } else {
            double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            double pi = fabs(dz);
            if (s < P->e2[0] || s >= P->e2[nb]) continue;
            if (!(pi < P->pimax)) continue;
            slot = cf_find64(P->e2, nb, s);
            if (P->ravg) sep = sqrt(s);
            if (kind == 1) slot = slot * npi + cf_find64(P->pe, npi, pi);
        }
        const size_t g = (size_t)e.z * nslot + slot;
        atomicAdd(hcnt + g, 1ull);
        double ww = 1.0;
        if (P->weighted) ww = __dmul_rn(cf_load(A.w, A.dtype, e.x), cf_load(B.w, B.dtype, e.y));
        if (P->weighted) atomicAdd(hw + g, ww);
        if (P->ravg) atomicAdd(hr + g, __dmul_rn(ww, sep));
    }
}

// CF_OPT_AUDIT, in place of the pair kernel: every pair of every work item goes to the FP64 recheck
// queue and nothing is binned in FP32, so the call returns the FP64 result of every evaluated pair.
// A warp takes items in turn; a lane takes i rows of the item and reserves each row's entries with
// one atomic.  Entries past the queue capacity are dropped: the host sees the count and repeats the
// call with a larger queue.
__global__ void cf_audit_kernel(const CfItem *__restrict__ items, const uint32_t *__restrict__ nitems_dev,
                                uint32_t items_cap, const uint32_t *__restrict__ orig, uint4 *__restrict__ queue,
                                unsigned long long *__restrict__ qcount, uint32_t qcap)
{
    const uint32_t n = min(*nitems_dev, items_cap);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n; t += nw) {
        const CfItem it = items[t];
        const uint32_t ic = it.cnt & 0xFFFFu, jc = it.cnt >> 16;
        const bool diag = (it.meta & CFI_ITEM_DIAG) != 0;
        const uint32_t jo = it.meta & CFI_ITEM_JOBMASK;
        for (uint32_t il = lane; il < ic; il += 32u) {
            const uint32_t j0 = diag ? il + 1u : 0u;      // within a cell paired with itself: j > i
            if (j0 >= jc) continue;
            const uint32_t cnt = jc - j0;
            const unsigned long long base = atomicAdd(qcount, (unsigned long long)cnt);
            const uint32_t oi = orig[it.ibeg + il];
            for (uint32_t k = 0; k < cnt; k++)
                if (base + k < qcap) queue[base + k] = make_uint4(oi, orig[it.jbeg + j0 + k], jo, 0u);
        }
    }
}

cudaError_t cfp_launch_audit(const CfItem *items, const uint32_t *nitems_dev, uint32_t items_cap,
                             const uint32_t *orig, uint4 *queue, unsigned long long *qcount, uint32_t qcap, int num_sms,
                             cudaStream_t st)
{
    cf_audit_kernel<<<num_sms * 4, 256, 0, st>>>(items, nitems_dev, items_cap, orig, queue, qcount, qcap);
    return cudaGetLastError();
}

cudaError_t cfp_launch_recheck(const CfDevPlan *plan, const CfSetDesc *sets, const CfJobDesc *jobs,
                               const uint4 *queue, const unsigned long long *qcount, uint32_t qcap,
                               unsigned long long *hcnt, double *hw, double *hr, int num_sms, cudaStream_t st)
{
    cf_recheck_kernel<<<num_sms * 2, 256, 0, st>>>(plan, sets, jobs, queue, qcount, qcap, hcnt, hw, hr);
    return cudaGetLastError();
}

// ---- pair-kernel dispatch ----
cudaError_t cfp_launch_r(const CfPairCfg &, const CfPairArgs &, int, cudaStream_t, int *, int *);
cudaError_t cfp_launch_rppi(const CfPairCfg &, const CfPairArgs &, int, cudaStream_t, int *, int *);
cudaError_t cfp_launch_wp(const CfPairCfg &, const CfPairArgs &, int, cudaStream_t, int *, int *);
cudaError_t cfp_launch_theta(const CfPairCfg &, const CfPairArgs &, int, cudaStream_t, int *, int *);
cudaError_t cfp_launch_mocks(const CfPairCfg &, const CfPairArgs &, int, cudaStream_t, int *, int *);

size_t cfp_pair_smem(const CfPairCfg &c, int warps)
{
    size_t b = cfpair::align16(2u * (uint32_t)c.nlut_words) + (size_t)c.nfine * 16;
    if (cfpair::warp_hist(c.kind)) b += cfpair::align16(4u * (uint32_t)c.nb);   // per rp bin ravg scales
    return b + (size_t)cfpair::warp_bytes(c.kind, c.weighted != 0, c.ravg != 0, c.lo != 0, c.ghist ? 0 : c.nslot,
                                          c.variant == 2) * warps;
}

cudaError_t cfp_launch_pair(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                            int *warps_out)
{
    switch (c.kind) {
    case 0: return cfp_launch_r(c, a, num_sms, st, grid_out, warps_out);
    case 1: return cfp_launch_rppi(c, a, num_sms, st, grid_out, warps_out);
    case 2: return cfp_launch_wp(c, a, num_sms, st, grid_out, warps_out);
    case 3: return cfp_launch_theta(c, a, num_sms, st, grid_out, warps_out);
    case 4: return cfp_launch_mocks(c, a, num_sms, st, grid_out, warps_out);
    }
    return cudaErrorInvalidValue;
}
