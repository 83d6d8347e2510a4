// cf_build.h -- launchers of the cell-build, work-list and pair-count kernels.
#pragma once
#include <cuda_runtime.h>

#include "cf_internal.h"

// per point set: 3 min keys, 3 max keys, bad, norm deviation, min |v|^2, smallest nonzero |w|,
// largest |w|, negative weights
#define CFB_BBOX_WORDS 12
#define CFB_ITEM_STAGE 256      // work items a block of the one-pass work list stages in shared memory
cudaError_t cfb_bbox(const CfSetDesc *sets, int nsets, int64_t nmax, unsigned long long *out, cudaStream_t st);
// fills out[nsets * CFB_BBOX_WORDS] with the starting values cfb_bbox reduces into
cudaError_t cfb_bbox_init(unsigned long long *out, int nsets, cudaStream_t st);
// key = cell * sub^3 + Morton sub-cell (sub = 1, 2, 4): the counting-sort key of every point
cudaError_t cfb_assign(const CfDevPlan *plan, const CfSetDesc *sets, int nsets, int64_t nmax, int sub,
                       uint32_t *count, uint32_t *key, uint32_t *slot, cudaStream_t st);
// origins of the angular grid's cells (3 per cell) from their (RA, DEC) boxes
cudaError_t cfb_ang_origins(const CfDevPlan *plan, int ncell, double *origin, float *origin32, cudaStream_t st);
int64_t cfb_scan_tmp_words(int64_t n);
// exclusive scan of n counts into out[0..n) and the total into out[n] (and *total_copy if given);
// tmp holds cfb_scan_tmp_words(n) words, *done must be 0 (a ticket counter).  every, if given,
// receives every[i >> every_shift] = out[i] for the multiples i of 2^every_shift up to n (the cell
// starts among the sub-cell starts: cell_start[c] = fstart[c * sub^3]).
cudaError_t cfb_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, uint32_t *done, cudaStream_t st,
                     uint32_t *total_copy = nullptr, uint32_t *every = nullptr, int every_shift = 0);
cudaError_t cfb_scatter(const CfDevPlan *plan, const CfSetDesc *sets, int nsets, int64_t nmax, int sub,
                        const uint32_t *fstart, const uint32_t *key, const uint32_t *slot, float4 *pa,
                        float4 *pb, float4 *plo, uint32_t *orig, cudaStream_t st);
// tight point bounding box per cell (6 floats: lo xyz, hi xyz, cell-relative), for cell-pair pruning;
// with gbox (6 floats per point) also the box of every 32-point group of a cell at its first point
cudaError_t cfb_cellbox(const uint32_t *cell_start, int64_t ncell_all, const float4 *pa, const float4 *pb, float *box,
                        float *gbox, cudaStream_t st);
// the units (job, i cell) whose i cell holds points, appended to live[] (nunits entries) at the
// zeroed counter *nlive
cudaError_t cfb_live_units(const CfDevPlan *plan, const CfSetDesc *sets, const CfJobDesc *jobs,
                           const uint32_t *cell_start, int64_t nunits, uint32_t *live, uint32_t *nlive,
                           cudaStream_t st);
// cbox: the boxes above, or nullptr to visit every stencil neighbour; gbox: the group boxes, or
// nullptr for j ranges over whole cells; live / nlive: the units to visit (cfb_live_units), or
// nullptr for all of them (with a list, mode 0 writes the counts of the listed units only: the
// caller zeroes the rest).  mode 0: per-unit item counts
// into counts[], their number in 64 bits added to *evaluated; mode 1: items at offsets[]; mode 2:
// count and emit in one pass, items reserved on the counter counts[0] (zeroed by the caller), their
// number added to *total64.  Modes 1 and 2 add the pairs the stored items hold to *evaluated.
cudaError_t cfb_items(const CfDevPlan *plan, const CfSetDesc *sets, const CfJobDesc *jobs, const CfStencil *stencil,
                      const uint32_t *cell_start, const float *cbox, const float *gbox, const uint32_t *live,
                      const uint32_t *nlive, int64_t nunits, int mode, uint32_t *counts, const uint32_t *offsets,
                      CfItem *items, uint32_t items_cap, unsigned long long *evaluated, unsigned long long *total64,
                      cudaStream_t st);
// work lists of a smaller capacity are taken in list order (CfPairArgs::order = NULL): the two
// ordering passes cost 12-15 us, the pair kernel saves 3-7 %, so they pay from about 0.3 ms of
// pair kernel (some 30,000 items)
#define CF_ORDER_MIN_ITEMS 40960u
// the order in which the pair kernel takes the work list: the indices of the items of each class
// (cf_item_class) together, classes in increasing order and each class in list order, so that the
// warps of an SM run one instance's code at a time.  order[] needs min(*nitems_dev, items_cap)
// entries; part[] CFI_ITEM_CLASSES words per block of the launch (cfb_order_blocks), no initial
// value.
inline int cfb_order_blocks(uint32_t items_cap, int num_sms)
{
    const int cap = num_sms > 0 ? 4 * num_sms : 4;
    const int64_t b = ((int64_t)items_cap + 255) / 256;
    return b < 1 ? 1 : (b > cap ? cap : (int)b);
}
cudaError_t cfb_order(const CfItem *items, const uint32_t *nitems_dev, uint32_t items_cap, uint32_t *order,
                      uint32_t *part, int num_sms, cudaStream_t st);
cudaError_t cfb_wsq(const CfSetDesc *sets, int nsets, int64_t nmax, double *out, cudaStream_t st);

// ---- pair counting ----
struct CfPairArgs {
    const CfDevPlan *plan;
    const uint16_t *lut;         // coarse LUT entries (global copy; staged into shared memory)
    const CfFine *fine;          // fine LUT entries
    const CfItem *items;
    const uint32_t *order;       // the items in the order they are taken (cfb_order; NULL: list order)
    const uint32_t *nitems_dev;  // item count written by the work-list scan
    uint32_t items_cap;          // items beyond this were not stored
    uint32_t qcap;
    uint32_t *cursor;
    const ulonglong2 *pa;        // (-X,-X | -Y,-Y)
    const ulonglong2 *pb;        // (-Z,-Z | w, w)
    const ulonglong2 *plo;       // FP64 residuals, two per point (may be NULL)
    const uint32_t *orig;
    unsigned long long *hcnt;    // [njobs][nslot]
    double *hw;                  // [njobs][nslot]
    double *hr;                  // [njobs][nslot]
    uint4 *queue;                // (orig i, orig j, job, 0)
    unsigned long long *qcount;  // queued pairs, 64-bit so that it cannot wrap (entries >= qcap are dropped)
    float L[3];                  // periodic sides (wrap axes)
    int nb, npi, nslot;
    int ghist;                   // 1: rp-pi / mocks add straight into hcnt/hw/hr (global atomics):
                                 // their per-warp histogram does not fit in shared memory
    float fxw;                   // rp-pi / mocks per-warp weight sums in fixed point (two 32-bit words
                                 // per slot, see cf_pair.cuh) at this power-of-two scale (0: FP64)
    float fxr;                   // nonzero: the ravg sums too, those of rp bin k at scale fxr_bin[k]
    double ifxw;                 // 1 / fxw
    float fxr_bin[CF_MAX_BINS];
};

// Static configuration of a pair-kernel launch (selects the template instance and the shared
// memory layout).
struct CfPairCfg {
    int kind;          // 0 r, 1 rppi, 2 wp, 3 theta, 4 mocks
    int weighted, ravg, wrap, lo;
    int ghist;         // see CfPairArgs::ghist (no per-warp histogram in shared memory)
    int nlut_words, nfine, nslot;
    int nb;            // r / rp / theta bins
    int warps;         // warps per CTA (0: automatic)
    int ctas_per_sm;   // 0: occupancy-derived
    int variant;       // 1 direct binning, 2 compacting ring (resolved from 0 by the caller)
};

// Shared-memory bytes of one CTA with `warps` warps.
size_t cfp_pair_smem(const CfPairCfg &c, int warps);

// Launch the persistent pair kernel.  Returns cudaErrorInvalidValue when no CTA shape fits in
// shared memory.  *grid_out receives the number of CTAs launched.
cudaError_t cfp_launch_pair(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st,
                            int *grid_out, int *warps_out);
// CF_OPT_AUDIT: queue every pair of every work item for the FP64 recheck (launched instead of the
// pair kernel).
cudaError_t cfp_launch_audit(const CfItem *items, const uint32_t *nitems_dev, uint32_t items_cap,
                             const uint32_t *orig, uint4 *queue, unsigned long long *qcount, uint32_t qcap, int num_sms,
                             cudaStream_t st);
cudaError_t cfp_launch_recheck(const CfDevPlan *plan, const CfSetDesc *sets, const CfJobDesc *jobs,
                               const uint4 *queue, const unsigned long long *qcount, uint32_t qcap,
                               unsigned long long *hcnt, double *hw, double *hr, int num_sms, cudaStream_t st);
