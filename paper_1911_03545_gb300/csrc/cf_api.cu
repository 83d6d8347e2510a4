// cf_api.cu -- context, device scratch, and the cf_count / cf_batch_* entry points.
//
// One call runs the whole path on the context's stream:
//   prepare (host): stage inputs, bbox/validate, plan grid + bands + tables (Sec. 4.1-4.2)
//   build  (device): assign -> scan -> scatter (Sec. 4.3), work list count -> scan (Sec. 4.2-4.3)
//   count  (device): emit work items -> persistent pair kernel (Sec. 4.4-4.7) -> FP64 recheck
//                    of near-edge pairs -> readback
//   finish (host): doubling and self pairs (Sec. 4.3, Appendix B), ravg (Sec. 6.5),
//                  wp (Eq. 2 with the analytic RR of Appendix B).
// The two device phases contain no host synchronisation, so the batched path can record them
// into a CUDA graph and replay it.
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "cf_api_internal.h"

namespace {

const char *status_name(int s)
{
    switch (s) {
    case CF_OK: return "ok";
    case CF_ERR_ARG: return "invalid argument";
    case CF_ERR_OOM: return "out of memory";
    case CF_ERR_CUDA: return "CUDA error";
    case CF_ERR_TIMEOUT: return "timeout";
    case CF_ERR_BUSY: return "busy";
    case CF_ERR_CANCELLED: return "cancelled";
    default: return "internal error";
    }
}

double dkey_to_double(unsigned long long k)
{
    unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// context helpers
// ---------------------------------------------------------------------------------------------
int CfCtx::fail(int status, const std::string &msg)
{
    err = std::string(status_name(status)) + ": " + msg;
    return status;
}

int CfCtx::cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return CF_OK;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(CF_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    return fail(CF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int CfCtx::ensure(int b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    Buf &B = buf[b];
    if (B.cap >= bytes) return CF_OK;
    size_t want = bytes + bytes / 4 + 256;
    size_t used_other = mem_used - B.cap;
    if (mem_cap && used_other + want > mem_cap) {
        want = bytes;
        if (used_other + want > mem_cap)
            return fail(CF_ERR_OOM, "device scratch would exceed the context's memory cap (" +
                                        std::to_string(used_other + want) + " > " + std::to_string(mem_cap) + " bytes)");
    }
    if (B.p) {
        cudaStreamSynchronize(stream);
        cudaFree(B.p);
        mem_used -= B.cap;
        B.p = nullptr;
        B.cap = 0;
    }
    gen++;
    cudaError_t e = cudaMalloc(&B.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        B.p = nullptr;
        return fail(CF_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
    }
    B.cap = want;
    mem_used += want;
    return CF_OK;
}

int CfCtx::ensure_host(size_t bytes)
{
    if (hpin_cap >= bytes) return CF_OK;
    if (hpin) {
        cudaStreamSynchronize(stream);
        cudaFreeHost(hpin);
    }
    hpin = nullptr;
    gen++;
    size_t want = bytes + bytes / 4 + 4096;
    if (cudaMallocHost(&hpin, want) != cudaSuccess) {
        cudaGetLastError();
        hpin_cap = 0;
        return fail(CF_ERR_OOM, "pinned host staging allocation failed");
    }
    hpin_cap = want;
    return CF_OK;
}

// Pinned staging for the per-call uploads: host-to-device copies from pinned memory are
// asynchronous, so the call need not wait for them (from pageable memory they may synchronise).
// The buffer is reused by the next call, which starts after this call's final synchronisation.
int CfCtx::ensure_upload(size_t bytes)
{
    if (hup_cap >= bytes) return CF_OK;
    if (hup) {
        cudaStreamSynchronize(stream);
        cudaFreeHost(hup);
    }
    hup = nullptr;
    size_t want = bytes + bytes / 4 + 65536;
    if (cudaMallocHost(&hup, want) != cudaSuccess) {
        cudaGetLastError();
        hup_cap = 0;
        return fail(CF_ERR_OOM, "pinned host staging allocation failed");
    }
    hup_cap = want;
    return CF_OK;
}

int CfCtx::ensure_aux()
{
    if (aux) return CF_OK;
    int rc;
    if ((rc = cuda(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming), "event"))) return rc;
    if ((rc = cuda(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming), "event"))) return rc;
    return cuda(cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking), "stream");
}

int CfCtx::ensure_bbox_host(size_t bytes)
{
    if (hbb_cap >= bytes) return CF_OK;
    if (hbb) {
        cudaStreamSynchronize(stream);
        cudaFreeHost(hbb);
    }
    hbb = nullptr;
    const size_t want = std::max<size_t>(bytes, 4096);
    if (cudaMallocHost(&hbb, want) != cudaSuccess) {
        cudaGetLastError();
        hbb_cap = 0;
        return fail(CF_ERR_OOM, "pinned host staging allocation failed");
    }
    hbb_cap = want;
    return CF_OK;
}

void CfCtx::drop_graph()
{
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    graph_exec = nullptr;
    graph = nullptr;
}

CfCtx::~CfCtx()
{
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (aux) cudaStreamDestroy(aux);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    for (auto &B : buf)
        if (B.p) cudaFree(B.p);
    if (hpin) cudaFreeHost(hpin);
    if (hup) cudaFreeHost(hup);
    if (hbb) cudaFreeHost(hbb);
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------------------------
// phases
// ---------------------------------------------------------------------------------------------
static int check_points(CfCtx *C, const cf_params *p, const cf_points *d)
{
    if (!d) return C->fail(CF_ERR_ARG, "point set is NULL");
    if (d->n < 0 || d->n >= (int64_t)1 << 31) return C->fail(CF_ERR_ARG, "point count out of range");
    if (d->dtype != CF_F32 && d->dtype != CF_F64) return C->fail(CF_ERR_ARG, "dtype must be CF_F32 or CF_F64");
    if (d->n > 0 && (!d->x || !d->y || !d->z)) return C->fail(CF_ERR_ARG, "coordinate pointer is NULL");
    if (p->weight == CF_W_PAIR_PRODUCT && d->n > 0 && !d->w)
        return C->fail(CF_ERR_ARG, "weights were requested but a point set has w == NULL");
    return CF_OK;
}

#define CF_TRY(x)              \
    do {                       \
        int rc_ = (x);         \
        if (rc_) return rc_;   \
    } while (0)
#define CF_CU(x, what) CF_TRY(C->cuda((x), what))

// the work list and the order the pair kernel takes it in (one index per item, then the ordering
// pass's per-block class sizes)
static int ensure_items(CfCtx *C, size_t cap)
{
    cap = std::max<size_t>(1, cap);
    CF_TRY(C->ensure(B_ITEMS, sizeof(CfItem) * cap));
    const size_t part = (size_t)CFI_ITEM_CLASSES * cfb_order_blocks((uint32_t)cap, C->num_sms);
    return C->ensure(B_ORDER, sizeof(uint32_t) * (cap + part));
}

// The bbox pass's readback (CFB_BBOX_WORDS per point set): reject non-finite values and periodic
// positions outside [0, L]; record each set's weight range and the union of the sets' boxes, the
// largest | |v|^2 - 1 | and the smallest |v|^2.
static int cf_check_bbox(CfCtx *C, CfRun &R, const unsigned long long *bb, double bbox[6], double &norm_dev,
                         double &vmin2)
{
    const cf_params *p = &R.p;
    const size_t bbw = CFB_BBOX_WORDS;
    for (int a = 0; a < 6; a++) bbox[a] = a < 3 ? INFINITY : -INFINITY;
    norm_dev = 0.0;
    vmin2 = INFINITY;
    R.wmin.assign(R.nsets, INFINITY);
    R.wmax.assign(R.nsets, 0.0);
    R.wneg = false;
    for (int s = 0; s < R.nsets; s++) {
        if (R.sets[s].n == 0) continue;
        const unsigned long long *b = bb + bbw * s;
        if (b[6]) return C->fail(CF_ERR_ARG, "non-finite coordinate or weight");
        if (R.sets[s].w) {
            if (b[9] != ~0ull) std::memcpy(&R.wmin[s], &b[9], 8);
            std::memcpy(&R.wmax[s], &b[10], 8);
            R.wneg = R.wneg || b[11] != 0;
        }
        double nd, r2;
        std::memcpy(&nd, &b[7], 8);
        std::memcpy(&r2, &b[8], 8);
        norm_dev = std::max(norm_dev, nd);
        vmin2 = std::min(vmin2, r2);
        for (int a = 0; a < 3; a++) {
            double lo = dkey_to_double(b[a]), hi = dkey_to_double(b[3 + a]);
            if (p->periodic && (lo < 0.0 || hi > p->box[a]))
                return C->fail(CF_ERR_ARG, "periodic positions must lie in [0, box] (axis " + std::to_string(a) + ")");
            bbox[a] = std::min(bbox[a], lo);
            bbox[3 + a] = std::max(bbox[3 + a], hi);
        }
    }
    for (int a = 0; a < 3; a++)
        if (!(bbox[a] <= bbox[3 + a])) { bbox[a] = 0.0; bbox[3 + a] = 0.0; }
    return CF_OK;
}

int cf_prepare(CfCtx *C, const cf_params *p, const std::vector<const cf_points *> &pts,
               const std::vector<CfJobDesc> &jobs, CfRun &R)
{
    std::string err;
    int rc = cfp_check_params(p, err);
    if (rc) return C->fail(rc, err);
    R.p = *p;
    R.edges.assign(p->edges, p->edges + p->nbins + 1);
    R.p.edges = R.edges.data();
    R.nsets = (int)pts.size();
    R.njobs = (int)jobs.size();
    R.jobs = jobs;
    if (R.nsets < 1 || R.nsets > CFI_MAX_SETS || R.njobs < 1 || R.njobs > (int)CFI_ITEM_JOBMASK)
        return C->fail(CF_ERR_ARG, "too many point sets or jobs");
    R.npts = 0;
    R.nmax = 0;
    bool any_f64 = false;
    size_t in_bytes = 0;
    R.pts.clear();
    for (int s = 0; s < R.nsets; s++) {
        CF_TRY(check_points(C, p, pts[s]));
        R.pts.push_back(*pts[s]);
        R.npts += pts[s]->n;
        R.nmax = std::max<int64_t>(R.nmax, pts[s]->n);
        any_f64 |= pts[s]->dtype == CF_F64;
        if (!pts[s]->on_device && pts[s]->n > 0)
            in_bytes += 4 * (((pts[s]->dtype == CF_F64 ? 8 : 4) * (size_t)pts[s]->n + 255) & ~(size_t)255);
    }
    if (R.npts >= ((int64_t)1 << 31)) return C->fail(CF_ERR_ARG, "more than 2^31 points in one call");
    for (auto &J : jobs)
        if (J.a < 0 || J.a >= R.nsets || J.b < 0 || J.b >= R.nsets) return C->fail(CF_ERR_ARG, "bad job");
    cudaStream_t st = C->stream;
    const int nsets = R.nsets, njobs = R.njobs;

    // a call that failed between its side-stream bbox pass and the join left that pass unjoined:
    // order it before this call's uploads
    if (C->aux_pending) {
        CF_CU(cudaStreamWaitEvent(st, C->ev_join, 0), "stream wait");
        C->aux_pending = false;
    }

    // ---- stage inputs (host arrays are copied; device arrays are used in place) ----
    if (in_bytes) CF_TRY(C->ensure(B_IN, in_bytes));
    R.sets.assign(nsets, CfSetDesc());
    {
        char *inbase = (char *)C->buf[B_IN].p;
        size_t inoff = 0;
        int64_t pb = 0;
        const bool wt = p->weight == CF_W_PAIR_PRODUCT;
        for (int s = 0; s < nsets; s++) {
            const cf_points *d = pts[s];
            CfSetDesc &S = R.sets[s];
            std::memset(&S, 0, sizeof(S));
            S.n = d->n;
            S.dtype = d->dtype;
            S.pbeg = pb;
            pb += d->n;
            if (d->on_device || d->n == 0) {
                S.x = d->x;
                S.y = d->y;
                S.z = d->z;
                S.w = wt ? d->w : nullptr;
                continue;
            }
            size_t bytes = (d->dtype == CF_F64 ? 8 : 4) * (size_t)d->n;
            const void *src[4] = {d->x, d->y, d->z, wt ? d->w : nullptr};
            const void **dst[4] = {&S.x, &S.y, &S.z, &S.w};
            for (int a = 0; a < 4; a++) {
                if (!src[a]) { *dst[a] = nullptr; continue; }
                char *q = inbase + inoff;
                CF_CU(cudaMemcpyAsync(q, src[a], bytes, cudaMemcpyHostToDevice, st), "input copy");
                *dst[a] = q;
                inoff += (bytes + 255) & ~(size_t)255;
            }
        }
    }

    // ---- bbox + validation (Sec. 4.1: the grid covers every data set of the call) ----
    // B_BBOX holds the pass's starting values (then its results) and, after them, the point sets'
    // descriptors: both go up in one copy from pinned memory
    const size_t bbw = CFB_BBOX_WORDS;
    const size_t soff = (8 * bbw * (size_t)nsets + 255) & ~(size_t)255;
    CF_TRY(C->ensure(B_BBOX, soff + sizeof(CfSetDesc) * nsets));
    CF_TRY(C->ensure_host(std::max<size_t>(soff + sizeof(CfSetDesc) * nsets, 4096)));
    {
        unsigned long long *init = (unsigned long long *)C->hpin;
        for (int s = 0; s < nsets; s++)
            for (size_t a = 0; a < bbw; a++) init[bbw * s + a] = (a < 3 || a == 8 || a == 9) ? ~0ull : 0ull;
        std::memcpy((char *)C->hpin + soff, R.sets.data(), sizeof(CfSetDesc) * nsets);
        CF_CU(cudaMemcpyAsync(C->buf[B_BBOX].p, C->hpin, soff + sizeof(CfSetDesc) * nsets, cudaMemcpyHostToDevice, st),
              "bbox init and sets");
    }
    R.bb_sets = (const CfSetDesc *)((char *)C->buf[B_BBOX].p + soff);
    // Periodic inputs whose sums need no weight range (no fixed-point per-warp sums) are planned from
    // the box alone; their bbox pass runs on a side stream beside the build, and its readback is
    // checked after the call's final synchronisation instead of being waited for here.  Invalid
    // data cannot fault in the meantime: cell indices clamp to the grid and a non-finite separation
    // fails every cut.
    const bool warp_sums = (p->kind == CF_DD_RPPI || p->kind == CF_DD_RPPI_MOCKS) &&
                           (p->weight == CF_W_PAIR_PRODUCT || p->output_ravg);
    R.bbox_deferred = p->periodic && !warp_sums && !C->capturing;
    R.bbox_aux = false;
    R.fused_items = false;
    cudaStream_t bst = st;
    if (R.bbox_deferred) {
        CF_TRY(C->ensure_aux());
        CF_TRY(C->ensure_bbox_host(8 * bbw * (size_t)nsets));
        CF_CU(cudaEventRecord(C->ev_fork, st), "event");
        C->aux_pending = true;
        CF_CU(cudaStreamWaitEvent(C->aux, C->ev_fork, 0), "stream wait");
        bst = C->aux;
        R.bbox_aux = true;
    }
    CF_CU(cfb_bbox(R.bb_sets, nsets, std::max<int64_t>(R.nmax, 1), (unsigned long long *)C->buf[B_BBOX].p, bst),
          "bbox kernel");
    C->launches = 1;
    double bbox[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    double norm_dev = 0.0;   // largest | |v|^2 - 1 | over the points
    double vmin2 = INFINITY;  // smallest |v|^2 over the points
    if (R.bbox_deferred) {
        CF_CU(cudaMemcpyAsync(C->hbb, C->buf[B_BBOX].p, 8 * bbw * (size_t)nsets, cudaMemcpyDeviceToHost, bst),
              "bbox readback");
        CF_CU(cudaEventRecord(C->ev_join, bst), "event");
        R.wmin.assign(nsets, INFINITY);
        R.wmax.assign(nsets, 0.0);
        R.wneg = false;
        for (int a = 0; a < 3; a++) {
            bbox[a] = 0.0;
            bbox[3 + a] = p->box[a];
        }
    } else {
        CF_CU(cudaMemcpyAsync(C->hpin, C->buf[B_BBOX].p, 8 * bbw * (size_t)nsets, cudaMemcpyDeviceToHost, st),
              "bbox readback");
        CF_CU(cudaStreamSynchronize(st), "bbox sync");
        CF_TRY(cf_check_bbox(C, R, (const unsigned long long *)C->hpin, bbox, norm_dev, vmin2));
    }

    // ---- plan ----
    const bool angular = p->kind == CF_DD_THETA && C->opt[CF_OPT_THETA_GRID] == 1;
    std::memcpy(R.bbox, bbox, sizeof(bbox));
    R.vmin2 = vmin2;
    R.angular = angular;
    if (angular && norm_dev > 2e-3)
        return C->fail(CF_ERR_ARG, "the angular grid needs unit vectors (|v| within 1e-3 of 1)");
    CfHostPlan &H = R.plan;
    int refine[3];
    for (int a = 0; a < 3; a++)
        refine[a] = p->refine[a] > 0 ? p->refine[a] : (C->opt[CF_OPT_REFINE] > 0 ? (int)C->opt[CF_OPT_REFINE] : 1);
    int tile = C->opt[CF_OPT_TILE] > 0 ? (int)std::min<int64_t>(128, std::max<int64_t>(32, C->opt[CF_OPT_TILE])) : 128;
    int jchunk = C->opt[CF_OPT_JCHUNK] > 0 ? (int)std::min<int64_t>(CFI_JMAX, C->opt[CF_OPT_JCHUNK]) : CFI_JMAX;
    // |v| of the point nearest the observer (its square was summed in float32 for float32 inputs:
    // a few roundings high or low)
    const double vmin = std::isfinite(vmin2) ? std::sqrt(vmin2) * (1.0 - 1e-6) : 0.0;
    {
        // the plan depends only on these: a repeated call on the same inputs reuses the previous
        // one (planning takes ~0.1 ms of host time while the device waits)
        std::string key;
        auto put = [&key](const void *v, size_t n) { key.append((const char *)v, n); };
        put(p, offsetof(cf_params, edges));
        put(&p->nbins, sizeof(cf_params) - offsetof(cf_params, nbins));
        put(p->edges, sizeof(double) * (size_t)(p->nbins + 1));
        put(bbox, sizeof(bbox));
        put(&R.npts, sizeof(R.npts));
        const int ints[6] = {any_f64 ? 1 : 0, refine[0] * 16 + refine[1] * 4 + refine[2], tile, jchunk, angular ? 1 : 0,
                             0};
        put(ints, sizeof(ints));
        put(&vmin, sizeof(vmin));
        if (key != C->plan_key) {
            C->plan_key.clear();
            rc = cfp_make_plan(p, bbox, R.npts, any_f64 ? 1 : 0, refine, tile, jchunk, &H, err, angular ? 1 : 0,
                               vmin);
            if (rc) return C->fail(rc, err);
            C->plan_key = key;
        }
    }
    CfDevPlan &D = H.d;
    D.nsets = nsets;
    D.njobs = njobs;
    R.ncell = D.g.ncell;
    for (int s = 0; s < nsets; s++) R.sets[s].cbeg = (int64_t)s * R.ncell;
    R.ncell_all = R.ncell * nsets;
    if (R.ncell_all >= ((int64_t)1 << 31)) return C->fail(CF_ERR_ARG, "too many cells");
    R.nst = D.g.nstencil;
    // points sort by (cell, Morton sub-cell): the finest order whose key array stays within about
    // twice the points (and 1M keys)
    {
        const int64_t want = C->opt[CF_OPT_CELL_ORDER];
        const int64_t lim = std::max<int64_t>(2 * R.npts, (int64_t)1 << 20);
        if (want == 1 || want == 2 || want == 4) R.sub = (int)want;
        else R.sub = R.ncell_all * 64 <= lim ? 4 : (R.ncell_all * 8 <= lim ? 2 : 1);
        R.nfine = R.ncell_all * R.sub * R.sub * R.sub;
        if (R.nfine >= ((int64_t)1 << 31)) return C->fail(CF_ERR_ARG, "too many cells");
    }
    R.nunit = (int64_t)njobs * R.ncell;      // work-list units: one per (job, i cell)
    if (R.nunit >= ((int64_t)1 << 31)) return C->fail(CF_ERR_ARG, "work list too large");
    R.np = std::max<int64_t>(R.npts, 1);
    // a grid with more cells than points (most of them empty): list the units with points first,
    // so that the work-list pass does not spend a warp iteration on each empty cell
    R.live_units = R.nunit >= 65536 && R.nunit > R.npts;
    R.nslot = (size_t)D.nslot;
    R.hsz = R.nslot * njobs;
    R.self_pairs = p->edges[0] == 0.0;

    // ---- device buffers (allocated here so that the device phases never allocate) ----
    // the angular grid's origins (3 per cell) are computed on the device by the build
    const size_t norigin = D.ang ? 3 * (size_t)D.g.ncell : H.origin.size();
    // The plan, its tables and the call's descriptors share one device block, filled from the
    // pinned staging by one copy: plan | LUT | fine entries | stencil | jobs | sets | bands |
    // origins (FP64) | origins (float32).  The angular grid's origins are computed on the device.
    const size_t piece[9] = {sizeof(CfDevPlan), sizeof(uint16_t) * H.lut.size(), sizeof(CfFine) * H.fine.size(),
                             sizeof(CfStencil) * H.stencil.size(), sizeof(CfJobDesc) * njobs,
                             sizeof(CfSetDesc) * nsets, sizeof(CfBand) * H.bands.size(), sizeof(double) * norigin,
                             sizeof(float) * norigin};
    size_t poff[10];
    poff[0] = 0;
    for (int k = 0; k < 9; k++) poff[k + 1] = poff[k] + ((std::max<size_t>(piece[k], 1) + 255) & ~(size_t)255);
    CF_TRY(C->ensure(B_PLANBLK, poff[9]));
    {
        char *blk = (char *)C->buf[B_PLANBLK].p;
        R.d_plan = (const CfDevPlan *)(blk + poff[0]);
        R.d_lut = (const uint16_t *)(blk + poff[1]);
        R.d_fine = (const CfFine *)(blk + poff[2]);
        R.d_stencil = (const CfStencil *)(blk + poff[3]);
        R.d_jobs = (const CfJobDesc *)(blk + poff[4]);
        R.d_sets = (const CfSetDesc *)(blk + poff[5]);
        D.band = (const CfBand *)(blk + poff[6]);
        R.d_origin = (double *)(blk + poff[7]);
        R.d_origin32 = (float *)(blk + poff[8]);
        D.origin = R.d_origin;
        D.origin32 = R.d_origin32;
    }
    CF_TRY(C->ensure(B_CNT, 4 * (size_t)(R.nfine + 1)));
    CF_TRY(C->ensure(B_FSTART, 4 * (size_t)(R.nfine + 1)));
    CF_TRY(C->ensure(B_CSTART, 4 * (size_t)(R.ncell_all + 1)));
    CF_TRY(C->ensure(B_CELLID, 4 * (size_t)R.np));
    CF_TRY(C->ensure(B_SLOT, 4 * (size_t)R.np));
    CF_TRY(C->ensure(B_PA, 16 * (size_t)R.np));
    CF_TRY(C->ensure(B_PB, 16 * (size_t)R.np));
    CF_TRY(C->ensure(B_ORIG, 4 * (size_t)R.np));
    CF_TRY(C->ensure(B_CBOX, 24 * (size_t)R.ncell_all));
    if (C->opt[CF_OPT_CELL_PRUNE] == 0 && C->opt[CF_OPT_BLOCK_PRUNE] == 1) CF_TRY(C->ensure(B_GBOX, 24 * (size_t)R.np));
    if (D.f64lo) CF_TRY(C->ensure(B_PLO, 32 * (size_t)R.np));
    CF_TRY(C->ensure(B_SCAN, 4 * (size_t)cfb_scan_tmp_words(std::max(R.nfine, R.nunit))));
    CF_TRY(C->ensure(B_ICNT, 4 * (size_t)std::max<int64_t>(R.nunit, 1)));
    CF_TRY(C->ensure(B_IOFF, 4 * (size_t)(R.nunit + 1)));
    if (R.live_units) CF_TRY(C->ensure(B_LIVE, 4 * (size_t)R.nunit));
    CF_TRY(C->ensure(B_OUT, readback_bytes(R)));
    R.qcap = C->opt[CF_OPT_QUEUE] > 0 ? (uint32_t)std::min<int64_t>(CF_MAX_ENTRIES, C->opt[CF_OPT_QUEUE])
                                      : C->qcap_default;
    CF_TRY(C->ensure(B_QUEUE, 16 * (size_t)R.qcap));
    CF_TRY(C->ensure_host(readback_bytes(R)));

    {
        // one upload through pinned staging (no wait for the transfer); the angular grid's origins
        // are left to the device
        const void *src[9] = {&D, H.lut.data(), H.fine.data(), H.stencil.data(), R.jobs.data(), R.sets.data(),
                              H.bands.data(), H.origin.data(), H.origin32.data()};
        const int npieces = D.ang ? 7 : 9;
        CF_TRY(C->ensure_upload(poff[npieces]));
        for (int k = 0; k < npieces; k++)
            if (piece[k]) std::memcpy((char *)C->hup + poff[k], src[k], piece[k]);
        CF_CU(cudaMemcpyAsync(C->buf[B_PLANBLK].p, C->hup, poff[npieces], cudaMemcpyHostToDevice, st), "plan upload");
    }

    // pair-kernel configuration
    std::memset(&R.cfg, 0, sizeof(R.cfg));
    R.cfg.kind = D.kind;
    R.cfg.weighted = D.weighted;
    R.cfg.ravg = D.ravg;
    R.cfg.wrap = D.g.wrap[0] | D.g.wrap[1] | D.g.wrap[2];
    R.cfg.lo = D.f64lo;
    R.cfg.nlut_words = D.nlut_words;
    R.cfg.nfine = D.nfine;
    R.cfg.nslot = D.nslot;
    R.cfg.nb = D.nb;
    R.cfg.warps = (int)C->opt[CF_OPT_WARPS];
    R.cfg.ctas_per_sm = (int)C->opt[CF_OPT_CTAS_PER_SM];
    // the mocks kind has the direct form only (a compacting form measured slower)
    R.cfg.variant = (C->opt[CF_OPT_VARIANT] == 2 && D.kind != CF_DD_RPPI_MOCKS) ? 2 : 1;
    R.items_cap = 0;
    return CF_OK;
}

size_t readback_bytes(const CfRun &R) { return OUT_HIST + 24 * R.hsz + 8 * (size_t)R.nsets; }

// bbox pass of a captured graph: starting values, the pass, its readback at R.bb_off
static int cf_enqueue_bbox(CfCtx *C, CfRun &R)
{
    cudaStream_t st = C->stream;
    unsigned long long *bb = (unsigned long long *)C->buf[B_BBOX].p;
    CF_CU(cfb_bbox_init(bb, R.nsets, st), "bbox init");
    CF_CU(cfb_bbox(R.bb_sets, R.nsets, std::max<int64_t>(R.nmax, 1), bb, st), "bbox kernel");
    CF_CU(cudaMemcpyAsync((char *)C->hpin + R.bb_off, bb, 8 * CFB_BBOX_WORDS * (size_t)R.nsets, cudaMemcpyDeviceToHost,
                          st), "bbox readback");
    C->launches += 2;
    return CF_OK;
}

// Whether new data of a replay still fits the captured plan: finite values, every set inside the
// box the grid was made for (which for periodic sets lies in [0, box]), for mocks no point nearer
// the observer than before, for the angular grid unit vectors.
static bool bbox_within(const CfRun &R, const unsigned long long *bb)
{
    for (int s = 0; s < R.nsets; s++) {
        if (R.sets[s].n == 0) continue;
        const unsigned long long *b = bb + CFB_BBOX_WORDS * s;
        if (b[6]) return false;
        for (int a = 0; a < 3; a++)
            if (!(dkey_to_double(b[a]) >= R.bbox[a] && dkey_to_double(b[3 + a]) <= R.bbox[3 + a])) return false;
        double nd, r2;
        std::memcpy(&nd, &b[7], 8);
        std::memcpy(&r2, &b[8], 8);
        if (R.p.kind == CF_DD_RPPI_MOCKS && !(r2 >= R.vmin2)) return false;
        if (R.angular && !(nd <= 2e-3)) return false;
    }
    return true;
}

// cell build + work-list count and scan (device only)
int cf_enqueue_build(CfCtx *C, CfRun &R)
{
    cudaStream_t st = C->stream;
    const CfDevPlan *dplan = R.d_plan;
    const CfSetDesc *dsets = R.d_sets;
    const CfJobDesc *djobs = R.d_jobs;
    uint32_t *cnt = (uint32_t *)C->buf[B_CNT].p, *cstart = (uint32_t *)C->buf[B_CSTART].p;
    char *out = (char *)C->buf[B_OUT].p;
    uint32_t *fstart = (uint32_t *)C->buf[B_FSTART].p;
    if (R.plan.d.ang) {
        CF_CU(cfb_ang_origins(dplan, R.plan.d.g.ncell, R.d_origin, R.d_origin32, st), "cell origins");
        C->launches += 1;
    }
    CF_CU(cudaMemsetAsync(cnt, 0, 4 * (size_t)R.nfine, st), "memset counts");
    CF_CU(cudaMemsetAsync(out, 0, OUT_HIST, st), "memset work-list counters");
    CF_CU(cfb_assign(dplan, dsets, R.nsets, R.np, R.sub, cnt, (uint32_t *)C->buf[B_CELLID].p,
                     (uint32_t *)C->buf[B_SLOT].p, st),
          "assign");
    // sub-cell starts, and the cell starts among them (sub^3 = 2^(3 log2 sub) sub-cells per cell)
    const int sub_shift = R.sub == 4 ? 6 : (R.sub == 2 ? 3 : 0);
    CF_CU(cfb_scan(cnt, fstart, R.nfine, (uint32_t *)C->buf[B_SCAN].p, (uint32_t *)(out + OUT_SCAN), st, nullptr,
                   cstart, sub_shift),
          "scan cells");
    CF_CU(cfb_scatter(dplan, dsets, R.nsets, R.np, R.sub, fstart, (uint32_t *)C->buf[B_CELLID].p,
                      (uint32_t *)C->buf[B_SLOT].p, (float4 *)C->buf[B_PA].p, (float4 *)C->buf[B_PB].p,
                      (float4 *)C->buf[B_PLO].p, (uint32_t *)C->buf[B_ORIG].p, st),
          "scatter");
    const float *cbox = nullptr;
    float *gbox = nullptr;
    if (C->opt[CF_OPT_CELL_PRUNE] == 0) {
        // and, when asked for, the boxes of the cells' 32-point groups
        gbox = C->opt[CF_OPT_BLOCK_PRUNE] == 1 ? (float *)C->buf[B_GBOX].p : nullptr;
        CF_CU(cfb_cellbox(cstart, R.ncell_all, (const float4 *)C->buf[B_PA].p, (const float4 *)C->buf[B_PB].p,
                          (float *)C->buf[B_CBOX].p, gbox, st),
              "cell boxes");
        cbox = (const float *)C->buf[B_CBOX].p;
        C->launches += 1;
    }
    R.cbox = cbox;
    R.gbox = gbox;
    C->launches += 4;    // assign, 2 scan, scatter
    if (R.fused_items) return CF_OK;    // the count pass writes the work list in one go
    uint32_t *icnt = (uint32_t *)C->buf[B_ICNT].p, *ioff = (uint32_t *)C->buf[B_IOFF].p;
    // the work list's length in 64 bits, next to its 32-bit scan (checked in cf_finish)
    unsigned long long *items64 = (unsigned long long *)(out + OUT_ITEMS64);
    const uint32_t *live = nullptr, *nlive = nullptr;
    if (R.live_units) {
        // the units with points (the count phase keeps the list: its memset starts past OUT_NLIVE);
        // the others count no items
        live = (const uint32_t *)C->buf[B_LIVE].p;
        nlive = (const uint32_t *)(out + OUT_NLIVE);
        CF_CU(cudaMemsetAsync(icnt, 0, 4 * (size_t)R.nunit, st), "memset item counts");
        CF_CU(cfb_live_units(dplan, dsets, djobs, cstart, R.nunit, (uint32_t *)live, (uint32_t *)nlive, st),
              "live units");
        C->launches += 1;
    }
    CF_CU(cfb_items(dplan, dsets, djobs, R.d_stencil, cstart, cbox, gbox, live, nlive, R.nunit, 0, icnt, nullptr,
                    nullptr, 0, items64, nullptr, st),
          "items count");
    CF_CU(cfb_scan(icnt, ioff, R.nunit, (uint32_t *)C->buf[B_SCAN].p, (uint32_t *)(out + OUT_SCAN + 4), st,
                   (uint32_t *)(out + OUT_NITEMS)),
          "scan items");
    C->launches += 3;    // items count, 2 scan
    return CF_OK;
}

// Power-of-two scale for the fixed-point sums of terms in [tmin, tmax] (tmin > 0): tmax * scale <
// 2^26, with 1/1024 of margin for the terms' FP32 rounding, so that the two 32-bit words a slot keeps
// stay exact for 2^18 terms between flushes, and tmin * scale >= 2^21, so that rounding a term to an
// integer moves it by at most 2^-22 of itself.  0 (FP64 sums) when no such scale exists.
static float fixed_scale(double tmin, double tmax)
{
    if (!(tmin > 1e-30) || !(tmax >= tmin) || !(tmax < 1e30)) return 0.f;
    int ex = 0;
    std::frexp(tmax * (1.0 + 1.0 / 1024.0), &ex);   // the largest term, with margin, is below 2^ex
    const double s = std::ldexp(1.0, 26 - ex);
    return tmin * s >= 2097152.0 ? (float)s : 0.f;
}

// Scales of the per-warp weight and ravg sums of rp-pi / mocks.  A term is w_i w_j (weights), rp
// (ravg) or w_i w_j rp (both).  Weight products lie between the products of the sets' smallest
// nonzero and largest |w| (zero products are exact); the rp of a pair in rp bin k lies within 1e-5
// of [e_k, e_k+1] (its FP32 value may sit a few roundings outside), so each rp bin's ravg sum has a
// scale of its own.  Negative weights (sums that may cancel) and, with ravg, a first edge of 0 keep
// FP64 for every sum of the call.
static void fixed_point_scales(const CfRun &R, bool weighted, bool ravg, CfPairArgs &A)
{
    A.fxw = A.fxr = 0.f;
    A.ifxw = 0.0;
    double pmin = 1.0, pmax = 1.0;
    if (weighted) {
        if (R.wneg) return;
        pmin = INFINITY;
        pmax = 0.0;
        for (const CfJobDesc &J : R.jobs) {
            pmax = std::max(pmax, R.wmax[J.a] * R.wmax[J.b]);
            const double lo = R.wmin[J.a] * R.wmin[J.b];
            if (std::isfinite(lo)) pmin = std::min(pmin, lo);
        }
        if (!std::isfinite(pmin)) pmin = pmax = 1.0;   // every product is 0
        A.fxw = fixed_scale(pmin, pmax);
    }
    bool rok = true;
    if (ravg) {
        for (int k = 0; k + 1 < (int)R.edges.size(); k++) {
            A.fxr_bin[k] = fixed_scale(R.edges[k] * (1.0 - 1e-5) * pmin, R.edges[k + 1] * (1.0 + 1e-5) * pmax);
            rok = rok && A.fxr_bin[k] != 0.f;
        }
        A.fxr = rok ? 1.f : 0.f;
    }
    // one form for every sum the call keeps: fixed point only where all of them allow it
    if ((weighted && A.fxw == 0.f) || (ravg && A.fxr == 0.f)) A.fxw = A.fxr = 0.f;
    if (A.fxw != 0.f) A.ifxw = 1.0 / (double)A.fxw;
}

// work items -> pair kernel -> recheck -> readback (device only; records ev[1..3] when `timed`)
int cf_enqueue_count(CfCtx *C, CfRun &R, bool timed)
{
    cudaStream_t st = C->stream;
    const CfDevPlan *dplan = R.d_plan;
    const CfSetDesc *dsets = R.d_sets;
    const CfJobDesc *djobs = R.d_jobs;
    const CfDevPlan &D = R.plan.d;
    char *out = (char *)C->buf[B_OUT].p;
    uint32_t *ioff = (uint32_t *)C->buf[B_IOFF].p;
    unsigned long long *evaluated = (unsigned long long *)(out + OUT_EVAL);
    const size_t hsz = R.hsz;
    unsigned long long *hcnt = (unsigned long long *)(out + OUT_HIST);
    double *hw = (double *)(out + OUT_HIST + 8 * hsz), *hr = (double *)(out + OUT_HIST + 16 * hsz);
    double *wsq = (double *)(out + OUT_HIST + 24 * hsz);
    // evaluated pairs, the work cursor, the queue length, the histograms and w^2 sums (and for the
    // one-pass work list its two length counters): one memset
    const size_t zero_from = R.fused_items ? 0 : OUT_EVAL;
    CF_CU(cudaMemsetAsync(out + zero_from, 0, readback_bytes(R) - zero_from, st), "memset");
    uint32_t *nitems_dev = ioff + R.nunit;
    const uint32_t *cstart = (const uint32_t *)C->buf[B_CSTART].p;
    const uint32_t *live = R.live_units ? (const uint32_t *)C->buf[B_LIVE].p : nullptr;
    const uint32_t *nlive = R.live_units ? (const uint32_t *)(out + OUT_NLIVE) : nullptr;
    if (R.fused_items) {
        nitems_dev = (uint32_t *)(out + OUT_NITEMS);
        if (R.live_units) {
            // the memset above cleared the list's count: list the units with points again
            CF_CU(cfb_live_units(dplan, dsets, djobs, cstart, R.nunit, (uint32_t *)live, (uint32_t *)nlive, st),
                  "live units");
            C->launches += 1;
        }
        CF_CU(cfb_items(dplan, dsets, djobs, R.d_stencil, cstart, R.cbox, R.gbox, live, nlive, R.nunit, 2,
                        nitems_dev, nullptr, (CfItem *)C->buf[B_ITEMS].p, R.items_cap, evaluated,
                        (unsigned long long *)(out + OUT_ITEMS64), st),
              "items");
    } else {
        CF_CU(cfb_items(dplan, dsets, djobs, R.d_stencil, cstart, R.cbox, R.gbox, live, nlive, R.nunit, 1,
                        (uint32_t *)C->buf[B_ICNT].p, ioff, (CfItem *)C->buf[B_ITEMS].p, R.items_cap, evaluated,
                        nullptr, st),
              "items emit");
    }
    // a short list is taken as it is: the two ordering passes would cost more than they save (the
    // capacity of a repeat call's list holds 25 % headroom)
    const bool ordered = R.items_cap >= CF_ORDER_MIN_ITEMS;
    if (ordered)
        CF_CU(cfb_order((const CfItem *)C->buf[B_ITEMS].p, nitems_dev, R.items_cap, (uint32_t *)C->buf[B_ORDER].p,
                        (uint32_t *)C->buf[B_ORDER].p + R.items_cap, C->num_sms, st),
              "work-list order");
    if (timed) CF_CU(cudaEventRecordWithFlags(C->ev[1], st, C->capturing ? cudaEventRecordExternal : 0), "event");
    CfPairArgs &A = R.args;
    std::memset(&A, 0, sizeof(A));
    A.plan = dplan;
    A.lut = R.d_lut;
    A.fine = R.d_fine;
    A.items = (const CfItem *)C->buf[B_ITEMS].p;
    A.order = ordered ? (const uint32_t *)C->buf[B_ORDER].p : nullptr;
    A.nitems_dev = nitems_dev;
    A.items_cap = R.items_cap;
    A.qcap = R.qcap;
    A.cursor = (uint32_t *)(out + OUT_CURSOR);
    A.qcount = (unsigned long long *)(out + OUT_QCOUNT);
    A.pa = (const ulonglong2 *)C->buf[B_PA].p;
    A.pb = (const ulonglong2 *)C->buf[B_PB].p;
    A.plo = (const ulonglong2 *)C->buf[B_PLO].p;
    A.orig = (const uint32_t *)C->buf[B_ORIG].p;
    A.hcnt = hcnt;
    A.hw = hw;
    A.hr = hr;
    A.queue = (uint4 *)C->buf[B_QUEUE].p;
    for (int a = 0; a < 3; a++) A.L[a] = D.g.wrap[a] ? (float)D.g.L[a] : 0.f;
    A.nb = D.nb;
    A.npi = D.npi;
    A.nslot = D.nslot;
    // rp-pi / mocks keep one histogram per warp in shared memory; when even one warp's does not
    // fit (many rp x pi slots, weights), they add straight into the global histograms instead
    const bool per_warp = D.kind == CF_DD_RPPI || D.kind == CF_DD_RPPI_MOCKS;
    if (per_warp && !R.cfg.ghist && cfp_pair_smem(R.cfg, 1) > (size_t)C->smem_optin) R.cfg.ghist = 1;
    if (R.cfg.ghist) R.cfg.variant = 1;       // that form is built direct only
    A.ghist = R.cfg.ghist;
    // their per-warp sums go to fixed point when the terms' range allows it; never in a
    // captured graph, whose replays bring new weights
    if (per_warp && !A.ghist && !C->capturing) fixed_point_scales(R, D.weighted != 0, R.cfg.ravg != 0, A);
    if (A.fxw != 0.f || A.fxr != 0.f) R.cfg.variant = 1;    // built direct only
    int grid = 0, warps = 0;
    if (R.items_cap > 0 && C->opt[CF_OPT_AUDIT]) {
        CF_CU(cfp_launch_audit(A.items, A.nitems_dev, A.items_cap, A.orig, A.queue, A.qcount, A.qcap, C->num_sms,
                               st), "audit");
    } else if (R.items_cap > 0) {
        cudaError_t e = cfp_launch_pair(R.cfg, A, C->num_sms, st, &grid, &warps);
        if (e == cudaErrorInvalidValue) return C->fail(CF_ERR_ARG, "histogram does not fit in shared memory");
        CF_CU(e, "pair kernel");
    }
    C->last_grid = grid;
    C->last_warps = warps;
    if (timed) CF_CU(cudaEventRecordWithFlags(C->ev[2], st, C->capturing ? cudaEventRecordExternal : 0), "event");
    CF_CU(cfp_launch_recheck(dplan, dsets, djobs, A.queue, A.qcount, R.qcap, A.hcnt, A.hw, A.hr, C->num_sms, st), "recheck");
    if (R.self_pairs && D.weighted) {
        CF_CU(cfb_wsq(dsets, R.nsets, R.np, wsq, st), "self-pair weights");
        C->launches++;
    }
    C->launches += 2 + (R.items_cap > 0 ? 1 : 0) + (ordered ? 2 : 0);   // items emit, recheck, pair, order
    if (timed) CF_CU(cudaEventRecordWithFlags(C->ev[3], st, C->capturing ? cudaEventRecordExternal : 0), "event");
    // the side stream's bbox pass joins here, so that the call's synchronisation covers it
    if (R.bbox_aux) {
        CF_CU(cudaStreamWaitEvent(st, C->ev_join, 0), "stream wait");
        C->aux_pending = false;
    }
    // readback: the whole B_OUT block (counters, histograms, w^2 sums) in one copy
    CF_CU(cudaMemcpyAsync(C->hpin, out, readback_bytes(R), cudaMemcpyDeviceToHost, st), "readback");
    return CF_OK;
}

// after the stream is synchronised: overflow checks (*retry = 1 queue, 2 items) and finalize
int cf_finish(CfCtx *C, CfRun &R, std::vector<CfJobResult> &res, int *retry)
{
    const char *h = (const char *)C->hpin;
    const unsigned long long qn = *(const unsigned long long *)(h + OUT_QCOUNT);
    const uint32_t nitems = *(const uint32_t *)(h + OUT_NITEMS);
    *retry = 0;
    // work items and queue entries are indexed in 32 bits, with headroom for the grid-stride
    // loops and the work cursor's overshoot
    if (*(const unsigned long long *)(h + OUT_ITEMS64) > CF_MAX_ENTRIES)
        return C->fail(CF_ERR_ARG, "the work list exceeds 2^32 - 2^20 items (fewer points per call, or a coarser grid)");
    // the audit queues every evaluated pair
    if (C->opt[CF_OPT_AUDIT] && *(const unsigned long long *)(h + OUT_EVAL) >= 0xF0000000ull)
        return C->fail(CF_ERR_ARG, "CF_OPT_AUDIT needs fewer than 2^32 - 2^28 evaluated pairs");
    if (qn > CF_MAX_ENTRIES)
        return C->fail(CF_ERR_ARG, "more than 2^32 - 2^20 pairs lie within the FP32 error bands of the edges "
                                   "(points on a lattice aligned with the edges?)");
    if (nitems > R.items_cap) {
        R.items_cap = nitems;
        *retry = 2;
        return CF_OK;
    }
    if (qn > R.qcap) {
        R.qcap = (uint32_t)std::min<uint64_t>(CF_MAX_ENTRIES, qn + qn / 4 + 1024);
        C->qcap_default = std::max(C->qcap_default, R.qcap);
        *retry = 1;
        return CF_OK;
    }
    const size_t nslot = R.nslot, hsz = R.hsz;
    const unsigned long long *hc = (const unsigned long long *)(h + OUT_HIST);
    const double *hw = (const double *)(h + OUT_HIST + 8 * hsz);
    const double *hr = (const double *)(h + OUT_HIST + 16 * hsz);
    const double *wsq = (const double *)(h + OUT_HIST + 24 * hsz);
    const CfDevPlan &D = R.plan.d;
    res.assign(R.njobs, CfJobResult());
    for (int j = 0; j < R.njobs; j++) {
        CfJobResult &Q = res[j];
        Q.npairs.assign(nslot, 0);
        Q.wsum.assign(nslot, 0.0);
        Q.rsum.assign(nslot, 0.0);
        const bool autoc = R.jobs[j].autoc != 0;
        const double mult = autoc ? 2.0 : 1.0;
        for (size_t k = 0; k < nslot; k++) {
            // Sec. 4.3: unique pairs were counted for an auto-correlation; double them
            Q.npairs[k] = hc[j * nslot + k] * (autoc ? 2ull : 1ull);
            Q.wsum[k] = D.weighted ? hw[j * nslot + k] * mult : (double)Q.npairs[k];
            Q.rsum[k] = hr[j * nslot + k] * mult;
        }
        if (autoc && R.self_pairs) {
            // Appendix B: the N self pairs, added once, in the first bin (first pi bin for rp-pi)
            int64_t n = R.sets[R.jobs[j].a].n;
            Q.npairs[0] += (uint64_t)n;
            Q.wsum[0] += D.weighted ? wsq[R.jobs[j].a] : (double)n;
        }
        Q.n1 = R.sets[R.jobs[j].a].n;
        Q.autoc = autoc;
    }
    C->stats.rechecked_pairs = qn;
    C->stats.evaluated_pairs = (int64_t) * (const unsigned long long *)(h + OUT_EVAL);
    C->stats.work_items = nitems;
    C->stats.cells = R.ncell;
    for (int a = 0; a < 3; a++) {
        C->stats.grid[a] = D.g.n[a];
        C->stats.refine[a] = D.g.k[a];
    }
    C->stats.ncat = R.njobs;
    C->stats.variant = R.cfg.variant;
    C->stats.fixed_sums = (R.args.fxw != 0.f ? 1 : 0) | (R.args.fxr != 0.f ? 2 : 0);
    C->stats.kernel_launches = C->launches;
    return CF_OK;
}

static void record_times(CfCtx *C, bool with_build)
{
    float ms = 0;
    if (with_build && cudaEventElapsedTime(&ms, C->ev[0], C->ev[1]) == cudaSuccess) C->stats.ms_build = ms;
    if (cudaEventElapsedTime(&ms, C->ev[1], C->ev[2]) == cudaSuccess) C->stats.ms_pair = ms;
    if (cudaEventElapsedTime(&ms, C->ev[2], C->ev[3]) == cudaSuccess) C->stats.ms_recheck = ms;
    cudaGetLastError();
}

int cf_run(CfCtx *C, const cf_params *p, const std::vector<const cf_points *> &pts, const std::vector<CfJobDesc> &jobs,
           std::vector<CfJobResult> &res)
{
    auto t0 = std::chrono::steady_clock::now();
    CfRun &R = C->run;
    C->drop_graph();
    CF_TRY(cf_prepare(C, p, pts, jobs, R));
    cudaStream_t st = C->stream;
    // the work list depends on the plan and on the pruning and order options
    const std::string ikey = C->plan_key + std::to_string(C->opt[CF_OPT_CELL_PRUNE]) + "/" +
                             std::to_string(C->opt[CF_OPT_CELL_ORDER]) + "/" +
                             std::to_string(C->opt[CF_OPT_BLOCK_PRUNE]);
    // a call on the same plan sized the work list before: take that size with headroom, count and
    // write the list in one pass, and let cf_finish run the count again in the rare case that the
    // list outgrew it
    R.fused_items = C->items_hint && C->items_key == ikey;
    CF_CU(cudaEventRecord(C->ev[0], st), "event");
    CF_TRY(cf_enqueue_build(C, R));
    if (R.fused_items) {
        R.items_cap = C->items_hint;
    } else {
        // size the work list from the device count (one small readback)
        CF_CU(cudaMemcpyAsync(C->hpin, (uint32_t *)C->buf[B_IOFF].p + R.nunit, 4, cudaMemcpyDeviceToHost, st),
              "items total");
        CF_CU(cudaStreamSynchronize(st), "items sync");
        R.items_cap = *(const uint32_t *)C->hpin;
    }
    CF_TRY(ensure_items(C, R.items_cap));
    for (int attempt = 0; attempt < 4; attempt++) {
        CF_TRY(cf_enqueue_count(C, R, true));
        CF_CU(cudaStreamSynchronize(st), "count sync");
        if (R.bbox_deferred && attempt == 0) {
            // the inputs' check that a periodic call did not wait for (its plan needs only L)
            double bb[6], nd, v2;
            CF_TRY(cf_check_bbox(C, R, (const unsigned long long *)C->hbb, bb, nd, v2));
        }
        int retry = 0;
        CF_TRY(cf_finish(C, R, res, &retry));
        if (!retry) {
            const uint32_t n = (uint32_t)C->stats.work_items;
            C->items_hint = (uint32_t)std::min<uint64_t>(CF_MAX_ENTRIES, (uint64_t)n + n / 4 + 1024);
            C->items_key = ikey;
            record_times(C, attempt == 0);
            C->stats.ms_total =
                (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            return CF_OK;
        }
        if (retry == 1) CF_TRY(C->ensure(B_QUEUE, 16 * (size_t)R.qcap));
        if (retry == 2) CF_TRY(ensure_items(C, R.items_cap));
    }
    return C->fail(CF_ERR_INTERNAL, "recheck queue kept overflowing");
}

void cf_write_result(const cf_params *p, const CfJobResult &Q, cf_result *out)
{
    if (!out) return;
    const size_t nslot = Q.npairs.size();
    if (out->npairs) std::memcpy(out->npairs, Q.npairs.data(), 8 * nslot);
    if (out->wsum) std::memcpy(out->wsum, Q.wsum.data(), 8 * nslot);
    if (out->ravg) {
        for (size_t k = 0; k < nslot; k++) {
            double den = p->weight == CF_W_PAIR_PRODUCT ? Q.wsum[k] : (double)Q.npairs[k];
            out->ravg[k] = (p->output_ravg && den > 0) ? Q.rsum[k] / den : 0.0;
        }
    }
    if (out->wp) {
        const int nb = p->nbins;
        if (p->kind == CF_WP && p->periodic && Q.autoc) {
            // Eq. (2) with 1 + xi = DD/RR (Sec. 2.1) and RR from density (N-1)/V (Appendix B):
            // wp = DD / (N (N-1) / V * pi (rp_hi^2 - rp_lo^2)) - 2 pimax
            const double V = p->box[0] * p->box[1] * p->box[2];
            const double n = (double)Q.n1;
            for (int k = 0; k < nb; k++) {
                double area = M_PI * (p->edges[k + 1] * p->edges[k + 1] - p->edges[k] * p->edges[k]);
                double rr = n * (n - 1) / V * area;
                out->wp[k] = rr > 0 ? (double)Q.npairs[k] / rr - 2.0 * p->pimax : 0.0;
            }
        } else {
            for (int k = 0; k < nb; k++) out->wp[k] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
extern "C" {

cf_status cf_create(void **ctx_out, int device, void *cuda_stream)
{
    if (!ctx_out) return CF_ERR_ARG;
    *ctx_out = nullptr;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return CF_ERR_CUDA;
    }
    CfCtx *C = new CfCtx();
    C->device = device;
    C->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&C->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&C->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    for (auto &e : C->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            delete C;
            cudaSetDevice(prev);
            return CF_ERR_CUDA;
        }
    }
    cudaSetDevice(prev);
    *ctx_out = C;
    return CF_OK;
}

cf_status cf_destroy(void *ctx)
{
    if (!ctx) return CF_ERR_ARG;
    CfCtx *C = (CfCtx *)ctx;
    DeviceGuard g(C->device);
    cudaStreamSynchronize(C->stream);
    delete C;
    return CF_OK;
}

const char *cf_last_error(const void *ctx)
{
    if (!ctx) return "null context";
    return ((const CfCtx *)ctx)->err.c_str();
}

cf_status cf_set_option(void *ctx, int option, int64_t value)
{
    if (!ctx) return CF_ERR_ARG;
    CfCtx *C = (CfCtx *)ctx;
    if (option < 1 || option >= CF_OPT_COUNT_) return (cf_status)C->fail(CF_ERR_ARG, "unknown option");
    if (value < 0) return (cf_status)C->fail(CF_ERR_ARG, "option values must be >= 0");
    C->opt[option] = value;
    if (option == CF_OPT_MEM_CAP) C->mem_cap = (size_t)value;
    return CF_OK;
}

cf_status cf_get_stats(const void *ctx, cf_stats *out)
{
    if (!ctx || !out) return CF_ERR_ARG;
    *out = ((const CfCtx *)ctx)->stats;
    return CF_OK;
}

cf_status cf_count(void *ctx, const cf_params *params, const cf_points *d1, const cf_points *d2, cf_result *out)
{
    if (!ctx) return CF_ERR_ARG;
    CfCtx *C = (CfCtx *)ctx;
    DeviceGuard g(C->device);
    if (!params) return (cf_status)C->fail(CF_ERR_ARG, "params is NULL");
    if (params->autocorr && d2) return (cf_status)C->fail(CF_ERR_ARG, "d2 must be NULL for an auto-correlation");
    if (!params->autocorr && !d2) return (cf_status)C->fail(CF_ERR_ARG, "d2 is required for a cross-correlation");
    std::vector<const cf_points *> pts{d1};
    std::vector<CfJobDesc> jobs(1);
    jobs[0] = {0, params->autocorr ? 0 : 1, params->autocorr ? 1 : 0, 0};
    if (!params->autocorr) pts.push_back(d2);
    std::vector<CfJobResult> res;
    int rc = cf_run(C, params, pts, jobs, res);
    if (rc) return (cf_status)rc;
    cf_write_result(params, res[0], out);
    return CF_OK;
}

static int batch_jobs(CfCtx *C, const cf_params *params, const cf_points *cats, int ncat,
                      std::vector<const cf_points *> &pts, std::vector<CfJobDesc> &jobs)
{
    if (!params || !cats || ncat < 1) return C->fail(CF_ERR_ARG, "params / cats / ncat invalid");
    if (!params->autocorr) return C->fail(CF_ERR_ARG, "batched counting is for auto-correlations");
    pts.resize(ncat);
    jobs.resize(ncat);
    for (int c = 0; c < ncat; c++) {
        pts[c] = &cats[c];
        jobs[c] = {c, c, 1, 0};
    }
    return CF_OK;
}

cf_status cf_batch_count(void *ctx, const cf_params *params, const cf_points *cats, int ncat, cf_result *outs)
{
    if (!ctx) return CF_ERR_ARG;
    CfCtx *C = (CfCtx *)ctx;
    DeviceGuard g(C->device);
    std::vector<const cf_points *> pts;
    std::vector<CfJobDesc> jobs;
    int rc = batch_jobs(C, params, cats, ncat, pts, jobs);
    if (rc) return (cf_status)rc;
    std::vector<CfJobResult> res;
    rc = cf_run(C, params, pts, jobs, res);
    if (rc) return (cf_status)rc;
    for (int c = 0; c < ncat; c++)
        if (outs) cf_write_result(params, res[c], &outs[c]);
    return CF_OK;
}

cf_status cf_batch_capture(void *ctx, const cf_params *params, const cf_points *cats, int ncat)
{
    if (!ctx) return CF_ERR_ARG;
    CfCtx *C = (CfCtx *)ctx;
    DeviceGuard g(C->device);
    std::vector<const cf_points *> pts;
    std::vector<CfJobDesc> jobs;
    int rc = batch_jobs(C, params, cats, ncat, pts, jobs);
    if (rc) return (cf_status)rc;
    for (int c = 0; c < ncat; c++)
        if (!cats[c].on_device) return (cf_status)C->fail(CF_ERR_ARG, "graph capture needs device-resident catalogues");
    // a normal run sizes every buffer (and checks the inputs); the graph then records the two
    // device phases with a work-list capacity 25% above the measured size
    std::vector<CfJobResult> res;
    rc = cf_run(C, params, pts, jobs, res);
    if (rc) return (cf_status)rc;
    CfRun &R = C->run;
    R.items_cap = R.items_cap + R.items_cap / 4 + 1024;
    // the graph sizes its work list here (one pass writes it) and runs its own bbox pass in line
    R.fused_items = true;
    R.bbox_aux = false;
    if ((rc = ensure_items(C, R.items_cap))) return (cf_status)rc;
    R.qcap = std::max(R.qcap, (uint32_t)std::min<int64_t>(CF_MAX_ENTRIES, C->stats.rechecked_pairs * 2 + 4096));
    if ((rc = C->ensure(B_QUEUE, 16 * (size_t)R.qcap))) return (cf_status)rc;
    // the graph also re-runs the bbox pass, read back past the results, so that a replay can
    // check that its new data still fit the plan
    R.bb_off = (readback_bytes(R) + 255) & ~(size_t)255;
    if ((rc = C->ensure_host(R.bb_off + 8 * CFB_BBOX_WORDS * (size_t)R.nsets))) return (cf_status)rc;
    cudaStream_t user = C->stream;
    cudaStreamSynchronize(user);
    C->drop_graph();
    // record on a context-owned stream (the legacy default stream cannot be captured); the
    // graph is launched on the context's own stream by cf_batch_replay
    if (!C->cap_stream && (rc = C->cuda(cudaStreamCreateWithFlags(&C->cap_stream, cudaStreamNonBlocking), "stream")))
        return (cf_status)rc;
    cudaStream_t st = C->cap_stream;
    if ((rc = C->cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture"))) return (cf_status)rc;
    C->capturing = true;
    C->stream = st;
    C->launches = 0;          // a replay reports the graph's own kernels
    int rc0 = cf_enqueue_bbox(C, R);
    int rc1 = rc0 ? rc0 : cf_enqueue_build(C, R);
    int rc2 = rc1 ? rc1 : cf_enqueue_count(C, R, true);
    C->stream = user;
    C->capturing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc2) {
        if (graph) cudaGraphDestroy(graph);
        return (cf_status)rc2;
    }
    if ((rc = C->cuda(e, "end capture"))) return (cf_status)rc;
    C->graph = graph;
    if ((rc = C->cuda(cudaGraphInstantiate(&C->graph_exec, graph, 0), "graph instantiate"))) {
        C->drop_graph();
        return (cf_status)rc;
    }
    C->graph_gen = C->gen;
    C->graph_ncat = ncat;
    return CF_OK;
}

cf_status cf_batch_replay(void *ctx, cf_result *outs, int ncat)
{
    if (!ctx) return CF_ERR_ARG;
    CfCtx *C = (CfCtx *)ctx;
    DeviceGuard g(C->device);
    if (!C->graph_exec) return (cf_status)C->fail(CF_ERR_ARG, "no captured batch on this context");
    if (ncat != C->graph_ncat) return (cf_status)C->fail(CF_ERR_ARG, "ncat differs from the captured batch");
    if (C->gen != C->graph_gen) {
        C->drop_graph();
        return (cf_status)C->fail(CF_ERR_INTERNAL, "device scratch changed since capture; capture again");
    }
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = C->stream;
    int rc;
    if ((rc = C->cuda(cudaGraphLaunch(C->graph_exec, st), "graph launch"))) return (cf_status)rc;
    if ((rc = C->cuda(cudaStreamSynchronize(st), "graph sync"))) return (cf_status)rc;
    CfRun &R = C->run;
    std::vector<CfJobResult> res;
    int retry = 0;
    if (!bbox_within(R, (const unsigned long long *)((const char *)C->hpin + R.bb_off))) retry = 3;
    else if ((rc = cf_finish(C, R, res, &retry))) return (cf_status)rc;
    if (retry) {
        // the new data left the captured plan's box (or are not finite), or the work list or the
        // recheck queue outgrew the captured capacity: count without the graph (same inputs,
        // checked and planned afresh) and drop the graph so that the next capture sizes it again
        std::vector<const cf_points *> pts;
        for (auto &q : R.pts) pts.push_back(&q);
        std::vector<CfJobDesc> jobs = R.jobs;
        cf_params p = R.p;
        std::vector<double> edges = R.edges;
        p.edges = edges.data();
        std::vector<cf_points> keep = R.pts;
        pts.clear();
        for (auto &q : keep) pts.push_back(&q);
        if ((rc = cf_run(C, &p, pts, jobs, res))) return (cf_status)rc;
    } else {
        record_times(C, false);
        C->stats.ms_build = 0;
    }
    for (int c = 0; c < ncat; c++)
        if (outs) cf_write_result(&R.p, res[c], &outs[c]);
    C->stats.ms_total = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return CF_OK;
}

}  // extern "C"
