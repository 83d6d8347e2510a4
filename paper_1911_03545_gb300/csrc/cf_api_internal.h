// cf_api_internal.h -- the context object and the shared host path of the entry points.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "cf.h"
#include "cf_build.h"
#include "cf_plan.h"

enum CfBuf {
    B_IN, B_SETS, B_BBOX, B_PLAN, B_LUT, B_FINE, B_STENCIL, B_JOBS, B_CNT, B_CSTART, B_CELLID, B_SLOT,
    B_PA, B_PB, B_PLO, B_ORIG, B_SCAN, B_ICNT, B_IOFF, B_ITEMS, B_HCNT, B_HW, B_HR, B_QUEUE, B_WSQ, B_MISC, B_ORIGIN,
    B_CBOX, B_FSTART, B_BANDS, B_ORIGIN32, B_OUT, B_PLANBLK, B_GBOX, B_ORDER, B_LIVE, B_COUNT_
};

// B_OUT: the counters and histograms one call reads back, laid out as the host copy of them (one
// device-to-host copy): work-list length (u32, also at the end of its scan), at OUT_NLIVE the number
// of units with points in their i cell (u32, when the work list visits only those), the same length in 64 bits,
// evaluated pairs, the pair kernel's work cursor (u32), recheck-queue length, then from OUT_HIST
// hcnt[hsz] (u64), hw[hsz], hr[hsz] (f64) and the sum of w^2 per point set (f64); at OUT_SCAN the
// tickets of the build's two scans.  The build zeroes the first OUT_HIST bytes, the count phase
// everything from OUT_EVAL on (from 0 for the one-pass work list), each with one memset.
#define OUT_NITEMS 0
#define OUT_NLIVE 4
#define OUT_ITEMS64 8
#define OUT_EVAL 16
#define OUT_CURSOR 24
#define OUT_QCOUNT 32
#define OUT_SCAN 40
#define OUT_HIST 64

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct CfJobResult {
    std::vector<unsigned long long> npairs;
    std::vector<double> wsum, rsum;
    int64_t n1 = 0;
    bool autoc = false;
};

// most work items and recheck-queue entries of one call: both are indexed in 32 bits, and the
// grid-stride loops and the work cursor run a few thousand past the end
constexpr uint64_t CF_MAX_ENTRIES = 0xFFF00000ull;   // 2^32 - 2^20

// State of one call between its phases (kept in the context so a captured graph can be replayed)
struct CfRun {
    cf_params p;
    std::vector<double> edges;
    std::vector<cf_points> pts;
    std::vector<CfSetDesc> sets;
    std::vector<CfJobDesc> jobs;
    CfHostPlan plan;
    int nsets = 0, njobs = 0;
    int64_t npts = 0, nmax = 0, np = 1, ncell = 0, ncell_all = 0, nst = 0, nunit = 0;
    const float *cbox = nullptr;   // cell boxes for pruning (nullptr: every stencil neighbour)
    const float *gbox = nullptr;   // 32-point group boxes for pruning inside cell pairs (or nullptr)
    int sub = 1;                   // Morton sub-cells per axis inside a cell (1, 2, 4)
    int64_t nfine = 0;             // ncell_all * sub^3 counting-sort keys
    size_t nslot = 0, hsz = 0;
    bool self_pairs = false;
    double bbox[6] = {0, 0, 0, 0, 0, 0};   // union of the sets' boxes the plan was made for
    double vmin2 = 0.0;            // smallest |v|^2 over the points (mocks: the plan's near-observer test)
    bool angular = false;          // DD(theta) on the angular grid (needs unit vectors)
    bool bbox_deferred = false;    // periodic call planned from L: its bbox is checked after the final sync
    bool fused_items = false;      // the work list is counted and written in one pass (size known)
    bool live_units = false;       // the work list visits only the units whose i cell holds points
    bool bbox_aux = false;         // the bbox pass runs on the side stream: join before the readback
    // the call's plan, tables and descriptors inside the B_PLANBLK device block
    const CfDevPlan *d_plan = nullptr;
    const uint16_t *d_lut = nullptr;
    const CfFine *d_fine = nullptr;
    const CfStencil *d_stencil = nullptr;
    const CfJobDesc *d_jobs = nullptr;
    const CfSetDesc *d_sets = nullptr;
    const CfSetDesc *bb_sets = nullptr;   // the sets' descriptors the bbox pass reads (in B_BBOX)
    double *d_origin = nullptr;
    float *d_origin32 = nullptr;
    size_t bb_off = 0;             // captured graph: offset of its bbox readback in pinned memory
    std::vector<double> wmin, wmax;   // per point set: smallest nonzero |w| (inf: none), largest |w|
    bool wneg = false;                // some weight is negative
    uint32_t qcap = 0, items_cap = 0;
    CfPairCfg cfg;
    CfPairArgs args;
};

struct CfCtx {
    struct Buf {
        void *p = nullptr;
        size_t cap = 0;
    };
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 1;
    int smem_optin = 0;            // largest dynamic shared memory of one CTA (opt-in)
    std::string plan_key;          // inputs of the plan held in run.plan (empty: none)
    std::string err;
    size_t mem_cap = 0, mem_used = 0;
    Buf buf[B_COUNT_];
    void *hpin = nullptr;
    size_t hpin_cap = 0;
    void *hbb = nullptr;           // pinned bbox readback checked after the final synchronisation
    size_t hbb_cap = 0;
    void *hup = nullptr;           // pinned staging of the plan, tables and descriptors uploaded per call
    size_t hup_cap = 0;
    uint32_t items_hint = 0;       // work-list capacity for the next call with plan `items_key`
    std::string items_key;
    int64_t opt[CF_OPT_COUNT_] = {0};
    uint32_t qcap_default = 1u << 20;
    cf_stats stats = {};
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    CfRun run;
    int last_grid = 0, last_warps = 0;
    int launches = 0;              // kernels launched by the current call
    uint64_t gen = 0;              // bumped whenever device or pinned scratch is reallocated
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_gen = 0;
    int graph_ncat = 0;
    bool capturing = false;
    cudaStream_t cap_stream = nullptr;   // stream used to record the batch graph
    cudaStream_t aux = nullptr;          // side stream of the deferred bbox pass (runs beside the build)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool aux_pending = false;            // side-stream work not yet joined into `stream`

    int fail(int status, const std::string &msg);
    int cuda(cudaError_t e, const char *what);
    int ensure(int b, size_t bytes);
    int ensure_host(size_t bytes);
    int ensure_upload(size_t bytes);
    int ensure_aux();
    int ensure_bbox_host(size_t bytes);
    void drop_graph();
    ~CfCtx();
};

size_t readback_bytes(const CfRun &R);
int cf_prepare(CfCtx *C, const cf_params *p, const std::vector<const cf_points *> &pts,
               const std::vector<CfJobDesc> &jobs, CfRun &R);
int cf_enqueue_build(CfCtx *C, CfRun &R);
int cf_enqueue_count(CfCtx *C, CfRun &R, bool timed);
int cf_finish(CfCtx *C, CfRun &R, std::vector<CfJobResult> &res, int *retry);
int cf_run(CfCtx *C, const cf_params *p, const std::vector<const cf_points *> &pts, const std::vector<CfJobDesc> &jobs,
           std::vector<CfJobResult> &res);
void cf_write_result(const cf_params *p, const CfJobResult &R, cf_result *out);
