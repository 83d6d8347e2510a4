/*
 * cf.h -- C ABI of the GB300 binned pair counter.
 *
 * Method: Sinha & Garrison, "Corrfunc -- a suite of blazing fast correlation functions on the
 * CPU" (arXiv:1911.03545).  The library counts pairs of points binned by separation over a
 * cell-list grid (Sec. 4.1-4.3), for the four pair counters of Table 1's theory rows plus the
 * angular counter and DD(rp, pi) of observed positions: DD(r), DD(rp, pi), wp(rp), DD(theta) and
 * DDrppi_mocks (Appendix A.2.1); auto or cross; periodic or not (mocks: not);
 * optionally with pair-product weights (Sec. 2.1, weight_func) and the mean separation per
 * bin ("ravg", Sec. 6.5).
 *
 * Result definition (what every entry point returns, bit-exact for counts):
 *   - a pair (i, j) is binned by its separation s in the half-open bin lo <= s < hi, compared in
 *     squared space against e*e evaluated in FP64 (Sec. 2.1 Code naivecorr, Sec. 4.7);
 *   - r^2 = dx^2+dy^2+dz^2, rp^2 = dx^2+dy^2, pi = |dz|, z is the line of sight (Appendix A.1);
 *     the separation arithmetic is FP64 on the given coordinates (float32 inputs are widened
 *     exactly), evaluated as ((dx*dx + dy*dy) + dz*dz) without fused multiply-add;
 *   - periodic separations use the minimum image: d = a - b; if d > L/2: d -= L;
 *     if d <= -L/2: d += L (Sec. 4.4, Code normal_pbc);
 *   - pi bins have width pimax/npibins on [0, pimax) (Appendix A.1 uses width 1); pairs with
 *     pi >= pimax are excluded; wp counts are the sum over pi bins (Appendix A.1);
 *   - mocks (Appendix A.2.1): s = v1 - v2, l = 0.5*(v1 + v2) per axis, then s.l, l.l and s.s as
 *     ((x + y) + z) sums of products, pi^2 = (s.l)^2 / l.l (0 when l.l = 0), rp^2 = s.s - pi^2
 *     (clamped at 0); a pair counts when pi^2 < pimax^2 and e0^2 <= rp^2 < e_n^2, in the rp bin
 *     of rp^2 and the pi bin of pi^2 against the squared pi edges (m * pimax/npibins)^2; ravg
 *     sums sqrt(rp^2);
 *   - theta edges are in degrees; a pair of unit vectors is binned by its chord |v1 - v2|
 *     against c = 2*sin(theta*(pi/360)), squared in FP64 (Appendix A.2.2, Sec. 4.7);
 *   - auto-correlations return ordered counts: every unordered pair counted twice, plus the N
 *     self pairs in the first bin when the first edge is 0 (Sec. 4.3, Appendix B), so that
 *     auto(D) == cross(D, D);
 *   - wsum = sum of w_i*w_j per bin; ravg = sum(w_i*w_j*s)/wsum (weighted) or sum(s)/npairs,
 *     0 for an empty bin; for theta s is the angle in degrees.  Both match an FP64 evaluation
 *     within 1e-6 relative.
 *
 * Conventions for every function:
 *   - all functions return a cf_status; nothing throws across the ABI; after an error the
 *     message is available from cf_last_error(ctx) and the context stays usable;
 *   - input arrays are borrowed for the duration of the call and never freed by the library;
 *     device inputs must be readable on the context's stream;
 *   - output arrays are caller-owned host memory;
 *   - a context is not thread safe: use one context per host thread (the server below owns its
 *     own worker thread and serialises access internally).
 */
#ifndef CF_GB300_H
#define CF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CF_OK = 0,
    CF_ERR_ARG = -1,        /* invalid argument (message says which) */
    CF_ERR_OOM = -2,        /* device memory exhausted or above the context's cap */
    CF_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    CF_ERR_TIMEOUT = -4,    /* a bounded wait expired */
    CF_ERR_BUSY = -5,       /* server: result not ready yet */
    CF_ERR_CANCELLED = -6,  /* server: request was cancelled */
    CF_ERR_INTERNAL = -7    /* an internal consistency check failed */
} cf_status;

/* CF_DD_RPPI_MOCKS: DD(rp, pi) of observed positions (Appendix A.2.1, the line of sight of Fisher
 * et al. 1994): for points v1, v2 seen from an observer at the origin, s = v1 - v2,
 * l = (v1 + v2) / 2, pi = |s.l| / |l|, rp^2 = s.s - pi^2; pi bins of width pimax / npibins on
 * 0 <= pi < pimax, rp bins from `edges`.  Cartesian inputs (convert RA, DEC, comoving distance
 * beforehand), non-periodic only. */
typedef enum { CF_DD_R = 0, CF_DD_RPPI = 1, CF_WP = 2, CF_DD_THETA = 3, CF_DD_RPPI_MOCKS = 4 } cf_kind;
typedef enum { CF_F32 = 0, CF_F64 = 1 } cf_dtype;
typedef enum { CF_W_NONE = 0, CF_W_PAIR_PRODUCT = 1 } cf_weight;

#define CF_MAX_BINS 252          /* r / rp / theta bins */
#define CF_MAX_PIBINS 252        /* pi bins */

/* Problem statement (Table 1; Sec. 4.1 grid; Sec. 4.2 refinement; Appendix A bins). */
typedef struct {
    int kind;            /* cf_kind */
    int autocorr;        /* 1: d2 must be NULL, count D1 x D1 (Sec. 4.3) */
    int periodic;        /* 1: minimum-image separations in a box [0, box[a]] per axis (Sec. 4.4) */
    double box[3];       /* periodic box side per axis; ignored if !periodic */
    const double *edges; /* host array of nbins+1 strictly increasing edges >= 0: r, rp, or theta in
                            degrees (<= 180) */
    int nbins;           /* 1 .. CF_MAX_BINS */
    double pimax;        /* CF_DD_RPPI / CF_WP / CF_DD_RPPI_MOCKS: pi cut (> 0) */
    int npibins;         /* CF_DD_RPPI / CF_WP / CF_DD_RPPI_MOCKS: number of pi bins of width
                            pimax/npibins */
    int refine[3];       /* refinement factor per axis (Sec. 4.2, 1..4); 0 = automatic */
    int output_ravg;     /* 1: compute ravg (Sec. 6.5) */
    int weight;          /* cf_weight; CF_W_PAIR_PRODUCT needs w in every point set */
} cf_params;

/* A point set.  Coordinates (and w) share one dtype.  For CF_DD_THETA x,y,z are unit vectors
 * (non-periodic only).  Periodic coordinates must lie in [0, box] (Sec. 4.4: the closed
 * interval); anything else, and any non-finite value, is CF_ERR_ARG. */
typedef struct {
    const void *x, *y, *z;
    const void *w;       /* NULL unless weighted */
    int64_t n;           /* >= 0, < 2^31 */
    int dtype;           /* cf_dtype */
    int on_device;       /* 1: device pointers on the context's device; 0: host pointers */
} cf_points;

/* Caller-owned host outputs of length
 * nout = nbins * (kind == CF_DD_RPPI || kind == CF_DD_RPPI_MOCKS ? npibins : 1),
 * row-major (rp bin, pi bin).  Any pointer may be NULL to skip that output. */
typedef struct {
    uint64_t *npairs;
    double *wsum;        /* sum of w_i*w_j (pair count when unweighted) */
    double *ravg;        /* needs output_ravg */
    double *wp;          /* CF_WP with periodic autocorr only: Eq. (2) with the analytic RR of
                            Appendix B (density (N-1)/V), nbins values */
} cf_result;

/* Statistics of the last cf_count / cf_batch_count call on a context. */
typedef struct {
    int64_t evaluated_pairs;   /* separations computed by the pair kernel (i x j per work item) */
    int64_t rechecked_pairs;   /* pairs within the FP32 error band of an edge, redone in FP64 */
    int64_t work_items;        /* (i tile, j range) items of the pair kernel */
    int64_t cells;             /* cells per catalogue */
    int grid[3];               /* cells per axis */
    int refine[3];             /* refinement used */
    int variant;               /* pair kernel variant used */
    int ncat;                  /* catalogues in the call */
    float ms_build;            /* cell build + work list (CUDA events) */
    float ms_pair;             /* pair kernel (CUDA events on the context stream) */
    float ms_recheck;          /* FP64 recheck + finalize */
    float ms_total;            /* whole call, host wall clock */
    int kernel_launches;       /* CUDA kernels this library launched for the call */
    int fixed_sums;            /* rp-pi / mocks: bit 0 weight sums, bit 1 ravg sums kept per warp in
                                  fixed point (each term within 2^-22 of itself); else FP64 */
} cf_stats;

/* Create a context on `device` (its current-device state is restored on return), issuing all
 * work on `cuda_stream` (a cudaStream_t, or NULL for the legacy default stream).  The context
 * owns device scratch, grown on demand and freed by cf_destroy. */
cf_status cf_create(void **ctx_out, int device, void *cuda_stream);
cf_status cf_destroy(void *ctx);
/* Message of the last failure on this context (static storage owned by the context). */
const char *cf_last_error(const void *ctx);

/* Options (0 = default).  CF_OPT_MEM_CAP caps the context's device scratch in bytes so that
 * a request above it fails with CF_ERR_OOM instead of allocating; CF_OPT_VARIANT pins the
 * pair-kernel variant; CF_OPT_TILE pins the i-tile size (32..128); CF_OPT_JCHUNK pins the
 * j range length per work item; CF_OPT_QUEUE sets the FP64 recheck queue capacity;
 * CF_OPT_CTAS_PER_SM sets the persistent grid; CF_OPT_AUDIT = 1 sends every pair the pair
 * kernel evaluates to the FP64 recheck instead of binning it in FP32, so the call returns the FP64
 * result of every evaluated pair: equal counts with and without it show that the FP32 path
 * misclassified nothing (the band audit; slow, and CF_ERR_ARG above 2^32 - 2^28 evaluated pairs,
 * as the queue's entries are indexed in 32 bits); CF_OPT_ITER_LIMIT is reserved and has no
 * effect (no kernel of this library waits on a flag: every device loop is bounded by its data);
 * CF_OPT_WARPS and CF_OPT_REFINE are the autotuner's knobs. */
typedef enum {
    CF_OPT_MEM_CAP = 1,
    CF_OPT_VARIANT = 2,
    CF_OPT_TILE = 3,
    CF_OPT_JCHUNK = 4,
    CF_OPT_QUEUE = 5,
    CF_OPT_CTAS_PER_SM = 6,
    CF_OPT_AUDIT = 7,
    CF_OPT_ITER_LIMIT = 8,
    CF_OPT_WARPS = 9,        /* warps per CTA of the pair kernel: up to 16 for the direct form with
                                weights or ravg, up to 8 otherwise (0 = as many as fit) */
    CF_OPT_REFINE = 10,      /* refinement factor used when params.refine is 0 */
    CF_OPT_CELL_PRUNE = 11,  /* 0 (default): skip cell pairs whose points' bounding boxes lie farther
                                apart than the largest edge (and pimax along z for rp-pi / wp);
                                1: visit every stencil neighbour.  Results are the same either way */
    CF_OPT_CELL_ORDER = 12,  /* points inside a cell are ordered by Morton sub-cell: 0 (default) picks
                                the sub-cells per axis (4, 2 or 1) from the cell count; 1, 2 or 4 pin
                                it.  Results are the same for every order */
    CF_OPT_THETA_GRID = 13,  /* DD(theta) cell list: 0 (default) a 3-D grid over the unit vectors,
                                1 declination bands x right-ascension cells (Sec. 4.1.2), for wide or
                                near-polar footprints.  Results are the same for both */
    CF_OPT_BLOCK_PRUNE = 14, /* 1: inside a cell pair kept by CF_OPT_CELL_PRUNE, test each i tile
                                against every group of 32 consecutive points of the j cell and give
                                the pair kernel only the runs of groups that may hold a pair within
                                the largest edge (or pimax): the late entry / early exit of Sec. 4.5
                                at group granularity; skipped pairs are not evaluated.  0 (default):
                                whole cells.  No effect with CF_OPT_CELL_PRUNE = 1.  Results are the
                                same either way */
    CF_OPT_COUNT_ = 15
} cf_option;
cf_status cf_set_option(void *ctx, int option, int64_t value);

/* Count pairs of one point set (autocorr) or two (cross).  d2 must be NULL for autocorr.
 * Synchronous: returns after the outputs are written.  Sec. 4.1-4.7 (method), Sec. 2.1
 * (result).  Limits: fewer than 2^31 points per call; at most 2^32 - 2^20 work items (i tile x
 * j range of a cell pair) and as many pairs within the FP32 error bands of the edges (the FP64
 * recheck queue), both counted in 64 bits and refused with CF_ERR_ARG beyond. */
cf_status cf_count(void *ctx, const cf_params *params, const cf_points *d1, const cf_points *d2,
                   cf_result *out);

/* Count `ncat` independent catalogues with the same params (autocorr only): one cell build
 * over all catalogues, one persistent pair-kernel launch over the concatenated work list.
 * outs[c] receives catalogue c's results.  cf_batch_capture counts once and records the device
 * part into a CUDA graph that cf_batch_replay re-launches on new data of the same sizes (same
 * pointers).  The graph re-runs the bounding-box pass: when the new data leave the box the
 * capture was planned for (or, for DD(rp, pi) of observed positions, come nearer the observer),
 * or the work list or recheck queue outgrow the captured capacity, the replay counts without
 * the graph, with every check of cf_batch_count (so invalid data fail with CF_ERR_ARG), and
 * drops the graph: the next replay then fails until the batch is captured again.  Weighted sums
 * of a replay are FP64 (cf_stats.fixed_sums = 0). */
cf_status cf_batch_count(void *ctx, const cf_params *params, const cf_points *cats, int ncat,
                         cf_result *outs);
cf_status cf_batch_capture(void *ctx, const cf_params *params, const cf_points *cats, int ncat);
cf_status cf_batch_replay(void *ctx, cf_result *outs, int ncat);

cf_status cf_get_stats(const void *ctx, cf_stats *out);

/* Host-only planning probe (needs no GPU): builds the plan that cf_count would use for
 * `params` over the bounding box bbox = {xlo, ylo, zlo, xhi, yhi, zhi} of `npoints` points
 * (any_f64 = 1 if any input is float64) and reports it.  bands_r (nbins+1 values) and bands_p
 * (npibins+1 values, rp-pi / wp / mocks) receive the FP32 error band of each squared edge / pi
 * edge (mocks: of each squared pi edge):
 * an FP32 value within a band of an edge is re-evaluated in FP64.  With nv > 0, `values` are
 * classified through the same lookup table the pair kernel uses (which = 0: squared r / rp /
 * chord; which = 1: |dz|, or pi^2 for mocks): classes[i] = bin index, 0xFE outside every bin, 0xFF within a band.
 * which = 2 / 3 classify the same way as the direct pair kernel does (an FP32 cut at the table's
 * tail, then the lookup without its upper clamp); 0xFD there would mean an index past the table.
 * Adding 4 to `which` plans DD(theta) on the angular grid (CF_OPT_THETA_GRID = 1): grid[] then
 * reports the bands, the most RA cells of a band, and 1. 
 * Grid and refinement: Sec. 4.1-4.2; bins in squared space: Sec. 4.7. */
typedef struct {
    int grid[3];
    int refine[3];
    int wrap[3];          /* axes with explicit minimum image (periodic, fewer than 2k+1 cells) */
    int nstencil;         /* neighbour offsets kept after pruning */
    int lut_cells[2];     /* coarse table cells: squared separation, |dz| */
    int fine_entries;
    double width[3];      /* cell width per axis */
    double theta_rel;     /* relative part of the FP32 separation error bound */
    double delta[3];      /* absolute part per axis */
} cf_plan_info;
cf_status cf_plan_probe(const cf_params *params, const double bbox[6], int64_t npoints, int any_f64,
                        cf_plan_info *info, double *bands_r, double *bands_p, int which, const float *values,
                        int64_t nv, uint32_t *classes);

/* Serving: continuous batching of autocorr requests with the same params.  A worker thread
 * admits requests while device memory (mem_budget_bytes) and slots (max_slots) allow, builds
 * their cell lists while earlier requests are counted, and counts every admitted request in
 * the next pair-kernel wave.  The inputs and the cf_result arrays of a request are borrowed:
 * they must stay valid until cf_server_poll has returned something other than CF_ERR_BUSY or
 * CF_ERR_TIMEOUT for its ticket, or until cf_server_cancel has returned CF_OK for it.  A wave
 * that fails is counted again one request at a time, so one bad catalogue fails only its own
 * request.  If no worker can create its CUDA context, pending and later requests fail with
 * CF_ERR_CUDA. */
cf_status cf_server_start(void **server_out, int device, const cf_params *params,
                          size_t mem_budget_bytes, int max_slots);
/* CF_ERR_ARG (invalid catalogue), CF_ERR_OOM (larger than the budget), CF_ERR_CANCELLED (stopping),
 * CF_ERR_CUDA (no worker), else CF_OK with *ticket set. */
cf_status cf_server_submit(void *server, const cf_points *cat, cf_result *out, uint64_t *ticket);
/* CF_OK: done (result written); CF_ERR_BUSY: not yet (timeout_ms == 0); CF_ERR_TIMEOUT; or the
 * request's own error status (CF_ERR_CANCELLED after a cancel).  Any status other than BUSY and
 * TIMEOUT retires the ticket. */
cf_status cf_server_poll(void *server, uint64_t ticket, int timeout_ms);
/* Withdraw a queued request: CF_OK, after which the library no longer references its inputs or
 * result arrays and cf_server_poll returns CF_ERR_CANCELLED for it.  CF_ERR_BUSY when the request
 * is already in a wave on the GPU: it cannot be withdrawn, its buffers stay in use, and
 * cf_server_poll returns its result.  CF_OK without effect when it has already finished.
 * CF_ERR_ARG for an unknown ticket. */
cf_status cf_server_cancel(void *server, uint64_t ticket);
cf_status cf_server_stop(void *server);
/* Message of the server's last failure, copied into storage owned by the calling thread (valid
 * until that thread's next call). */
const char *cf_server_last_error(const void *server);

/* ---- allocation-free count (the paper has no counterpart) ----
 * For callers that cannot allocate device memory: code running inside another framework's memory
 * pool (every byte must come from that pool), plugins where allocation is forbidden, and programs
 * that must not allocate after start-up because an allocation can synchronise the device.
 * cf_count_noalloc allocates nothing (no cudaMalloc, cudaFree, pinned memory or allocating
 * library call).  Inputs and outputs are the caller's DEVICE arrays: d1 (and d2 for a cross
 * count) with on_device = 1; npairs / wsum / ravg of nbins * (npibins for CF_DD_RPPI and
 * CF_DD_RPPI_MOCKS) entries (any
 * may be NULL).  Results follow the definition at the top of this file (counts exact, sums
 * within 1e-6 relative).  The work is enqueued on `cuda_stream` and the function returns without
 * waiting; the outputs are ready when the stream reaches that point.
 * It evaluates every pair in FP64 without a cell list, so it suits small inputs (cost ~ N1*N2).
 * Its only scratch is a fixed array of CF_NOALLOC_SCRATCH_BYTES in the library image, present on
 * every device that loads the library until the process exits; histograms are limited to
 * CF_NOALLOC_MAX_SLOTS slots (nbins, or nbins*npibins for rp-pi and mocks): larger requests return
 * CF_ERR_ARG.  The first call on a device looks up the array's device address with that device
 * current: make that first call before any stream capture.  All calls share the array and each
 * call clears it first, so calls whose GPU work overlaps (other streams, or unordered host
 * threads) race and must not be issued.  Status: CF_ERR_ARG for invalid or oversized input,
 * CF_ERR_CUDA for a failed launch or no current device. */
#define CF_NOALLOC_MAX_SLOTS 2048
#define CF_NOALLOC_SCRATCH_BYTES 65536
cf_status cf_count_noalloc(const cf_params *params, const cf_points *d1, const cf_points *d2, uint64_t *npairs,
                           double *wsum, double *ravg, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
