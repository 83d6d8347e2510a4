// cf_internal.h -- descriptors shared by the host planner and the CUDA kernels.
//
// Data layout in device memory (one call = a set of point sets and a set of jobs):
//   point set s (a catalogue, or one side of a cross count) is scattered into cell order by a
//   counting sort (Sec. 4.3: particles of a cell are stored contiguously).  For every point p
//   (global index over all sets) we keep
//     pa[p] = float4(-X, -X, -Y, -Y)   pb[p] = float4(-Z, -Z, w, w)
//   where X = x - o(cell) is the cell-relative coordinate (Sec. 4.4's shift trick applied per
//   cell), stored negated and duplicated so that one packed f32x2 add forms two separations.
//   For mocks the second copies hold the absolute position instead: pa = (-X, x, -Y, y),
//   pb = (-Z, z, w, w) with x, y, z rounded to float32.
//     plo[2p] = float4(-Xlo, -Xlo, -Ylo, -Ylo), plo[2p+1] = float4(-Zlo, -Zlo, 0, 0)
//   (float64 inputs with ravg only: x - o = X + Xlo; for mocks the second copies hold the low
//   parts of the absolute position, x = float(x) + xlo)
//     orig[p] = index of the point in its input arrays
//   cell_start[set cell offset + c] .. [c+1] delimit a cell's points.
//   A work item is one (i tile, j range, shift) triple of a cell pair (Sec. 4.3).
#pragma once
#include <stdint.h>

#include "cf.h"

#define CFI_MAX_SETS 4096
#define CFI_MAX_STENCIL 4096
#define CFI_LUT_MAX 8192          // coarse LUT cells (2 B each)
#define CFI_LUT_TARGET 4096       // preferred coarse cells per table
#define CFI_FINE_MAX 1024         // fine LUT entries (16 B each)
#define CFI_CLS_OUT 0xFEu         // class: outside every bin
#define CFI_CLS_AMB 0xFFu         // class: within the FP32 error band of an edge
#define CFI_FINE_FLAG 0x100u      // coarse entry >= this: index of a fine entry + flag
#define CFI_JMAX 512              // longest j range of a work item (9-bit j in a candidate)

// Pair-kernel item (48 bytes, three 16-byte loads)
struct CfItem {
    uint32_t ibeg;     // first i point (global sorted index)
    uint32_t jbeg;     // first j point
    uint32_t cnt;      // icnt (low 16) | jcnt (high 16)
    uint32_t meta;     // job (low 20 bits) | diag (bit 30)
    float s[3];        // shift hi:  x_i - x_j = (X_i + s + slo) - X_j
    float pad0;
    float slo[3];      // shift lo
    float pad1;
};
#define CFI_ITEM_DIAG (1u << 30)
#define CFI_ITEM_JOBMASK 0xFFFFFu

// The pair-kernel instance an item runs in (the kernel dispatches on the same thresholds): 0 an
// i tile of more than 96 points (four slots per lane), 1 a cell with itself, 2 a tile of 65-96
// points (three slots), 3 one of 33-64 (two), 4 one of at most 32 (one).  The work list is handed
// to the pair kernel in this order of classes.  (The mocks kind runs classes 0 and 2 in its
// four-slot instance.)
#define CFI_ITEM_CLASSES 5
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t cf_item_class(uint32_t cnt, uint32_t meta)
{
    if (meta & CFI_ITEM_DIAG) return 1u;
    const uint32_t ic = cnt & 0xFFFFu;
    return ic > 96u ? 0u : (ic > 64u ? 2u : (ic > 32u ? 3u : 4u));
}

// A point set (input view + where its sorted points and cells live)
struct CfSetDesc {
    const void *x, *y, *z, *w;   // device pointers of the input arrays
    int64_t n;
    int dtype;                   // 0 f32, 1 f64
    int pad;
    int64_t pbeg;                // first sorted point of this set
    int64_t cbeg;                // first cell of this set in cell_start
};

// A job: count set a (i side) against set b (j side) into histogram slot block `job`
struct CfJobDesc {
    int a, b;
    int autoc;
    int pad;
};

// Coarse/fine bin lookup on the bit pattern of a non-negative float (Sec. 4.7: bins are found
// on squared separations; the bit pattern of a positive float is monotone in its value).
struct CfLut {
    uint32_t base;     // bits of the start of coarse cell 0
    uint32_t shift;    // log2 of a coarse cell width in bit space
    uint32_t last;     // index of the last coarse cell (values above clamp here)
    uint32_t coff;     // offset of the coarse entries in the shared LUT array (in words)
    uint32_t foff;     // offset of the fine entries (in 16-byte units from the fine base)
    uint32_t tail;     // bits from which every value is outside all bins
    uint32_t pad[2];
};

struct CfFine {        // class of v: byte seg of `code`, seg = (v >= t1) + (v >= t2)
    uint32_t t1, t2, code, pad;
};

// Grid parameters (Sec. 4.1 Eq. 3 cell index; Sec. 4.2 refinement)
struct CfGrid {
    int n[3];
    int ncell;
    double lo[3];
    double width[3];
    double inv[3];         // n / extent
    double L[3];           // periodic side (0 when not periodic)
    int periodic;
    int wrap[3];           // explicit minimum image on this axis
    int k[3];
    int nstencil;
};

struct CfStencil {         // neighbour offset per axis; wrap axes enumerate targets (i+d) mod n
    int d[3];
    int pad;
};

#define CFI_MAX_ANG_K 4           // refinement of the angular grid (bands searched: 2k + 1)

// One DEC band of the angular grid (DD(theta) alternative cell list): DEC in [dlo, dhi),
// nra RA cells of width w (radians) over [0, 2 pi), cells base .. base + nra - 1.  da[d] is the RA
// half-width to search in band b + d - k: 2 asin(sin(t / 2) / cos dm) with dm the largest |DEC| of
// both bands (haversine bound), or -1 when every RA cell is searched
struct CfBand {
    double dlo, dhi, w;
    double inv_w;                      // 1 / w
    double da[2 * CFI_MAX_ANG_K + 1];  // RA half-width searched in band b + d - k (negative: every cell)
    int nra, base;
};

// Everything the kernels need for one call
struct CfDevPlan {
    CfGrid g;
    int kind;              // 0 r, 1 rppi, 2 wp, 3 theta, 4 mocks (rp-pi of observed positions)
    int nb;                // r / rp / theta bins
    int npi;               // pi bins (1 for r, theta, wp)
    int nslot;             // nb * npi for rppi and mocks, nb otherwise
    int weighted, ravg, f64lo;
    int nsets, njobs;
    int tile;              // max i tile (64 or 128)
    int jchunk;            // max j range per item
    CfLut lr, lp;          // r/rp/chord LUT, and pi LUT (rppi/wp)
    int nlut_words;        // coarse words (both LUTs)
    int nfine;             // fine entries (both LUTs)
    double pimax;
    const double *origin;  // device table of cell origins: axis a, index i at origin[ooff[a] + i]
                           // (angular grid: cell c at origin[3 c + a])
    int ooff[3];
    int ang;               // 1: angular grid (theta): DEC bands x RA cells instead of the 3-D grid
    int nband;
    const CfBand *band;    // device table of the bands
    double adlo, ah;       // lowest band edge and band height (radians)
    double tsearch;        // neighbour-search angle (radians): the largest edge, widened
    float cut_r;           // candidate cut on the FP32 squared separation (above the last band);
                           // mocks: on rp^2 in the form (s.s - cut_r) l.l < (s.l)^2
    float cut_p;           // candidate cut on the FP32 |dz| (rp-pi / wp); mocks: on pi^2 in the
                           // form (s.l)^2 < cut_p l.l
    float near2;           // mocks: a candidate whose FP32 l.l is below this goes to the FP64
                           // recheck when its s.s - cut_r is below cut_su (0: no candidate can be)
    float cut_su;
    double smax2;          // mocks: largest |s|^2 of a counted pair (rmax^2 + pimax^2, widened)
    // float32 helpers of the cell build (the FP64 pipe runs at a small fraction of the FP32 rate):
    const float *origin32; // float32 copies of `origin` (exact: origins are multiples of the float32
                           // spacing at their cell's magnitude)
    float inv32[3], lo32[3];   // n / extent and the lower corner per axis, float32
    float cguard[3];       // a float32 cell coordinate within cguard of an integer is recomputed in FP64
    float pmargin[3];      // cell-pair pruning in float32: each gap is shrunk by this (its rounding)
    float e2max32, zmax32; // the largest squared separation / |dz| of a counted pair, rounded up
    double e2[CF_MAX_BINS + 1];     // squared edges (FP64, host-computed)
    double pe[CF_MAX_PIBINS + 1];   // pi edges (mocks: squared pi edges)
};
