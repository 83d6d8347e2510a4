// cf_plan.h -- host-side planning: validation, grid, stencil, FP32 error bands, bin LUTs.
#pragma once
#include <string>
#include <vector>

#include "cf_internal.h"

struct CfHostPlan {
    CfDevPlan d;                       // copied to device memory for the kernels
    std::vector<uint16_t> lut;         // coarse LUT entries (class or fine flag | index): r-like LUT then pi LUT
    std::vector<CfFine> fine;          // fine LUT entries (both LUTs)
    std::vector<CfStencil> stencil;    // neighbour offsets after pruning
    std::vector<double> origin;        // cell origins per axis (see cfp_origin), n0 + n1 + n2 values
                                       // (angular grid: 3 per cell)
    std::vector<float> origin32;       // the same origins as float32 (exact)
    std::vector<CfBand> bands;         // angular grid: the DEC bands
    double W[3];                       // largest separation a counted pair can have, per axis
    double band_r[CF_MAX_BINS + 1];    // FP32 error band of each squared edge
    double band_p[CF_MAX_PIBINS + 1];  // FP32 error band of each pi edge
    double theta_rel, delta[3], M[3];  // error model terms (for diagnostics)
    double eta;                        // mocks: bound on |error of l| / |l| (diagnostics)
};

// Validate the parameters alone (no point data).  Returns 0 or CF_ERR_ARG with a message.
int cfp_check_params(const cf_params *p, std::string &err);

// Squared edges (r, rp: e*e; theta: (2 sin(theta pi/360))^2) and pi edges, FP64.
void cfp_edges(const cf_params *p, double *e2, double *pe);

// Build the plan.  bbox = {xlo, ylo, zlo, xhi, yhi, zhi} over every point set of the call;
// npoints = total points (caps the grid); f64 = any float64 input; refine = requested factors
// (0 = automatic); tile = max i tile (64 or 128); jchunk = max j range per work item.
// angular = 1 (DD(theta) only): DEC bands x RA cells instead of the 3-D grid over unit vectors.
// vmin (mocks only): a lower bound on |v| over the points (negative: derived from bbox).
int cfp_make_plan(const cf_params *p, const double bbox[6], int64_t npoints, int f64,
                  const int refine[3], int tile, int jchunk, CfHostPlan *out, std::string &err,
                  int angular = 0, double vmin = -1.0);

// Origin of cell i on an axis starting at lo with cell width w.  For float32 coordinates x in
// the cell, x - origin is exact in float32: the origin is a multiple of the float32 spacing at
// the cell's largest magnitude and lies between 0 and every x of the cell (0 itself for a cell
// that straddles 0).
double cfp_origin(double lo, double width, int i);

// Bits of the smallest float >= v (v >= 0), and of the smallest float > v.
uint32_t cfp_float_ceil_bits(double v);
uint32_t cfp_float_above_bits(double v);
