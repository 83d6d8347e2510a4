/*
 * cf_oracle.c -- plain FP64 CPU oracle for binned pair counts.
 *
 * TEST INFRASTRUCTURE.  This file defines what the GPU path must reproduce; it is used only
 * by tests/, by __graft_entry__.smoke() and by bench.py's CPU-baseline leg.  It shares no
 * code with the CUDA library and must never be linked into it.
 *
 * What it computes (Sinha & Garrison, "Corrfunc", arXiv:1911.03545):
 *   - Sec. 2.1, Code "naivecorr": a double loop over pairs; a pair whose separation lies
 *     outside [min, max) is skipped, otherwise its bin count is incremented and the pair
 *     weight w_i*w_j (Sec. 2.1, weight_func) added to the bin's weight sum.
 *   - Appendix A.1, Eq. (sep): r^2 = dx^2+dy^2+dz^2, rp^2 = dx^2+dy^2, pi = |dz|, with z the
 *     line of sight.  rp bins come from the edges array; pi bins are of unit width on
 *     [0, pimax] (Appendix A.1); wp counts include every pair with pi < pimax.
 *   - Appendix A.2.2 / Sec. 4.7: angular bins are compared in a monotone transform of theta
 *     instead of theta itself; here the chord length |v1 - v2| of the given unit vectors.
 *   - Appendix A.2.1 (observed or mock galaxies, the line of sight of Fisher et al.): for
 *     positions v1, v2 seen from an observer at the origin, s = v1 - v2, l = (v1 + v2) / 2,
 *     pi = s.l / |l|, rp^2 = s.s - pi^2; rp bins from the edges, pi bins as above.
 *   - Sec. 4.4, Code "normal_pbc": periodic separations use the minimum image, subtracting
 *     first and then wrapping once in each direction.
 *   - Sec. 4.3 and Appendix B: auto-correlations count each unordered pair once and double
 *     the totals; if the first bin starts at 0 the N self-pairs are added once.
 *
 * Arithmetic fixed here where the paper is silent:
 *   - bins are half-open, lo <= s < hi, compared in squared space against e2 = e*e (FP64);
 *   - the squared separation is evaluated as ((dx*dx + dy*dy) + dz*dz), no fused multiply-add
 *     (the file is compiled with -ffp-contract=off);
 *   - theta edges are in degrees; chord edge c = 2*sin(theta*(pi/360)), e2 = c*c;
 *   - pi edges p_m = m*(pimax/npibins) for m < npibins, p_npibins = pimax;
 *   - ravg sums sqrt(s) (weighted by w_i*w_j when weights are given); for theta it sums the
 *     angle in degrees, 2*asin(chord/2)*(180/pi);
 *   - mocks: each dot product is ((a.x*b.x + a.y*b.y) + a.z*b.z); pi is compared in squared
 *     space, pi^2 = (s.l * s.l) / (l.l) against the squared pi edges (0 when l = 0);
 *     rp^2 = s.s - pi^2, taken as 0 when rounding makes it negative; positions are Cartesian
 *     with the observer at the origin and never periodic.
 *
 * Modes:
 *   OR_BRUTE  every pair (i<j for auto), the definition;
 *   OR_ZWIN   the paper's z-sorted late-entry / early-exit pruning (Sec. 4.6): the second set
 *             is sorted by z and only j with z inside a window slightly wider than the
 *             maximum z separation are visited.  A pair outside the window has |dz| >= zmax,
 *             so its squared separation (a sum of non-negative rounded terms, rounding being
 *             monotone) is >= zmax^2 and it would be rejected anyway: the result is
 *             bit-identical to OR_BRUTE;
 *   OR_ROWS   for each i in [row_lo, row_hi) every ordered pair (i, j): j over all of the
 *             second set (cross), or all j != i plus the self pair when the first edge is 0
 *             (auto).  No doubling.  Summed over all rows this equals the full auto result.
 *   OR_ZROWS  OR_ROWS with OR_ZWIN's window: the same pairs of the same rows, only j inside the
 *             z window visited; bit-identical to OR_ROWS for the reason given for OR_ZWIN.  It
 *             times the z-window oracle on a sample of rows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_R 0
#define OR_RPPI 1
#define OR_WP 2
#define OR_THETA 3
#define OR_MOCKS 4

#define OR_BRUTE 0
#define OR_ZWIN 1
#define OR_ROWS 2
#define OR_ZROWS 3

typedef struct {
    int kind;
    int autocorr;
    int periodic;
    double box[3];
    const double *edges;
    int nbins;
    double pimax;
    int npibins;
    int weighted;
    int ravg;
} or_params;

typedef struct {
    int kind, periodic, nbins, npi, weighted, ravg;
    double box[3];
    double e2[1025];     /* squared r / rp / chord edges */
    double pe[1025];     /* pi edges */
    double pe2[1025];    /* squared pi edges (mocks) */
    double pimax, pimax2;
} or_plan;

static int or_nout(const or_plan *p)
{
    return (p->kind == OR_RPPI || p->kind == OR_MOCKS) ? p->nbins * p->npi : p->nbins;
}

/* Sec. 4.4, Code normal_pbc: subtract, then wrap once each way. */
static double or_sep(double a, double b, int periodic, double L)
{
    double d = a - b;
    if (periodic) {
        if (d > 0.5 * L) d -= L;
        if (d <= -0.5 * L) d += L;
    }
    return d;
}

/* Largest k with e[k] <= s, for s already known to lie in [e[0], e[n]). */
static int or_find(const double *e, int n, double s)
{
    int k = n - 1;             /* Sec. 4.7: scan from the outermost bin inwards */
    while (k > 0 && s < e[k]) k--;
    return k;
}

/* Bin one pair.  Returns the output slot, or -1 if the pair falls outside every bin; *sep is
 * the separation used for ravg. */
static int or_bin_pair(const or_plan *p, double xi, double yi, double zi, double xj, double yj,
                       double zj, double *sep)
{
    int nb = p->nbins;
    if (p->kind == OR_MOCKS) {
        /* Appendix A.2.1: s = v1 - v2, l = (v1 + v2) / 2, pi = s.l / |l|, rp^2 = s.s - pi^2 */
        double sx = xi - xj, sy = yi - yj, sz = zi - zj;
        double lx = 0.5 * (xi + xj), ly = 0.5 * (yi + yj), lz = 0.5 * (zi + zj);
        double sl = sx * lx + sy * ly;
        sl = sl + sz * lz;
        double ll = lx * lx + ly * ly;
        ll = ll + lz * lz;
        double ss = sx * sx + sy * sy;
        ss = ss + sz * sz;
        double pi2 = ll > 0.0 ? (sl * sl) / ll : 0.0;
        double rp2 = ss - pi2;
        if (rp2 < 0.0) rp2 = 0.0;
        if (!(pi2 < p->pimax2)) return -1;
        if (rp2 < p->e2[0] || rp2 >= p->e2[nb]) return -1;
        int k = or_find(p->e2, nb, rp2);
        if (p->ravg) *sep = sqrt(rp2);
        return k * p->npi + or_find(p->pe2, p->npi, pi2);
    }
    double dx = or_sep(xi, xj, p->periodic, p->box[0]);
    double dy = or_sep(yi, yj, p->periodic, p->box[1]);
    double dz = or_sep(zi, zj, p->periodic, p->box[2]);
    if (p->kind == OR_R || p->kind == OR_THETA) {
        double s = dx * dx + dy * dy;
        s = s + dz * dz;
        if (s < p->e2[0] || s >= p->e2[nb]) return -1;
        int k = or_find(p->e2, nb, s);
        if (p->ravg) {
            double c = sqrt(s);
            *sep = p->kind == OR_THETA ? 2.0 * asin(0.5 * c) * (180.0 / M_PI) : c;
        }
        return k;
    }
    /* OR_RPPI / OR_WP */
    double s = dx * dx + dy * dy;
    double pi = fabs(dz);
    if (s < p->e2[0] || s >= p->e2[nb]) return -1;
    if (!(pi < p->pimax)) return -1;
    int k = or_find(p->e2, nb, s);
    if (p->ravg) *sep = sqrt(s);
    if (p->kind == OR_WP) return k;
    int m = or_find(p->pe, p->npi, pi);
    return k * p->npi + m;
}

static int or_make_plan(const or_params *in, or_plan *p)
{
    memset(p, 0, sizeof(*p));
    if (in->nbins < 1 || in->nbins > 1024) return -1;
    p->kind = in->kind;
    p->periodic = in->periodic;
    p->nbins = in->nbins;
    p->weighted = in->weighted;
    p->ravg = in->ravg;
    for (int a = 0; a < 3; a++) p->box[a] = in->box[a];
    for (int k = 0; k <= in->nbins; k++) {
        double e = in->edges[k];
        if (in->kind == OR_THETA) {
            double c = 2.0 * sin(e * (M_PI / 360.0));
            p->e2[k] = c * c;
        } else {
            p->e2[k] = e * e;
        }
    }
    p->npi = 1;
    if (in->kind == OR_MOCKS && in->periodic) return -1;
    if (in->kind == OR_RPPI || in->kind == OR_WP || in->kind == OR_MOCKS) {
        if (in->npibins < 1 || in->npibins > 1024 || !(in->pimax > 0)) return -1;
        p->npi = in->npibins;
        p->pimax = in->pimax;
        p->pimax2 = in->pimax * in->pimax;
        double dpi = in->pimax / in->npibins;
        for (int m = 0; m < in->npibins; m++) p->pe[m] = (double)m * dpi;
        p->pe[in->npibins] = in->pimax;
        for (int m = 0; m <= in->npibins; m++) p->pe2[m] = p->pe[m] * p->pe[m];
    }
    return 0;
}

/* z-window half width: the largest |dz| a counted pair can have. */
static double or_zmax(const or_plan *p)
{
    if (p->kind == OR_RPPI || p->kind == OR_WP) return p->pimax;
    /* mocks: a pair with |dz| >= 1.001 Rsep (Rsep^2 = rmax^2 + pimax^2) has s.s >= 1.002 Rsep^2, so
     * either pi^2 >= pimax^2 or rp^2 > rmax^2, with margins far above the rounding */
    if (p->kind == OR_MOCKS) return 1.001 * sqrt(p->e2[p->nbins] + p->pimax2);
    return sqrt(p->e2[p->nbins]);
}

typedef struct {
    const double *z;
    int64_t i;
} or_zkey;

static int or_zcmp(const void *a, const void *b)
{
    const or_zkey *u = (const or_zkey *)a, *v = (const or_zkey *)b;
    if (u->z[u->i] < v->z[v->i]) return -1;
    if (u->z[u->i] > v->z[v->i]) return 1;
    return (u->i > v->i) - (u->i < v->i);
}

/* First position in the z-sorted order whose z is >= v. */
static int64_t or_lower(const double *zs, int64_t n, double v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (zs[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

int or_count(const or_params *in, int64_t n1, const double *x1, const double *y1, const double *z1,
             const double *w1, int64_t n2, const double *x2, const double *y2, const double *z2,
             const double *w2, int mode, int nthreads, int64_t row_lo, int64_t row_hi,
             uint64_t *npairs, double *wsum, double *rsum)
{
    or_plan P;
    if (or_make_plan(in, &P) != 0) return -1;
    const int autoc = in->autocorr;
    if (autoc) { n2 = n1; x2 = x1; y2 = y1; z2 = z1; w2 = w1; }
    const int nout = or_nout(&P);
    for (int k = 0; k < nout; k++) { npairs[k] = 0; wsum[k] = 0; rsum[k] = 0; }
    const int rowwise = (mode == OR_ROWS || mode == OR_ZROWS);   /* ordered pairs of a row range */
    if (!rowwise) { row_lo = 0; row_hi = n1; }
    if (row_lo < 0) row_lo = 0;
    if (row_hi > n1) row_hi = n1;

    /* z-sorted view of the second set for OR_ZWIN */
    int64_t *order = NULL;
    double *zs = NULL;
    double zmax = or_zmax(&P);
    double Lz = P.box[2];
    int use_window = (mode == OR_ZWIN || mode == OR_ZROWS);
    if (use_window && P.periodic && 2.0 * zmax * (1.0 + 1e-9) >= 0.5 * Lz) use_window = 0;
    if (use_window) {
        or_zkey *keys = (or_zkey *)malloc(sizeof(or_zkey) * (size_t)(n2 > 0 ? n2 : 1));
        order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n2 > 0 ? n2 : 1));
        zs = (double *)malloc(sizeof(double) * (size_t)(n2 > 0 ? n2 : 1));
        if (!keys || !order || !zs) { free(keys); free(order); free(zs); return -2; }
        for (int64_t j = 0; j < n2; j++) { keys[j].z = z2; keys[j].i = j; }
        qsort(keys, (size_t)n2, sizeof(or_zkey), or_zcmp);
        for (int64_t j = 0; j < n2; j++) { order[j] = keys[j].i; zs[j] = z2[keys[j].i]; }
        free(keys);
    }
    /* widen the window a little so rounding of its bounds or of dz never drops a pair */
    double zabs = fabs(Lz);
    for (int64_t j = 0; use_window && j < n2; j++) if (fabs(z2[j]) > zabs) zabs = fabs(z2[j]);
    for (int64_t i = 0; use_window && i < n1; i++) if (fabs(z1[i]) > zabs) zabs = fabs(z1[i]);
    double zwin = zmax * (1.0 + 1e-9) + 1e-12 * (zabs + 1.0);

#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int status = 0;
#pragma omp parallel
    {
        uint64_t *hc = (uint64_t *)calloc((size_t)nout, sizeof(uint64_t));
        double *hw = (double *)calloc((size_t)nout, sizeof(double));
        double *hr = (double *)calloc((size_t)nout, sizeof(double));
        if (!hc || !hw || !hr) {
#pragma omp atomic write
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = row_lo; i < row_hi; i++) {
                double xi = x1[i], yi = y1[i], zi = z1[i];
                double wi = w1 ? w1[i] : 1.0;
                /* candidate ranges [a, b) over the (possibly sorted) second set */
                int64_t ra[3], rb[3];
                int nr = 0;
                if (!use_window) {
                    ra[0] = (rowwise || !autoc) ? 0 : i + 1;
                    rb[0] = n2;
                    nr = 1;
                } else {
                    double lo = zi - zwin, hi = zi + zwin;
                    ra[nr] = or_lower(zs, n2, lo); rb[nr] = or_lower(zs, n2, hi); nr++;
                    if (P.periodic && lo < 0) {
                        ra[nr] = or_lower(zs, n2, lo + Lz); rb[nr] = n2; nr++;
                    }
                    if (P.periodic && hi > Lz) {
                        ra[nr] = 0; rb[nr] = or_lower(zs, n2, hi - Lz); nr++;
                    }
                }
                for (int q = 0; q < nr; q++) {
                    for (int64_t t = ra[q]; t < rb[q]; t++) {
                        int64_t j = use_window ? order[t] : t;
                        if (autoc) {
                            if (rowwise) { if (j == i) continue; }
                            else if (j <= i) continue;
                        }
                        double sep = 0.0;
                        int k = or_bin_pair(&P, xi, yi, zi, x2[j], y2[j], z2[j], &sep);
                        if (k < 0) continue;
                        double ww = wi * (w2 ? w2[j] : 1.0);
                        hc[k] += 1;
                        hw[k] += ww;
                        if (P.ravg) hr[k] += (P.weighted ? ww : 1.0) * sep;
                    }
                }
                /* Appendix B: the self pair of i, counted once, when the first bin starts at 0 */
                if (autoc && rowwise && in->edges[0] == 0.0) {
                    double sep = 0.0;
                    int k = or_bin_pair(&P, xi, yi, zi, xi, yi, zi, &sep);
                    if (k >= 0) { hc[k] += 1; hw[k] += wi * wi; }
                }
            }
#pragma omp critical
            {
                for (int k = 0; k < nout; k++) { npairs[k] += hc[k]; wsum[k] += hw[k]; rsum[k] += hr[k]; }
            }
        }
        free(hc); free(hw); free(hr);
    }
    free(order);
    free(zs);
    if (status) return status;

    if (autoc && !rowwise) {
        /* Sec. 4.3: unique pairs were counted; double them */
        for (int k = 0; k < nout; k++) { npairs[k] *= 2; wsum[k] *= 2.0; rsum[k] *= 2.0; }
        /* Appendix B: add the N self pairs once if the first bin starts at 0 */
        if (in->edges[0] == 0.0 && n1 > 0) {
            double sep = 0.0;
            int k = or_bin_pair(&P, x1[0], y1[0], z1[0], x1[0], y1[0], z1[0], &sep);
            if (k >= 0) {
                double sw = 0.0;
                for (int64_t i = 0; i < n1; i++) sw += w1 ? w1[i] * w1[i] : 1.0;
                npairs[k] += (uint64_t)n1;
                wsum[k] += sw;
            }
        }
    }
    return 0;
}

/* Squared edges exactly as the oracle compares against them (for tests that need them). */
int or_squared_edges(int kind, const double *edges, int nbins, double *e2)
{
    for (int k = 0; k <= nbins; k++) {
        double e = edges[k];
        if (kind == OR_THETA) {
            double c = 2.0 * sin(e * (M_PI / 360.0));
            e2[k] = c * c;
        } else {
            e2[k] = e * e;
        }
    }
    return 0;
}
