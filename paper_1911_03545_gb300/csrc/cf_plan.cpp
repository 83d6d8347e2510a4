// cf_plan.cpp -- host planning for the pair counter.
//
//  * grid: Sec. 4.1 (cells of width >= the largest separation, n = floor(extent / Rmax)),
//    Sec. 4.2 (k sub-cells per Rmax cell, (2k+1) neighbours per axis);
//  * stencil: Sec. 4.3 (cell pairs that may hold a pair within range); offsets whose cell gap
//    alone exceeds the range are dropped (the minimum cell-pair separation of Sec. 7);
//  * FP32 error bands and the bin lookup: Sec. 4.7 finds bins on squared separations; here the
//    lookup runs on the FP32 bit pattern, and every value within the proven FP32 error of an
//    edge is classed "ambiguous" and re-evaluated in FP64 by the recheck kernel.
#include "cf_plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace {

const double U32 = 5.9604644775390625e-08;   // 2^-24, FP32 unit roundoff
const double U64 = 1.1102230246251565e-16;   // 2^-53
const double SAFETY = 4.0;                    // margin on the first-order error bound

double ulp32_of_magnitude(double m)
{
    // spacing of float32 values of magnitude <= m (power of two), m > 0
    int e;
    std::frexp(m * (1.0 + 1.0 / 1048576.0), &e);   // m = f * 2^e, f in [0.5, 1)
    return std::ldexp(1.0, e - 24);
}

bool all_finite(const double *v, int n)
{
    for (int i = 0; i < n; i++)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

double cfp_origin(double lo_axis, double width, int i)
{
    double lo = lo_axis + (double)i * width;
    double hi = lo + width;
    if (lo <= 0.0 && hi >= 0.0) return 0.0;
    double m = std::max(std::fabs(lo), std::fabs(hi)) * (1.0 + 1.0 / 1048576.0);
    int e;
    std::frexp(m, &e);
    double q = std::ldexp(1.0, e - 24);
    if (lo > 0.0) return std::floor(lo / q) * q;
    return std::ceil(hi / q) * q;
}

uint32_t cfp_float_ceil_bits(double v)
{
    if (!(v > 0)) return 0u;
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}

uint32_t cfp_float_above_bits(double v)
{
    if (v < 0) return 0u;
    float f = (float)v;
    if ((double)f <= v) f = std::nextafter(f, INFINITY);
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}

int cfp_check_params(const cf_params *p, std::string &err)
{
    if (!p) { err = "params is NULL"; return CF_ERR_ARG; }
    if (p->kind < CF_DD_R || p->kind > CF_DD_RPPI_MOCKS) { err = "unknown kind"; return CF_ERR_ARG; }
    if (p->nbins < 1 || p->nbins > CF_MAX_BINS) { err = "nbins must be in [1, 252]"; return CF_ERR_ARG; }
    if (!p->edges) { err = "edges is NULL"; return CF_ERR_ARG; }
    if (!all_finite(p->edges, p->nbins + 1)) { err = "edges must be finite"; return CF_ERR_ARG; }
    if (p->edges[0] < 0) { err = "edges must be >= 0"; return CF_ERR_ARG; }
    for (int k = 0; k < p->nbins; k++)
        if (!(p->edges[k + 1] > p->edges[k])) { err = "edges must be strictly increasing"; return CF_ERR_ARG; }
    if (p->kind == CF_DD_THETA) {
        if (p->periodic) { err = "DD(theta) is non-periodic"; return CF_ERR_ARG; }
        if (p->edges[p->nbins] > 180.0) { err = "theta edges must be <= 180 degrees"; return CF_ERR_ARG; }
    }
    if (p->kind == CF_DD_RPPI_MOCKS && p->periodic) { err = "DD(rp, pi) of mocks is non-periodic"; return CF_ERR_ARG; }
    if (p->kind == CF_DD_RPPI || p->kind == CF_WP || p->kind == CF_DD_RPPI_MOCKS) {
        if (!(std::isfinite(p->pimax) && p->pimax > 0)) { err = "pimax must be finite and > 0"; return CF_ERR_ARG; }
        if (p->npibins < 1 || p->npibins > CF_MAX_PIBINS) { err = "npibins must be in [1, 252]"; return CF_ERR_ARG; }
    }
    if (p->periodic) {
        for (int a = 0; a < 3; a++)
            if (!(std::isfinite(p->box[a]) && p->box[a] > 0)) { err = "periodic box sides must be finite and > 0"; return CF_ERR_ARG; }
    }
    for (int a = 0; a < 3; a++)
        if (p->refine[a] < 0 || p->refine[a] > 4) { err = "refine factors must be in [0, 4]"; return CF_ERR_ARG; }
    if (p->weight != CF_W_NONE && p->weight != CF_W_PAIR_PRODUCT) { err = "unknown weight type"; return CF_ERR_ARG; }
    return CF_OK;
}

void cfp_edges(const cf_params *p, double *e2, double *pe)
{
    for (int k = 0; k <= p->nbins; k++) {
        double e = p->edges[k];
        if (p->kind == CF_DD_THETA) {
            double c = 2.0 * std::sin(e * (M_PI / 360.0));
            e2[k] = c * c;
        } else {
            e2[k] = e * e;
        }
    }
    if (p->kind == CF_DD_RPPI || p->kind == CF_WP || p->kind == CF_DD_RPPI_MOCKS) {
        double dpi = p->pimax / p->npibins;
        for (int m = 0; m < p->npibins; m++) pe[m] = (double)m * dpi;
        pe[p->npibins] = p->pimax;
        // mocks bin pi^2 against the squared edges (Appendix A.2.1 gives pi through s.l / |l|)
        if (p->kind == CF_DD_RPPI_MOCKS)
            for (int m = 0; m <= p->npibins; m++) pe[m] = pe[m] * pe[m];
    }
}

namespace {

// ---------------------------------------------------------------------------------------
// Bin lookup tables
// ---------------------------------------------------------------------------------------
struct Seg { uint32_t start; uint32_t cls; };
static_assert(CFI_FINE_FLAG + CFI_FINE_MAX <= 0x10000u, "coarse table entries are 16-bit");

// Class function over float bit patterns for edges E[0..m] with bands B: half-open bins
// [E_k, E_k+1) -> class k; below E_0 -> OUT (or bin 0 when E_0 == 0); at or above E_m -> OUT;
// within a band -> AMB.
std::vector<Seg> make_segments(const double *E, const double *B, int m)
{
    struct Iv { uint32_t a, b; };
    std::vector<Iv> amb;
    std::vector<uint32_t> pts;
    for (int k = 0; k <= m; k++) {
        if (k == 0 && E[0] == 0.0) continue;          // nothing lies below 0: no band needed
        uint32_t a = cfp_float_ceil_bits(E[k] - B[k]);
        uint32_t b = cfp_float_above_bits(E[k] + B[k]);
        amb.push_back({a, b});
        pts.push_back(a);
        pts.push_back(b);
    }
    pts.push_back(0u);
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    auto classify = [&](uint32_t v) -> uint32_t {
        for (auto &iv : amb)
            if (v >= iv.a && v < iv.b) return CFI_CLS_AMB;
        float f;
        std::memcpy(&f, &v, 4);
        double x = (double)f;
        if (x < E[0]) return CFI_CLS_OUT;
        if (x >= E[m]) return CFI_CLS_OUT;
        int k = m - 1;
        while (k > 0 && x < E[k]) k--;
        return (uint32_t)k;
    };
    std::vector<Seg> segs;
    for (uint32_t s : pts) {
        uint32_t c = classify(s);
        if (segs.empty() || segs.back().cls != c) segs.push_back({s, c});
    }
    return segs;
}

// Build coarse + fine tables for the segment list.  Returns false if no cell width <= the
// table limit separates the breakpoints into cells of at most three segments.
bool build_lut(const std::vector<Seg> &segs, CfLut &L, std::vector<uint16_t> &words,
               std::vector<CfFine> &fine)
{
    if (segs.size() < 2) return false;
    uint32_t lo = segs[1].start;                  // first class change
    uint32_t hi = segs.back().start;              // last class change
    // the finest cell width whose table holds <= CFI_LUT_TARGET cells: cells that contain an
    // edge need the fine entry, so narrow cells keep that slower path rare
    int s0 = 0;
    while (s0 < 23 && ((((uint64_t)hi - (((uint64_t)lo >> s0) << s0)) >> s0) + 2) > (uint64_t)CFI_LUT_TARGET) s0++;
    for (int s = s0; s >= 0; s--) {
        uint64_t w = 1ull << s;
        uint64_t base = ((uint64_t)lo >> s) << s;
        base = base >= w ? base - w : 0;
        uint64_t last = ((uint64_t)hi - base) >> s;
        if (last + 1 > (uint64_t)CFI_LUT_MAX) return false;
        std::vector<uint16_t> cw(last + 1);
        std::vector<CfFine> fw;
        bool ok = true;
        size_t si = 0;                            // segment containing the cell start
        for (uint64_t c = 0; c <= last && ok; c++) {
            uint64_t c0 = base + c * w, c1 = c0 + w;
            while (si + 1 < segs.size() && segs[si + 1].start <= c0) si++;
            // segments starting strictly inside (c0, c1)
            std::vector<Seg> inside;
            for (size_t t = si + 1; t < segs.size() && segs[t].start < c1; t++) inside.push_back(segs[t]);
            if (c == last) {
                // values above the table clamp to this cell: it must end in the final class
                for (size_t t = si + 1; t < segs.size(); t++)
                    if (segs[t].start >= c1) { ok = false; break; }
            }
            if (inside.empty()) {
                cw[c] = (uint16_t)segs[si].cls;
            } else if (inside.size() <= 2) {
                CfFine f;
                f.t1 = inside[0].start;
                f.t2 = inside.size() > 1 ? inside[1].start : 0xFFFFFFFFu;
                uint32_t c2 = inside.size() > 1 ? inside[1].cls : inside[0].cls;
                f.code = segs[si].cls | (inside[0].cls << 8) | (c2 << 16);
                f.pad = 0;
                cw[c] = (uint16_t)(CFI_FINE_FLAG + (uint32_t)(fine.size() + fw.size()));
                fw.push_back(f);
                if (fine.size() + fw.size() > CFI_FINE_MAX) ok = false;
            } else {
                ok = false;
            }
        }
        if (!ok) continue;
        L.base = (uint32_t)base;
        L.shift = (uint32_t)s;
        L.last = (uint32_t)last;
        L.coff = (uint32_t)words.size();
        L.foff = 0;
        L.tail = segs.back().start;
        words.insert(words.end(), cw.begin(), cw.end());
        fine.insert(fine.end(), fw.begin(), fw.end());
        return true;
    }
    return false;
}

}  // namespace

namespace {

// range of cos (c = 1) or sin (c = 0) over the angle interval [a0, a1] (a1 - a0 <= 2 pi)
void trig_range(double a0, double a1, int c, double &mn, double &mx)
{
    auto f = [&](double a) { return c ? std::cos(a) : std::sin(a); };
    mn = std::min(f(a0), f(a1));
    mx = std::max(f(a0), f(a1));
    // extrema at multiples of pi / 2 inside the interval
    const double q = M_PI / 2;
    for (double k = std::ceil(a0 / q); k * q <= a1; k += 1.0) {
        const double v = f(k * q);
        mn = std::min(mn, v);
        mx = std::max(mx, v);
    }
}

}  // namespace

int cfp_make_plan(const cf_params *p, const double bbox[6], int64_t npoints, int f64,
                  const int refine[3], int tile, int jchunk, CfHostPlan *out, std::string &err, int angular,
                  double vmin)
{
    CfHostPlan &H = *out;
    std::memset(&H.d, 0, sizeof(H.d));
    H.lut.clear();
    H.fine.clear();
    H.stencil.clear();
    CfDevPlan &D = H.d;
    D.kind = p->kind;
    D.nb = p->nbins;
    D.npi = (p->kind == CF_DD_RPPI || p->kind == CF_DD_RPPI_MOCKS) ? p->npibins : 1;
    D.nslot = D.nb * D.npi;
    D.weighted = p->weight == CF_W_PAIR_PRODUCT;
    D.ravg = p->output_ravg != 0;
    D.f64lo = (f64 && D.ravg) ? 1 : 0;
    D.tile = tile;
    D.jchunk = jchunk;
    D.pimax = p->pimax;
    cfp_edges(p, D.e2, D.pe);
    const bool rppi_like = p->kind == CF_DD_RPPI || p->kind == CF_WP;
    const bool mocks = p->kind == CF_DD_RPPI_MOCKS;
    // mocks: a counted pair has |s|^2 = rp^2 + pi^2 < rmax^2 + pimax^2 along no fixed axis
    const double S2 = mocks ? D.e2[D.nb] + p->pimax * p->pimax : 0.0;
    D.smax2 = S2 * (1.0 + 1e-6);

    // ---- largest separation per axis (cell width before refinement), Sec. 4.1 ----
    double rmax = std::sqrt(D.e2[D.nb]);      // r, rp or chord
    if (mocks) rmax = std::sqrt(S2);
    H.W[0] = H.W[1] = rmax;
    H.W[2] = rppi_like ? p->pimax : rmax;

    // ---- grid, Sec. 4.1 Eq. (3) and Sec. 4.2 ----
    CfGrid &G = D.g;
    G.periodic = p->periodic ? 1 : 0;
    double extent[3];
    for (int a = 0; a < 3; a++) {
        int k = refine[a] > 0 ? refine[a] : 1;
        G.k[a] = k;
        if (p->periodic) {
            G.lo[a] = 0.0;
            extent[a] = p->box[a];
            G.L[a] = p->box[a];
        } else {
            G.lo[a] = bbox[a];
            extent[a] = bbox[3 + a] - bbox[a];
            if (!(extent[a] > 0)) extent[a] = H.W[a] > 0 ? H.W[a] : 1.0;
            G.L[a] = 0.0;
        }
        double nb = std::floor(extent[a] / H.W[a]);
        if (!(nb >= 1)) nb = 1;
        if (nb > 1e6) nb = 1e6;
        G.n[a] = (int)nb * k;
    }
    // cap the number of cells (tiny separations in a large volume): a cell wider than the
    // largest separation stays correct, it only holds more points
    double cap = std::max(1048576.0, 8.0 * (double)npoints);
    for (int it = 0; it < 64; it++) {
        double tot = (double)G.n[0] * G.n[1] * G.n[2];
        if (tot <= cap) break;
        int a = 0;
        for (int b = 1; b < 3; b++) if (G.n[b] > G.n[a]) a = b;
        G.n[a] = std::max(G.k[a], (int)(G.n[a] * 0.8));
    }
    G.ncell = G.n[0] * G.n[1] * G.n[2];
    H.origin.clear();
    for (int a = 0; a < 3; a++) {
        G.width[a] = extent[a] / G.n[a];
        G.inv[a] = G.n[a] / extent[a];
        G.wrap[a] = (p->periodic && G.n[a] < 2 * G.k[a] + 1) ? 1 : 0;
        D.ooff[a] = (int)H.origin.size();
        for (int i = 0; i < G.n[a]; i++) H.origin.push_back(cfp_origin(G.lo[a], G.width[a], i));
    }

    // ---- stencil, Sec. 4.2-4.3 ----
    std::vector<int> off[3];
    for (int a = 0; a < 3; a++) {
        if (G.wrap[a]) for (int d = 0; d < G.n[a]; d++) off[a].push_back(d);
        else for (int d = -G.k[a]; d <= G.k[a]; d++) off[a].push_back(d);
    }
    auto gap = [&](int a, int d) -> double {
        if (G.wrap[a]) return 0.0;
        int g = std::abs(d) - 1;
        if (g <= 0) return 0.0;
        return g * G.width[a] * (1.0 - 1e-9);
    };
    for (int dx : off[0])
        for (int dy : off[1])
            for (int dz : off[2]) {
                double gx = gap(0, dx), gy = gap(1, dy), gz = gap(2, dz);
                bool keep;
                if (rppi_like) keep = (gx * gx + gy * gy < D.e2[D.nb] * (1 + 1e-6)) && (gz < p->pimax * (1 + 1e-6));
                else keep = gx * gx + gy * gy + gz * gz < (mocks ? S2 : D.e2[D.nb]) * (1 + 1e-6);
                if (keep) H.stencil.push_back({{dx, dy, dz}, 0});
            }
    if ((int)H.stencil.size() > CFI_MAX_STENCIL) { err = "stencil too large"; return CF_ERR_ARG; }
    G.nstencil = (int)H.stencil.size();

    // ---- angular grid for DD(theta) (Sec. 4.1.2: declination bands, right-ascension cells) ----
    // Bands of height >= tmax / k over the data's declinations; in each band RA cells at least
    // tmax / k wide at the band's edge nearest a pole.  Each cell's origin comes from the analytic
    // box of its (RA, DEC) patch on the unit sphere, widened for unit vectors stored in float32.
    double Mang[3] = {0.0, 0.0, 0.0};
    H.bands.clear();
    D.ang = (angular && p->kind == CF_DD_THETA) ? 1 : 0;
    if (D.ang) {
        const double t = p->edges[p->nbins] * (M_PI / 180.0);
        // chords are taken between the given vectors: with |v| up to 1e-3 off unit length a pair a
        // little beyond t in angle can still be below the largest chord edge
        const double tw = t * (1.0 + 2e-3) + 1e-9;
        const int k = std::min(G.k[0], CFI_MAX_ANG_K);
        G.k[0] = G.k[1] = G.k[2] = k;
        // declinations of the normalised vectors: z / |v| differs from z by <= 1.5e-3 |z|
        const double zlo = std::max(-1.0, bbox[2] - 2e-3 * std::fabs(bbox[2]) - 1e-6);
        const double zhi = std::min(1.0, bbox[5] + 2e-3 * std::fabs(bbox[5]) + 1e-6);
        const double dlo = std::asin(zlo), dhi = std::asin(zhi);
        int nband = (int)std::floor((dhi - dlo) / tw);
        nband = std::max(1, std::min(nband, 100000)) * k;
        const double h = (dhi - dlo) / nband;
        double cap = std::max(1048576.0, 8.0 * (double)npoints);
        // RA cells of a band: at least tw / k wide where the band is narrowest (its poleward edge)
        auto nra_of = [&](double blo, double bhi, double scale) {
            const double dm = std::max(std::fabs(blo), std::fabs(bhi));
            double n = std::floor(2 * M_PI * std::cos(std::min(dm, M_PI / 2)) / tw * scale);
            return (int)std::max(1.0, std::min(n, 1e6)) * k;
        };
        double scale = 1.0;
        for (int it = 0; it < 64; it++) {
            double tot = 0;
            for (int b = 0; b < nband; b++) tot += nra_of(dlo + b * h, dlo + (b + 1) * h, scale);
            if (tot <= cap) break;
            scale *= 0.8;
        }
        // The cells' origins are computed on the device (cf_ang_origin_kernel) from the same
        // boxes; here only a bound on how far a cell's points lie from its origin, per band: the
        // box is at most (cos range) + cos_max * min(w, 2) wide in x and y (|d cos a| <= |d a|) and
        // the z range of the band in z, widened like the boxes, plus one float32 spacing.
        int base = 0;
        H.origin.clear();
        double ext[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < nband; b++) {
            CfBand B;
            std::memset(&B, 0, sizeof(B));
            B.dlo = dlo + b * h;
            B.dhi = (b == nband - 1) ? dhi : dlo + (b + 1) * h;
            B.nra = nra_of(B.dlo, B.dhi, scale);
            B.w = 2 * M_PI / B.nra;
            B.base = base;
            base += B.nra;
            H.bands.push_back(B);
            double cmin, cmax, zmn, zmx;
            trig_range(B.dlo, B.dhi, 1, cmin, cmax);
            trig_range(B.dlo, B.dhi, 0, zmn, zmx);
            cmin = std::max(cmin, 0.0);
            const double wxy = (cmax - cmin) + cmax * std::min(B.w, 2.0);
            const double widen = 2.0 * (1e-3 * 1.0 + 2e-6) + 1e-7;
            ext[0] = std::max(ext[0], wxy + widen);
            ext[1] = std::max(ext[1], wxy + widen);
            ext[2] = std::max(ext[2], (zmx - zmn) + widen);
        }
        if (base <= 0 || (double)base > 2e9) { err = "angular grid too large"; return CF_ERR_ARG; }
        const double sh = std::sin(0.5 * tw);
        for (int b = 0; b < nband; b++) {
            CfBand &B = H.bands[b];
            B.inv_w = 1.0 / B.w;
            for (int d = 0; d <= 2 * CFI_MAX_ANG_K; d++) {
                const int b2 = b + d - k;
                B.da[d] = -1.0;
                if (d > 2 * k || b2 < 0 || b2 >= nband) continue;
                const CfBand &O = H.bands[b2];
                const double dm = std::max(std::max(std::fabs(B.dlo), std::fabs(B.dhi)),
                                           std::max(std::fabs(O.dlo), std::fabs(O.dhi)));
                const double cm = std::cos(std::min(dm, 0.5 * M_PI));
                if (sh < cm) B.da[d] = 2.0 * std::asin(sh / cm) * (1.0 + 1e-9) + 1e-12;
            }
        }
        D.nband = nband;
        D.adlo = dlo;
        D.ah = h;
        D.tsearch = tw;
        int maxra = 0;
        for (auto &B : H.bands) maxra = std::max(maxra, B.nra);
        G.n[0] = nband;
        G.n[1] = maxra;
        G.n[2] = 1;
        G.ncell = base;
        G.nstencil = 0;
        H.stencil.clear();
        for (int a = 0; a < 3; a++) {
            G.wrap[a] = 0;
            G.width[a] = ext[a];
            D.ooff[a] = 0;
            // |X_i + S| = |x_i - o_j| <= |x_i - x_j| + |x_j - o_j| for pairs near an edge
            Mang[a] = ext[a] + 2.0 * std::sin(tw / 2) * 1.01;
        }
    }

    // ---- float32 helpers of the cell build ----
    // The build's cell index, cell-relative coordinates and cell-pair pruning run in float32 for
    // float32 inputs; these bounds keep every decision the FP64 one (or a conservative one).
    H.origin32.assign(H.origin.begin(), H.origin.end());   // exact: snapped to the float32 grid
    {
        auto ceilf32 = [](double v) {
            const uint32_t b = cfp_float_ceil_bits(v);
            float f;
            std::memcpy(&f, &b, 4);
            return f;
        };
        for (int a = 0; a < 3; a++) {
            const double amax = D.ang ? 1.01 : std::max(std::fabs(G.lo[a]), std::fabs(G.lo[a] + extent[a]));
            D.inv32[a] = (float)G.inv[a];
            D.lo32[a] = (float)G.lo[a];
            // t32 = fl(fl(x - lo32) * inv32) is within 2^-24 (inv |lo| + 3 n + 1) of the exact cell
            // coordinate (x - lo) * n / extent of a point inside the grid; the kernel redoes in
            // FP64 any t32 within four times that of an integer (a cell boundary)
            D.cguard[a] = ceilf32(4 * U32 * (G.inv[a] * std::fabs(G.lo[a]) + 3.0 * G.n[a] + 1.0));
            // the gap of two cell boxes under a shift, fl(fl(b_i + s) - b_j) with
            // s = fl(fl(o_i - o_j) - fl(delta)), carries at most 6 roundings at magnitudes up to
            // 2 amax + 2 L + 4 w (and fl(delta) is within 2^-24 L of delta); on top of the FP64
            // form's margin of 1e-5 w
            D.pmargin[a] = ceilf32(1e-5 * G.width[a] + 8 * U32 * (2 * amax + 2 * G.L[a] + 4 * G.width[a]));
        }
        // squared gaps summed in float32 are within 3 roundings below the exact sum of the shrunk
        // gaps' squares: prune only at or above the bound raised by 2^-20
        D.e2max32 = ceilf32((mocks ? D.smax2 : D.e2[D.nb]) * (1.0 + 1.0 / 1048576.0));
        D.zmax32 = ceilf32(p->pimax * (1.0 + 1.0 / 1048576.0));
    }

    // ---- FP32 error model: a per-axis bound on the separation's error, then a band per edge ----
    // stored cell-relative coordinates X are exact for float32 inputs (snapped origins);
    // float64 inputs round to float32 (epsX), or keep a lo part when ravg is requested.
    const double u = U32;
    const bool precise = D.ravg;
    for (int a = 0; a < 3; a++) {
        double amax = D.ang ? 1.01 : std::max(std::fabs(G.lo[a]), std::fabs(G.lo[a] + extent[a]));
        double Q = ulp32_of_magnitude(std::max(amax, 1e-300));
        double M = D.ang ? Mang[a] : (G.wrap[a] ? (extent[a] + 2 * G.width[a]) : ((G.k[a] + 1) * G.width[a]));
        M = M * 1.001 + 4 * Q;
        double epsX = 0;
        if (f64) epsX = D.f64lo ? (2 * U64 * 2 * amax + u * u * (G.width[a] + 2 * Q)) : (u * (G.width[a] + 2 * Q) + 2 * U64 * amax);
        double wrapterm = G.wrap[a] ? u * G.L[a] : 0.0;
        double truth = 2 * U64 * (M + G.L[a] + amax);
        double delta;
        if (precise) delta = 4 * u * u * M + 2 * epsX + wrapterm + truth;
        else delta = u * M + u * M + 2 * epsX + wrapterm + truth;
        H.delta[a] = delta;
        H.M[a] = M;
    }
    H.theta_rel = precise ? 2 * u : u;
    auto band_sq = [&](double E, int naxes, double th, const double *delta) -> double {
        double d = std::sqrt(E) * 1.01 + 1e-300;
        double sumD = 0, quad = 0;
        for (int a = 0; a < naxes; a++) {
            sumD += delta[a];
            quad += (th * d + delta[a]) * (th * d + delta[a]);
        }
        double chain = (naxes == 3 ? 3 : 2) * u * E;
        return SAFETY * (2 * th * E + 2 * d * sumD + quad + chain + 4 * U64 * E);
    };
    int naxes = rppi_like ? 2 : 3;
    for (int k = 0; k <= D.nb; k++) H.band_r[k] = band_sq(D.e2[k], naxes, H.theta_rel, H.delta);
    if (rppi_like) {
        for (int m = 0; m <= p->npibins; m++)
            H.band_p[m] = SAFETY * (H.theta_rel * D.pe[m] + H.delta[2] + 4 * U64 * D.pe[m]);
    }
    H.eta = 0.0;
    D.near2 = 0.0f;
    D.cut_su = 0.0f;
    if (mocks) {
        // Error model of the mocks kernel (Appendix A.2.1 evaluated in FP32).  Per pair: s from
        // the cell-relative coordinates (per-axis error <= delta, Dl2 its 2-norm), l = A_i - s/2
        // from the float32 absolute position A_i; the binned values are pi^2 = (s.l)^2 / l.l and
        // rp^2 = |s x A_i|^2 / l.l (s x A_i = s x l exactly).  A candidate with l.l below
        // near2 = S^2 goes to the FP64 recheck, so every other one has |l| >= 0.999 S and
        // |A_i| <= 1.51 |l|.  Both values divide
        // by l.l through one reciprocal (<= 2 ulp) and a product.
        double Dl = 0.0, Dl2 = 0.0;
        for (int a = 0; a < 3; a++) {
            Dl += H.delta[a];
            Dl2 += H.delta[a] * H.delta[a];
        }
        Dl2 = std::sqrt(Dl2);
        const double uA = f64 ? u : 0.0;
        const double S = std::sqrt(S2);
        const double lmin = 0.999 * S;
        const double eta = (uA + u) + (0.5 * uA * S + 0.5 * Dl2) / lmin;   // |error of l| / |l|
        if (!(eta < 1e-4)) {
            err = "coordinates too large for the FP32 mocks kernel at these separations";
            return CF_ERR_ARG;
        }
        H.eta = eta;
        const double ell = (2 * eta + eta * eta + 3 * u) * 1.01;          // relative error of l.l
        const double aA = 1.51;                                          // |A_i| / |l|
        const double truth = 64 * U64;                    // the FP64 evaluation's own error / S^2
        const double pm2 = p->pimax * p->pimax;
        // |pi^2 - its FP32 value| for pi <= pimx, |s| <= Sx, rp <= rpx.  To first order the error
        // of s enters as 2 pi (eps . l/|l|) and that of l as 2 pi (rp_vec . dl) / |l|; the dot
        // product's rounding as 2 pi 3u |s|; l.l, the square and the division relatively.
        auto epi = [&](double pimx, double Sx, double rpx) {
            const double e1 = (Dl2 + rpx * eta + 3 * u * Sx) * 1.001;
            const double e2nd = Dl2 + Sx * eta + 3 * u * Sx;
            return (2 * pimx * e1 + e2nd * e2nd + pimx * pimx * ell) * (1 + 6 * u) + 6 * u * pimx * pimx;
        };
        // |rp^2 - its FP32 value| for rp <= rpx, |s| <= Sx: |c - its FP32 value| <= g |l| with
        // c = s x A_i (input errors |eps||A| + |s||dA|; each component a difference of two rounded
        // products, rounded), then |c|^2's chain (3u), the reciprocal (4u) and product (u), l.l
        auto erp = [&](double rpx, double Sx) {
            const double g = aA * (Dl2 + Sx * uA + 2 * u * (Sx + Dl2) * 1.001) + u * rpx;
            return 2 * rpx * g + g * g + rpx * rpx * (8 * u + ell);
        };
        for (int k = 0; k <= D.nb; k++) {
            const double Sk = std::sqrt(D.e2[k] + pm2) * 1.001;
            H.band_r[k] = SAFETY * erp(std::sqrt(D.e2[k]) * 1.0001, Sk) * 1.001 + truth * Sk * Sk;
        }
        const double rpm = std::sqrt(D.e2[D.nb] + H.band_r[D.nb]) * 1.001;
        for (int m = 0; m <= p->npibins; m++) {
            const double Sm = std::sqrt(rpm * rpm + D.pe[m]) * 1.001;
            H.band_p[m] = SAFETY * epi(std::sqrt(D.pe[m]) * 1.0001 + 1e-300, Sm, rpm) + truth * Sm * Sm;
        }
        // Candidate cuts in the multiplied form (s.s - cut_r) l.l < (s.l)^2 < cut_p l.l, loose by
        // twice the error of that form: s.s (input error, the chain from -cut_r), pi^2 as above
        // with the full |s| in place of rp, and the form's own roundings.
        const double Cbound = 1.1 * S2;
        auto ess = [&](double Sx) {
            const double a = Sx + Dl;
            return 2 * Sx * Dl + Dl * Dl + 3 * u * (Cbound + a * a) + u * a * a;
        };
        const double Smax = S * 1.001;
        const double ecut = ess(Smax) + epi(p->pimax * 1.001, Smax, Smax) + u * (D.e2[D.nb] + S2);
        const double Cr = D.e2[D.nb] + 2 * SAFETY * ecut + 8 * u * S2;
        const double Cp = pm2 + 2 * H.band_p[p->npibins] + 8 * u * pm2;
        D.cut_r = (float)Cr;
        if ((double)D.cut_r < Cr) D.cut_r = std::nextafter(D.cut_r, INFINITY);
        D.cut_p = (float)Cp;
        if ((double)D.cut_p < Cp) D.cut_p = std::nextafter(D.cut_p, INFINITY);
        // Near the observer: a candidate with |s| up to the stencil's reach may have a midpoint
        // within S of the origin unless every point is at least that far plus half the reach.
        double reach = 0.0;
        for (int a = 0; a < 3; a++) reach += ((G.k[a] + 1) * G.width[a]) * ((G.k[a] + 1) * G.width[a]);
        reach = std::sqrt(reach) * 1.001;
        if (vmin < 0.0) {
            double g2 = 0.0;
            for (int a = 0; a < 3; a++) {
                const double gap = std::max(0.0, std::max(bbox[a], -bbox[3 + a]));
                g2 += gap * gap;
            }
            vmin = std::sqrt(g2) * (1.0 - 1e-12);
        }
        if (!(vmin - 0.5 * reach >= 1.01 * S)) {
            D.near2 = (float)S2;
            // s.s - cut_r of a near candidate that may count: s.s <= S^2 (1 + 1e-4) + 2 ess(S)
            const double su = S2 * (1 + 1e-4) + 2 * ess(S) - (double)D.cut_r;
            D.cut_su = (float)su;
            if ((double)D.cut_su < su) D.cut_su = std::nextafter(D.cut_su, INFINITY);
        }
    }
    // ---- lookup tables ----
    {
        auto segs = make_segments(D.e2, H.band_r, D.nb);
        if (!build_lut(segs, D.lr, H.lut, H.fine)) {
            err = "bin edges too close together for the FP32 lookup table";
            return CF_ERR_ARG;
        }
    }
    if (rppi_like || mocks) {
        std::vector<double> pe(D.pe, D.pe + p->npibins + 1);
        std::vector<double> bp(H.band_p, H.band_p + p->npibins + 1);
        int m = p->npibins;
        if (p->kind == CF_WP) { pe = {0.0, p->pimax}; bp = {0.0, H.band_p[p->npibins]}; m = 1; }
        auto segs = make_segments(pe.data(), bp.data(), m);
        if (!build_lut(segs, D.lp, H.lut, H.fine)) {
            err = "pi bins too narrow for the FP32 lookup table";
            return CF_ERR_ARG;
        }
    }
    // candidate cuts of the pair kernel's first phase: the FP32 value at which the final
    // "outside every bin" segment of each table starts
    if (!mocks) {
        float f;
        std::memcpy(&f, &D.lr.tail, 4);
        D.cut_r = f;
        if (rppi_like) std::memcpy(&f, &D.lp.tail, 4);
        else f = INFINITY;
        D.cut_p = f;
    }
    D.nlut_words = (int)H.lut.size();
    D.nfine = (int)H.fine.size();
    return CF_OK;
}

// Host emulation of the kernel's table lookup (same arithmetic as lut_class in cf_pair.cuh).
uint32_t cfp_lut_class(const CfHostPlan &H, int which, uint32_t vb)
{
    const CfLut &L = (which & 1) ? H.d.lp : H.d.lr;
    if (which & 2) {
        // the direct pair kernel: an FP32 cut at the tail, then the lookup without upper clamp
        // (lut_class_in in cf_pair.cuh); 0xFD flags an index past the table
        if (vb >= L.tail) return CFI_CLS_OUT;
        const uint32_t idx = (std::max(vb, L.base) - L.base) >> L.shift;
        if (idx > L.last) return 0xFDu;
        uint32_t c = H.lut[L.coff + idx];
        if (c >= CFI_FINE_FLAG) {
            const CfFine &f = H.fine[c - CFI_FINE_FLAG];
            uint32_t seg = (vb >= f.t1 ? 1u : 0u) + (vb >= f.t2 ? 1u : 0u);
            c = (f.code >> (8u * seg)) & 0xFFu;
        }
        return c;
    }
    int t = (int)(vb - L.base);
    t = t > 0 ? t : 0;
    uint32_t idx = std::min((uint32_t)t >> L.shift, L.last);
    uint32_t c = H.lut[L.coff + idx];
    if (c >= CFI_FINE_FLAG) {
        const CfFine &f = H.fine[c - CFI_FINE_FLAG];
        uint32_t seg = (vb >= f.t1 ? 1u : 0u) + (vb >= f.t2 ? 1u : 0u);
        c = (f.code >> (8u * seg)) & 0xFFu;
    }
    return c;
}

extern "C" cf_status cf_plan_probe(const cf_params *params, const double bbox[6], int64_t npoints, int any_f64,
                                   cf_plan_info *info, double *bands_r, double *bands_p, int which,
                                   const float *values, int64_t nv, uint32_t *classes)
{
    if (!params || !bbox) return CF_ERR_ARG;
    std::string err;
    if (cfp_check_params(params, err) != CF_OK) return CF_ERR_ARG;
    const bool rppi_like = params->kind == CF_DD_RPPI || params->kind == CF_WP || params->kind == CF_DD_RPPI_MOCKS;
    if (which < 0 || which > 7) return CF_ERR_ARG;
    const int angular = (which & 4) ? 1 : 0;
    which &= 3;
    if ((which & 1) && !rppi_like && nv > 0) return CF_ERR_ARG;
    CfHostPlan *H = new CfHostPlan();
    int refine[3];
    for (int a = 0; a < 3; a++) refine[a] = params->refine[a] > 0 ? params->refine[a] : 1;
    int rc = cfp_make_plan(params, bbox, npoints, any_f64, refine, 128, 512, H, err, angular);
    if (rc) {
        delete H;
        return (cf_status)rc;
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        for (int a = 0; a < 3; a++) {
            info->grid[a] = H->d.g.n[a];
            info->refine[a] = H->d.g.k[a];
            info->wrap[a] = H->d.g.wrap[a];
            info->width[a] = H->d.g.width[a];
            info->delta[a] = H->delta[a];
        }
        info->nstencil = H->d.g.nstencil;
        info->lut_cells[0] = (int)H->d.lr.last + 1;
        info->lut_cells[1] = rppi_like ? (int)H->d.lp.last + 1 : 0;
        info->fine_entries = (int)H->fine.size();
        info->theta_rel = H->theta_rel;
    }
    if (bands_r)
        for (int k = 0; k <= params->nbins; k++) bands_r[k] = H->band_r[k];
    if (bands_p && rppi_like)
        for (int m = 0; m <= params->npibins; m++) bands_p[m] = H->band_p[m];
    for (int64_t i = 0; i < nv; i++) {
        uint32_t b;
        std::memcpy(&b, values + i, 4);
        classes[i] = cfp_lut_class(*H, which, b);
    }
    delete H;
    return CF_OK;
}
