// margin.cu -- the proven error margin of the FP32 distance filter.
//
// Grid frame (frame 0).  The search-and-refine kernel evaluates, for a
// query p of home cell c and a candidate q of an adjacent cell, in FP32 with
// round-to-nearest:
//     o_j  = fl(fl(c_j + 1/2) * w32)                 home cell centre, w32 = fl32(w)
//     z_j  = fl(y_j - o_j)                           y_j = fl32(fl64(x_j - g_min_j))
//     pp   = fma chain of z_p,j^2,  qq = fma chain of z_q,j^2
//     s32  = fma(m_{d-1}, z_q,d-1, ... fma(m_0, z_q,0, fl(qq + pp)))   m_j = -2 z_p,j
// i.e. s32 ~ |z_p|^2 + |z_q|^2 - 2 z_p . z_q = |z_p - z_q|^2.  The exact
// member test is s64 <= E2 = fl64(eps^2) on the FP64 sum of Section III.
// Bounds (u = 2^-24, v = 2^-53, X_j = g_max_j - g_min_j, U = max_j |g_j|):
//  (a) stored coordinate: |y_j - (x_j - g_min_j)| <= rho_j = X_j (u + v + uv) + 2^-150;
//  (b) a point of cell c satisfies |x_j - g_min_j - (c_j + 1/2) w| <= (1/2 + 3vU) w
//      (the cell index is floor of the FP64 quotient, relative error <= 3v);
//      one of an adjacent cell: <= (3/2 + 3vU) w;
//  (c) |o_j - (c_j + 1/2) w| <= 3.1 u (X_j + w);
//  so |z_p,j| <= Rp_j = (1+u)((1/2 + 3vU) w + rho_j + 3.1u(X_j + w)) and
//     |z_q,j| <= Rq_j likewise with 3/2;
//  (d) |(z_p,j - z_q,j) - (x_p,j - x_q,j)| <= eta_j = 2 rho_j + u (Rp_j + Rq_j)(1+u),
//      so | |z_p - z_q| - |Delta| | <= H = |eta|;
//  (e) expanded evaluation: |s32 - |z_p - z_q|^2| <= E = g_d (Rp^2 + Rq^2)
//      + g_{d+1} (Rp + Rq)^2 (1 + g_{d+1}) + (3d+2) 2^-149, g_k = k u / (1 - k u),
//      Rp = |(Rp_j)|, Rq = |(Rq_j)|;
//  (f) the FP64 value: |s64 - |Delta|^2| <= g64 |Delta|^2 + a64, g64 = (d+3)v/(1-(d+3)v).
// Hence, with R2 = sqrt((E2 + a64) / (1 - g64)) and R1 = sqrt((E2 - a64) / (1 + g64)):
//     s64 <= E2  =>  |Delta| <= R2  =>  s32 <= (R2 + H)^2 + E =: hi
//     s32 <= lo := (R1 - H)^2 - E  =>  |Delta| <= R1  =>  s64 <= E2.
// hi is rounded up and lo down to FP32 after a relative safety factor of
// 2^-20 that covers the rounding of this host computation.
//
// Cell frame (frame 1).  The records hold coordinates relative to a frame
// that repeats every four cells: with K_j = floor(c_j / 4) for the point's
// own cell c_j and T_j = fl64(4 K_j w),
//     y_j  = fl32(fl64(fl64(x_j - g_min_j) - T_j)),      0 <=~ y_j <~ 4 w,
// and the home cell centre is o_j = fl(fl((c_j mod 4) + 1/2) * w32).  A
// candidate of an adjacent cell may lie in the neighbouring frame (K differs
// by dK in {-1, 0, 1}); the kernel undoes that with
//     k = rint(fl(z_raw * inv4)),  z = z_raw - 4 w32 k,    inv4 = fl32(1 / (4 w32)),
// which is exact (Sterbenz: |z_raw| is within a factor 2 of 4 w32 when
// k != 0) and gives k = -dK while the home-frame value stays below 2 w in
// magnitude.  The error no longer grows with the extent X_j except through
// FP64 roundings:
//  (a') P_j = x_j - g_min_j - 4 K_j w lies in [(m - 3vU) w, (m + 1 + 3vU) w]
//       with m = c_j mod 4; |fl(x_j - g_min_j) - T_j - P_j| <= v (2 X_j + w);
//       so |fl(x_j - g_min_j) - T_j| <= Y_j = (4 + 3vU) w + v (2 X_j + w) and
//       |y_j - P_j| <= rho_j = v (2 X_j + w) + v Y_j + u (1 + v) Y_j + 2^-150;
//  (c') |o_j - (m + 1/2) w| <= oerr = 3.1 u (4 w);
//  Rp_j = (1+u)((1/2 + 3vU) w + rho_j + oerr); before the wrap
//  |z_raw,j| <= Zr_j = (1+u)((15/2 + 3vU) w + rho_j + oerr); after it
//  Rq_j = (3/2 + 3vU) w + rho_j + oerr + u Zr_j + 4 u w, the last term for the
//  frame step 4 w32 against 4 w;
//  (d') eta_j = 2 rho_j + u (Rp_j + Zr_j) + 4 u w (o cancels in z_p - z_q).
// The wrap is valid when every Rq_j < 1.99 w; (e), (f), hi and lo as above.
//
// Frame choice (automatic): the grid frame needs no wrap step in the kernel
// and is kept while its band is below 2^-10 E2; otherwise the frame with
// the narrower band; FP64 arithmetic when neither has a usable margin.
//
// Difference form (points of more than 8 dimensions).  The kernel stores
// y_j = fl32(fl64(x_j - fmin_j)) for every dimension (fmin_j = min_j - eps,
// X_j = fmax_j - fmin_j) and evaluates t_j = fl(y_p,j - y_q,j) and s32 as
// two fma chains, one over the even and one over the odd coordinates,
//     s_e = fma(t_j, t_j, ... ) (j even),  s_o likewise (j odd),  s32 = fl(s_e + s_o).
//  (a) |y_j - (x_j - fmin_j)| <= rho_j = X_j (u + v + uv) + 2^-150;
//  (b) |t_j - Delta_j| <= 2 rho_j + u (|Delta_j| + 2 rho_j);
//  (c) every term is non-negative, and each t_j^2 passes through at most
//      ceil(d/2) + 1 <= d roundings (its fma, the later fmas of its chain,
//      the final add), each a factor within (1 +- u): so
//      (1 - g_d) |t|^2 <= s32 <= (1 + g_d) |t|^2, for any grouping of the sum.
// Member: |Delta| <= R2, each |Delta_j| <= R2, so |t| <= R2 + H2 with
// H2 = |(2 rho_j + u (R2 + 2 rho_j))_j| and hi = (1 + g_d)(R2 + H2)^2.
// Conversely s32 <= lo = (1 - g_d)(R1 - H1)^2 gives |t| <= T = R1 - H1, each
// |Delta_j| <= (T + 2 rho_j (1 + u)) / (1 - u) <= D_j (T <= R1), and
// |Delta| <= T + H1 <= R1 with H1 = |(2 rho_j + u (D_j + 2 rho_j))_j|.
//
// Expanded form for points of more than 8 dimensions (the kernel of those
// points).  The grid covers six of the d dimensions; the kernel evaluates
// the grid frame's expanded sum over all d coordinates with the origin o_j
// at the home cell centre in a grid dimension (o_j as in the grid frame)
// and at the middle of the data range in the others, o_j = fl32(X_j / 2):
//     z_j = fl(y_j - o_j),  y_j = fl32(fl64(x_j - fmin_j)),
//     pp, qq as fma chains of z^2, s32 = fl(qq + pp) followed by the fma
//     terms m_j z_q,j, m_j = -2 z_p,j, in two chains (even and odd j)
//     added at the end: every term passes through at most d / 2 + 2 <= d + 1
//     roundings, which the bound (e) allows in any grouping.
// Bounds (a)-(f) hold per dimension with Rp_j, Rq_j as in the grid frame
// for a grid dimension (U = the largest grid dimension's cell count), and
// for the others |y_j - o_j| <= (1 + 2u) X_j / 2 + rho_j, so
// Rp_j = Rq_j = (1 + u)((1 + 2u) X_j / 2 + rho_j).
#include <cmath>

#include "sj_internal.cuh"

namespace sj {

namespace {

struct FrameMargin {
    bool ok = false;
    float lo32 = -1.0f, hi32 = 0.0f;
};

// The expanded-form bound from per-dimension bounds (the sums of squares
// over dimensions of eta_j, Rp_j and Rq_j; derivation above): hi and lo in
// FP32, rounded outward, or no margin when `valid` is false, the inputs are
// out of range or the band is wider than half of E2.
FrameMargin margin_tail(int d, double E2, float w32, bool valid, double Xmax, double H2, double Rp2,
                        double Rq2) {
    FrameMargin fm;
    const double u = std::ldexp(1.0, -24), v = std::ldexp(1.0, -53);
    const double safety = std::ldexp(1.0, -20);
    const double H = std::sqrt(H2) * (1.0 + safety);
    const double Rp = std::sqrt(Rp2) * (1.0 + safety), Rq = std::sqrt(Rq2) * (1.0 + safety);
    auto gam = [&](int k) { return k * u / (1.0 - k * u); };
    const double E = (gam(d) * (Rp * Rp + Rq * Rq) +
                      gam(d + 1) * (Rp + Rq) * (Rp + Rq) * (1.0 + gam(d + 1)) +
                      (3.0 * d + 2.0) * std::ldexp(1.0, -149)) *
                     (1.0 + safety);
    const double g64 = (d + 3) * v / (1.0 - (d + 3) * v);
    const double a64 = 2.0 * d * std::ldexp(1.0, -1074);
    if (!valid || !std::isfinite(E2) || !(Xmax < std::ldexp(1.0, 60)) ||
        E2 < std::ldexp(1.0, -100) || !((Rp + Rq) * (Rp + Rq) < std::ldexp(1.0, 100)) ||
        !(w32 > 0.0f) || !std::isfinite(4.0f * w32))
        return fm;
    const double R2 = std::sqrt((E2 + a64) / (1.0 - g64)) * (1.0 + safety);
    const double hi = ((R2 + H) * (R2 + H) + E) * (1.0 + safety);
    float hi32 = (float)hi;
    if ((double)hi32 < hi) hi32 = std::nextafter(hi32, INFINITY);
    float lo32 = -1.0f;
    const double R1 = std::sqrt((E2 - a64) / (1.0 + g64)) * (1.0 - safety);
    if (R1 > H) {
        const double lo = ((R1 - H) * (R1 - H) - E) * (1.0 - safety);
        if (lo > 0.0) {
            lo32 = (float)lo;
            if ((double)lo32 > lo) lo32 = std::nextafter(lo32, -INFINITY);
        }
    }
    // a band wider than half of E2 makes the filter pointless: compute in FP64
    if ((double)hi32 - (lo32 > 0.0f ? (double)lo32 : 0.0) > 0.5 * E2) return fm;
    fm.ok = true;
    fm.lo32 = lo32;
    fm.hi32 = hi32;
    return fm;
}

FrameMargin frame_margin(const Geometry &g, int frame) {
    const double u = std::ldexp(1.0, -24), v = std::ldexp(1.0, -53);
    const int d = g.d;
    const double w = g.w;
    double U = 0.0;
    for (int j = 0; j < d; ++j) U = std::fmax(U, (double)g.ng[j]);
    double H2 = 0.0, Rp2 = 0.0, Rq2 = 0.0, Xmax = 0.0;
    bool wrap_ok = true;
    for (int j = 0; j < d; ++j) {
        const double X = (g.gmax[j] - g.gmin[j]) * (1.0 + 4.0 * v);
        Xmax = std::fmax(Xmax, X);
        double rp, rq, eta;
        if (frame == SJ_FRAME_GRID) {
            const double rho = X * (u + v + u * v) + std::ldexp(1.0, -150);
            const double oerr = 3.1 * u * (X + w);
            rp = (1.0 + u) * ((0.5 + 3.0 * v * U) * w + rho + oerr);
            rq = (1.0 + u) * ((1.5 + 3.0 * v * U) * w + rho + oerr);
            eta = 2.0 * rho + u * (rp + rq) * (1.0 + u);
        } else {
            const double Y = (4.0 + 3.0 * v * U) * w + v * (2.0 * X + w);
            const double rho =
                v * (2.0 * X + w) + v * Y + u * (1.0 + v) * Y + std::ldexp(1.0, -150);
            const double oerr = 3.1 * u * 4.0 * w;
            rp = (1.0 + u) * ((0.5 + 3.0 * v * U) * w + rho + oerr);
            const double zr = (1.0 + u) * ((7.5 + 3.0 * v * U) * w + rho + oerr);
            rq = (1.5 + 3.0 * v * U) * w + rho + oerr + u * zr + 4.0 * u * w;
            eta = 2.0 * rho + u * (rp + zr) + 4.0 * u * w;
            if (!(rq < 1.99 * w)) wrap_ok = false;
        }
        H2 += eta * eta;
        Rp2 += rp * rp;
        Rq2 += rq * rq;
    }
    return margin_tail(d, g.E2, (float)w, wrap_ok, Xmax, H2, Rp2, Rq2);
}

double band_of(const FrameMargin &m) {
    return (double)m.hi32 - (m.lo32 > 0.0f ? (double)m.lo32 : 0.0);
}

}  // namespace

bool fp32_margin_diff(int d, double eps, const double *fmin, const double *fmax, float *lo32,
                      float *hi32) {
    const double u = std::ldexp(1.0, -24), v = std::ldexp(1.0, -53);
    const double safety = std::ldexp(1.0, -20);
    const double E2 = eps * eps;
    const double gd = d * u / (1.0 - d * u);
    const double g64 = (d + 3) * v / (1.0 - (d + 3) * v);
    const double a64 = 2.0 * d * std::ldexp(1.0, -1074);
    *lo32 = -1.0f;
    *hi32 = 0.0f;
    if (!std::isfinite(E2) || E2 < std::ldexp(1.0, -100)) return false;
    const double R2 = std::sqrt((E2 + a64) / (1.0 - g64)) * (1.0 + safety);
    const double R1 = std::sqrt((E2 - a64) / (1.0 + g64)) * (1.0 - safety);
    double h2 = 0.0, h1 = 0.0;
    for (int j = 0; j < d; ++j) {
        const double X = (fmax[j] - fmin[j]) * (1.0 + 4.0 * v);
        if (!(X < std::ldexp(1.0, 60))) return false;
        const double rho = X * (u + v + u * v) + std::ldexp(1.0, -150);
        const double e2 = 2.0 * rho + u * (R2 + 2.0 * rho);
        const double Dj = (R1 + 2.0 * rho * (1.0 + u)) / (1.0 - u);
        const double e1 = 2.0 * rho + u * (Dj + 2.0 * rho);
        h2 += e2 * e2;
        h1 += e1 * e1;
    }
    const double H2 = std::sqrt(h2) * (1.0 + safety), H1 = std::sqrt(h1) * (1.0 + safety);
    const double hi = (1.0 + gd) * (R2 + H2) * (R2 + H2) * (1.0 + safety);
    float h = (float)hi;
    if ((double)h < hi) h = std::nextafter(h, INFINITY);
    float l = -1.0f;
    if (R1 > H1) {
        const double lo = (1.0 - gd) * (R1 - H1) * (R1 - H1) * (1.0 - safety);
        if (lo > 0.0) {
            l = (float)lo;
            if ((double)l > lo) l = std::nextafter(l, -INFINITY);
        }
    }
    if (!std::isfinite(h) || (double)h - (l > 0.0f ? (double)l : 0.0) > 0.5 * E2) return false;
    *lo32 = l;
    *hi32 = h;
    return true;
}

bool fp32_margin_hd(int d, double eps, const double *fmin, const double *fmax, const int *grid,
                    float *lo32, float *hi32, float *mid32) {
    const double u = std::ldexp(1.0, -24), v = std::ldexp(1.0, -53);
    const double E2 = eps * eps;
    const double w = eps * (1.0 + std::ldexp(1.0, -16));
    *lo32 = -1.0f;
    *hi32 = 0.0f;
    double U = 0.0;
    for (int j = 0; j < d; ++j)
        if (grid[j]) U = std::fmax(U, std::floor((fmax[j] - fmin[j]) / w) + 1.0);
    double H2 = 0.0, Rp2 = 0.0, Rq2 = 0.0, Xmax = 0.0;
    for (int j = 0; j < d; ++j) {
        const double X = (fmax[j] - fmin[j]) * (1.0 + 4.0 * v);
        Xmax = std::fmax(Xmax, X);
        const double rho = X * (u + v + u * v) + std::ldexp(1.0, -150);
        double rp, rq;
        if (grid[j]) {
            // bounded by the home cell and its neighbours, as in the grid frame
            const double oerr = 3.1 * u * (X + w);
            rp = (1.0 + u) * ((0.5 + 3.0 * v * U) * w + rho + oerr);
            rq = (1.0 + u) * ((1.5 + 3.0 * v * U) * w + rho + oerr);
            mid32[j] = 0.0f;
        } else {
            // anywhere in the data range: origin at its middle
            mid32[j] = (float)(0.5 * (fmax[j] - fmin[j]));
            rp = rq = (1.0 + u) * ((1.0 + 2.0 * u) * 0.5 * X + rho);
        }
        const double eta = 2.0 * rho + u * (rp + rq) * (1.0 + u);
        H2 += eta * eta;
        Rp2 += rp * rp;
        Rq2 += rq * rq;
    }
    const FrameMargin m = margin_tail(d, E2, (float)w, U < 2147483648.0, Xmax, H2, Rp2, Rq2);
    if (!m.ok) return false;
    *lo32 = m.lo32;
    *hi32 = m.hi32;
    return true;
}

void fp32_margin(Geometry &g, int frame_mode) {
    g.fp32_ok = 0;
    g.frame = SJ_FRAME_GRID;
    g.lo32 = -1.0f;
    g.hi32 = 0.0f;
    g.w32 = (float)g.w;
    g.w4 = 4.0f * g.w32;
    g.inv_w4 = (float)(1.0 / (4.0 * (double)g.w32));
    const FrameMargin m0 = frame_margin(g, SJ_FRAME_GRID), m1 = frame_margin(g, SJ_FRAME_CELL);
    int pick = -1;
    if (frame_mode == SJ_FRAME_GRID) {
        pick = m0.ok ? SJ_FRAME_GRID : -1;
    } else if (frame_mode == SJ_FRAME_CELL) {
        pick = m1.ok ? SJ_FRAME_CELL : -1;
    } else if (m0.ok && band_of(m0) <= std::ldexp(g.E2, -10)) {
        pick = SJ_FRAME_GRID;
    } else if (m1.ok && (!m0.ok || band_of(m1) < band_of(m0))) {
        pick = SJ_FRAME_CELL;
    } else if (m0.ok) {
        pick = SJ_FRAME_GRID;
    }
    if (pick < 0) return;
    const FrameMargin &m = pick == SJ_FRAME_CELL ? m1 : m0;
    g.frame = pick;
    g.lo32 = m.lo32;
    g.hi32 = m.hi32;
    g.fp32_ok = 1;
}

}  // namespace sj

namespace {

sj_status margin_entry(int d, double eps, const double *gmin, const double *gmax, int frame,
                       float *w32, float *lo, float *hi) {
    if (d < 1 || d > sj::kMaxDim || !gmin || !gmax || !(eps > 0.0) || !std::isfinite(eps) ||
        (frame != SJ_FRAME_GRID && frame != SJ_FRAME_CELL))
        return SJ_EINVAL;
    sj::Geometry g;
    g.d = d;
    g.eps = eps;
    g.E2 = eps * eps;
    g.w = eps * (1.0 + std::ldexp(1.0, -16));
    for (int j = 0; j < d; ++j) {
        g.gmin[j] = gmin[j];
        g.gmax[j] = gmax[j];
        const double cells = std::floor((gmax[j] - gmin[j]) / g.w) + 1.0;
        if (!(cells < 2147483648.0)) return SJ_ERANGE;
        g.ng[j] = (int64_t)cells;
    }
    sj::fp32_margin(g, frame);
    if (w32) *w32 = g.w32;
    if (lo) *lo = g.lo32;
    if (hi) *hi = g.hi32;
    return g.fp32_ok ? SJ_OK : SJ_ERANGE;
}

}  // namespace

extern "C" sj_status sj_fp32_margin(int d, double eps, const double *gmin, const double *gmax,
                                    float *w32, float *lo, float *hi) {
    return margin_entry(d, eps, gmin, gmax, SJ_FRAME_GRID, w32, lo, hi);
}

extern "C" sj_status sj_fp32_margin_frame(int d, double eps, const double *gmin,
                                          const double *gmax, int frame, float *w32, float *lo,
                                          float *hi) {
    return margin_entry(d, eps, gmin, gmax, frame, w32, lo, hi);
}

extern "C" sj_status sj_fp32_margin_hd(int d, double eps, const double *fmin, const double *fmax,
                                       const int *grid, float *lo, float *hi, float *mid) {
    if (d < 1 || d > sj::kMaxPointDim || !fmin || !fmax || !grid || !(eps > 0.0) || !std::isfinite(eps))
        return SJ_EINVAL;
    float l = -1.0f, h = 0.0f, md[sj::kMaxPointDim] = {};
    const bool ok = sj::fp32_margin_hd(d, eps, fmin, fmax, grid, &l, &h, md);
    if (lo) *lo = l;
    if (hi) *hi = h;
    if (mid)
        for (int j = 0; j < d; ++j) mid[j] = md[j];
    return ok ? SJ_OK : SJ_ERANGE;
}

extern "C" sj_status sj_fp32_margin_diff(int d, double eps, const double *fmin,
                                         const double *fmax, float *lo, float *hi) {
    if (d < 1 || d > sj::kMaxPointDim || !fmin || !fmax || !(eps > 0.0) || !std::isfinite(eps))
        return SJ_EINVAL;
    float l = -1.0f, h = 0.0f;
    const bool ok = sj::fp32_margin_diff(d, eps, fmin, fmax, &l, &h);
    if (lo) *lo = l;
    if (hi) *hi = h;
    return ok ? SJ_OK : SJ_ERANGE;
}
