// margin.cu -- the proven error margin of the FP32 distance filter.
//
// The search-and-refine kernel evaluates, for a query p of home cell c and
// a candidate q of an adjacent cell, in FP32 with round-to-nearest:
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
#include <cmath>

#include "sj_internal.cuh"

namespace sj {

void fp32_margin(Geometry &g) {
    const double u = std::ldexp(1.0, -24), v = std::ldexp(1.0, -53);
    const int d = g.d;
    const double w = g.w;
    double U = 0.0;
    for (int j = 0; j < d; ++j) U = std::fmax(U, (double)g.ng[j]);
    double H2 = 0.0, Rp2 = 0.0, Rq2 = 0.0, Xmax = 0.0;
    for (int j = 0; j < d; ++j) {
        const double X = (g.gmax[j] - g.gmin[j]) * (1.0 + 4.0 * v);
        Xmax = std::fmax(Xmax, X);
        const double rho = X * (u + v + u * v) + std::ldexp(1.0, -150);
        const double oerr = 3.1 * u * (X + w);
        const double rp = (1.0 + u) * ((0.5 + 3.0 * v * U) * w + rho + oerr);
        const double rq = (1.0 + u) * ((1.5 + 3.0 * v * U) * w + rho + oerr);
        const double eta = 2.0 * rho + u * (rp + rq) * (1.0 + u);
        H2 += eta * eta;
        Rp2 += rp * rp;
        Rq2 += rq * rq;
    }
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

    g.fp32_ok = 0;
    g.lo32 = -1.0f;
    g.hi32 = 0.0f;
    g.w32 = (float)w;
    if (!std::isfinite(g.E2) || !(Xmax < std::ldexp(1.0, 60)) || g.E2 < std::ldexp(1.0, -100) ||
        !((Rp + Rq) * (Rp + Rq) < std::ldexp(1.0, 100)) || !std::isfinite(g.w32))
        return;
    const double R2 = std::sqrt((g.E2 + a64) / (1.0 - g64)) * (1.0 + safety);
    const double hi = ((R2 + H) * (R2 + H) + E) * (1.0 + safety);
    float hi32 = (float)hi;
    if ((double)hi32 < hi) hi32 = std::nextafter(hi32, INFINITY);
    float lo32 = -1.0f;
    const double R1 = std::sqrt((g.E2 - a64) / (1.0 + g64)) * (1.0 - safety);
    if (R1 > H) {
        const double lo = ((R1 - H) * (R1 - H) - E) * (1.0 - safety);
        if (lo > 0.0) {
            lo32 = (float)lo;
            if ((double)lo32 > lo) lo32 = std::nextafter(lo32, -INFINITY);
        }
    }
    // a band wider than half of E2 makes the filter pointless: compute in FP64
    if ((double)hi32 - (lo32 > 0.0f ? (double)lo32 : 0.0) > 0.5 * g.E2) return;
    g.lo32 = lo32;
    g.hi32 = hi32;
    g.fp32_ok = 1;
}

}  // namespace sj

extern "C" sj_status sj_fp32_margin(int d, double eps, const double *gmin, const double *gmax,
                                    float *w32, float *lo, float *hi) {
    if (d < 1 || d > sj::kMaxDim || !gmin || !gmax || !(eps > 0.0) || !std::isfinite(eps))
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
    sj::fp32_margin(g);
    if (w32) *w32 = g.w32;
    if (lo) *lo = g.lo32;
    if (hi) *hi = g.hi32;
    return g.fp32_ok ? SJ_OK : SJ_ERANGE;
}
