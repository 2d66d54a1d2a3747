// Host-side planning of the exp / psi actions, shared by the problem path
// (engine.cu) and the allocation-free action (noalloc.cu): the real shift mu
// that minimises the row-sum bound of t (A_s - mu I) (the shift of Sec. 3.4
// written as exp(M) = e^{i t mu} exp(i t (A_s - mu I))), and the Taylor plan
// (sub-steps S, degree m) that meets a truncation tolerance for that bound.
#include <algorithm>
#include <cmath>

#include "mxp_internal.h"

namespace mxp {

using cd = std::complex<double>;

// nu(mu) = t * max over (one class per axis, kappa in {kmin, kmax}) of
//          sum_d (|wp_d| + |wm_d|) + |kappa (1 + i s) - sum_d wc_d - mu|.
// This bounds ||t (A_s - mu I)||_inf from above (|.| is convex in kappa, so
// the extreme values of kappa bound every cell of a class).
static double nu_of_mu(const AxisClasses *cls, int dim, const double kap[2], cd z, double t, double mu)
{
    const size_t n0 = cls[0].off.size(), n1 = dim > 1 ? cls[1].off.size() : 1,
                 n2 = dim > 2 ? cls[2].off.size() : 1;
    double best = 0;
    for (size_t a = 0; a < n0; ++a)
        for (size_t b = 0; b < n1; ++b)
            for (size_t c = 0; c < n2; ++c) {
                double off = cls[0].off[a];
                cd wcs = cls[0].wc[a];
                if (dim > 1) { off += cls[1].off[b]; wcs += cls[1].wc[b]; }
                if (dim > 2) { off += cls[2].off[c]; wcs += cls[2].wc[c]; }
                for (int q = 0; q < 2; ++q) best = std::max(best, off + std::abs(kap[q] * z - wcs - mu));
            }
    return t * best;
}

ShiftChoice choose_shift(const AxisClasses *cls, int dim, double kmin, double kmax, double shift_s, double t)
{
    const double kap[2] = {kmin, kmax};
    const cd z(1.0, shift_s);
    // nu(mu) is convex: golden-section search between the extreme real parts of
    // kappa - sum_d wc_d, where its minimiser lies
    double lo = 1e300, hi = -1e300;
    const size_t n0 = cls[0].off.size(), n1 = dim > 1 ? cls[1].off.size() : 1,
                 n2 = dim > 2 ? cls[2].off.size() : 1;
    for (size_t a = 0; a < n0; ++a)
        for (size_t b = 0; b < n1; ++b)
            for (size_t c = 0; c < n2; ++c) {
                double wr = cls[0].wc[a].real();
                if (dim > 1) wr += cls[1].wc[b].real();
                if (dim > 2) wr += cls[2].wc[c].real();
                for (int q = 0; q < 2; ++q) {
                    lo = std::min(lo, kap[q] - wr);
                    hi = std::max(hi, kap[q] - wr);
                }
            }
    const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
    double a = lo, b = hi;
    double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
    double f1 = nu_of_mu(cls, dim, kap, z, t, x1), f2 = nu_of_mu(cls, dim, kap, z, t, x2);
    for (int it = 0; it < 200 && (b - a) > 1e-12 * (std::abs(a) + std::abs(b) + 1); ++it) {
        if (f1 < f2) { b = x2; x2 = x1; f2 = f1; x1 = b - gr * (b - a); f1 = nu_of_mu(cls, dim, kap, z, t, x1); }
        else { a = x1; x1 = x2; f1 = f2; x2 = a + gr * (b - a); f2 = nu_of_mu(cls, dim, kap, z, t, x2); }
    }
    ShiftChoice out;
    out.mu = 0.5 * (a + b);
    out.nu = nu_of_mu(cls, dim, kap, z, t, out.mu);
    return out;
}

TaylorPlan make_plan(double nu, double tol, double theta_max, int kmult)
{
    TaylorPlan best;
    best.nu = nu;
    if (!(nu > 0)) {
        best.S = 1;
        best.m = kmult;
        return best;
    }
    const int Smin = std::max(1, (int)std::ceil(nu / theta_max));
    long best_cost = -1;
    for (int S = Smin; S <= 4 * Smin + 8; ++S) {
        const double th = nu / S;
        const double lt = std::log(tol);
        int m = 1;
        for (; m < 400; ++m) {
            const double lg = std::log((double)S) + (m + 1) * std::log(th) - std::lgamma(m + 2.0) + th;
            if (lg <= lt) break;
        }
        if (kmult > 1) m = ((m + kmult - 1) / kmult) * kmult;
        const long cost = (long)m * S;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best.S = S;
            best.m = m;
        }
    }
    return best;
}

}  // namespace mxp

extern "C" int mxp_taylor_plan(double nu, double tol, double theta_max, int kmult, int *S, int *m)
{
    if (!S || !m || !(nu >= 0) || !(tol > 0 && tol < 1) || !(theta_max > 0) || kmult < 1) return 0;
    const mxp::TaylorPlan pl = mxp::make_plan(nu, tol, theta_max, kmult);
    *S = pl.S;
    *m = pl.m;
    return 1;
}
