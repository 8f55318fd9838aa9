// Host FP64 parameter solve of the P-LBM (arXiv 2504.15018, Secs. IV-V).
//
//  - EOS: Peng-Robinson in lattice units and the paper's Eq. EOS.
//  - Coexistence by the equal-area rule (the mechanical-stability condition of Sec. IV at
//    eps = 2 in the diffusive limit): int_{rho_v}^{rho_l} (p - p0) / rho^2 drho = 0,
//    p(rho_v) = p(rho_l) = p0.  Spinodals by a log-spaced scan + bisection on p',
//    roots by bisection, the area by composite 8-point Gauss-Legendre quadrature,
//    p0 by bisection (the area decreases monotonically in p0).
//  - Multiphase SI unit converter (Sec. V, Eqs. unit, unit2) and Eqs. thickness,
//    surface_tension (Sec. IV, r = 1; f_gamma with rho_1 = rho_v, rho_2 = rho_l).
#include <cmath>
#include <cstring>

#include "plb.h"
#include "plb_host.h"

namespace plb {

PrConstants pr_constants(const plb_eos_params &e) {
    PrConstants c;
    c.Tc = 0.0778 * e.a / (0.45724 * e.b * e.R);
    const double m = 0.37464 + 1.54226 * e.omega - 0.26992 * e.omega * e.omega;
    const double g = 1.0 + m * (1.0 - std::sqrt(e.T_over_Tc));
    c.alpha = g * g;
    c.RT = e.R * e.T_over_Tc * c.Tc;
    c.aalpha = e.a * c.alpha;
    return c;
}

// p_EOS(rho) without p_scale.
double eos_pressure_host(const plb_eos_params &e, double rho) {
    if (e.kind == PLB_EOS_PR) {
        const PrConstants c = pr_constants(e);
        const double br = e.b * rho;
        return rho * c.RT / (1.0 - br) - c.aalpha * rho * rho / (1.0 + 2.0 * br - br * br);
    }
    const double sr = std::sqrt(rho), sv = std::sqrt(e.rho_v), rv = e.rho_v, rl = e.rho_l;
    const double r2 = rho * rho;
    return e.pc_over_rhoc3 * (2.0 * r2 * rho + (rv - 2.0 * rl) * r2 - 3.0 * sv * r2 * sr + 2.0 * sv * rl * rho * sr +
                              sv * rl * rl * sr);
}

namespace {

double rho_upper(const plb_eos_params &e) {
    return e.kind == PLB_EOS_PR ? 0.999999 / e.b : 4.0 * e.rho_l;
}

double dpdrho(const plb_eos_params &e, double r) {
    const double h = 1e-6 * r;
    return (eos_pressure_host(e, r + h) - eos_pressure_host(e, r - h)) / (2.0 * h);
}

// root of g on [lo, hi] by bisection, g(lo) and g(hi) of opposite sign
template <class Fn> double bisect(Fn g, double lo, double hi, int iters = 200) {
    double glo = g(lo);
    for (int k = 0; k < iters; ++k) {
        const double mid = 0.5 * (lo + hi);
        const double gm = g(mid);
        if ((gm < 0.0) == (glo < 0.0)) {
            lo = mid;
            glo = gm;
        } else {
            hi = mid;
        }
        if (hi - lo <= 1e-16 * std::fabs(hi)) break;
    }
    return 0.5 * (lo + hi);
}

bool spinodals(const plb_eos_params &e, double &s1, double &s2) {
    const double top = rho_upper(e);
    const int n = 4000;
    double prev_r = top * 1e-6, prev_d = dpdrho(e, prev_r);
    bool have1 = false;
    for (int k = 1; k <= n; ++k) {
        const double r = top * std::pow(10.0, -6.0 + 6.0 * k / n) * (1.0 - 1e-9);
        const double d = dpdrho(e, r);
        if (!have1 && prev_d > 0.0 && d <= 0.0) {
            s1 = bisect([&](double x) { return dpdrho(e, x); }, prev_r, r);
            have1 = true;
        } else if (have1 && prev_d < 0.0 && d >= 0.0) {
            s2 = bisect([&](double x) { return dpdrho(e, x); }, prev_r, r);
            return true;
        }
        prev_r = r;
        prev_d = d;
    }
    return false;
}

// int_a^b g(r) dr with 8-point Gauss-Legendre on m panels
template <class Fn> double gauss_legendre(Fn g, double a, double b, int m) {
    static const double x8[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double w8[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    const double h = (b - a) / m;
    double sum = 0.0;
    for (int k = 0; k < m; ++k) {
        const double c = a + (k + 0.5) * h, r = 0.5 * h;
        for (int j = 0; j < 4; ++j) sum += w8[j] * r * (g(c - r * x8[j]) + g(c + r * x8[j]));
    }
    return sum;
}

}  // namespace

int solve_coexistence(const plb_eos_params &e, double &rho_v, double &rho_l, double &p0) {
    if (e.kind == PLB_EOS_PAPER) {
        rho_v = e.rho_v;
        rho_l = e.rho_l;
        p0 = e.pc_over_rhoc3 * e.rho_v * e.rho_l * e.rho_l;
        return PLB_OK;
    }
    double s1 = 0, s2 = 0;
    if (!spinodals(e, s1, s2)) return PLB_EINVAL;   // supercritical: no coexistence
    const double top = rho_upper(e);
    const double p_hi = eos_pressure_host(e, s1);
    const double p_lo = std::fmax(eos_pressure_host(e, s2), 0.0);
    auto roots = [&](double pp, double &rv, double &rl) {
        rv = bisect([&](double r) { return eos_pressure_host(e, r) - pp; }, 0.0, s1);
        rl = bisect([&](double r) { return eos_pressure_host(e, r) - pp; }, s2, top);
    };
    auto area = [&](double pp) {
        double rv, rl;
        roots(pp, rv, rl);
        auto g = [&](double r) { return (eos_pressure_host(e, r) - pp) / (r * r); };
        // panels split at the spinodals; the vapour branch is graded geometrically
        double sum = 0.0;
        double a = rv;
        for (int k = 0; k < 24; ++k) {
            const double b = rv * std::pow(s1 / rv, (k + 1) / 24.0);
            sum += gauss_legendre(g, a, b, 8);
            a = b;
        }
        sum += gauss_legendre(g, s1, s2, 256);
        sum += gauss_legendre(g, s2, rl, 256);
        return sum;
    };
    double lo = p_lo + 1e-12 * (p_hi - p_lo), hi = p_hi - 1e-12 * (p_hi - p_lo);
    // area(lo) > 0 > area(hi); shrink lo toward p_lo until the bracket holds
    double lo_try = 0.5 * (lo + hi);
    while (area(lo_try) < 0.0 && lo_try - lo > 1e-14 * p_hi) lo_try = lo + 0.1 * (lo_try - lo);
    if (area(lo_try) < 0.0) return PLB_EINVAL;
    p0 = bisect(area, lo_try, hi, 200);
    roots(p0, rho_v, rho_l);
    return PLB_OK;
}

namespace {
double f_xi(double rho, double rv, double rl) {
    const double sr = std::sqrt(rho), sv = std::sqrt(rv), sl = std::sqrt(rl);
    return std::log(sr - sv) / (rl - rv) - std::log(sl - sr) / (2.0 * sl * (sl - sv)) -
           std::log(sr + sl) / (2.0 * sl * (sv + sl));
}
double f_gamma(double rho, double rv, double rl) {
    return rho * rho / 4.0 - rl / 2.0 * rho - std::sqrt(rv) / 3.0 * rho * std::sqrt(rho) + std::sqrt(rv) * rl * std::sqrt(rho);
}
}  // namespace

int si_convert(const double si[6], const double lat[3], double xi, double out[11]) {
    const double rho_v = si[0], rho_l = si[1], nu_v = si[2], nu_l = si[3], gamma = si[4], L = si[5];
    const double L_lat = lat[0], tau_l = lat[1], rho_l_lat = lat[2];
    if (!(rho_v > 0 && rho_l > rho_v && nu_v > 0 && nu_l > 0 && gamma >= 0 && L > 0 && L_lat > 0 && tau_l > 0.5 &&
          rho_l_lat > 0 && xi > 0))
        return PLB_EINVAL;
    const double nu_l_lat = (tau_l - 0.5) / 3.0;
    const double C_L = L / L_lat;                              // Eq. unit
    const double C_T = C_L * C_L * nu_l_lat / nu_l;
    const double C_M = C_L * C_L * C_L * rho_l / rho_l_lat;
    const double C_U = C_L / C_T;                              // Eq. unit2
    const double C_VF = C_M / (C_L * C_L * C_T * C_T);
    const double C_g = C_M / (C_T * C_T);
    const double rv = rho_v / (C_M / (C_L * C_L * C_L));
    const double rl = rho_l_lat;
    const double tau_v = 3.0 * nu_v * C_T / (C_L * C_L) + 0.5;
    const double g_lat = gamma / C_g;
    const double r1 = rv + 0.33 * (rl - rv), r2 = rv + 0.67 * (rl - rv);
    const double df = f_xi(r1, rv, rl) - f_xi(r2, rv, rl);
    const double P = df * df / (6.0 * xi * xi);                // Eq. thickness
    const double kappa = std::sqrt(27.0 / (2.0 * P)) * g_lat / (f_gamma(rv, rv, rl) - f_gamma(rl, rv, rl));  // Eq. surface_tension
    const double vals[11] = {C_L, C_T, C_M, C_U, C_VF, C_g, rv, tau_v, g_lat, P, kappa};
    std::memcpy(out, vals, sizeof(vals));
    return PLB_OK;
}

}  // namespace plb
