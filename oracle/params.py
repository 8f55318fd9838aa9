"""FP64 parameter solve of the P-LBM (arXiv 2504.15018, Secs. IV-V, Apps. A-B).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy / scipy,
written from the paper's formulas; shares nothing with the library's C++
parameter solve, which it checks.

Contents:
  - Eq. EOS (the paper's equation of state) and the Peng-Robinson EOS
    (Peng & Robinson 1976, lattice units, the second EOS kind);
  - the Maxwell equal-area construction (the mechanical stability condition
    of Sec. IV with eps = 2 and psi -> sqrt(rho), i.e. int (p - p0)/rho^2 = 0);
  - the finite-psi mechanical-stability densities of Sec. IV for any eps;
  - Eq. thickness (p_c / rho_c^3 from the interface width xi, f_xi of Sec. IV),
    Eq. surface_tension (kappa from gamma, f_gamma of App. B with rho_1 = rho_v,
    rho_2 = rho_l);
  - the SI unit converter, Eqs. unit and unit2 (Sec. V);
  - the analytic planar profile of App. A and the analytic gamma of App. B;
  - the sharp-interface layered Poiseuille profile used for the plates test
  - the diffuse-interface channel flow (viscosity varying with the App. A density profile)
    and the linear relaxation-time interpolation of Sec. VI
    (the paper does not print its analytic solution; this is the textbook one).
"""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import integrate, optimize

# ------------------------------------------------------------------ EOS


def pr_Tc(a: float, b: float, R: float = 1.0) -> float:
    """Critical temperature of the Peng-Robinson EOS: a = 0.45724 R^2 Tc^2/pc, b = 0.0778 R Tc/pc."""
    return 0.0778 * a / (0.45724 * b * R)


def pr_alpha(T: float, Tc: float, omega: float) -> float:
    m = 0.37464 + 1.54226 * omega - 0.26992 * omega ** 2
    return (1.0 + m * (1.0 - math.sqrt(T / Tc))) ** 2


def pr_pressure(rho, a: float, b: float, R: float, omega: float, T: float):
    rho = np.asarray(rho, dtype=np.float64)
    al = pr_alpha(T, pr_Tc(a, b, R), omega)
    return rho * R * T / (1.0 - b * rho) - a * al * rho ** 2 / (1.0 + 2.0 * b * rho - (b * rho) ** 2)


def pr_pc(a: float, b: float, R: float = 1.0) -> float:
    """Critical pressure pc = 0.0778 R Tc / b."""
    return 0.0778 * R * pr_Tc(a, b, R) / b


def pr_chemical_potential(rho, a: float, b: float, R: float, omega: float, T: float):
    """Chemical potential of the PR fluid up to a T-only constant, from its Helmholtz energy:
    mu = df/drho with f = rho R T ln(rho/(1 - b rho)) + a alpha rho /(2 sqrt2 b) ln((1+(1-sqrt2) b rho)/(1+(1+sqrt2) b rho)).
    Closed form; independent of the numerical Maxwell construction."""
    rho = np.asarray(rho, dtype=np.float64)
    al = pr_alpha(T, pr_Tc(a, b, R), omega)
    s2 = math.sqrt(2.0)
    br = b * rho
    f_over_rho = R * T * np.log(rho / (1.0 - br)) + a * al / (2.0 * s2 * b) * np.log(
        (1.0 + (1.0 - s2) * br) / (1.0 + (1.0 + s2) * br))
    p = pr_pressure(rho, a, b, R, omega, T)
    # mu = (f + p) / rho  with f = rho * f_over_rho  ->  mu = f_over_rho + p / rho
    return f_over_rho + p / rho


def paper_pressure(rho, rho_v: float, rho_l: float, P: float):
    """Eq. EOS with P = p_c / rho_c^3."""
    rho = np.asarray(rho, dtype=np.float64)
    sv = math.sqrt(rho_v)
    return P * (2.0 * rho ** 3 + (rho_v - 2.0 * rho_l) * rho ** 2 - 3.0 * sv * rho ** 2.5
                + 2.0 * sv * rho_l * rho ** 1.5 + sv * rho_l ** 2 * rho ** 0.5)


# ----------------------------------------------------- coexistence densities


def _spinodals(p, rho_max: float):
    """Local maximum (rho_s1) and minimum (rho_s2) of p(rho) on (0, rho_max)."""
    grid = np.linspace(rho_max * 1e-4, rho_max, 20001)
    vals = p(grid)
    dv = np.diff(vals)
    i1 = int(np.argmax(dv < 0))                 # first descending step: near the local max
    i2 = i1 + int(np.argmax(dv[i1:] > 0))       # next ascending step: near the local min
    s1 = optimize.minimize_scalar(lambda r: -p(r), bounds=(grid[max(i1 - 2, 0)], grid[i1 + 2]),
                                  method="bounded", options={"xatol": 1e-14}).x
    s2 = optimize.minimize_scalar(p, bounds=(grid[max(i2 - 2, 0)], grid[min(i2 + 2, len(grid) - 1)]),
                                  method="bounded", options={"xatol": 1e-14}).x
    return float(s1), float(s2)


def coexistence(p, rho_max: float, weight=None):
    """Densities (rho_v, rho_l) and p0 with p(rho_v) = p(rho_l) = p0 and
    int_{rho_v}^{rho_l} (p - p0) weight(rho) drho = 0.

    weight(rho) = 1/rho^2 is the Maxwell equal-area rule (Sec. IV with eps = 2 in the
    diffusive limit psi ~ sqrt(rho)); other weights give the finite-psi
    mechanical-stability condition."""
    if weight is None:
        weight = lambda r: 1.0 / r ** 2
    s1, s2 = _spinodals(p, rho_max)
    p_hi = float(p(s1))
    p_lo = max(float(p(s2)), 1e-9 * p_hi)

    def roots(p0):
        rv = optimize.brentq(lambda r: p(r) - p0, 1e-300, s1, xtol=1e-300, rtol=1e-15)
        rl = optimize.brentq(lambda r: p(r) - p0, s2, rho_max, xtol=1e-15, rtol=1e-15)
        return rv, rl

    def area(p0):
        rv, rl = roots(p0)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val, _ = integrate.quad(lambda r: (p(r) - p0) * weight(r), rv, rl, epsabs=1e-15, epsrel=1e-13,
                                    limit=400, points=[s1, s2])
        return val

    # area(p0) decreases with p0: walk the lower end down until the bracket holds
    hi = p_hi - 1e-12 * (p_hi - p_lo)
    lo = 0.5 * (p_lo + p_hi)
    while area(lo) < 0.0:
        if lo <= p_lo * 1.000001:
            raise ValueError("no coexistence pressure in the spinodal range")
        lo = max(p_lo, p_lo + 0.1 * (lo - p_lo)) if lo - p_lo > 1e-12 * p_hi else p_lo * 1.000001
    p0 = optimize.brentq(area, lo, hi, xtol=1e-16, rtol=1e-15)
    rv, rl = roots(p0)
    return rv, rl, p0


def pr_maxwell(a: float, b: float, R: float, omega: float, T: float):
    p = lambda r: pr_pressure(r, a, b, R, omega, T)
    return coexistence(p, 0.999 / b)


def mechanical_stability(p_scaled, G: float = -1.0, eps: float = 2.0, rho_max: float = 10.0, h: float = 1e-7):
    """Coexistence densities of the finite-psi condition of Sec. IV:
    int (p - p0) psi'(rho) / psi^(1+eps) drho = 0 with psi = sqrt(2 (p - rho/3)/G)."""
    psi = lambda r: math.sqrt(2.0 * (p_scaled(r) - r / 3.0) / G)
    dpsi = lambda r: (psi(r + h * r) - psi(r - h * r)) / (2.0 * h * r)
    weight = lambda r: dpsi(r) / psi(r) ** (1.0 + eps)
    return coexistence(p_scaled, rho_max, weight)


# ------------------------------------------------------- Sec. IV parameters


def f_xi(rho, rho_v: float, rho_l: float):
    """f_xi of Sec. IV / App. A."""
    sr, sv, sl = np.sqrt(rho), math.sqrt(rho_v), math.sqrt(rho_l)
    return (np.log(sr - sv) / (rho_l - rho_v)
            - np.log(sl - sr) / (2.0 * sl * (sl - sv))
            - np.log(sr + sl) / (2.0 * sl * (sv + sl)))


def f_gamma(rho, rho_v: float, rho_l: float):
    """f_gamma of App. B (rho_1 = rho_v, rho_2 = rho_l)."""
    return rho ** 2 / 4.0 - rho_l / 2.0 * rho - math.sqrt(rho_v) / 3.0 * rho ** 1.5 + math.sqrt(rho_v) * rho_l * rho ** 0.5


def interface_densities(rho_v: float, rho_l: float):
    return rho_v + 0.33 * (rho_l - rho_v), rho_v + 0.67 * (rho_l - rho_v)


def P_from_thickness(xi: float, rho_v: float, rho_l: float, r: float = 1.0) -> float:
    """Eq. thickness: p_c/rho_c^3 = (f_xi(rho_I1) - f_xi(rho_I2))^2 / (6 r xi^2)."""
    r1, r2 = interface_densities(rho_v, rho_l)
    return (f_xi(r1, rho_v, rho_l) - f_xi(r2, rho_v, rho_l)) ** 2 / (6.0 * r * xi ** 2)


def thickness_from_P(P: float, rho_v: float, rho_l: float, r: float = 1.0) -> float:
    """App. A: xi = sqrt(rho_c^3/(6 r p_c)) |f_xi(rho_I1) - f_xi(rho_I2)| (absolute value taken)."""
    r1, r2 = interface_densities(rho_v, rho_l)
    return math.sqrt(1.0 / (6.0 * r * P)) * abs(f_xi(r1, rho_v, rho_l) - f_xi(r2, rho_v, rho_l))


def kappa_from_gamma(gamma: float, P: float, rho_v: float, rho_l: float, r: float = 1.0) -> float:
    """Eq. surface_tension: kappa = sqrt(27/(2 r P)) gamma / (f_gamma(rho_v) - f_gamma(rho_l))."""
    return math.sqrt(27.0 / (2.0 * r * P)) * gamma / (f_gamma(rho_v, rho_v, rho_l) - f_gamma(rho_l, rho_v, rho_l))


def gamma_analytic(kappa: float, P: float, rho_v: float, rho_l: float, r: float = 1.0) -> float:
    """App. B: gamma = sqrt(2 r P / 27) kappa (f_gamma(rho_v) - f_gamma(rho_l))."""
    return math.sqrt(2.0 * r * P / 27.0) * kappa * (f_gamma(rho_v, rho_v, rho_l) - f_gamma(rho_l, rho_v, rho_l))


def planar_profile(x, x0: float, P: float, rho_v: float, rho_l: float, r: float = 1.0):
    """App. A, Eq. analytical_interface: sqrt(6 r P) x + C0 = f_xi(rho), solved for rho.

    f_xi rises from -inf at rho_v to +inf at rho_l, so rho increases with x; the
    constant C0 is fixed so that rho(x0) = (rho_v + rho_l)/2."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    k = math.sqrt(6.0 * r * P)
    rm = 0.5 * (rho_v + rho_l)
    C0 = f_xi(rm, rho_v, rho_l) - k * x0
    out = np.empty_like(x)
    lo, hi = rho_v * (1 + 1e-15) + 1e-300, rho_l * (1 - 1e-15)
    for j, xx in enumerate(x):
        target = k * xx + C0
        g = lambda rr: f_xi(rr, rho_v, rho_l) - target
        a, b = lo, hi
        if g(a) > 0:
            out[j] = rho_v
            continue
        if g(b) < 0:
            out[j] = rho_l
            continue
        out[j] = optimize.brentq(g, a, b, xtol=1e-15, rtol=1e-15)
    return out


def diffusive_gamma(p, rho_v: float, rho_l: float, p0: float, kappa: float = 1.0, r: float = 1.0):
    """App. A/B applied to any EOS in the diffusive limit (eps = 2):
    z^2 = 6 r rho int_{rho_v}^{rho} (p - p0)/rho'^2 drho'  (from Eq. EDO with p_xx = p0),
    gamma = kappa/(9 r) int z d sqrt(rho)."""
    def z(rr):
        val, _ = integrate.quad(lambda s: (p(s) - p0) / s ** 2, rho_v, rr, epsabs=1e-15, epsrel=1e-12, limit=200)
        return math.sqrt(max(6.0 * r * rr * val, 0.0))
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        val, _ = integrate.quad(lambda s: z(s * s), math.sqrt(rho_v), math.sqrt(rho_l), epsabs=1e-14,
                                epsrel=1e-10, limit=200)
    return kappa / (9.0 * r) * val


# ------------------------------------------------------------ unit converter


def si_converter(*, rho_v_phs: float, rho_l_phs: float, nu_v_phs: float, nu_l_phs: float, gamma_phs: float,
                 L_phs: float, L_lat: float, tau_l: float, rho_l_lat: float, xi_lat: float):
    """Eqs. unit and unit2 of Sec. V plus the Sec. IV parameter formulas (r = 1)."""
    nu_l_lat = (tau_l - 0.5) / 3.0
    C_L = L_phs / L_lat
    C_T = C_L ** 2 * nu_l_lat / nu_l_phs
    C_M = C_L ** 3 * rho_l_phs / rho_l_lat
    C_U = C_L / C_T
    C_VF = C_M / (C_L ** 2 * C_T ** 2)
    C_gamma = C_M / C_T ** 2
    C_rho = C_M / C_L ** 3
    rho_v_lat = rho_v_phs / C_rho
    nu_v_lat = nu_v_phs * C_T / C_L ** 2
    tau_v = 3.0 * nu_v_lat + 0.5
    gamma_lat = gamma_phs / C_gamma
    P = P_from_thickness(xi_lat, rho_v_lat, rho_l_lat)
    kappa = kappa_from_gamma(gamma_lat, P, rho_v_lat, rho_l_lat)
    return dict(C_L=C_L, C_T=C_T, C_M=C_M, C_U=C_U, C_VF=C_VF, C_gamma=C_gamma, rho_v=rho_v_lat,
                rho_l=rho_l_lat, tau_l=tau_l, tau_v=tau_v, gamma_lat=gamma_lat, P=P, kappa=kappa)


# --------------------------------------------------------- layered Poiseuille


def layered_poiseuille(y, layers, F: float):
    """Steady u_x(y) for body force F between no-slip walls at y = y_walls[0], y_walls[1].

    layers: list of (y_lo, y_hi, mu) covering [y_wall_lo, y_wall_hi] in order.
    In each layer mu u'' = -F; u = 0 at both walls; u and mu u' continuous at
    interfaces.  Solved as one linear system for (A_k, B_k) in u = -F y^2/(2 mu_k) + A_k y + B_k."""
    n = len(layers)
    Amat = np.zeros((2 * n, 2 * n))
    rhs = np.zeros(2 * n)
    row = 0
    y0, _, mu0 = layers[0]
    Amat[row, 0], Amat[row, 1] = y0, 1.0
    rhs[row] = F * y0 ** 2 / (2 * mu0)
    row += 1
    for k in range(n - 1):
        yi = layers[k][1]
        mk, mk1 = layers[k][2], layers[k + 1][2]
        # continuity of u
        Amat[row, 2 * k], Amat[row, 2 * k + 1] = yi, 1.0
        Amat[row, 2 * k + 2], Amat[row, 2 * k + 3] = -yi, -1.0
        rhs[row] = F * yi ** 2 / (2 * mk) - F * yi ** 2 / (2 * mk1)
        row += 1
        # continuity of mu u'
        Amat[row, 2 * k] = mk
        Amat[row, 2 * k + 2] = -mk1
        rhs[row] = 0.0  # mu(-F y/mu) cancels on both sides
        row += 1
    yn, mun = layers[-1][1], layers[-1][2]
    Amat[row, 2 * n - 2], Amat[row, 2 * n - 1] = yn, 1.0
    rhs[row] = F * yn ** 2 / (2 * mun)
    coef = np.linalg.solve(Amat, rhs)
    y = np.asarray(y, dtype=np.float64)
    u = np.zeros_like(y)
    for k, (lo, hi, mu) in enumerate(layers):
        m = (y >= lo) & (y <= hi)
        u[m] = -F * y[m] ** 2 / (2 * mu) + coef[2 * k] * y[m] + coef[2 * k + 1]
    return u


# --------------------------------------------------------- diffuse-interface channel flow


def tau_of_rho(rho, tau_v: float, tau_l: float, rho_v: float, rho_l: float):
    """Sec. VI: tau = tau_v + (rho - rho_v) / (rho_l - rho_v) (tau_l - tau_v), the weight clamped to
    [0, 1] outside [rho_v, rho_l]."""
    wgt = np.clip((np.asarray(rho, dtype=np.float64) - rho_v) / (rho_l - rho_v), 0.0, 1.0)
    return tau_v + wgt * (tau_l - tau_v)


def channel_flow(y, mu, F: float, y_lo: float, y_hi: float, breaks=()):
    """Steady u_x(y) of a body-force-driven flow between no-slip walls at y_lo and y_hi when the
    dynamic viscosity varies across the channel (mu: callable of y).

    The x-momentum balance d/dy (mu du/dy) = -F integrates to mu u' = -F (y - y_s), with y_s the
    height of zero shear; u(y_lo) = 0 gives u(y) = -F int_{y_lo}^{y} (s - y_s) / mu(s) ds and
    u(y_hi) = 0 fixes y_s = int s / mu / int 1 / mu over the channel.  For a piecewise constant
    mu this is the layered Poiseuille solution; for constant mu, the Poiseuille parabola.
    breaks: heights where mu changes fast (the interfaces), passed to the quadrature."""
    pts = sorted(b for b in breaks if y_lo < b < y_hi)

    def q(fn, a, b):
        inner = [p for p in pts if a < p < b]
        val, _ = integrate.quad(fn, a, b, points=inner or None, epsabs=0.0, epsrel=1e-12, limit=400)
        return val

    inv = q(lambda s: 1.0 / mu(s), y_lo, y_hi)
    ys = q(lambda s: s / mu(s), y_lo, y_hi) / inv
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    order = np.argsort(y)
    out = np.empty_like(y)
    acc, prev = 0.0, y_lo
    for j in order:
        acc += q(lambda s: (s - ys) / mu(s), prev, y[j])
        prev = y[j]
        out[j] = -F * acc
    return out
