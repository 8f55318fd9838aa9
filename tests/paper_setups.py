"""Set-ups of the paper's Sec. VI benchmarks in lattice units, shared by the oracle tests and the
GPU tests: R134a at 30 C (Table I), the unit converter (Eqs. unit, unit2, thickness,
surface_tension), the App. A planar profile and the diffuse-interface channel flow."""
from __future__ import annotations

import numpy as np

from oracle import params as pp

R134A = dict(rho_v_phs=37.5, rho_l_phs=1187.0, nu_v_phs=0.339e-6, nu_l_phs=0.158e-6)
GAMMA_R134A = 7.58e-3


def converter(n_lat, tau_l, L=10e-6, xi_cells=None, gamma=GAMMA_R134A):
    """Conversion for a length L resolved by n_lat cells; xi = 1.5 dx at 100 cells per 10 um
    (Tables II and IV: xi = 1.5 k dx on grid k)."""
    if xi_cells is None:
        xi_cells = 1.5 * n_lat / 100.0
    return pp.si_converter(**R134A, gamma_phs=gamma, L_phs=L, L_lat=n_lat, tau_l=tau_l, rho_l_lat=1.187,
                           xi_lat=xi_cells)


def relative_norms(num, ana):
    """Eq. relative_norms: L1, L2 and L_inf of num - ana relative to ana."""
    e = num - ana
    return (np.abs(e).sum() / np.abs(ana).sum(), np.sqrt((e ** 2).sum()) / np.sqrt((ana ** 2).sum()),
            np.abs(e).max() / np.abs(ana).max())


def plates(ny, tau_l=0.56, F_si=1e6):
    """Sec. VI.D: liquid in the lower half, vapour in the upper half, no-slip walls at y = -1/2 and
    ny - 1/2, body force F_si along x.  Returns the lattice parameters, the App. A density profile
    across the interface at y = ny/2 - 1/2 (liquid below) and the steady diffuse-interface
    velocity, mu(y) = rho(y) (tau(rho(y)) - 1/2) / 3 with tau interpolated as in Sec. VI."""
    c = converter(ny, tau_l)
    rv, rl, P = c["rho_v"], c["rho_l"], c["P"]
    yc = ny / 2 - 0.5
    y = np.arange(ny, dtype=float)
    prof = lambda yy: pp.planar_profile(-np.asarray(yy, dtype=float), -yc, P, rv, rl)

    def mu(s):
        r = prof(s)[0]
        return r * (pp.tau_of_rho(r, c["tau_v"], tau_l, rv, rl) - 0.5) / 3.0

    F = F_si / c["C_VF"]
    u = pp.channel_flow(y, mu, F, -0.5, ny - 0.5, breaks=(yc,))
    return dict(c, F=F, tau_l=tau_l, rho=prof(y), u=u, nu_l=(tau_l - 0.5) / 3.0)


def planar(nx, tau_l=0.56):
    """Sec. VI.A: vapour outside, liquid in the middle half of a periodic row of nx cells,
    interfaces at nx/4 - 1/2 and 3 nx/4 - 1/2 with the App. A profile."""
    c = converter(nx, tau_l)
    rv, rl, P = c["rho_v"], c["rho_l"], c["P"]
    x = np.arange(nx, dtype=float)
    rho = np.where(x < nx / 2, pp.planar_profile(x, nx / 4 - 0.5, P, rv, rl),
                   pp.planar_profile(-x, -(3 * nx / 4 - 0.5), P, rv, rl))
    return dict(c, rho=rho)


def galilean_steps(k, t1=7.91e-6, t2=31.6e-6):
    """Sec. VI.C on grid k (Table II): steps at rest, then steps after the velocity jump."""
    c = converter(100 * k, 0.56)
    n1, n2 = round(t1 / c["C_T"]), round(t2 / c["C_T"])
    return n1, n2 - n1, 0.1 / c["C_U"]


def equilibrium(c, w, rho, u):
    """Eq. Single_Phase_EDF for every cell, (Q, N): c (Q, d), w (Q,), rho (N,), u (d, N)."""
    cu = c @ u
    usq = (u ** 2).sum(0)
    return w[:, None] * rho[None, :] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * usq[None, :])


def balanced_init_oracle(P, lattice, rho, u0=None):
    """Start at rest (or at u0) in the sense of Eq. Momentum: f^eq(rho, u0 - F / (2 rho)), so the
    physical velocity (sum f c + F/2) / rho is u0 from the first step (the library's
    plb_init_physical).  F is read back through the oracle's own moments of f^eq(rho, u0)."""
    import oracle
    f = oracle.init(P, rho, u0)
    _, u, _ = oracle.moments(P, f)
    base = np.zeros_like(u) if u0 is None else np.asarray(u0, dtype=float)
    c, w = oracle.velocity_set(lattice)
    return np.ascontiguousarray(equilibrium(c[:, :u.shape[0]].astype(float), w, rho, 2 * base - u).T)
