"""Pins of the oracle's FP64 parameter solve against what the paper and the
mathematics fix: printed kappa values and conversion tables (Sec. VI), closed
forms of the EOSs, the App. A profile ODE and the App. B surface tension."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import params as pp

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")))
R134A = dict(rho_v_phs=37.5, rho_l_phs=1187.0, nu_v_phs=0.339e-6, nu_l_phs=0.158e-6)
PR = dict(a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.327)


def _convert(N, tau_l, gamma=7.58e-3, L=10e-6, xi_cells=1.5):
    return pp.si_converter(**R134A, gamma_phs=gamma, L_phs=L, L_lat=N, tau_l=tau_l, rho_l_lat=1.187,
                           xi_lat=xi_cells)


@pytest.mark.parametrize("case", GOLDEN["kappa"]["cases"])
def test_kappa_matches_printed_values(case):
    """Sec. VI.B: kappa from Eq. surface_tension at Delta x = 0.1 um, xi = 1.5 Delta x."""
    c = _convert(100, case["tau_l"], gamma=case["gamma_mN_m"] * 1e-3)
    assert round(c["kappa"], case["digits"]) == pytest.approx(case["kappa"], abs=0.5 * 10 ** -case["digits"])


@pytest.mark.parametrize("table,tau_l", [("table_planar", 0.56), ("table_droplet", 0.62), ("table_plates", 0.56)])
def test_conversion_tables(table, tau_l):
    """Tables II-IV: Delta t, C_U, C_gamma (and C_VF) from Eqs. unit / unit2, Delta x = 10 um / N."""
    t = GOLDEN[table]
    Ns = t.get("N_x", t.get("N_y"))
    for k, N in enumerate(Ns):
        c = _convert(N, tau_l)
        dt = c["C_T"]
        if "dt_ps" in t:
            assert dt * 1e12 == pytest.approx(t["dt_ps"][k], rel=2e-3)
        else:
            assert dt * 1e9 == pytest.approx(t["dt_ns"][k], rel=3e-3)
        assert c["C_U"] == pytest.approx(t["C_U"][k], rel=1e-3)
        assert c["C_gamma"] == pytest.approx(t["C_gamma"][k], abs=0.006)
        if "C_VF_TN_m3" in t:
            assert c["C_VF"] / 1e12 == pytest.approx(t["C_VF_TN_m3"][k], rel=1e-3)


def test_kappa_is_resolution_independent_under_diffusive_scaling():
    """xi = 1.5 k Delta x_k and Delta t ~ Delta x^2: kappa stays 1.026 on every grid of Table II."""
    ks = [_convert(100 * k, 0.56, xi_cells=1.5 * k)["kappa"] for k in range(1, 6)]
    assert np.allclose(ks, ks[0], rtol=1e-12)
    assert round(ks[0], 3) == 1.026


def test_paper_eos_closed_forms():
    """Eq. EOS: p(rho_v) = p(rho_l) = P rho_v rho_l^2 and the Maxwell area vanishes (Sec. IV)."""
    rv, rl, P = 0.0375, 1.187, 0.0439932
    p0 = P * rv * rl ** 2
    assert pp.paper_pressure(rv, rv, rl, P) == pytest.approx(p0, rel=1e-13)
    assert pp.paper_pressure(rl, rv, rl, P) == pytest.approx(p0, rel=1e-13)
    area, _ = integrate.quad(lambda r: (pp.paper_pressure(r, rv, rl, P) - p0) / r ** 2, rv, rl, epsabs=1e-16,
                             epsrel=1e-13)
    assert abs(area) < 1e-13
    # the generic Maxwell solver recovers the densities the EOS was built around
    cv, cl, cp0 = pp.coexistence(lambda r: pp.paper_pressure(r, rv, rl, P), 3.0)
    assert cv == pytest.approx(rv, rel=1e-8) and cl == pytest.approx(rl, rel=1e-9)
    assert cp0 == pytest.approx(p0, rel=1e-9)


def test_pr_critical_point():
    """PR at T = Tc: dp/drho = d2p/drho2 = 0 at the critical density, pc = 0.0778 R Tc / b
    (to the rounding of the published constants 0.45724 and 0.0778)."""
    Tc = pp.pr_Tc(PR["a"], PR["b"])
    assert Tc == pytest.approx(0.0729220, abs=1e-7)
    p = lambda r: float(pp.pr_pressure(r, PR["a"], PR["b"], PR["R"], PR["omega"], Tc))
    rho = np.linspace(0.5, 4.0, 350001)
    vals = pp.pr_pressure(rho, PR["a"], PR["b"], PR["R"], PR["omega"], Tc)
    d1 = np.gradient(vals, rho)
    i = int(np.argmin(np.abs(d1)))
    rc = rho[i]
    h = 1e-3
    d2 = (p(rc + h) - 2 * p(rc) + p(rc - h)) / h ** 2
    assert abs(d1[i]) < 2e-5 and abs(d2) < 2e-4
    assert p(rc) == pytest.approx(pp.pr_pc(PR["a"], PR["b"]), rel=2e-4)


@pytest.mark.parametrize("t_ratio,rv_ref,rl_ref", [(0.7, 0.057929, 8.059209), (0.8, 0.201851, 7.182058),
                                                   (0.9, 0.587209, 5.889068)])
def test_pr_maxwell_equal_chemical_potential(t_ratio, rv_ref, rl_ref):
    """Maxwell construction = equal pressure and equal chemical potential (closed-form PR Helmholtz energy)."""
    T = t_ratio * pp.pr_Tc(PR["a"], PR["b"])
    rv, rl, p0 = pp.pr_maxwell(PR["a"], PR["b"], PR["R"], PR["omega"], T)
    mu = pp.pr_chemical_potential(np.array([rv, rl]), PR["a"], PR["b"], PR["R"], PR["omega"], T)
    assert abs(mu[0] - mu[1]) < 1e-12
    p = pp.pr_pressure(np.array([rv, rl]), PR["a"], PR["b"], PR["R"], PR["omega"], T)
    assert p == pytest.approx([p0, p0], rel=1e-12)
    assert rv == pytest.approx(rv_ref, abs=2e-6) and rl == pytest.approx(rl_ref, abs=2e-6)


def test_mechanical_stability_reduces_to_maxwell_in_diffusive_limit():
    """Sec. IV: with eps = 2 and psi ~ sqrt(rho) (p_scale -> 0) the condition is the Maxwell rule."""
    T = 0.8 * pp.pr_Tc(PR["a"], PR["b"])
    rv, rl, _ = pp.pr_maxwell(PR["a"], PR["b"], PR["R"], PR["omega"], T)
    prev = None
    for s in (1.0, 0.25, 0.0625, 1.0 / 256):
        ps = lambda r, s=s: s * pp.pr_pressure(r, PR["a"], PR["b"], PR["R"], PR["omega"], T)
        mv, ml, _ = pp.mechanical_stability(ps, -1.0, 2.0, rho_max=0.999 / PR["b"])
        gap = abs(mv - rv) / rv
        if prev is not None:
            assert gap < prev / 3.0     # second order in Delta x (s ~ Delta x^2)
        prev = gap
    assert prev < 1e-3


def test_gamma_closed_form_matches_quadrature():
    """App. B closed form vs numerical quadrature of the App. A profile (two independent routes)."""
    rv, rl = 0.0375, 1.187
    P = pp.P_from_thickness(1.5, rv, rl)
    p = lambda r: pp.paper_pressure(r, rv, rl, P)
    p0 = P * rv * rl ** 2
    for kappa in (0.5, 1.0, 2.0):
        g_closed = pp.gamma_analytic(kappa, P, rv, rl)
        g_quad = pp.diffusive_gamma(p, rv, rl, p0, kappa)
        assert g_closed == pytest.approx(g_quad, rel=1e-7)


def test_profile_solves_interface_ode_and_has_width_xi():
    """App. A: d sqrt(rho)/dx = -sqrt(6 P)(sqrt(rho) - sqrt(rho_v))(rho - rho_l); 33-67 % width = xi."""
    rv, rl, xi = 0.0375, 1.187, 3.0
    P = pp.P_from_thickness(xi, rv, rl)
    assert pp.thickness_from_P(P, rv, rl) == pytest.approx(xi, rel=1e-13)
    x = np.linspace(-6, 6, 1201)
    rho = pp.planar_profile(x, 0.0, P, rv, rl)
    s = np.sqrt(rho)
    z_num = np.gradient(s, x)
    z_ana = -math.sqrt(6 * P) * (s - math.sqrt(rv)) * (rho - rl)
    assert np.max(np.abs(z_num[5:-5] - z_ana[5:-5])) < 1e-4 * np.max(np.abs(z_ana))
    r1, r2 = pp.interface_densities(rv, rl)
    x1 = np.interp(r1, rho, x)
    x2 = np.interp(r2, rho, x)
    assert abs(x2 - x1) == pytest.approx(xi, rel=1e-4)


def test_layered_poiseuille():
    """One layer is the textbook parabola; two layers keep u and mu u' continuous."""
    y = np.linspace(-0.5, 15.5, 161)
    u = pp.layered_poiseuille(y, [(-0.5, 15.5, 2.0)], 1e-5)
    assert np.allclose(u, 1e-5 / (2 * 2.0) * (y + 0.5) * (15.5 - y), rtol=1e-12, atol=1e-18)
    layers = [(-0.5, 5.5, 3.0), (5.5, 15.5, 0.2)]
    yy = np.array([5.5 - 1e-9, 5.5 + 1e-9])
    uu = pp.layered_poiseuille(yy, layers, 1e-5)
    assert uu[0] == pytest.approx(uu[1], rel=1e-6)
    h = 1e-4
    dl = (pp.layered_poiseuille([5.5], layers[:1] + [(5.5, 15.5, 0.2)], 1e-5)[0]
          - pp.layered_poiseuille([5.5 - h], layers, 1e-5)[0]) / h
    dr = (pp.layered_poiseuille([5.5 + h], layers, 1e-5)[0] - pp.layered_poiseuille([5.5], layers, 1e-5)[0]) / h
    assert 3.0 * dl == pytest.approx(0.2 * dr, rel=1e-3)


def test_channel_flow_with_constant_viscosity_is_the_poiseuille_parabola():
    y = np.linspace(-0.5, 31.5, 65)
    u = pp.channel_flow(y, lambda s: 0.7, 3e-6, -0.5, 31.5)
    assert np.allclose(u, 3e-6 / (2 * 0.7) * (y + 0.5) * (31.5 - y), rtol=1e-10, atol=1e-15)


def test_channel_flow_tends_to_the_layered_solution_as_the_interface_sharpens():
    """mu(y) = tanh blend of 3.0 (below 10.5) and 0.2 (above) over a width W: the profile
    approaches the two-layer closed form, with an error that falls in proportion to W."""
    ys = np.linspace(-0.5, 31.5, 33)
    sharp = pp.layered_poiseuille(ys, [(-0.5, 10.5, 3.0), (10.5, 31.5, 0.2)], 1e-5)
    errs = []
    for W in (0.25, 0.125, 0.0625):
        mu = lambda s, W=W: 0.2 + 2.8 * 0.5 * (1 - math.tanh((s - 10.5) / W))
        u = pp.channel_flow(ys, mu, 1e-5, -0.5, 31.5, breaks=(10.5,))
        errs.append(np.max(np.abs(u - sharp)) / np.max(sharp))
    assert errs[2] < 0.015
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_tau_interpolation_hits_both_phases_and_clamps():
    t = pp.tau_of_rho(np.array([0.1, 4.0, 0.05, 9.0, 2.05]), 0.62, 0.56, 0.1, 4.0)
    assert np.allclose(t, [0.62, 0.56, 0.62, 0.56, 0.59])
