"""The paper's own benchmarks (Sec. VI) on the GPU through the C ABI, with the paper's EOS
(Eq. EOS) parametrised from SI units by the converter (Eqs. unit, unit2, thickness,
surface_tension) for R134a (Table I):
  - planar interface, grids 1-5 of Table II: the equilibrium profile converges to the
    analytic App. A profile at second order in the relative norms of Eq. relative_norms;
  - static droplet, Table III: maximum spurious velocity against the printed values and
    its decay with resolution (third order in lattice units, Sec. VI.B)."""
import math

import numpy as np
import pytest

from oracle import params as pp

pytestmark = pytest.mark.gpu

R134A = dict(rho_v_phs=37.5, rho_l_phs=1187.0, nu_v_phs=0.339e-6, nu_l_phs=0.158e-6)


def converter(k, tau_l, L=10e-6, gamma=7.58e-3):
    return pp.si_converter(**R134A, gamma_phs=gamma, L_phs=L, L_lat=100 * k, tau_l=tau_l, rho_l_lat=1.187,
                           xi_lat=1.5 * k)


def relative_norms(num, ana):
    e = num - ana
    return (np.abs(e).sum() / np.abs(ana).sum(), np.sqrt((e ** 2).sum()) / np.sqrt((ana ** 2).sum()),
            np.abs(e).max() / np.abs(ana).max())


def _planar(k, precision, tau=1.0, steps_per_k2=16000):
    import paper_2504_15018_gb300 as plb
    c = converter(k, 0.56)
    rv, rl, P = c["rho_v"], c["rho_l"], c["P"]
    nx = 100 * k
    x = np.arange(nx, dtype=float)
    ana = np.where(x < 50 * k, pp.planar_profile(x, 25 * k - 0.5, P, rv, rl),
                   pp.planar_profile(-x, -(75 * k - 0.5), P, rv, rl))
    opts = plb.make_opts(precision=precision, kappa=c["kappa"])
    if tau != 1.0:
        opts.tau_v, opts.tau_rho_v, opts.tau_rho_l = c["tau_v"], rv, rl
    lat = plb.Lattice(plb.PLB_D2Q9, (nx, 2, 1), plb.paper_eos(rv, rl, P), tau=tau, G=-1.0, eps=2.0, opts=opts)
    lat.init(np.tile(ana, 2))
    lat.step(steps_per_k2 * k * k)
    lat.status()
    rho = lat.moments()[0].reshape(2, nx).mean(axis=0)
    return relative_norms(rho, ana)


def test_planar_interface_converges_second_order():
    """Sec. VI.A: Nx = 100 k, xi = 1.5 k Delta x, k = 1..5 (Table II), FP64; the converged
    profile against App. A (Eq. analytical_interface).  tau = 1: the static equilibrium is
    reached faster than with the paper's tau_l = 0.56 (equilibration ~ L^2 / nu)."""
    norms = [_planar(k, 0) for k in range(1, 6)]
    for k, n in enumerate(norms, 1):
        print(f"fp64 grid {k}: L1 {n[0]:.3e} L2 {n[1]:.3e} Linf {n[2]:.3e}")
    for j in range(3):
        orders = [math.log(norms[k][j] / norms[k + 1][j]) / math.log((k + 2) / (k + 1)) for k in range(4)]
        print(f"  norm {j}: orders {[round(o, 2) for o in orders]}")
        assert min(orders) > 1.8, orders


def test_planar_interface_fp32_converges_second_order_on_grids_1_to_3():
    """FP32 storage on grids 1-3 (up to 144000 steps): the error norms fall at second order like
    FP64's and stay within 10 % of them.  The FP32 collision weights sum to exactly one, so the
    only mass change left is the rounding of the per-cell sums; in a steady planar state that
    rounding repeats every step (about 2e-9 of the mass per step here), which moves the
    interfaces slightly and is why FP32 is not closer to FP64 on grid 3."""
    n64, n32 = [], []
    for k in (1, 2, 3):
        n64.append(_planar(k, 0))
        n32.append(_planar(k, 1))
        print(f"grid {k}: L2 fp64 {n64[-1][1]:.4e} fp32 {n32[-1][1]:.4e}")
    for k in range(3):
        assert n32[k][1] < 1.1 * n64[k][1]
    orders = [math.log(n32[k][1] / n32[k + 1][1]) / math.log((k + 2) / (k + 1)) for k in range(2)]
    print(f"  fp32 L2 orders {[round(o, 2) for o in orders]}")
    assert min(orders) > 1.8, orders


def _droplet_umax(k, precision=0):
    import paper_2504_15018_gb300 as plb
    from paper_2504_15018_gb300 import inputs
    c = converter(k, 0.62)
    rv, rl, P = c["rho_v"], c["rho_l"], c["P"]
    n = 100 * k
    R = 25 * k                                   # D = 5 um in a 10 um box
    dims = (n, n, 1)
    x, y, _ = inputs.grid_coords(dims)
    r = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2)
    rho = pp.planar_profile(R - r, 0.0, P, rv, rl)    # App. A profile across the interface
    opts = plb.make_opts(precision=precision, kappa=c["kappa"], tau_v=c["tau_v"], tau_rho_v=rv, tau_rho_l=rl)
    lat = plb.Lattice(plb.PLB_D2Q9, dims, plb.paper_eos(rv, rl, P), tau=0.62, G=-1.0, eps=2.0, opts=opts)
    lat.init(rho)
    steps = 40000 * k * k
    lat.step(steps)
    lat.status()
    u1 = lat.reduce(plb.PLB_UMAX)[0]
    lat.step(steps // 4)
    u2 = lat.reduce(plb.PLB_UMAX)[0]
    return u2, abs(u2 - u1) / u2, c


def test_spurious_currents_table3():
    """Sec. VI.B, Table III (D = 5 um, tau_l = 0.62): the paper prints a maximum spurious
    velocity of 2.6e-3 lattice units on grid 1 and 2.2e-5 on grid 5, decaying at third order in
    lattice units.  The paper does not state gamma for this test; R134a's 7.58 mN/m is used,
    so the printed value is an approximate pin (factor 3)."""
    u1, drift1, c1 = _droplet_umax(1)
    u2, drift2, c2 = _droplet_umax(2)
    print(f"grid 1: umax {u1:.3e} (kappa {c1['kappa']:.3f}, still changing {drift1:.1%}); "
          f"grid 2: umax {u2:.3e} (kappa {c2['kappa']:.3f}); lattice-unit order {math.log2(u1 / u2):.2f}")
    assert 2.6e-3 / 3 < u1 < 2.6e-3 * 3
    assert math.log2(u1 / u2) > 2.3
