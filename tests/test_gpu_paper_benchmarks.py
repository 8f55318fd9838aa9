"""The paper's own benchmarks (Sec. VI) on the GPU through the C ABI, with the paper's EOS
(Eq. EOS) parametrised from SI units by the converter (Eqs. unit, unit2, thickness,
surface_tension) for R134a (Table I):
  - planar interface, grids 1-5 of Table II: the equilibrium profile converges to the
    analytic App. A profile at second order in the relative norms of Eq. relative_norms;
  - static droplet, Table III: maximum spurious velocity against the printed values and
    its decay with resolution (third order in lattice units, Sec. VI.B);
  - Galilean invariance, Sec. VI.C: the planar interface set in uniform motion; the velocity
    error against the uniform field converges at second order;
  - two-phase flow between parallel plates, Sec. VI.D (Table IV grids): the velocity profile
    converges at second order to the diffuse-interface channel flow."""
import math

import numpy as np
import pytest

from oracle import params as pp

pytestmark = pytest.mark.gpu

from paper_setups import converter as _conv, relative_norms, plates, galilean_steps, equilibrium


def converter(k, tau_l):
    return _conv(100 * k, tau_l)


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


def _galilean(k, precision=0):
    import paper_2504_15018_gb300 as plb
    from paper_setups import planar
    s = planar(100 * k)
    n1, n2, U = galilean_steps(k)
    nx = 100 * k
    opts = plb.make_opts(precision=precision, kappa=s["kappa"], tau_v=s["tau_v"], tau_rho_v=s["rho_v"],
                         tau_rho_l=s["rho_l"])
    lat = plb.Lattice(plb.PLB_D2Q9, (nx, 2, 1), plb.paper_eos(s["rho_v"], s["rho_l"], s["P"]), tau=0.56, G=-1.0,
                      eps=2.0, opts=opts)
    lat.init(np.tile(s["rho"], 2), physical=True)
    lat.step(n1)
    # the velocity jump: every cell's equilibrium part moves by U, the rest is kept (the effect
    # of a one-step force rho U)
    c, w = plb.plb_velocity_set(plb.PLB_D2Q9)
    c = c[:, :2].astype(float)
    f = lat.populations()
    rho, u, _ = lat.moments()
    u2 = u.copy()
    u2[0] += U
    lat.set_populations(f - equilibrium(c, w, rho, u) + equilibrium(c, w, rho, u2))
    lat.step(n2)
    lat.status()
    _, u, _ = lat.moments()
    ux = u[0].reshape(2, nx).mean(0)
    return relative_norms(ux, np.full(nx, U)), U


def test_galilean_invariance_converges_second_order():
    """Sec. VI.C: the planar interface of Sec. VI.A (Table II grids) at rest until 7.91 us, then
    moved at U_x = 0.1 m/s until 31.6 us.  The phases drift relative to each other through the
    interface error; the error of u_x against the uniform U_x falls at second order.  The start
    is balanced (plb_init_physical: physical velocity zero); with f = f^eq(rho, 0) the sound
    waves from the initial F/(2 rho) velocity dominate the error on grids 3-5."""
    norms = []
    for k in range(1, 6):
        n, U = _galilean(k)
        norms.append(n)
        print(f"galilean fp64 grid {k}: U {U:.4e} L1 {n[0]:.3e} L2 {n[1]:.3e} Linf {n[2]:.3e}")
    for j in range(3):
        orders = [math.log(norms[k][j] / norms[k + 1][j]) / math.log((k + 2) / (k + 1)) for k in range(4)]
        print(f"  norm {j}: orders {[round(o, 2) for o in orders]}")
        assert min(orders) > 1.7, orders


def _plates(k, precision=0, steps_factor=0.5):
    import paper_2504_15018_gb300 as plb
    ny = 100 * k
    s = plates(ny)
    nx = 2 if precision != 0 else 5 * k
    opts = plb.make_opts(precision=precision, kappa=s["kappa"], tau_v=s["tau_v"], tau_rho_v=s["rho_v"],
                         tau_rho_l=s["rho_l"], wall_y=1, body_force=(s["F"], 0.0, 0.0))
    lat = plb.Lattice(plb.PLB_D2Q9, (nx, ny, 1), plb.paper_eos(s["rho_v"], s["rho_l"], s["P"]), tau=s["tau_l"],
                      G=-1.0, eps=2.0, opts=opts)
    u0 = np.zeros((2, nx * ny))
    u0[0] = np.repeat(s["u"], nx)
    lat.init(np.repeat(s["rho"], nx), u0, physical=True)
    steps = int(steps_factor * (ny / 2) ** 2 / s["nu_l"])
    lat.step(steps // 2)
    _, u, _ = lat.moments()
    half = relative_norms(u[0].reshape(ny, nx).mean(1), s["u"])
    lat.step(steps - steps // 2)
    lat.status()
    _, u, _ = lat.moments()
    return relative_norms(u[0].reshape(ny, nx).mean(1), s["u"]), half, s


def test_two_phase_plates_converge_second_order():
    """Sec. VI.D on the Table IV grids (Nx = 5 k, Ny = 100 k, F = 1e6 N/m^3, R134a): FP64 velocity
    profiles against the diffuse-interface channel flow, second order in all three norms.
    FP32 is reported: the body force is 1.6e-8 in lattice units on grid 1 and falls as k^-3,
    below one FP32 ulp of the liquid populations, so part of each step's forcing is rounded
    away and the FP32 profile error is larger than FP64's (grid 1 asserted within 40 %)."""
    norms = []
    for k in range(1, 6):
        n, half, s = _plates(k)
        norms.append(n)
        print(f"plates fp64 grid {k}: F {s['F']:.3e} umax {s['u'].max():.3e} L1 {n[0]:.3e} L2 {n[1]:.3e} "
              f"Linf {n[2]:.3e} (L2 at half time {half[1]:.3e})")
        assert abs(half[1] / n[1] - 1) < 0.1            # steady
    for j in range(3):
        orders = [math.log(norms[k][j] / norms[k + 1][j]) / math.log((k + 2) / (k + 1)) for k in range(4)]
        print(f"  norm {j}: orders {[round(o, 2) for o in orders]}")
        assert min(orders) > 1.8, orders
    for k in (1, 2, 3):
        n32, _, _ = _plates(k, precision=1)
        print(f"plates fp32 grid {k}: L2 {n32[1]:.3e} (fp64 {norms[k - 1][1]:.3e})")
        if k == 1:
            assert n32[1] < 1.4 * norms[0][1]


# Sec. VI.B, Young-Laplace test: (gamma [N/m], tau_l) of the five cases; kappa follows from
# Eq. surface_tension through the converter (1.026 / 0.923 / 1.140 / 0.0923 / 5.698 printed)
LAPLACE_CASES = [(0.0758e-3, 0.68), (0.758e-3, 0.68), (7.58e-3, 0.56), (75.8e-3, 0.52), (379e-3, 0.52)]
LAPLACE_RADII = (15, 20, 25, 30, 35)


def _young_laplace(precision):
    """All 25 droplets (5 surface tensions x 5 radii) in one batch: 150 x 150 cells over
    15 um (dx = 0.1 um, xi = 1.5 dx), paper EOS, tau(rho) interpolation."""
    import paper_2504_15018_gb300 as plb
    from paper_2504_15018_gb300 import inputs
    from paper_setups import converter as conv
    n = 150
    insts, fields, meta = [], [], []
    x, y, _ = inputs.grid_coords((n, n, 1))
    r = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2)
    for gamma, tau_l in LAPLACE_CASES:
        c = conv(n, tau_l, L=15e-6, xi_cells=1.5, gamma=gamma)
        for R in LAPLACE_RADII:
            opts = plb.make_opts(precision=precision, kappa=c["kappa"], tau_v=c["tau_v"], tau_rho_v=c["rho_v"],
                                 tau_rho_l=c["rho_l"])
            insts.append(plb.make_instance((n, n, 1), plb.paper_eos(c["rho_v"], c["rho_l"], c["P"]), tau=tau_l,
                                           opts=opts))
            fields.append(pp.planar_profile(R - r, 0.0, c["P"], c["rho_v"], c["rho_l"]))
            meta.append((gamma, c))
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, rho in enumerate(fields):
        b.init(k, rho)
    b.step(30000)
    b.status()
    acc = np.zeros((len(insts), 4))
    for _ in range(10):
        b.step(200)
        for k in range(len(insts)):
            acc[k] += (b.reduce(k, plb.PLB_MASS)[0],
                       b.reduce(k, plb.PLB_MEAN_RHO, (n // 2 - 4, n // 2 - 4, 0), (n // 2 + 5, n // 2 + 5, 1))[0],
                       b.reduce(k, plb.PLB_MEAN_RHO, (0, 0, 0), (9, 9, 1))[0],
                       b.reduce(k, plb.PLB_UMAX)[0])
    acc /= 10
    b.status()
    out = []
    for j, (gamma, tau_l) in enumerate(LAPLACE_CASES):
        rows = []
        for i in range(len(LAPLACE_RADII)):
            k = j * len(LAPLACE_RADII) + i
            c = meta[k][1]
            mass, r_in, r_out, umax = acc[k]
            dP = pp.paper_pressure(r_in, c["rho_v"], c["rho_l"], c["P"]) - \
                pp.paper_pressure(r_out, c["rho_v"], c["rho_l"], c["P"])
            Rm = math.sqrt((mass - r_out * n * n) / (math.pi * (r_in - r_out)))
            rows.append((Rm, float(dP), umax))
        rows = np.array(rows)
        A = np.stack([1.0 / rows[:, 0], np.ones(len(rows))], axis=1)
        g_fit, _ = np.linalg.lstsq(A, rows[:, 1], rcond=None)[0]
        out.append((gamma, tau_l, meta[j * len(LAPLACE_RADII)][1]["kappa"], g_fit,
                    meta[j * len(LAPLACE_RADII)][1]["gamma_lat"], rows))
    return out


def test_young_laplace_five_surface_tensions():
    """Sec. VI.B: Delta P R against the surface tension imposed through Eq. surface_tension, per
    droplet (the Young-Laplace line through the origin), for the droplets that start at
    R0 = 20, 25, 30 cells (the R0 = 15 droplets shrink to R ~ 11-12, the R0 = 35 ones feel their
    periodic images).  As in the paper: close agreement for kappa near 1 at tau_l 0.68 / 0.56
    (within 5 %), less for tau_l = 0.52 (capillary oscillations barely damped) and for the
    kappa = 0.0923 and 5.698 cases.  FP32 fits the same gamma as FP64 within 1 %."""
    res64 = _young_laplace(0)
    res32 = _young_laplace(1)
    tols = {0.0758e-3: 0.6, 0.758e-3: 0.05, 7.58e-3: 0.05, 75.8e-3: 0.25, 379e-3: 0.2}
    ok = True
    for (gamma, tau_l, kappa, g64, g_lat, rows), r32 in zip(res64, res32):
        ratio = rows[1:4, 0] * rows[1:4, 1] / g_lat
        print(f"gamma {gamma * 1e3:.4g} mN/m tau_l {tau_l} kappa {kappa:.4g}: imposed {g_lat:.5e}; "
              f"dP R / gamma at R0 = 20, 25, 30: {np.round(ratio, 4).tolist()}; fit fp64 {g64:.5e} "
              f"fp32 {r32[3]:.5e} ({(r32[3] / g64 - 1) * 100:+.3f} %); umax {rows[:, 2].max():.2e}")
        for R, dP, um in rows:
            print(f"    R {R:.3f} dP {dP:.5e} gamma/R {g_lat / R:.5e} umax {um:.2e}")
        ok &= abs(r32[3] / g64 - 1) < 0.01
        ok &= bool(np.all(np.abs(ratio - 1) < tols[gamma]))
    assert ok


def test_young_laplace_kappa_0_0923_improves_with_resolution():
    """Sec. VI.B: the gamma_1 = 0.0758 mN/m case (kappa = 0.0923) repeated at dx = 0.05 um,
    xi = 3 dx (dt = 0.95 ns at tau_l = 0.68) agrees better with the imposed surface tension than
    at dx = 0.1 um.  FP32 (which fits the same gamma as FP64 at dx = 0.1 um)."""
    coarse = _young_laplace_case(0.0758e-3, 0.68, 150, 1.5, (20, 25, 30), 30000)
    fine = _young_laplace_case(0.0758e-3, 0.68, 300, 3.0, (40, 50, 60), 120000)
    ec, ef = np.abs(coarse - 1).max(), np.abs(fine - 1).max()
    print(f"dP R / gamma: dx 0.1 um {np.round(coarse, 4).tolist()}, dx 0.05 um {np.round(fine, 4).tolist()}")
    assert ef < ec


def _young_laplace_case(gamma, tau_l, n, xi_cells, radii, steps):
    import paper_2504_15018_gb300 as plb
    from paper_2504_15018_gb300 import inputs
    from paper_setups import converter as conv
    c = conv(n, tau_l, L=15e-6, xi_cells=xi_cells, gamma=gamma)
    x, y, _ = inputs.grid_coords((n, n, 1))
    r = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2)
    opts = plb.make_opts(precision=1, kappa=c["kappa"], tau_v=c["tau_v"], tau_rho_v=c["rho_v"], tau_rho_l=c["rho_l"])
    insts = [plb.make_instance((n, n, 1), plb.paper_eos(c["rho_v"], c["rho_l"], c["P"]), tau=tau_l, opts=opts)
             for _ in radii]
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, R in enumerate(radii):
        b.init(k, pp.planar_profile(R - r, 0.0, c["P"], c["rho_v"], c["rho_l"]))
    b.step(steps)
    acc = np.zeros((len(radii), 3))
    h = n // 30
    for _ in range(10):
        b.step(steps // 150)
        for k in range(len(radii)):
            acc[k] += (b.reduce(k, plb.PLB_MASS)[0],
                       b.reduce(k, plb.PLB_MEAN_RHO, (n // 2 - h, n // 2 - h, 0), (n // 2 + h + 1, n // 2 + h + 1, 1))[0],
                       b.reduce(k, plb.PLB_MEAN_RHO, (0, 0, 0), (2 * h + 1, 2 * h + 1, 1))[0])
    b.status()
    acc /= 10
    out = []
    for mass, r_in, r_out in acc:
        dP = pp.paper_pressure(r_in, c["rho_v"], c["rho_l"], c["P"]) - pp.paper_pressure(r_out, c["rho_v"], c["rho_l"],
                                                                                        c["P"])
        Rm = math.sqrt((mass - r_out * n * n) / (math.pi * (r_in - r_out)))
        out.append(float(dP) * Rm / c["gamma_lat"])
    return np.array(out)
