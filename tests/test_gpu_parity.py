"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs (small grids that still span several thread blocks and a ragged tail).

FP64 storage: max relative error <= 1e-12 on every population after 1000 steps.
FP32 / FP16-shifted storage: tolerances derived from the storage rounding (see the
test docstrings)."""
import numpy as np
import pytest

from gpu_cases import make_lattice, max_rel_err, maxwell, oracle_params, run_both, case_fields, direction_map
import oracle

pytestmark = pytest.mark.gpu

RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.3, s_m=1.5)

FP64_CASES = {
    "d2q9_bgk_periodic_droplet": dict(lattice=0, dims=(37, 29, 1), kappa=1.3, fext=(1e-6, -2e-6, 0)),
    "d2q9_mrt_walls_slab_taurho": dict(lattice=0, dims=(24, 20, 1), wall=True, mrt=True, rates=RATES, tau=0.8,
                                       tau_v=1.1, shape="slab", fext=(1e-5, 0, 0), t_ratio=0.85),
    "d2q9_bgk_paper_eos_G": dict(lattice=0, dims=(45, 3, 1), eos="paper", rho_v=0.0375, rho_l=1.187, P=0.0439932,
                                 tau=0.56, tau_v=0.6287, shape="slab", kappa=1.026, G=-2.5),
    "d3q19_bgk_periodic_droplet": dict(lattice=1, dims=(13, 11, 9), kappa=0.7, t_ratio=0.75),
    "d3q19_mrt_walls_slab": dict(lattice=1, dims=(10, 12, 8), wall=True, mrt=True, rates=RATES, shape="slab",
                                 fext=(2e-6, 0, 1e-6)),
    "d3q19_mrt_periodic_droplet_u0": dict(lattice=1, dims=(12, 9, 11), mrt=True, rates=RATES, u0=(0.02, -0.01, 0.015),
                                          tau=0.9),
    # wetting walls: psi on the wall nodes fixed at psi(wall_rho)
    "d2q9_bgk_wetting_walls": dict(lattice=0, dims=(26, 22, 1), wall=True, shape="slab", wall_rho=1.2,
                                   fext=(2e-6, 0, 0)),
    "d3q19_mrt_wetting_walls": dict(lattice=1, dims=(11, 14, 8), wall=True, mrt=True, rates=RATES, shape="slab",
                                    wall_rho=0.9),
}

# Even nx: FP32 / FP16S storage runs the two-cells-per-thread kernels on these.
PAIR_CASES = {
    "d2q9_bgk_even_droplet": dict(lattice=0, dims=(36, 29, 1), kappa=1.3, fext=(1e-6, -2e-6, 0)),
    "d2q9_mrt_even_walls_taurho": dict(lattice=0, dims=(24, 20, 1), wall=True, mrt=True, rates=RATES, tau=0.8,
                                       tau_v=1.1, shape="slab", fext=(1e-5, 0, 0), t_ratio=0.85),
    "d3q19_mrt_even_walls": dict(lattice=1, dims=(10, 12, 8), wall=True, mrt=True, rates=RATES, shape="slab",
                                 fext=(2e-6, 0, 1e-6)),
    "d3q19_bgk_even_droplet_u0": dict(lattice=1, dims=(12, 9, 11), u0=(0.02, -0.01, 0.015), tau=0.9, kappa=0.8),
    "d2q9_bgk_two_wide": dict(lattice=0, dims=(2, 17, 1), shape="slab", wall=True, fext=(1e-5, 0, 0)),
}


@pytest.mark.parametrize("name", list(FP64_CASES))
def test_fp64_population_parity_1000_steps(name):
    """Max relative error <= 1e-12 on every population after 1000 steps.  The FP64 kernels
    evaluate every term in the order the equations write it, with one rounding per product
    and per sum, so they round as the oracle does; the dynamics of the tau_l = 0.56 case
    amplify a 1e-16 perturbation by about 1e5 in 1000 steps, so only such an evaluation
    meets the bound on every case.  The number of populations that differ at all is printed."""
    case = dict(FP64_CASES[name], precision=0)
    ref, got, lat, _ = run_both(case, 1000)
    err = max_rel_err(ref, got)
    print(f"{name}: max rel err {err:.3e}, populations differing from the oracle: "
          f"{int(np.count_nonzero(got != ref))} of {got.size}")
    assert err <= 1e-12


@pytest.mark.parametrize("name", ["d2q9_bgk_periodic_droplet", "d3q19_mrt_walls_slab"])
def test_fp64_parity_at_odd_step_counts(name):
    """Both AA parities and the switch between them (1, 2, 3 and 7 steps)."""
    for steps in (1, 2, 3, 7):
        ref, got, _, _ = run_both(dict(FP64_CASES[name], precision=0), steps)
        assert max_rel_err(ref, got) <= 1e-12, steps


@pytest.mark.parametrize("name", ["d2q9_bgk_periodic_droplet", "d3q19_mrt_periodic_droplet_u0",
                                  "d3q19_mrt_walls_slab"] + list(PAIR_CASES))
def test_fp32_population_parity(name):
    """FP32 storage and arithmetic: each step rounds a population through about 8 FP32
    operations of relative error 2^-24; accumulated linearly over 200 steps that bounds the
    deviation from FP64 by 200 * 8 * 2^-24 = 9.5e-5 relative."""
    steps = 200
    ref, got, _, _ = run_both(dict({**FP64_CASES, **PAIR_CASES}[name], precision=1), steps)
    err = max_rel_err(ref, got)
    print(f"{name} fp32: max rel err {err:.3e}")
    assert err <= steps * 8 * 2.0 ** -24


@pytest.mark.parametrize("name", ["d2q9_bgk_periodic_droplet", "d3q19_mrt_periodic_droplet_u0",
                                  "d2q9_mrt_even_walls_taurho", "d3q19_mrt_even_walls"])
def test_fp16s_population_parity(name):
    """FP16 storage of f_i - w_i rho_ref (rho_ref = rho_v): each store rounds the deviation by
    at most half an ulp, <= 2^-11 of its magnitude <= 2^-11 w_i rho_l.  Independent roundings
    over n steps add like a random walk: bound sqrt(n) * 2^-11 relative to w_i rho_l.  The
    horizon is 50 steps: later, the relaxing interfaces of the walled slab amplify any
    perturbation (FP32 and the one-cell-per-thread FP16 kernel grow the same way), and FP16 is
    assessed on the macroscopic results instead (tests/test_gpu_precision.py)."""
    case = dict({**FP64_CASES, **PAIR_CASES}[name], precision=2)
    steps = 50
    ref, got, _, _ = run_both(case, steps)
    rho, _, rv, rl = case_fields(case)
    c_w = np.abs(ref).max(axis=1, keepdims=True)          # ~ w_i rho_l per direction
    err = float(np.max(np.abs(got - ref) / c_w))
    print(f"{name} fp16s: max err / (w_i rho_l) {err:.3e}")
    assert err <= np.sqrt(steps) * 2.0 ** -11


@pytest.mark.parametrize("name", ["d2q9_mrt_even_walls_taurho", "d3q19_mrt_even_walls", "d2q9_bgk_periodic_droplet"])
def test_fp16s_stochastic_rounding_parity(name):
    """FP16 storage with stochastic rounding: each store errs by less than one ulp,
    2^-10 of the deviation <= 2^-10 w_i rho_l, with zero mean; over n steps the errors add like
    a random walk: bound sqrt(n) * 2^-10 relative to w_i rho_l."""
    case = dict({**FP64_CASES, **PAIR_CASES}[name], precision=2, fp16_rounding=1)
    steps = 50
    ref, got, _, _ = run_both(case, steps)
    c_w = np.abs(ref).max(axis=1, keepdims=True)
    err = float(np.max(np.abs(got - ref) / c_w))
    print(f"{name} fp16s-sr: max err / (w_i rho_l) {err:.3e}")
    assert err <= np.sqrt(steps) * 2.0 ** -10


def test_moments_parity():
    """rho, u and p of the library against the oracle's moments of the same populations."""
    case = dict(FP64_CASES["d2q9_bgk_periodic_droplet"], precision=0)
    ref, got, lat, P = run_both(case, 300)
    r, u, p = lat.moments()
    inv = np.argsort(direction_map(0))
    ro, uo, po = oracle.moments(P, np.ascontiguousarray(got.T[:, inv]))
    assert np.max(np.abs(r - ro) / ro) < 1e-14
    assert np.max(np.abs(u - uo)) < 1e-15
    # p = p_EOS(rho) is a difference of two terms each smaller than rho (PR: rho R T / (1 - b rho)
    # and a alpha rho^2 / (...)); in the liquid they cancel to p ~ rho / 500, so the rounding
    # bound is relative to rho, not to p
    assert np.max(np.abs(p - po) / ro) < 1e-14


def test_reductions_against_oracle_fields():
    import paper_2504_15018_gb300 as plb
    case = dict(FP64_CASES["d3q19_mrt_walls_slab"], precision=0)
    ref, got, lat, P = run_both(case, 50)
    inv = np.argsort(direction_map(1))
    ro, uo, po = oracle.moments(P, np.ascontiguousarray(got.T[:, inv]))
    umag = np.sqrt((uo ** 2).sum(0))
    assert lat.reduce(plb.PLB_MASS)[0] == pytest.approx(ro.sum(), rel=1e-13)
    assert np.allclose(lat.reduce(plb.PLB_MOMENTUM), (ro * uo).sum(1), rtol=1e-10, atol=1e-15)
    assert lat.reduce(plb.PLB_UMAX)[0] == pytest.approx(umag.max(), rel=1e-11)
    assert lat.reduce(plb.PLB_UL1)[0] == pytest.approx(umag.sum(), rel=1e-11)
    assert lat.reduce(plb.PLB_UL2)[0] == pytest.approx(np.sqrt((umag ** 2).sum()), rel=1e-11)
    nx, ny, nz = case["dims"]
    lo, hi = (2, 3, 1), (7, 9, 5)
    box = np.zeros((nz, ny, nx), bool)
    box[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = True
    box = box.reshape(-1)
    assert lat.reduce(plb.PLB_MEAN_RHO, lo, hi)[0] == pytest.approx(ro[box].mean(), rel=1e-13)
    assert lat.reduce(plb.PLB_MEAN_P, lo, hi)[0] == pytest.approx(po[box].mean(), rel=1e-12)


def test_checkpoint_restart_is_bit_exact():
    case = dict(FP64_CASES["d3q19_mrt_walls_slab"], precision=1)
    rho, u0, rv, rl = case_fields(case)
    a = make_lattice(case, rv, rl)
    a.init(rho, u0)
    a.step(41)
    state = a.get_state()
    a.step(40)
    fa = a.populations()
    b = make_lattice(case, rv, rl)
    b.set_state(state)
    assert b.time == 41
    b.step(40)
    assert np.array_equal(fa, b.populations())


def test_set_populations_round_trip():
    case = dict(FP64_CASES["d2q9_bgk_periodic_droplet"], precision=0)
    rho, u0, rv, rl = case_fields(case)
    lat = make_lattice(case, rv, rl)
    lat.init(rho, u0)
    lat.step(3)                       # odd parity: swapped layout
    f = lat.populations()
    lat.set_populations(f)
    assert np.array_equal(lat.populations(), f)
    lat.step(5)
    other = make_lattice(case, rv, rl)
    other.init(rho, u0)
    other.step(8)
    assert max_rel_err(other.populations(), lat.populations()) < 1e-14


def test_psi_domain_and_invalid_inputs_are_reported():
    import paper_2504_15018_gb300 as plb
    case = dict(lattice=0, dims=(16, 8, 1), precision=1)
    rv, rl, _ = maxwell(0.8)
    lat = make_lattice(case, rv, rl)
    rho = np.full(128, 2.0)
    rho[37] = 10.2                    # near 1/b: p_EOS > rho/3, psi undefined
    lat.init(rho)
    lat.step(1)
    with pytest.raises(plb.PlbError) as e:
        lat.status()
    assert e.value.code == plb.PLB_EPSI_DOMAIN
    bad = np.full(128, 2.0)
    bad[5] = np.nan
    with pytest.raises(plb.PlbError) as e:
        lat.init(bad)
    assert e.value.code == plb.PLB_EINVAL
    lat.init(np.full(128, 2.0))       # re-init clears the flag
    lat.step(2)
    lat.status()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_init_reports_the_first_invalid_value(precision):
    """rho0 and u0 are checked on the device as plb_init reads them, over staging chunks of up
    to 2^18 x 19 cells: the error names the first invalid index (rho0 before u0), and a
    later valid plb_init gives the same populations as a lattice never given bad input."""
    import paper_2504_15018_gb300 as plb
    dims = (2 * 640, 640, 1)                       # 819,200 cells: several chunks with u0
    n = dims[0] * dims[1]
    rv, rl, _ = maxwell(0.8)
    case = dict(lattice=0, dims=dims, precision=precision)
    rng = np.random.default_rng(5)
    rho = rv * rng.uniform(1.0, 1.02, n)            # vapour with small noise: stable for a few steps
    u0 = rng.uniform(-0.01, 0.01, (2, n))
    lat = make_lattice(case, rv, rl)
    for bad_rho, bad_u, want in (({700_001: -1.0, 812_345: np.nan}, {}, "rho0[700001]"),
                                 ({5: 0.0}, {(1, 3): np.inf}, "rho0[5]"),
                                 ({}, {(1, 9): np.nan, (0, 800_000): -np.inf}, f"u0[{800_000}]"),
                                 ({n - 1: np.inf}, {}, f"rho0[{n - 1}]")):
        r, u = rho.copy(), u0.copy()
        for k, v in bad_rho.items():
            r[k] = v
        for (a, k), v in bad_u.items():
            u[a, k] = v
        with pytest.raises(plb.PlbError) as e:
            lat.init(r, u)
        assert e.value.code == plb.PLB_EINVAL
        assert want in str(e.value), str(e.value)
    lat.init(rho, u0)
    lat.step(3)
    lat.status()
    ref = make_lattice(case, rv, rl)
    ref.init(rho, u0)
    ref.step(3)
    assert np.array_equal(lat.populations(), ref.populations())


@pytest.mark.parametrize("name", ["d2q9_bgk_periodic_droplet", "d3q19_mrt_walls_slab", "d3q19_mrt_periodic_droplet_u0"])
def test_init_physical_matches_the_balanced_oracle_start(name):
    """plb_init_physical: f^eq(rho0, u0 - F/(2 rho0)) against the same start built from the
    oracle's own force, and the velocity of Eq. Momentum equal to u0 at t = 0."""
    from paper_setups import balanced_init_oracle
    case = dict(FP64_CASES[name], precision=0)
    rho, u0, rv, rl = case_fields(case)
    P = oracle_params(case, rv, rl)
    ref = balanced_init_oracle(P, case["lattice"], rho, u0)[:, direction_map(case["lattice"])].T
    lat = make_lattice(case, rv, rl)
    lat.init(rho, u0, physical=True)
    lat.status()
    got = lat.populations()
    assert max_rel_err(ref, got) < 1e-13
    _, u, _ = lat.moments()
    d = 2 if case["lattice"] == 0 else 3
    want = np.zeros((d, rho.size)) if u0 is None else u0
    assert np.max(np.abs(u[:d] - want)) < 1e-15
    # FP32 storage: the same start to FP32 rounding
    lat32 = make_lattice(dict(case, precision=1), rv, rl)
    lat32.init(rho, u0, physical=True)
    _, u32, _ = lat32.moments()
    assert np.max(np.abs(u32[:d] - want)) < 1e-6


@pytest.mark.parametrize("name", ["d2q9_bgk_wetting_walls", "d3q19_mrt_wetting_walls"])
def test_wetting_walls_fp32_pair_path_and_rejections(name):
    """Wetting walls on the two-cell FP32 path (even nx) against the oracle after 200 steps
    (linear FP32 accumulation bound), and the arguments the library refuses."""
    import paper_2504_15018_gb300 as plb
    case = dict(FP64_CASES[name], precision=1)
    case["dims"] = (case["dims"][0] + case["dims"][0] % 2,) + tuple(case["dims"][1:])
    ref, got, _, _ = run_both(case, 200)
    assert max_rel_err(ref, got) <= 200 * 8 * 2.0 ** -24
    with pytest.raises(plb.PlbError) as e:                       # wetting needs walls
        plb.Lattice(0, (16, 16, 1), plb.pr_eos(0.8), opts=plb.make_opts(wall_rho=1.0))
    assert e.value.code == plb.PLB_EINVAL
    with pytest.raises(plb.PlbError) as e:                       # psi undefined at this density
        plb.Lattice(0, (16, 16, 1), plb.pr_eos(0.8), opts=plb.make_opts(wall_y=1, wall_rho=10.4))
    assert e.value.code == plb.PLB_EINVAL
