"""Single-pass stepping (PLB_STREAM_FUSED): psi of each tile and its halo formed in shared
memory, force, collision and push streaming in one kernel, two population copies.  The
per-cell arithmetic is the code of the two-pass in-place (AA) kernels, so after any number of
steps both give the same populations bit for bit where both use the same collision form (D3Q19
with FP32 storage collides in moment space in the single pass and pair by pair in the two-pass
kernels, equal to rounding); ragged tiles (nx, ny not multiples of the 64 x 16 tile, nz not a
multiple of the z chunk), walls, one-row and two-column lattices, BGK and MRT, FP32, FP16S and
FP16S with stochastic rounding are covered.  Readouts, state and
the balanced start work on the current copy."""
import numpy as np
import pytest

from gpu_cases import case_fields, make_lattice

pytestmark = pytest.mark.gpu

RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.3, s_m=1.5)
CASES = {
    "d3q19_fp32_mrt_walls_ragged": dict(lattice=1, dims=(70, 20, 9), wall=True, shape="slab", mrt=True, rates=RATES,
                                        fext=(2e-6, 0, 0), precision=1),
    "d3q19_fp32_bgk_zchunks": dict(lattice=1, dims=(64, 48, 40), u0=(0.02, -0.01, 0.015), precision=1),
    "d3q19_fp32_mrt_one_plane": dict(lattice=1, dims=(18, 10, 1), mrt=True, rates=RATES, precision=1),
    "d2q9_fp32_bgk_droplet": dict(lattice=0, dims=(130, 67, 1), precision=1),
    "d2q9_fp32_mrt_walls_taurho": dict(lattice=0, dims=(96, 20, 1), wall=True, shape="slab", mrt=True, rates=RATES,
                                       tau=0.8, tau_v=1.1, fext=(1e-5, 0, 0), precision=1),
    "d2q9_fp32_two_wide": dict(lattice=0, dims=(2, 40, 1), shape="slab", precision=1),
    "d2q9_fp32_one_row": dict(lattice=0, dims=(66, 1, 1), shape="slab", precision=1),
    "d3q19_fp16s_mrt_walls": dict(lattice=1, dims=(34, 18, 12), wall=True, shape="slab", mrt=True, rates=RATES,
                                  precision=2),
    "d3q19_fp16s_sr_mrt_walls": dict(lattice=1, dims=(34, 18, 12), wall=True, shape="slab", mrt=True, rates=RATES,
                                     precision=2, fp16_rounding=1),
    # nx / 4 a multiple of 32 and several row segments: whole warps of the four-cell FP16 psi
    # pass and of the staged kernel along x
    "d3q19_fp16s_mrt_walls_wide": dict(lattice=1, dims=(256, 18, 6), wall=True, shape="slab", mrt=True,
                                       rates=RATES, precision=2),
    "d3q19_fp16s_sr_bgk_wide": dict(lattice=1, dims=(128, 20, 5), u0=(0.02, -0.01, 0.015), precision=2,
                                    fp16_rounding=1),
    "d2q9_fp16s_bgk_droplet": dict(lattice=0, dims=(80, 70, 1), precision=2),
    "d3q19_fp32_mrt_wetting_walls": dict(lattice=1, dims=(24, 20, 10), wall=True, shape="slab", mrt=True,
                                         rates=RATES, wall_rho=0.9, precision=1),
    "d2q9_fp16s_bgk_wetting_walls": dict(lattice=0, dims=(66, 34, 1), wall=True, shape="slab", wall_rho=1.2,
                                         precision=2),
}


def _pair(name, steps, physical=False):
    case = CASES[name]
    rho, u0, rv, rl = case_fields(case)
    out = []
    for streaming in (0, 1):
        lat = make_lattice(dict(case, streaming=streaming), rv, rl)
        lat.init(rho, u0, physical=physical)
        lat.step(steps)
        lat.status()
        out.append(lat)
    return out


def _moment_form_differs(case):
    """D3Q19 with FP32 storage: the single pass collides in moment space, the two-pass kernels
    pair by pair (FP16 storage uses the moment form in both, D2Q9 the pair form in both)."""
    return case["lattice"] == 1 and case["precision"] == 1


def _assert_same(case, a, b, steps):
    if _moment_form_differs(case):
        # the same update in FP32 with another rounding order: within the linear accumulation
        # bound of the oracle comparison, steps * 8 * 2^-24 (relative)
        err = float(np.max(np.abs(b - a) / np.abs(a)))
        assert err <= steps * 8 * 2.0 ** -24, err
    else:
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name", list(CASES))
def test_fused_matches_the_two_pass_kernels(name):
    """Bit for bit where both use the same collision form, else to rounding."""
    case = CASES[name]
    aa, fu = _pair(name, 7)
    _assert_same(case, aa.populations(), fu.populations(), 7)
    aa.step(6)
    fu.step(6)
    _assert_same(case, aa.populations(), fu.populations(), 13)
    assert fu.time == 13


@pytest.mark.parametrize("name,steps", [("d3q19_fp32_mrt_walls_ragged", 100), ("d2q9_fp32_mrt_walls_taurho", 100),
                                        ("d3q19_fp16s_mrt_walls", 50), ("d3q19_fp16s_sr_mrt_walls", 50)])
def test_fused_against_the_oracle(name, steps):
    """The single pass compared with the FP64 oracle directly: FP32 within the linear
    accumulation bound steps * 8 * 2^-24 (relative), FP16S within sqrt(steps) * 2^-11 (2^-10 with
    stochastic rounding) of w_i rho_l, as for the two-pass kernels."""
    from gpu_cases import max_rel_err, run_both
    case = dict(CASES[name], streaming=1)
    ref, got, _, _ = run_both(case, steps)
    if case["precision"] == 1:
        err = max_rel_err(ref, got)
        bound = steps * 8 * 2.0 ** -24
    else:
        err = float(np.max(np.abs(got - ref) / np.abs(ref).max(axis=1, keepdims=True)))
        bound = np.sqrt(steps) * 2.0 ** (-10 if case.get("fp16_rounding") else -11)
    print(f"{name} single pass, {steps} steps: error {err:.3e} (bound {bound:.2e})")
    assert err <= bound


def test_fused_readouts_state_and_balanced_start():
    import paper_2504_15018_gb300 as plb
    aa, fu = _pair("d3q19_fp16s_mrt_walls", 5, physical=True)
    for a, b in zip(aa.moments(), fu.moments()):
        assert np.array_equal(a, b)
    for what in (plb.PLB_MASS, plb.PLB_MOMENTUM, plb.PLB_UMAX, plb.PLB_UL2):
        assert np.array_equal(aa.reduce(what), fu.reduce(what))
    assert np.array_equal(aa.reduce(plb.PLB_MEAN_P, (2, 3, 1), (9, 11, 5)), fu.reduce(plb.PLB_MEAN_P, (2, 3, 1), (9, 11, 5)))
    # FP32 storage: the two collision forms round differently; u (about 1e-5 here) is a sum of
    # populations of order one, so its difference is absolute, at the populations' rounding
    aa, fu = _pair("d3q19_fp32_mrt_walls_ragged", 5, physical=True)
    for a, b in zip(aa.moments(), fu.moments()):
        assert np.allclose(a, b, rtol=1e-5, atol=1e-6)
    st = fu.get_state()
    fu.step(4)
    f4 = fu.populations()
    fu.set_state(st)
    fu.step(4)
    assert np.array_equal(fu.populations(), f4)
    f = fu.populations()
    fu.set_populations(f)
    assert np.array_equal(fu.populations(), f)


def test_fused_needs_fp32_arithmetic_even_nx_and_no_batch():
    import paper_2504_15018_gb300 as plb
    from gpu_cases import maxwell
    rv, rl, _ = maxwell(0.8)
    for prec, dims in ((0, (16, 8, 4)), (1, (15, 8, 4))):
        o = plb.make_opts(precision=prec, streaming=plb.PLB_STREAM_FUSED)
        with pytest.raises(plb.PlbError) as e:
            plb.Lattice(plb.PLB_D3Q19, dims, plb.pr_eos(0.8), opts=o)
        assert e.value.code == plb.PLB_EUNSUPPORTED
    o = plb.make_opts(precision=1, streaming=plb.PLB_STREAM_FUSED)
    with pytest.raises(plb.PlbError) as e:
        plb.Batch(plb.PLB_D2Q9, [plb.make_instance((16, 16, 1), plb.pr_eos(0.8), opts=o)])
    assert e.value.code == plb.PLB_EINVAL
