"""The allocation-free entry point plb_step_pairs_static, for callers that cannot
allocate device memory (a plugin given only its buffers by another framework, or a
real-time loop where cudaMalloc is not allowed).  Its scratch is a fixed device array
inside the library; this checks, through the C ABI, that two calls in a row produce the
same stored populations as the ordinary plb_create / plb_step path (the same kernels and
the same stochastic-rounding counter, so the results must agree bit for bit), and that
oversize lattices are refused."""
import numpy as np
import pytest

from gpu_cases import case_fields, make_lattice

pytestmark = pytest.mark.gpu

RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.3, s_m=1.5)
CASES = {
    "d2q9_fp32_droplet": dict(lattice=0, dims=(37, 29, 1), kappa=1.3, precision=1, fext=(1e-6, -2e-6, 0)),
    "d3q19_fp32_mrt_walls": dict(lattice=1, dims=(10, 12, 8), wall=True, mrt=True, rates=RATES, shape="slab",
                                 precision=1, fext=(2e-6, 0, 1e-6)),
    "d2q9_fp64_mrt_taurho": dict(lattice=0, dims=(24, 20, 1), wall=True, mrt=True, rates=RATES, tau=0.8, tau_v=1.1,
                                 shape="slab", precision=0, t_ratio=0.85),
    # FP16-shifted storage, round-to-nearest and stochastic rounding (the noise of step t is
    # drawn from the counter t: the t0 argument must carry it across calls)
    "d2q9_fp16s_even_droplet": dict(lattice=0, dims=(36, 29, 1), kappa=1.3, precision=2, fext=(1e-6, -2e-6, 0)),
    "d2q9_fp16s_sr_even_droplet": dict(lattice=0, dims=(36, 29, 1), kappa=1.3, precision=2, fext=(1e-6, -2e-6, 0),
                                       fp16_rounding=1),
    "d3q19_fp16s_sr_mrt_walls": dict(lattice=1, dims=(10, 12, 8), wall=True, mrt=True, rates=RATES,
                                     shape="slab", precision=2, fext=(2e-6, 0, 1e-6), fp16_rounding=1),
}

_NP_DTYPE = {0: np.float64, 1: np.float32, 2: np.float16}


def _stored(lat):
    """The lattice's stored populations as a (Q, N) array of the storage type (natural layout
    at even parity), taken from its raw checkpoint state."""
    buf = lat.get_state()
    prec = int(lat.opts.precision)
    raw = np.frombuffer(buf[64:].tobytes(), dtype=_NP_DTYPE[prec])
    pstride = raw.size // lat.Q
    return raw.reshape(lat.Q, pstride)[:, :lat.n].copy()


@pytest.mark.parametrize("name", list(CASES))
def test_static_scratch_matches_the_allocating_path(name):
    import torch

    import paper_2504_15018_gb300 as plb

    case = CASES[name]
    rho, u0, rv, rl = case_fields(case)
    ref = make_lattice(case, rv, rl)
    ref.init(rho, u0)
    dtype = {0: torch.float64, 1: torch.float32, 2: torch.float16}[case["precision"]]
    pops = torch.from_numpy(_stored(ref)).to(dtype=dtype, device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    npairs = 3
    for _ in range(2):                     # two calls in a row share the static scratch
        t0 = ref.time
        ref.step(2 * npairs)
        plb.plb_step_pairs_static(case["lattice"], ref.dims, plb.pr_eos(case.get("t_ratio", 0.8)),
                                  case.get("tau", 1.0), -1.0, 2.0, ref.opts, pops.data_ptr(), npairs, t0,
                                  stream.cuda_stream)
        got = pops.cpu().numpy()
        want = _stored(ref)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), \
            float(np.max(np.abs(got.astype(np.float64) - want.astype(np.float64))))


def test_static_scratch_rejects_oversize_lattices():
    import torch

    import paper_2504_15018_gb300 as plb

    dims = (256, 256, 64)                  # padded psi field far above the 8 MiB scratch
    opts = plb.make_opts(precision=plb.PLB_FP32)
    pops = torch.zeros(256, dtype=torch.float32, device="cuda")
    with pytest.raises(plb.PlbError) as e:
        plb.plb_step_pairs_static(plb.PLB_D3Q19, dims, plb.pr_eos(0.8), 1.0, -1.0, 2.0, opts, pops.data_ptr(), 1, 0,
                                  torch.cuda.current_stream().cuda_stream)
    assert e.value.code == plb.PLB_ENOMEM
    assert "static scratch" in str(e.value)
