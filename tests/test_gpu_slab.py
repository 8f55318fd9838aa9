"""Slab decomposition (plb_slab_*): one D3Q19 lattice split along z into slabs, each a handle
with two ghost planes, stepped with the psi pass, the psi-halo exchange, the collide pass and
the population exchange; after every even number of steps the owned planes must equal the
same planes of the whole lattice stepped by plb_step, bit for bit.  Here all slabs live on
one GPU and the exchange is the library's device-to-device copy (plb_slab_exchange); the
same plan drives a multi-process exchange (tests/test_slab_schedule.py)."""
import numpy as np
import pytest

from gpu_cases import make_lattice, maxwell
from paper_2504_15018_gb300 import inputs

pytestmark = pytest.mark.gpu

RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.3, s_m=1.5)
CASES = {
    "fp64_mrt_walls_2": dict(dims=(24, 20, 16), precision=0, wall=True, mrt=True, rates=RATES,
                             fext=(2e-6, 0.0, 1e-6), split=(7,)),
    "fp32_mrt_walls_3": dict(dims=(24, 20, 16), precision=1, wall=True, mrt=True, rates=RATES,
                             fext=(2e-6, 0.0, 1e-6), split=(5, 11)),
    "fp32_bgk_periodic_odd_nx": dict(dims=(23, 18, 12), precision=1, kappa=1.2, split=(6,)),
    "fp16s_mrt_walls_2": dict(dims=(24, 20, 16), precision=2, wall=True, mrt=True, rates=RATES,
                              fext=(2e-6, 0.0, 1e-6), split=(9,)),
    "fp16s_sr_mrt_walls_2": dict(dims=(24, 20, 16), precision=2, wall=True, mrt=True, rates=RATES,
                                 fext=(2e-6, 0.0, 1e-6), split=(8,), fp16_rounding=1),
}


def _field(dims, wall, rv, rl):
    nx, ny, nz = dims
    if wall:
        rho = inputs.slab(dims, 1, ny // 4, 3 * ny // 4, rl, rv, 3.0, periodic=False)
    else:
        rho = inputs.droplet(dims, (nx / 2 - 0.3, ny / 2 + 0.2, nz / 2 + 0.4), min(dims) / 4, rv, rl, 3.0)
    return inputs.add_noise(rho, inputs.MASTER_SEED + 400, 1e-4)


@pytest.mark.parametrize("name", list(CASES))
def test_slabs_equal_the_whole_lattice(name):
    import paper_2504_15018_gb300 as plb
    case = dict(CASES[name], lattice=1)
    nx, ny, nz = case["dims"]
    rv, rl, _ = maxwell(0.8)
    rho = _field(case["dims"], case.get("wall", False), rv, rl)
    whole = make_lattice(case, rv, rl)
    whole.init(rho)
    rho3 = rho.reshape(nz, ny, nx)
    cuts = (0,) + tuple(case["split"]) + (nz,)
    slabs = []
    for z0, z1 in zip(cuts[:-1], cuts[1:]):
        m = z1 - z0
        planes = np.arange(z0 - 1, z1 + 1) % nz            # ghost, owned planes, ghost
        lat = make_lattice(dict(case, dims=(nx, ny, m + 2)), rv, rl)
        lat.init(rho3[planes].reshape(-1))
        plb.plb_slab_bind(lat.h, z0)
        slabs.append((z0, z1, lat))
    with pytest.raises(plb.PlbError):                      # slabs are stepped pass by pass
        slabs[0][2].step(1)
    n = len(slabs)
    for step in range(1, 41):
        whole.step(1)
        for pass_ in (0, 1):
            for _, _, lat in slabs:
                plb.plb_slab_pass(lat.h, pass_)
            for k in range(n):                             # lower slab k, upper slab k + 1 (periodic)
                plb.plb_slab_exchange(slabs[k][2].h, slabs[(k + 1) % n][2].h, pass_)
        if step in (2, 16, 40):
            whole.status()
            ref = whole.populations().reshape(19, nz, ny, nx)
            for z0, z1, lat in slabs:
                lat.status()
                got = lat.populations().reshape(19, z1 - z0 + 2, ny, nx)[:, 1:-1]
                assert np.array_equal(got, ref[:, z0:z1]), (step, z0, float(np.max(np.abs(got - ref[:, z0:z1]))))
    print(f"{name}: {n} slabs equal the whole lattice bit for bit after 40 steps")


def test_slab_arguments_are_checked():
    import paper_2504_15018_gb300 as plb
    rv, rl, _ = maxwell(0.8)
    d2 = make_lattice(dict(lattice=0, dims=(16, 16, 1), precision=1), rv, rl)
    with pytest.raises(plb.PlbError) as e:
        plb.plb_slab_bind(d2.h, 0)
    assert e.value.code == plb.PLB_EUNSUPPORTED
    a = make_lattice(dict(lattice=1, dims=(16, 12, 6), precision=1), rv, rl)
    b = make_lattice(dict(lattice=1, dims=(16, 12, 6), precision=2), rv, rl)
    a.init(np.full(16 * 12 * 6, rv))
    b.init(np.full(16 * 12 * 6, rv))
    plb.plb_slab_bind(a.h, 0)
    plb.plb_slab_bind(b.h, 4)
    with pytest.raises(plb.PlbError):                      # collide before psi
        plb.plb_slab_pass(a.h, 1)
    plb.plb_slab_pass(a.h, 0)
    plb.plb_slab_pass(b.h, 0)
    with pytest.raises(plb.PlbError):                      # different precisions
        plb.plb_slab_exchange(a.h, b.h, 0)
