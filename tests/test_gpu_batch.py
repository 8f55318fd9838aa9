"""Batched lattices in one persistent launch (plb_batch_*): every instance of a batch must
evolve exactly as the same lattice stepped alone (the per-cell update is the same code), for
uneven sizes, odd and even nx (two-cell and one-cell paths), walls, per-instance EOS and tau,
both AA parities, graph replay and autotuned tilings.  A barrier whose arrivals are withheld
must end in PLB_ETIMEOUT, not a hang."""
import numpy as np
import pytest

import oracle
from gpu_cases import maxwell, oracle_params, direction_map
from paper_2504_15018_gb300 import inputs

pytestmark = pytest.mark.gpu

RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.3, s_m=1.5)


def _instances(lattice, specs, precision, mrt):
    import paper_2504_15018_gb300 as plb
    out, fields = [], []
    for k, sp in enumerate(specs):
        t = sp.get("t_ratio", 0.8)
        rv, rl, _ = maxwell(t)
        kw = dict(precision=precision, collision=plb.PLB_MRT if mrt else plb.PLB_BGK,
                  wall_y=int(sp.get("wall", False)), kappa=sp.get("kappa", 1.0),
                  body_force=sp.get("fext", (0.0, 0.0, 0.0)), **RATES)
        if sp.get("tau_v"):
            kw.update(tau_v=sp["tau_v"], tau_rho_v=rv, tau_rho_l=rl)
        if sp.get("wall_rho"):
            kw.update(wall_rho=sp["wall_rho"])
        opts = plb.make_opts(**kw)
        dims = sp["dims"]
        out.append(plb.make_instance(dims, plb.pr_eos(t), tau=sp.get("tau", 1.0), opts=opts))
        if sp.get("shape") == "slab":
            rho = inputs.slab(dims, 1, dims[1] // 4, 3 * dims[1] // 4, rl, rv, 3.0, periodic=not sp.get("wall"))
        else:
            c = [d / 2 for d in dims[:(2 if lattice == 0 else 3)]]
            rho = inputs.droplet(dims, c, min(dims[:(2 if lattice == 0 else 3)]) / 4, rv, rl, 3.0)
        rho = inputs.add_noise(rho, inputs.MASTER_SEED + 200 + k, 1e-4)
        u0 = None
        if sp.get("u0"):
            d = 2 if lattice == 0 else 3
            u0 = np.zeros((d, rho.size))
            for a in range(d):
                u0[a] = sp["u0"][a]
        fields.append((rho, u0))
    return out, fields


def _alone(lattice, inst, rho, u0, steps):
    import paper_2504_15018_gb300 as plb
    lat = plb.Lattice(lattice, tuple(inst.dims), inst.eos, inst.tau, inst.G, inst.eps, opts=inst.opts)
    lat.init(rho, u0)
    lat.step(steps)
    return lat.populations()


D2_SPECS = [
    dict(dims=(64, 48, 1), t_ratio=0.72),
    dict(dims=(37, 29, 1), t_ratio=0.85, kappa=1.3),                       # odd nx: one cell per thread
    dict(dims=(96, 20, 1), t_ratio=0.8, wall=True, shape="slab", fext=(1e-5, 0, 0), tau_v=1.2),
    dict(dims=(34, 66, 1), t_ratio=0.9, u0=(0.03, -0.02)),
    dict(dims=(2, 9, 1), t_ratio=0.8, wall=True, shape="slab"),
]


@pytest.mark.parametrize("precision,mrt", [(1, False), (1, True), (2, False), (0, True)])
def test_batch_matches_instances_stepped_alone(precision, mrt):
    import paper_2504_15018_gb300 as plb
    insts, fields = _instances(0, D2_SPECS, precision, mrt)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    b.configure(tile_cells=256)          # several tiles per instance
    b.step(7)
    b.step(6)                            # odd then even launch lengths; second call replays no graph
    b.step(7)                            # graph replay of the 7-step launch
    b.status()
    for k, (rho, u0) in enumerate(fields):
        want = _alone(0, insts[k], rho, u0, 20)
        got = b.populations(k)
        assert np.array_equal(got, want), (k, float(np.max(np.abs(got - want))))


def test_batch_d3q19_mrt_walls():
    import paper_2504_15018_gb300 as plb
    specs = [dict(dims=(16, 12, 10), wall=True, shape="slab", fext=(2e-6, 0, 0)),
             dict(dims=(13, 11, 9), t_ratio=0.75),
             dict(dims=(20, 8, 6), u0=(0.02, 0.0, -0.01), t_ratio=0.85)]
    insts, fields = _instances(1, specs, 1, True)
    b = plb.Batch(plb.PLB_D3Q19, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    b.configure(tile_cells=200)
    b.step(9)
    b.status()
    for k, (rho, u0) in enumerate(fields):
        assert np.array_equal(b.populations(k), _alone(1, insts[k], rho, u0, 9)), k


def test_batch_fp64_instance_against_oracle():
    import paper_2504_15018_gb300 as plb
    insts, fields = _instances(0, D2_SPECS[:3], 0, True)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    b.step(300)
    b.status()
    k = 2
    spec = D2_SPECS[k]
    rv, rl, _ = maxwell(spec["t_ratio"])
    case = dict(lattice=0, dims=spec["dims"], wall=True, mrt=True, rates=RATES, fext=spec["fext"], tau_v=1.2,
                t_ratio=spec["t_ratio"])
    P = oracle_params(case, rv, rl)
    ref = oracle.run(P, oracle.init(P, fields[k][0]), 300)[:, direction_map(0)].T
    got = b.populations(k)
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-12


def test_autotune_picks_a_valid_tiling_and_keeps_the_dynamics():
    import paper_2504_15018_gb300 as plb
    insts, fields = _instances(0, D2_SPECS, 1, False)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    before = plb.plb_batch_launch_counts(b.b)
    tile, bps, ms = b.autotune(2)
    assert tile in (512, 1024, 2048, 4096, 8192, 16384) and 1 <= bps <= 4 and ms > 0
    # every candidate (6 tile sizes x each resident count up to the occupancy limit, at most 4)
    # runs 2 warm-up and 2 timed steps, two plb_batch_step(2) calls: its new tiling drops the
    # graphs, so the warm-up call captures one and the timed call replays it
    after = plb.plb_batch_launch_counts(b.b)
    calls = (after["graph_launches"] + after["direct_launches"]) - (before["graph_launches"] +
                                                                    before["direct_launches"])
    ncand = calls // 2
    assert calls == 2 * ncand and ncand % 6 == 0 and 1 <= ncand // 6 <= 4, (before, after)
    assert plb.plb_batch_time(b.b) == ncand * (2 + 2)
    assert after["graph_captures"] - before["graph_captures"] == ncand, (before, after)
    assert after["direct_launches"] == before["direct_launches"], (before, after)
    b.step(3)
    b.status()
    total = plb.plb_batch_time(b.b)
    for k, (rho, u0) in enumerate(fields):
        assert np.array_equal(b.populations(k), _alone(0, insts[k], rho, u0, total)), k


def test_steps_are_captured_once_and_replayed_as_graphs():
    """On the batch's own (non-default) stream, the first plb_batch_step(n) for a given n is
    captured and instantiated as a CUDA graph, later calls with the same n replay it, and a new
    n is captured once more; nothing is launched directly.  Replays give the same populations
    as lone lattices stepped by plb_step."""
    import paper_2504_15018_gb300 as plb
    insts, fields = _instances(0, D2_SPECS[:3], 1, False)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    assert plb.plb_batch_launch_counts(b.b) == {"graph_captures": 0, "graph_launches": 0, "direct_launches": 0}
    for _ in range(3):
        b.step(4)
    b.step(1)
    b.step(4)
    b.status()
    assert plb.plb_batch_launch_counts(b.b) == {"graph_captures": 2, "graph_launches": 5, "direct_launches": 0}
    for k, (rho, u0) in enumerate(fields):
        assert np.array_equal(b.populations(k), _alone(0, insts[k], rho, u0, 17)), k


def test_withheld_barrier_arrival_times_out_with_an_error():
    import paper_2504_15018_gb300 as plb
    insts, fields = _instances(0, D2_SPECS[:2], 1, False)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    b.configure(spin_limit=2000)            # ~1 ms of polling
    plb.plb_batch_withhold_arrivals(b.b, 1)
    b.step(3)
    with pytest.raises(plb.PlbError) as e:
        b.status()
    assert e.value.code == plb.PLB_ETIMEOUT
    plb.plb_batch_reset_error(b.b)
    for k, (rho, u0) in enumerate(fields):   # the context is still usable
        b.init(k, rho, u0)
    b.configure(spin_limit=0)
    b.step(4)
    b.status()
    for k, (rho, u0) in enumerate(fields):
        assert np.array_equal(b.populations(k), _alone(0, insts[k], rho, u0, 4)), k


def test_views_refuse_stepping():
    import paper_2504_15018_gb300 as plb
    insts, fields = _instances(0, D2_SPECS[:1], 1, False)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    b.init(0, *fields[0])
    view = plb.plb_batch_instance(b.b, 0)
    with pytest.raises(plb.PlbError) as e:
        plb.plb_step(view, 1)
    assert e.value.code == plb.PLB_EINVAL


def test_batch_init_physical_matches_a_single_lattice():
    import paper_2504_15018_gb300 as plb
    insts, fields = _instances(0, D2_SPECS[:4], 1, True)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0, physical=True)
    b.step(5)
    b.status()
    for k, (rho, u0) in enumerate(fields):
        lat = plb.Lattice(0, tuple(insts[k].dims), insts[k].eos, insts[k].tau, insts[k].G, insts[k].eps,
                          opts=insts[k].opts)
        lat.init(rho, u0, physical=True)
        lat.step(5)
        assert np.array_equal(b.populations(k), lat.populations()), k


def _batch96():
    """The 96 uneven D2Q9 instances of the batched workload (FP32, MRT, tau = 1), as bench.py
    builds them."""
    import paper_2504_15018_gb300 as plb
    desc = inputs.batched_d2q9_instances(96)
    insts, fields = [], []
    for d in desc:
        side = d["side"]
        eos = plb.pr_eos(d["T_over_Tc"])
        rv, rl, _ = plb.plb_solve_params(eos)
        opts = plb.make_opts(precision=plb.PLB_FP32, collision=plb.PLB_MRT, s_e=1.19, s_eps=1.4, s_q=1.2,
                             s_pi=1.4, s_m=1.98)
        insts.append(plb.make_instance((side, side, 1), eos, tau=1.0, opts=opts))
        dims = (side, side, 1)
        u0 = None
        if d["kind"] == "planar":
            rho = inputs.slab(dims, 1, side // 4, 3 * side // 4, rl, rv, 4.0)
        else:
            rho = inputs.droplet(dims, (side / 2, side / 2), d["radius"], rv, rl, 4.0)
            if d["kind"] == "translating":
                u0 = np.zeros((2, side * side))
                u0[0], u0[1] = d["velocity"]
        fields.append((rho, u0))
    return desc, insts, fields


def _centroid(rho, side, floor):
    """Periodic (circular-mean) centroid of the density above floor, per axis."""
    m = np.clip(rho.reshape(side, side) - floor, 0.0, None)
    ang = 2 * np.pi * np.arange(side) / side
    out = []
    for w in (m.sum(axis=0), m.sum(axis=1)):            # x then y
        out.append(np.arctan2((w * np.sin(ang)).sum(), (w * np.cos(ang)).sum()) * side / (2 * np.pi))
    return np.array(out)


def test_batch96_workload_matches_lone_instances_and_translates_droplets():
    """The full 96-instance workload in one batch, 1000 steps: the smallest and largest
    instances and one of each kind evolve bit for bit as when stepped alone, and every
    translating droplet's centroid moves by U t (within 2 % of the distance travelled plus a
    quarter cell: the Galilean error of the interface)."""
    import paper_2504_15018_gb300 as plb
    desc, insts, fields = _batch96()
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    b.configure(tile_cells=1024)
    steps = 1000
    b.step(steps)
    b.status()
    sides = [d["side"] for d in desc]
    sample = {int(np.argmin(sides)), int(np.argmax(sides))}
    for kind in ("static", "translating", "planar"):
        sample.add(next(k for k, d in enumerate(desc) if d["kind"] == kind))
    for k in sorted(sample):
        assert np.array_equal(b.populations(k), _alone(0, insts[k], *fields[k], steps)), k
    checked = 0
    for k, d in enumerate(desc):
        if d["kind"] != "translating" or d["radius"] < 10:
            continue
        side = d["side"]
        rv, rl, _ = plb.plb_solve_params(insts[k].eos)
        floor = 0.5 * (rv + rl)
        c0 = _centroid(fields[k][0], side, floor)
        rho = b.moments(k)[0]
        c1 = _centroid(rho, side, floor)
        want = np.array(d["velocity"]) * steps
        err = np.abs((c1 - c0 - want + side / 2) % side - side / 2).max()
        assert err < 0.02 * np.abs(want).max() + 0.25, (k, c1 - c0, want)
        checked += 1
    assert checked >= 3


def test_batch_with_wetting_walls_matches_instances_stepped_alone():
    """Instances with wetting walls (the wall rows of their psi fields filled at creation) next
    to neutral-wall and periodic ones."""
    import paper_2504_15018_gb300 as plb
    specs = [dict(dims=(40, 24, 1), wall=True, shape="slab", wall_rho=1.2, fext=(1e-5, 0, 0)),
             dict(dims=(37, 20, 1), wall=True, shape="slab", wall_rho=0.6, t_ratio=0.75),
             dict(dims=(32, 32, 1), wall=True, shape="slab"),
             dict(dims=(30, 26, 1), t_ratio=0.85)]
    insts, fields = _instances(0, specs, 1, True)
    b = plb.Batch(plb.PLB_D2Q9, insts)
    for k, (rho, u0) in enumerate(fields):
        b.init(k, rho, u0)
    b.configure(tile_cells=256)
    b.step(11)
    b.status()
    for k, (rho, u0) in enumerate(fields):
        assert np.array_equal(b.populations(k), _alone(0, insts[k], rho, u0, 11)), k
