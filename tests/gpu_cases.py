"""Shared helpers of the GPU tests: one parity case runs the same seeded input through
the oracle and through the C ABI, and maps directions by velocity vector."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import params as pp
from paper_2504_15018_gb300 import inputs

PR_A, PR_B, PR_OMEGA = 2.0 / 49.0, 2.0 / 21.0, 0.327
TC = pp.pr_Tc(PR_A, PR_B)


def maxwell(t_ratio):
    return pp.pr_maxwell(PR_A, PR_B, 1.0, PR_OMEGA, t_ratio * TC)


def direction_map(lattice):
    """perm[i_lib] = oracle direction with the same velocity vector."""
    import paper_2504_15018_gb300 as plb
    c, _ = plb.plb_velocity_set(lattice)
    oc, _ = oracle.velocity_set(lattice)
    perm = []
    for v in c.tolist():
        perm.append([tuple(o) for o in oc.tolist()].index(tuple(v)))
    return np.array(perm)


def case_fields(case):
    """Seeded initial density (and velocity) of a parity case."""
    lattice, dims = case["lattice"], case["dims"]
    if case.get("eos", "pr") == "pr":
        rv, rl, _ = maxwell(case.get("t_ratio", 0.8))
    else:
        rv, rl = case["rho_v"], case["rho_l"]
    shape = case.get("shape", "droplet")
    nx, ny, nz = dims
    if shape == "droplet":
        center = (nx / 2 - 0.3, ny / 2 + 0.2) if lattice == 0 else (nx / 2 - 0.3, ny / 2 + 0.2, nz / 2 + 0.1)
        rho = inputs.droplet(dims, center, min(d for d in dims if d > 1) / 4, rv, rl, 3.0,
                             periodic=not case.get("wall", False))
    else:
        rho = inputs.slab(dims, 1, ny // 4, 3 * ny // 4, rl, rv, 3.0, periodic=not case.get("wall", False))
    rho = inputs.add_noise(rho, inputs.MASTER_SEED + 100, 1e-4)
    u0 = None
    if case.get("u0"):
        d = 2 if lattice == 0 else 3
        u0 = np.zeros((d, rho.size))
        for a, v in enumerate(case["u0"][:d]):
            u0[a] = v
    return rho, u0, rv, rl


def oracle_params(case, rv, rl):
    if case.get("eos", "pr") == "pr":
        eos = dict(kind="pr", a=PR_A, b=PR_B, R=1.0, omega=PR_OMEGA, T=case.get("t_ratio", 0.8) * TC)
    else:
        eos = dict(kind="paper", rho_v=rv, rho_l=rl, P=case["P"])
    return oracle.make_params(case["lattice"], case["dims"], wall_y=case.get("wall", False), eos=eos,
                              G=case.get("G", -1.0), eps=case.get("eps", 2.0), kappa=case.get("kappa", 1.0),
                              tau=case.get("tau", 1.0), tau_v=case.get("tau_v"), tau_rho=(rv, rl),
                              mrt=case.get("mrt", False), rates=case.get("rates"), fext=case.get("fext", (0, 0, 0)),
                              p_scale=case.get("p_scale", 1.0), wall_rho=case.get("wall_rho", 0.0))


def make_lattice(case, rv, rl):
    import paper_2504_15018_gb300 as plb
    if case.get("eos", "pr") == "pr":
        eos = plb.pr_eos(case.get("t_ratio", 0.8), p_scale=case.get("p_scale", 1.0))
    else:
        eos = plb.paper_eos(rv, rl, case["P"], p_scale=case.get("p_scale", 1.0))
    kw = dict(kappa=case.get("kappa", 1.0), precision=case.get("precision", plb.PLB_FP64),
              collision=plb.PLB_MRT if case.get("mrt") else plb.PLB_BGK, wall_y=int(case.get("wall", False)),
              body_force=case.get("fext", (0, 0, 0)))
    if case.get("tau_v") is not None:
        kw.update(tau_v=case["tau_v"], tau_rho_v=rv, tau_rho_l=rl)
    if case.get("rates"):
        kw.update(case["rates"])
    if case.get("rho_ref"):
        kw.update(rho_ref=case["rho_ref"])
    if case.get("fp16_rounding"):
        kw.update(fp16_rounding=case["fp16_rounding"])
    if case.get("streaming"):
        kw.update(streaming=case["streaming"])
    if case.get("wall_rho"):
        kw.update(wall_rho=case["wall_rho"])
    return plb.Lattice(case["lattice"], case["dims"], eos, tau=case.get("tau", 1.0), G=case.get("G", -1.0),
                       eps=case.get("eps", 2.0), opts=plb.make_opts(**kw))


def run_both(case, steps):
    """(oracle f (N, Q) in library direction order transposed to (Q, N), library f (Q, N), lattice)."""
    rho, u0, rv, rl = case_fields(case)
    P = oracle_params(case, rv, rl)
    fo = oracle.run(P, oracle.init(P, rho, u0), steps)
    lat = make_lattice(case, rv, rl)
    lat.init(rho, u0)
    lat.step(steps)
    lat.status()
    fl = lat.populations()
    perm = direction_map(case["lattice"])
    return fo[:, perm].T.copy(), fl, lat, P


def max_rel_err(ref, got):
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)))
