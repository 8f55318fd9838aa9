"""The oracle's FP64 arithmetic against a 50-digit replay.

A separate implementation of the time step in mpmath at 50 significant digits (density,
Peng-Robinson pressure and psi of Eq. Interaction_Potential, the M1 / M2 stencils and the
Shan-Chen force with the eps / kappa terms of Eq. interactionForce, Guo forcing, BGK or MRT
collision, push streaming with halfway bounce-back and mirrored psi at walls), started from the
same FP64 inputs, agrees with the C oracle to 1e-14 relative on every population after 20
steps: the oracle loses no accuracy beyond FP64 rounding, which the 1e-12 parity bound of the
FP64 GPU path relies on.  Both implementations read the paper the same way (the tests of
test_oracle_step.py pin that reading); this test pins the rounding only."""
import numpy as np
import mpmath as mp
import pytest

import oracle
from oracle import params as pp
from paper_2504_15018_gb300 import inputs

PR = dict(a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.327)


def _velocities(lattice):
    if lattice == oracle.D2Q9:
        vel = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]
        w = {0: mp.mpf(4) / 9, 1: mp.mpf(1) / 9, 2: mp.mpf(1) / 36}
        om = {1: mp.mpf(1) / 3, 2: mp.mpf(1) / 12}
    else:
        vel = [(0, 0, 0)] + [v for a in range(3) for v in (tuple(int(k == a) for k in range(3)),
                                                           tuple(-int(k == a) for k in range(3)))]
        for a, b in ((0, 1), (0, 2), (1, 2)):
            for sa in (1, -1):
                for sb in (1, -1):
                    v = [0, 0, 0]
                    v[a], v[b] = sa, sb
                    vel.append(tuple(v))
        w = {0: mp.mpf(1) / 3, 1: mp.mpf(1) / 18, 2: mp.mpf(1) / 36}
        om = {1: mp.mpf(1) / 6, 2: mp.mpf(1) / 12}
    c2 = [sum(x * x for x in v) for v in vel]
    return vel, [w[k] for k in c2], [om.get(k, mp.mpf(0)) for k in c2]


def _basis(lattice, vel):
    """Rows of the orthogonal MRT bases (Lallemand & Luo 2000; d'Humieres et al. 2002) and the
    kind of each row: 'e', 'eps', 'q', 'pi', 'm', or None (stress and conserved rows: 1/tau)."""
    rows = []
    for x, y, z in vel:
        c2 = x * x + y * y + z * z
        if lattice == oracle.D2Q9:
            rows.append([1, -4 + 3 * c2, 4 - mp.mpf(21) / 2 * c2 + mp.mpf(9) / 2 * c2 * c2, x, (-5 + 3 * c2) * x, y,
                         (-5 + 3 * c2) * y, x * x - y * y, x * y])
        else:
            rows.append([1, 19 * c2 - 30, (21 * c2 * c2 - 53 * c2 + 24) / mp.mpf(2), x, (5 * c2 - 9) * x, y,
                         (5 * c2 - 9) * y, z, (5 * c2 - 9) * z, 3 * x * x - c2, (3 * c2 - 5) * (3 * x * x - c2),
                         y * y - z * z, (3 * c2 - 5) * (y * y - z * z), x * y, y * z, x * z, (y * y - z * z) * x,
                         (z * z - x * x) * y, (x * x - y * y) * z])
    M = mp.matrix(rows).T
    kinds = ([None, "e", "eps", None, "q", None, "q", None, None] if lattice == oracle.D2Q9 else
             [None, "e", "eps", None, "q", None, "q", None, "q", None, "pi", None, "pi", None, None, None,
              "m", "m", "m"])
    return M, kinds


def _replay(lattice, dims, rho0, *, tau, kappa, eps, G, fext, wall, mrt, rates, T, steps):
    mp.mp.dps = 50
    vel, W, OM = _velocities(lattice)
    q, d = len(vel), (2 if lattice == oracle.D2Q9 else 3)
    opp = [vel.index(tuple(-x for x in v)) for v in vel]
    nx, ny, nz = dims
    n = nx * ny * nz
    idx = lambda x, y, z: x + nx * (y + ny * z)
    a, b, R, omg, T = (mp.mpf(v) for v in (PR["a"], PR["b"], PR["R"], PR["omega"], T))
    Tc = mp.mpf(0.0778) * a / (mp.mpf(0.45724) * b * R)
    m_om = mp.mpf(0.37464) + mp.mpf(1.54226) * omg - mp.mpf(0.26992) * omg ** 2
    alpha = (1 + m_om * (1 - mp.sqrt(T / Tc))) ** 2
    pres = lambda r: r * R * T / (1 - b * r) - a * alpha * r ** 2 / (1 + 2 * b * r - (b * r) ** 2)
    tau, kappa, eps, G = (mp.mpf(v) for v in (tau, kappa, eps, G))
    fext = [mp.mpf(v) for v in fext]
    if mrt:
        M, kinds = _basis(lattice, vel)
        norm2 = [sum(M[k, i] ** 2 for i in range(q)) for k in range(q)]
        rate = [mp.mpf(rates["s_" + k]) if k else 1 / tau for k in kinds]
    f = [[W[i] * mp.mpf(float(rho0[s])) for i in range(q)] for s in range(n)]
    for _ in range(steps):
        rho = [sum(fs) for fs in f]
        psi = [mp.sqrt(2 * (pres(r) - r / 3) / G) for r in rho]
        fnew = [[None] * q for _ in range(n)]
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    s = idx(x, y, z)
                    fs = f[s]

                    def psi_at(v):
                        yn = y + v[1]
                        if wall:
                            yn = -1 - yn if yn < 0 else (2 * ny - 1 - yn if yn >= ny else yn)
                        else:
                            yn %= ny
                        return psi[idx((x + v[0]) % nx, yn, (z + v[2]) % nz)]
                    M1 = [mp.mpf(0)] * 3
                    M2 = [[mp.mpf(0)] * 3 for _ in range(3)]
                    sc = [mp.mpf(0)] * 3
                    for i, v in enumerate(vel):
                        pn = psi_at(v)
                        for al in range(3):
                            M1[al] += 3 * W[i] * pn * v[al]
                            sc[al] += OM[i] * pn * v[al]
                            for be in range(3):
                                M2[al][be] += 9 * W[i] * pn * (v[al] * v[be] - (mp.mpf(1) / 3 if al == be else 0))
                    tr = sum(M2[be][be] for be in range(d))
                    F = [mp.mpf(0)] * 3
                    for al in range(d):
                        m21 = sum(M1[be] * M2[al][be] for be in range(d))
                        F[al] = (-G * psi[s] * sc[al] - G / 12 * (-3 * eps + 2 * kappa - 2) * m21
                                 + G / 6 * (kappa - 1) * M1[al] * tr + fext[al])
                    r = rho[s]
                    u = [(sum(fs[i] * vel[i][al] for i in range(q)) + F[al] / 2) / r for al in range(3)]
                    uu = sum(x_ * x_ for x_ in u)
                    uF = sum(u[al] * F[al] for al in range(3))
                    feq, Ft = [], []
                    for i, v in enumerate(vel):
                        cu = sum(v[al] * u[al] for al in range(3))
                        cF = sum(v[al] * F[al] for al in range(3))
                        feq.append(W[i] * r * (1 + 3 * cu + mp.mpf(9) / 2 * cu * cu - mp.mpf(3) / 2 * uu))
                        Ft.append(W[i] * (3 * cF + 9 * cu * cF - 3 * uF))
                    if not mrt:
                        post = [fs[i] - (fs[i] - feq[i]) / tau + (1 - 1 / (2 * tau)) * Ft[i] for i in range(q)]
                    else:
                        corr = []
                        for k in range(q):
                            mneq = sum(M[k, i] * (fs[i] - feq[i]) for i in range(q))
                            mf = sum(M[k, i] * Ft[i] for i in range(q))
                            corr.append(((1 - rate[k] / 2) * mf - rate[k] * mneq) / norm2[k])
                        post = [fs[i] + sum(M[k, i] * corr[k] for k in range(q)) for i in range(q)]
                    for i, v in enumerate(vel):
                        yn = y + v[1]
                        if wall and (yn < 0 or yn >= ny):
                            fnew[s][opp[i]] = post[i]
                        else:
                            fnew[idx((x + v[0]) % nx, yn % ny, (z + v[2]) % nz)][i] = post[i]
        f = fnew
    return vel, f


CASES = {
    "d2q9_bgk_periodic": dict(lattice=oracle.D2Q9, dims=(6, 6, 1), wall=False, mrt=False, tau=0.9, kappa=1.3),
    "d2q9_mrt_walls": dict(lattice=oracle.D2Q9, dims=(6, 6, 1), wall=True, mrt=True, tau=1.0, kappa=0.8),
    "d3q19_bgk_periodic": dict(lattice=oracle.D3Q19, dims=(4, 4, 4), wall=False, mrt=False, tau=0.8, kappa=1.1),
    "d3q19_mrt_walls": dict(lattice=oracle.D3Q19, dims=(4, 4, 4), wall=True, mrt=True, tau=1.0, kappa=1.0),
}
RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.3, s_m=1.5)


@pytest.mark.parametrize("name", list(CASES))
def test_oracle_matches_a_50_digit_replay(name):
    c = CASES[name]
    T = 0.8 * pp.pr_Tc(PR["a"], PR["b"])
    x, y, z = inputs.grid_coords(c["dims"])
    rho0 = 7.3 + 0.2 * np.sin(2 * np.pi * x / c["dims"][0]) * np.cos(2 * np.pi * (y + 0.3) / c["dims"][1]) \
        + 0.05 * np.sin(2 * np.pi * z / c["dims"][2])
    fext = (1e-4, -5e-5, 2e-5) if c["lattice"] == oracle.D3Q19 else (1e-4, -5e-5, 0.0)
    steps = 20
    P = oracle.make_params(c["lattice"], c["dims"], wall_y=c["wall"], eos=dict(kind="pr", **PR, T=T), G=-1.0,
                           eps=2.0, kappa=c["kappa"], tau=c["tau"], mrt=c["mrt"], rates=RATES, fext=fext)
    fo = oracle.run(P, oracle.init(P, rho0), steps)
    vel, fm = _replay(c["lattice"], c["dims"], rho0, tau=c["tau"], kappa=c["kappa"], eps=2.0, G=-1.0, fext=fext,
                      wall=c["wall"], mrt=c["mrt"], rates=RATES, T=T, steps=steps)
    oc, _ = oracle.velocity_set(c["lattice"])
    perm = [vel.index(tuple(int(k) for k in v)) for v in oc.tolist()]      # oracle direction -> replay index
    ref = np.array([[float(fm[s][perm[j]]) for j in range(len(perm))] for s in range(len(fm))])
    err = float(np.max(np.abs(fo - ref) / np.abs(ref)))
    moved = float(np.max(np.abs(ref - oracle.init(P, rho0)) / np.abs(ref)))
    print(f"{name}: max rel err vs 50-digit replay {err:.2e} (populations moved {moved:.1e})")
    assert moved > 1e-6                 # the state evolved: forces and collisions were exercised
    assert err <= 1e-14
