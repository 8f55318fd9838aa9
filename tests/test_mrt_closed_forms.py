"""The D3Q19 pair kernels relax the ten non-hydrodynamic (ghost) moments of
g = f - f^eq + F~/2 without forming g per population: the ghost moments of f^eq and of the
Guo term F~ (Sec. II) enter in closed form (collide_emit in the CUDA sources).  This checks
those closed forms against the oracle's own equilibrium, Guo bracket and d'Humieres et al.
(2002) rows on random cell states, with and without the FP16 storage shift (stored value
h = f - w rho_ref, drho = sum_i h_i).  With v = j - F/2 and P_a = u_a v_a:
  m_e(g)   = m_e(h)   + 11 drho - 19 u.v        m_eps(g) = m_eps(h) - 3 drho + 5.5 u.v
  m_pixx(g) = m_pixx(h) + P_x - (P_y + P_z)/2    m_piww(g) = m_piww(h) + (P_y - P_z)/2
  m_q(g)   = m_q(h)   + (2/3) j                 m_m(g)   = m_m(h)"""
import numpy as np
import pytest

import oracle

# rows of the oracle's D3Q19 basis: rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww,
# pxy, pyz, pxz, mx, my, mz
GHOST_ROWS = {"e": 1, "eps": 2, "qx": 4, "qy": 6, "qz": 8, "pixx": 10, "piww": 12, "mx": 16, "my": 17, "mz": 18}


@pytest.mark.parametrize("rho_ref", [0.0, 0.7, 7.2])
def test_d3q19_ghost_moments_of_g_in_closed_form(rho_ref):
    c, w = oracle.velocity_set(oracle.D3Q19)
    M, _ = oracle.mrt_matrix(oracle.D3Q19)
    rng = np.random.default_rng(11)
    for _ in range(50):
        f = w * rng.uniform(0.1, 8.0) * (1.0 + 0.2 * rng.standard_normal(19))
        F = 1e-2 * rng.standard_normal(3)
        rho = f.sum()
        j = c.T @ f
        u = (j + F / 2) / rho                                   # Eq. Momentum
        # Guo term at tau = 1 is (1 - 1/2) x bracket = F~/2
        g = f - oracle.feq(oracle.D3Q19, rho, u) + oracle.guo(oracle.D3Q19, 1.0, F, u)
        h = f - w * rho_ref
        drho = h.sum()
        P = u * (j - F / 2)
        uv = P.sum()
        mh = M @ h
        closed = {"e": mh[1] + 11 * drho - 19 * uv, "eps": mh[2] - 3 * drho + 5.5 * uv,
                  "qx": mh[4] + 2 / 3 * j[0], "qy": mh[6] + 2 / 3 * j[1], "qz": mh[8] + 2 / 3 * j[2],
                  "pixx": mh[10] + P[0] - (P[1] + P[2]) / 2, "piww": mh[12] + (P[1] - P[2]) / 2,
                  "mx": mh[16], "my": mh[17], "mz": mh[18]}
        mg = M @ g
        for name, row in GHOST_ROWS.items():
            assert abs(closed[name] - mg[row]) <= 1e-12 * (1.0 + abs(mg[row]) + rho), (name, closed[name], mg[row])


def test_closed_forms_fail_with_a_dropped_term():
    """The check is sharp: dropping the u.v term of m_e (a plausible slip) is detected."""
    c, w = oracle.velocity_set(oracle.D3Q19)
    M, _ = oracle.mrt_matrix(oracle.D3Q19)
    f = w * 1.3 * (1.0 + 0.1 * np.arange(19) / 19)
    F = np.array([0.01, -0.02, 0.005])
    rho, j = f.sum(), c.T @ f
    u = (j + F / 2) / rho
    g = f - oracle.feq(oracle.D3Q19, rho, u) + oracle.guo(oracle.D3Q19, 1.0, F, u)
    wrong = (M @ f)[1] + 11 * rho          # m_e(f) + 11 drho without -19 u.v (rho_ref = 0)
    assert abs(wrong - (M @ g)[1]) > 1e-6
