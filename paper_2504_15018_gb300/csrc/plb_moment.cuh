// D3Q19 collision carried out entirely in moment space (BGK and MRT with Guo forcing), for
// the pair kernels of FP16-shifted storage, whose fused pass is bound by arithmetic.
//
// With g = f - f^eq + Ft/2 (Ft the bracket of Eq. Guo_Forcing_Scheme), the MRT update
// f* = f - M^-1 S (m - m^eq) + M^-1 (I - S/2) M Ft of Sec. II is f* = f + Ft - M^-1 S M g.
// Row by row of the d'Humieres et al. (2002) basis M (norms n_k = |M_k|^2):
//   rho* = rho                       j* = j + F
//   m*_k = m_k + (M Ft)_k - s_k m_k(g)    for the 15 other rows (BGK: s_k = 1/tau),
// and f*_i = sum_k M_ki m*_k / n_k.  The moments of f^eq (second order) and of Ft are closed
// forms in rho, u and F; with v = j - F/2 (so rho u = j + F/2) and P_a = u_a v_a they give
//   m_e(g)    = m_e    + 11 drho - 19 u.v           (M Ft)_e    = 38 u.F
//   m_eps(g)  = m_eps  -  3 drho + 5.5 u.v          (M Ft)_eps  = -11 u.F
//   m_q(g)    = m_q    + (2/3) j                    (M Ft)_q    = -(2/3) F
//   m_3pxx(g) = m_3pxx - (2 P_x - P_y - P_z)        (M Ft)_3pxx = 2 (2 u_x F_x - u_y F_y - u_z F_z)
//   m_3pixx(g)= m_3pixx + (2 P_x - P_y - P_z) / 2   (M Ft)_3pixx = -(2 u_x F_x - u_y F_y - u_z F_z)
//   m_pww(g)  = m_pww  - (P_y - P_z)                (M Ft)_pww  = 2 (u_y F_y - u_z F_z)
//   m_piww(g) = m_piww + (P_y - P_z) / 2            (M Ft)_piww = -(u_y F_y - u_z F_z)
//   m_pxy(g)  = m_pxy  - (u_x j_y - u_y F_x / 2)    (M Ft)_pxy  = u_x F_y + u_y F_x  (and yz, xz)
//   m_m(g)    = m_m                                 (M Ft)_m    = 0
// in terms of the stored values h (h = f, or f - w rho_ref with the FP16 shift) and
// drho = sum_i h_i: the shift's moments (1, -11, 3 on rho, e, eps, zero elsewhere) cancel from
// every m(g).  The moments come from the opposite-pair sums s_r = h_i + h_i' and differences
// d_r = h_i - h_i', and the back-projection is formed as even (E_r) and odd (O_r) parts per pair,
// h*_i = E_r + O_r, h*_i' = E_r - O_r, with sums shared across velocity classes.
#pragma once
#include "plb_step.cuh"

namespace plb {

// emit(ic, v) receives the new stored value of population decltype(ic)::value.
template <int MRT, bool SHIFT, class T, class Emit>
__device__ __forceinline__ void collide_moments_d3q19(const KParams &p, const T *f, const T F[3], Emit &&emit) {
    using L = D3Q19;
    using R = typename ScalarOf<T>::type;
    const Phys<R> &q = phys<R>(p);
    static_assert(L::cx(1) == 1 && L::cy(3) == 1 && L::cz(5) == 1 && L::cx(7) == 1 && L::cy(7) == 1 &&
                      L::cx(9) == 1 && L::cy(9) == -1 && L::cx(11) == 1 && L::cz(11) == 1 && L::cx(13) == 1 &&
                      L::cz(13) == -1 && L::cy(15) == 1 && L::cz(15) == 1 && L::cy(17) == 1 && L::cz(17) == -1,
                  "pair order assumed below: 0-2 axes x, y, z; 3, 4: (1, +-1, 0); 5, 6: (1, 0, +-1); 7, 8: (0, 1, +-1)");
    // ---- moments of the stored values
    T s[9], d[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        s[r] = f[2 * r + 1] + f[2 * r + 2];
        d[r] = f[2 * r + 1] - f[2 * r + 2];
    }
    const T Dxy = s[3] + s[4], Dxz = s[5] + s[6], Dyz = s[7] + s[8];
    const T s12 = s[1] + s[2];
    const T Sax = s[0] + s12;                  // axis links
    const T Dxyz = Dxy + Dxz;
    const T Sed = Dxyz + Dyz;                  // edge links
    const T drho = f[0] + (Sax + Sed);
    const T m_e = mad(T(-30), f[0], mad(T(-11), Sax, T(8) * Sed));
    const T m_eps = mad(T(12), f[0], mad(T(-4), Sax, Sed));
    const T Tt = mad(T(-2), Dyz, Dxyz);       // Dxy + Dxz - 2 Dyz
    const T m_3pxx = mad(T(2), s[0], Tt - s12);
    const T m_3pixx = mad(T(-4), s[0], mad(T(2), s12, Tt));
    const T V = s[1] - s[2], U = Dxy - Dxz;
    const T m_pww = V + U, m_piww = mad(T(-2), V, U);
    const T m_pxy = s[3] - s[4], m_pxz = s[5] - s[6], m_pyz = s[7] - s[8];
    const T Pxy = d[3] + d[4], Qxy = d[3] - d[4];
    const T Pxz = d[5] + d[6], Qxz = d[5] - d[6];
    const T Pyz = d[7] + d[8], Qyz = d[7] - d[8];
    const T Ex = Pxy + Pxz, Ey = Qxy + Pyz, Ez = Qxz + Qyz;
    const T j[3] = {d[0] + Ex, d[1] + Ey, d[2] + Ez};
    const T m_q[3] = {mad(T(-4), d[0], Ex), mad(T(-4), d[1], Ey), mad(T(-4), d[2], Ez)};
    const T m_m[3] = {Pxy - Pxz, Pyz - Qxy, Qxz - Qyz};
    // ---- macroscopic quantities (Eqs. Density, Momentum) and tau(rho)
    const T rho = SHIFT ? drho + T(q.rho_ref) : drho;
    const T irho = fdiv(T(1), rho);
    const T u[3] = {mad(T(0.5), F[0], j[0]) * irho, mad(T(0.5), F[1], j[1]) * irho,
                    mad(T(0.5), F[2], j[2]) * irho};
    const T om = omega_of<T>(p, rho);
    const T UF[3] = {u[0] * F[0], u[1] * F[1], u[2] * F[2]};
    const T uF = UF[0] + UF[1] + UF[2];
    const T P[3] = {u[0] * mad(T(-0.5), F[0], j[0]), u[1] * mad(T(-0.5), F[1], j[1]),
                    u[2] * mad(T(-0.5), F[2], j[2])};
    const T uv = P[0] + P[1] + P[2];
    // rates: BGK relaxes every non-conserved row with omega
    const T s_e = MRT ? T(q.s_rate[1]) : om, s_eps = MRT ? T(q.s_rate[2]) : om, s_q = MRT ? T(q.s_rate[3]) : om;
    const T s_pi = MRT ? T(q.s_rate[4]) : om, s_m = MRT ? T(q.s_rate[5]) : om;
    // ---- post-collision moments over their norms, a_k = m*_k / n_k
    const T a_rho = T(1.0 / 19.0) * drho;
    T a_j[3], a_q[3], a_m[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a_j[c] = T(0.1) * (j[c] + F[c]);
        const T gq = mad(T(2.0 / 3.0), j[c], m_q[c]);
        a_q[c] = T(1.0 / 40.0) * mad(-s_q, gq, mad(T(-2.0 / 3.0), F[c], m_q[c]));
        a_m[c] = T(1.0 / 8.0) * mad(-s_m, m_m[c], m_m[c]);
    }
    const T ge = mad(T(11), drho, mad(T(-19), uv, m_e));
    const T a_e = T(1.0 / 2394.0) * mad(-s_e, ge, mad(T(38), uF, m_e));
    const T geps = mad(T(-3), drho, mad(T(5.5), uv, m_eps));
    const T a_eps = T(1.0 / 252.0) * mad(-s_eps, geps, mad(T(-11), uF, m_eps));
    const T X3 = mad(T(2), P[0], -(P[1] + P[2]));
    const T Y3 = mad(T(2), UF[0], -(UF[1] + UF[2]));
    const T a_3pxx = T(1.0 / 36.0) * mad(-om, m_3pxx - X3, mad(T(2), Y3, m_3pxx));
    const T a_3pixx = T(1.0 / 72.0) * mad(-s_pi, mad(T(0.5), X3, m_3pixx), m_3pixx - Y3);
    const T X2 = P[1] - P[2], Y2 = UF[1] - UF[2];
    const T a_pww = T(1.0 / 12.0) * mad(-om, m_pww - X2, mad(T(2), Y2, m_pww));
    const T a_piww = T(1.0 / 24.0) * mad(-s_pi, mad(T(0.5), X2, m_piww), m_piww - Y2);
    auto a_off = [&](const T &m, int a, int b) {
        // m_ab(g) = m_ab - (u_a j_b - u_b F_a / 2), (M Ft)_ab = u_a F_b + u_b F_a
        const T ubFa = u[b] * F[a];
        const T g = m - mad(T(-0.5), ubFa, u[a] * j[b]);
        return T(0.25) * mad(-om, g, m + mad(u[a], F[b], ubFa));
    };
    const T a_pxy = a_off(m_pxy, 0, 1), a_pyz = a_off(m_pyz, 1, 2), a_pxz = a_off(m_pxz, 0, 2);
    // ---- back-projection h*_i = sum_k M_ki a_k
    emit(std::integral_constant<int, 0>{}, mad(T(-30), a_e, mad(T(12), a_eps, a_rho)));
    const T Pa = mad(T(-11), a_e, mad(T(-4), a_eps, a_rho));      // axis links: rho, e, eps rows
    const T Pb = mad(T(8), a_e, a_rho + a_eps);                    // edge links
    auto pair = [&](auto rc, const T &E, const T &O) {
        constexpr int r = decltype(rc)::value;
        emit(std::integral_constant<int, 2 * r + 1>{}, E + O);
        emit(std::integral_constant<int, 2 * r + 2>{}, E - O);
    };
    pair(std::integral_constant<int, 0>{}, mad(T(2), a_3pxx, mad(T(-4), a_3pixx, Pa)), mad(T(-4), a_q[0], a_j[0]));
    {
        const T C = mad(T(2), a_3pixx, Pa - a_3pxx), Dw = mad(T(-2), a_piww, a_pww);
        pair(std::integral_constant<int, 1>{}, C + Dw, mad(T(-4), a_q[1], a_j[1]));
        pair(std::integral_constant<int, 2>{}, C - Dw, mad(T(-4), a_q[2], a_j[2]));
    }
    const T X = a_3pxx + a_3pixx, Wp = a_pww + a_piww;
    const T Jq[3] = {a_j[0] + a_q[0], a_j[1] + a_q[1], a_j[2] + a_q[2]};
    {
        const T B = (Pb + X) + Wp, O1 = Jq[0] + a_m[0], O2 = Jq[1] - a_m[1];
        pair(std::integral_constant<int, 3>{}, B + a_pxy, O1 + O2);
        pair(std::integral_constant<int, 4>{}, B - a_pxy, O1 - O2);
    }
    {
        const T B = (Pb + X) - Wp, O1 = Jq[0] - a_m[0], O2 = Jq[2] + a_m[2];
        pair(std::integral_constant<int, 5>{}, B + a_pxz, O1 + O2);
        pair(std::integral_constant<int, 6>{}, B - a_pxz, O1 - O2);
    }
    {
        const T B = mad(T(-2), X, Pb), O1 = Jq[1] + a_m[1], O2 = Jq[2] - a_m[2];
        pair(std::integral_constant<int, 7>{}, B + a_pyz, O1 + O2);
        pair(std::integral_constant<int, 8>{}, B - a_pyz, O1 - O2);
    }
}

}  // namespace plb
