// Plain FP64 evaluation of the per-cell arithmetic of one P-LBM step (Sec. II): every
// quantity is formed term by term in the order the equations write it, with one rounding
// per product and per sum (the FP64 kernels are compiled with -fmad=false), so that two
// correct FP64 evaluations of the step round identically.
//
//  - Eq. Density / Momentum: rho = sum_i f_i, rho u = sum_i f_i c_i + F/2, sums over the
//    velocities in the order of Eq. VelocitySet (D2Q9); D3Q19, which the paper does not
//    give, uses the storage order (rest, the six axis links, the twelve edge links).
//  - Eq. Interaction_Potential: psi = sqrt(2 (p_EOS - rho/3) / G).
//  - M1_a = sum_i w_i psi(x + c_i) c_ia / c_s^2, M2_ab = sum_i w_i psi(x + c_i)
//    (c_ia c_ib - c_s^2 d_ab) / c_s^4 (Sec. II), with 1/c_s^2 = 3 and 1/c_s^4 = 9 exact.
//  - Eq. Shan_Chen_Force and Eq. interactionForce (eps term read as in Eq.
//    New_Pressure_Tensor: -G/12 (2 kappa - 2 - 3 eps)).
//  - Eq. Single_Phase_EDF, Eq. Guo_Forcing_Scheme, Eq. LBE (BGK), and its moment-space
//    form f* = f - M^-1 S M (f - f^eq) + M^-1 (I - S/2) M Ft (MRT; bases of Lallemand & Luo
//    2000 for D2Q9 and d'Humieres et al. 2002 for D3Q19, every row of M evaluated, the
//    conserved rows relaxed with 1/tau like the stress rows).
// Zero terms (a zero velocity component or basis coefficient) are skipped: adding an exact
// zero to a sum that starts at +0 changes no bit.
#pragma once
#include "plb_device.cuh"

namespace plb {
namespace plain {

constexpr double CS2 = 1.0 / 3.0;   // c_s^2 (Eq. VelocitySet); 1/c_s^2 = 3, 1/c_s^4 = 9

// Storage slot of the n-th velocity in the summation order.
template <class L> struct Order;
template <> struct Order<D2Q9> {
    // Eq. VelocitySet: rest, (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1)
    __host__ __device__ static constexpr int slot(int n) {
        constexpr int t[9] = {0, 1, 3, 2, 4, 5, 8, 6, 7};
        return t[n];
    }
};
template <> struct Order<D3Q19> {
    __host__ __device__ static constexpr int slot(int n) { return n; }
};

template <class L> __host__ __device__ constexpr int cc(int n, int a) {
    return a == 0 ? L::cx(Order<L>::slot(n)) : (a == 1 ? L::cy(Order<L>::slot(n)) : L::cz(Order<L>::slot(n)));
}

// Shan-Chen weights omega(|c|^2) of Eq. Shan_Chen_Force (D3Q19: 3 w_i).
template <class L> __host__ __device__ constexpr double omega_sc(int n) {
    const int c2 = cc<L>(n, 0) * cc<L>(n, 0) + cc<L>(n, 1) * cc<L>(n, 1) + cc<L>(n, 2) * cc<L>(n, 2);
    if (c2 == 0) return 0.0;
    if (L::Q == 9) return c2 == 1 ? 1.0 / 3.0 : 1.0 / 12.0;
    return c2 == 1 ? 1.0 / 6.0 : 1.0 / 12.0;
}

// c_a c_b - c_s^2 d_ab.
template <class L> __host__ __device__ constexpr double cc2(int n, int a, int b) {
    return (double)(cc<L>(n, a) * cc<L>(n, b)) - (a == b ? CS2 : 0.0);
}

// Rows of the orthogonal moment bases, all Q of them, at velocity n of the summation order.
template <class L> __host__ __device__ constexpr double basis(int k, int n) {
    const double x = cc<L>(n, 0), y = cc<L>(n, 1), z = cc<L>(n, 2), c2 = x * x + y * y + z * z;
    if (L::Q == 9) {
        // rho, e, eps, jx, qx, jy, qy, pxx, pxy
        return k == 0 ? 1.0
             : k == 1 ? -4.0 + 3.0 * c2
             : k == 2 ? 4.0 - 10.5 * c2 + 4.5 * c2 * c2
             : k == 3 ? x
             : k == 4 ? (-5.0 + 3.0 * c2) * x
             : k == 5 ? y
             : k == 6 ? (-5.0 + 3.0 * c2) * y
             : k == 7 ? x * x - y * y
                      : x * y;
    }
    // rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz
    return k == 0 ? 1.0
         : k == 1 ? 19.0 * c2 - 30.0
         : k == 2 ? (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0
         : k == 3 ? x
         : k == 4 ? (5.0 * c2 - 9.0) * x
         : k == 5 ? y
         : k == 6 ? (5.0 * c2 - 9.0) * y
         : k == 7 ? z
         : k == 8 ? (5.0 * c2 - 9.0) * z
         : k == 9 ? 3.0 * x * x - c2
         : k == 10 ? (3.0 * c2 - 5.0) * (3.0 * x * x - c2)
         : k == 11 ? y * y - z * z
         : k == 12 ? (3.0 * c2 - 5.0) * (y * y - z * z)
         : k == 13 ? x * y
         : k == 14 ? y * z
         : k == 15 ? x * z
         : k == 16 ? (y * y - z * z) * x
         : k == 17 ? (z * z - x * x) * y
                   : (x * x - y * y) * z;
}

template <class L> __host__ __device__ constexpr double basis_norm2(int k) {
    double s = 0.0;
    for (int n = 0; n < L::Q; ++n) s += basis<L>(k, n) * basis<L>(k, n);
    return s;
}

// Relaxation rate of row k: 0 = 1/tau (conserved and stress rows), else the Phys::s_rate kind.
template <class L> __host__ __device__ constexpr int rate_kind(int k) {
    if (L::Q == 9) return k == 1 ? 1 : k == 2 ? 2 : (k == 4 || k == 6) ? 3 : 0;
    return k == 1 ? 1 : k == 2 ? 2 : (k == 4 || k == 6 || k == 8) ? 3 : (k == 10 || k == 12) ? 4
         : (k >= 16) ? 5 : 0;
}

// Pressure of the EOS times p_scale: Peng & Robinson (1976) or Eq. EOS, as written.
__host__ __device__ inline double pressure(const PlainPhys &q, int eos_kind, double rho) {
    double pr;
    if (eos_kind == 0) {
        const double br = q.b * rho;
        pr = rho * q.R * q.T / (1.0 - br) - q.a_alpha * rho * rho / (1.0 + 2.0 * br - br * br);
    } else {
        const double sr = sqrt(rho);
        pr = q.P * (2.0 * rho * rho * rho + q.rv_2rl * rho * rho - q.sv3 * rho * rho * sr + q.sv2rl * rho * sr +
                    q.svrlrl * sr);
    }
    return q.p_scale * pr;
}

// The argument 2 (p - rho/3) / G of the square root of Eq. Interaction_Potential.
__host__ __device__ inline double psi_arg(const PlainPhys &q, int eos_kind, double rho) {
    return 2.0 * (pressure(q, eos_kind, rho) - rho / 3.0) / q.G;
}

// rho of Eq. Density.
template <class L> __device__ __forceinline__ double density(const double *f) {
    double r = 0.0;
    Unroll<0, L::Q>::run([&](auto nc) { r = r + f[Order<L>::slot(decltype(nc)::value)]; });
    return r;
}

// psi of Eq. Interaction_Potential; raises the device flags on a domain error.
__device__ __forceinline__ double psi(const KParams &p, double rho) {
    if (!(rho > 0.0) || !(rho < INFINITY)) {
        atomicOr(p.flags, FLAG_NONFINITE);
        return 0.0;
    }
    const double arg = psi_arg(p.pl, p.eos_kind, rho);
    if (!(arg >= 0.0)) {
        atomicOr(p.flags, FLAG_PSI_DOMAIN);
        return 0.0;
    }
    return sqrt(arg);
}

// Total force density at a cell (Eqs. Shan_Chen_Force, interactionForce, plus the body
// force) from the padded psi field; pc points at the cell's psi.
template <class L, class Pol>
__device__ __forceinline__ void force(const KParams &p, const double *__restrict__ pc, double F[3]) {
    constexpr int D = L::D;
    const PlainPhys &q = p.pl;
    const int sy = p.px, sz = p.px * p.py;
    double M1[3] = {0.0, 0.0, 0.0}, sc[3] = {0.0, 0.0, 0.0};
    double M2[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    Unroll<0, L::Q>::run([&](auto nc) {
        constexpr int n = decltype(nc)::value;
        constexpr int c[3] = {cc<L>(n, 0), cc<L>(n, 1), cc<L>(n, 2)};
        const double pn = Pol::ro(pc + (c[0] + c[1] * sy + c[2] * sz));
        const double wp = L::w(Order<L>::slot(n)) * pn;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (c[a] != 0) M1[a] = M1[a] + wp * (double)c[a] * 3.0;
#pragma unroll
            for (int b = a; b < D; ++b)
                if (cc2<L>(n, a, b) != 0.0) M2[a][b] = M2[a][b] + wp * cc2<L>(n, a, b) * 9.0;
        }
        if (n > 0) {
#pragma unroll
            for (int a = 0; a < D; ++a)
                if (c[a] != 0) sc[a] = sc[a] + omega_sc<L>(n) * pn * (double)c[a];
        }
    });
    const double psi0 = Pol::ro(pc);
    double trM2 = 0.0;
#pragma unroll
    for (int b = 0; b < D; ++b) trM2 = trM2 + M2[b][b];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= D) {
            F[a] = 0.0;
            continue;
        }
        const double Fsc = -q.G * psi0 * sc[a];
        double M1M2 = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) M1M2 = M1M2 + M1[b] * (a <= b ? M2[a][b] : M2[b][a]);
        const double Fint = Fsc - q.K1 * M1M2 + q.K2 * M1[a] * trM2;
        F[a] = Fint + q.fext[a];
    }
}

// f^eq_n of Eq. Single_Phase_EDF, n in the summation order.
template <class L, int n> __device__ __forceinline__ double feq(double rho, const double u[3]) {
    constexpr int D = L::D;
    double cu = 0.0, quad = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (cc<L>(n, a) > 0) cu = cu + u[a];
        if (cc<L>(n, a) < 0) cu = cu - u[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
            if (cc2<L>(n, a, b) != 0.0) quad = quad + cc2<L>(n, a, b) * u[a] * u[b];
    return L::w(Order<L>::slot(n)) * rho * (1.0 + cu * 3.0 + quad * 4.5);
}

// The bracket of Eq. Guo_Forcing_Scheme (without 1 - 1/(2 tau)), n in the summation order.
template <class L, int n> __device__ __forceinline__ double guo(const double F[3], const double u[3]) {
    constexpr int D = L::D;
    double cF = 0.0, quad = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (cc<L>(n, a) > 0) cF = cF + F[a];
        if (cc<L>(n, a) < 0) cF = cF - F[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
            if (cc2<L>(n, a, b) != 0.0) quad = quad + cc2<L>(n, a, b) * F[a] * u[b];
    return L::w(Order<L>::slot(n)) * (cF * 3.0 + quad * 9.0);
}

// In place: pre-collision populations f (storage slots) -> post-collision populations.
template <class L, int MRT> __device__ __forceinline__ void collide(const KParams &p, double *f, const double F[3]) {
    constexpr int Q = L::Q, D = L::D;
    const PlainPhys &q = p.pl;
    const double rho = density<L>(f);
    double u[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double m = 0.0;
        Unroll<0, Q>::run([&](auto nc) {
            constexpr int n = decltype(nc)::value;
            if (cc<L>(n, a) > 0) m = m + f[Order<L>::slot(n)];
            if (cc<L>(n, a) < 0) m = m - f[Order<L>::slot(n)];
        });
        u[a] = (m + F[a] / 2.0) / rho;
    }
    double tau = q.tau_l;
    if (p.var_tau) {
        double wgt = (rho - q.tau_rho_v) / q.d_rho;
        if (wgt < 0.0) wgt = 0.0;
        if (wgt > 1.0) wgt = 1.0;
        tau = q.tau_v + wgt * q.d_tau;
    }
    if constexpr (!MRT) {
        const double kg = 1.0 - 1.0 / (2.0 * tau);
        Unroll<0, Q>::run([&](auto nc) {
            constexpr int n = decltype(nc)::value;
            constexpr int i = Order<L>::slot(n);
            const double fe = feq<L, n>(rho, u);
            const double Fi = kg * guo<L, n>(F, u);
            f[i] = f[i] - (f[i] - fe) / tau + Fi;
        });
    } else {
        double fneq[Q], Ft[Q], dmf[Q];
        Unroll<0, Q>::run([&](auto nc) {
            constexpr int n = decltype(nc)::value;
            fneq[n] = f[Order<L>::slot(n)] - feq<L, n>(rho, u);
            Ft[n] = guo<L, n>(F, u);
        });
        const double s_tau = 1.0 / tau;
        Unroll<0, Q>::run([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            double mneq = 0.0, mf = 0.0;
            Unroll<0, Q>::run([&](auto nc) {
                constexpr int n = decltype(nc)::value;
                constexpr double m = basis<L>(k, n);
                if (m != 0.0) {
                    mneq = mneq + m * fneq[n];
                    mf = mf + m * Ft[n];
                }
            });
            const double s = rate_kind<L>(k) == 0 ? s_tau : q.s_rate[rate_kind<L>(k)];
            const double dm = s * mneq;
            const double mF = (1.0 - s / 2.0) * mf;
            dmf[k] = mF - dm;
        });
        Unroll<0, Q>::run([&](auto nc) {
            constexpr int n = decltype(nc)::value;
            double corr = 0.0;
            Unroll<0, Q>::run([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr double mi = basis<L>(k, n) / basis_norm2<L>(k);
                if (mi != 0.0) corr = corr + mi * dmf[k];
            });
            f[Order<L>::slot(n)] = f[Order<L>::slot(n)] + corr;
        });
    }
}

// f = f^eq(rho, u) of Eq. Single_Phase_EDF into storage slots (initialisation).
template <class L> __device__ __forceinline__ void equilibrium(double rho, const double u[3], double *f) {
    Unroll<0, L::Q>::run([&](auto nc) {
        constexpr int n = decltype(nc)::value;
        f[Order<L>::slot(n)] = feq<L, n>(rho, u);
    });
}

}  // namespace plain
}  // namespace plb
