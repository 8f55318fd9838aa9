/*
 * Plain, slow FP64 CPU oracle of one time step of the pseudo-potential lattice
 * Boltzmann method (P-LBM) of "On the consistency of pseudo-potential lattice
 * Boltzmann methods" (arXiv 2504.15018).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no source with the CUDA library.
 *
 * Every routine below follows the paper's equations in their printed order,
 * with Delta x = Delta t = 1 (lattice units, r = 1, Sec. V):
 *   Eq. LBE                 f_i(t+1, x+c_i) - f_i(t, x) = -(f_i - f_i^eq)/tau + F_i'
 *   Eq. VelocitySet         D2Q9 velocities c_i and weights w_i, c_s^2 = 1/3
 *   Eq. Single_Phase_EDF    second-order equilibrium f_i^eq
 *   Eq. Shan_Chen_Force     F^SC = -G psi(x) sum_{i>0} omega(|c_i|^2) psi(x+c_i) c_i
 *   Eq. Interaction_Potential  psi = sqrt(2 (p_EOS - rho/3) / G)
 *   Eq. interactionForce    F^int = F^SC - G/12 (3 eps/2 + 2 kappa - 2) M1_b M2_ab
 *                                        + G/6 (kappa - 1) M1_a M2_bb
 *   M^(1), M^(2)            weighted first / second moments of psi (Sec. II)
 *   Eq. Guo_Forcing_Scheme  F_i' = w_i (1 - 1/(2 tau)) (c_i.F/c_s^2 + (c_ia c_ib - c_s^2 d_ab) F_a u_b / c_s^4)
 *   Eq. Density, Momentum   rho = sum f_i,  rho u = sum f_i c_i + F/2
 *   Sec. VI (tau)           tau = tau_v + (rho - rho_v)/(rho_l - rho_v) (tau_l - tau_v)
 *   Eq. EOS                 the paper's own equation of state
 *
 * Readings where the paper is silent (each one is a documented design reading):
 *   - D3Q19 uses the standard weights 1/3, 1/18, 1/36 and omega = 3 w_i
 *     (omega(1) = 1/6, omega(2) = 1/12), so that F^SC = -G psi M^(1) on both lattices.
 *   - The Peng-Robinson EOS (Peng & Robinson 1976) in lattice units is the second EOS kind.
 *   - MRT is the moment-space generalisation of BGK with the orthogonal bases of
 *     Lallemand & Luo (2000, D2Q9) and d'Humieres et al. (2002, D3Q19):
 *       f* = f - M^-1 S (M f - M f^eq) + M^-1 (I - S/2) M Ft,
 *     Ft_i = w_i (c_i.F/c_s^2 + (c_ia c_ib - c_s^2 d_ab) F_a u_b / c_s^4);
 *     with S = I / tau this is exactly the BGK update with Guo forcing.
 *   - Solid walls are halfway bounce-back at y = -1/2 and y = ny - 1/2; psi on a wall
 *     node equals psi on the fluid node it mirrors (y = -1 <-> 0, y = ny <-> ny - 1).
 *     With wall_rho > 0 the wall nodes instead carry psi(wall_rho), the pseudo-potential of
 *     a prescribed wall density (wetting walls: wall_rho near rho_l wets, near rho_v does not).
 *   - The tau interpolation weight is clamped to [0, 1].
 *   - Eq. interactionForce and Eq. New_Pressure_Tensor disagree on the eps term: the
 *     continuum limit of -G/12 (3 eps/2) M1_b M2_ab adds +G/16 eps (d psi)^2 to p_ab,
 *     while Eq. New_Pressure_Tensor (and the Maxwell rule at eps = 2, Sec. IV) needs
 *     -G/8 eps (d psi)^2, i.e. the force term +G/4 eps M1_b M2_ab.  With the printed
 *     coefficient the planar coexistence densities follow the mechanical-stability
 *     condition with exponent -eps/2 instead of eps.  The default reading therefore
 *     uses -G/12 (2 kappa - 2 - 3 eps) M1_b M2_ab; eps_printed = 1 keeps the printed one.
 *   - Streaming is a plain push into a second array (no in-place scheme).
 *
 * Layout of the oracle's population array: f[cell * Q + i] with
 * cell = x + nx * (y + ny * z).  Build with -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ORC_MUTANT (tests only, default 0): builds with a planted mistake, one per value, so that
 * tests/test_oracle_mutants.py can check that some pin fails on each.  0 is the oracle. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EPSI_DOMAIN 2
#define ORC_ENONFINITE 3

typedef struct {
    int lattice;              /* 0 = D2Q9, 1 = D3Q19 */
    int nx, ny, nz;           /* nz = 1 for D2Q9 */
    int wall_y;               /* 1: bounce-back walls bounding y; 0: periodic in y */
    int eos_kind;             /* 0 = Peng-Robinson, 1 = paper's EOS (Eq. EOS) */
    double pr_a, pr_b, pr_R, pr_omega, pr_T;   /* PR constants, absolute temperature */
    double pe_rho_v, pe_rho_l, pe_P;           /* paper EOS: rho_v, rho_l, p_c/rho_c^3 */
    double p_scale;           /* factor on p_EOS (Delta t^2 / Delta x^2 in Eq. Interaction_Potential) */
    double G, eps, kappa;
    double tau_l, tau_v, tau_rho_v, tau_rho_l; /* tau(rho) interpolation of Sec. VI */
    int mrt;                  /* 0 = BGK, 1 = MRT */
    double s_e, s_eps, s_q, s_pi, s_m;         /* MRT rates of the non-hydrodynamic moments */
    double fext[3];           /* external body force density */
    int eps_printed;          /* 1: eps coefficient exactly as printed in Eq. interactionForce (3 eps / 2);
                                 0: the reading that realises Eq. New_Pressure_Tensor (-3 eps), see below */
    double wall_rho;          /* > 0: psi on wall nodes = psi(wall_rho); <= 0: mirror of the fluid row */
} orc_params;

/* ---------------------------------------------------------------- lattices */

/* D2Q9 in the order of Eq. VelocitySet. */
static const int C2[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
/* D3Q19: rest, 6 axis links, 12 edge links. */
static const int C3[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static int lat_q(int lattice) { return lattice == 0 ? 9 : 19; }
static int lat_d(int lattice) { return lattice == 0 ? 2 : 3; }
static const int (*lat_c(int lattice))[3] { return lattice == 0 ? C2 : C3; }

static double lat_w(int lattice, int i) {
    const int *c = lat_c(lattice)[i];
    int c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    if (lattice == 0) return c2 == 0 ? 4.0 / 9.0 : (c2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    return c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

/* Shan-Chen weights omega(|c_i|^2). */
static double lat_omega(int lattice, int i) {
    const int *c = lat_c(lattice)[i];
    int c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    if (c2 == 0) return 0.0;
    if (lattice == 0) return c2 == 1 ? 1.0 / 3.0 : (ORC_MUTANT == 10 ? 1.0 / 6.0 : 1.0 / 12.0);
    return c2 == 1 ? 1.0 / 6.0 : 1.0 / 12.0;
}

static int lat_opposite(int lattice, int i) {
    const int (*c)[3] = lat_c(lattice);
    int q = lat_q(lattice);
    for (int j = 0; j < q; ++j)
        if (c[j][0] == -c[i][0] && c[j][1] == -c[i][1] && c[j][2] == -c[i][2]) return j;
    return -1;
}

/* c_s^2 = 1/3 in lattice units (Eq. VelocitySet).  Its inverse powers are the exact numbers
 * 1/c_s^2 = 3 and 1/c_s^4 = 9, so the formulas below multiply by them rather than divide by the
 * rounded FP64 value of 1/3, which would add a rounding the equations do not have. */
static const double CS2 = 1.0 / 3.0;
static const double INV_CS2 = 3.0;
static const double INV_CS4 = 9.0;

int orc_velocity_set(int lattice, int *c_out, double *w_out) {
    if (lattice != 0 && lattice != 1) return -1;
    int q = lat_q(lattice);
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3 * i + a] = lat_c(lattice)[i][a];
        w_out[i] = lat_w(lattice, i);
    }
    return q;
}

/* ---------------------------------------------------------- equation of state */

/* Peng & Robinson (1976): p = rho R T/(1 - b rho) - a alpha(T) rho^2/(1 + 2 b rho - b^2 rho^2),
 * alpha = [1 + m (1 - sqrt(T/Tc))]^2, m = 0.37464 + 1.54226 w - 0.26992 w^2,
 * Tc = 0.0778 a / (0.45724 b R). */
static double pr_pressure(const orc_params *P, double rho) {
    double Tc = 0.0778 * P->pr_a / (0.45724 * P->pr_b * P->pr_R);
    double m = 0.37464 + 1.54226 * P->pr_omega - 0.26992 * P->pr_omega * P->pr_omega;
    double g = 1.0 + m * (1.0 - sqrt(P->pr_T / Tc));
    double alpha = g * g;
    double br = P->pr_b * rho;
    return rho * P->pr_R * P->pr_T / (1.0 - br) - P->pr_a * alpha * rho * rho / (1.0 + 2.0 * br - br * br);
}

/* Eq. EOS: p = (p_c/rho_c^3) [2 rho^3 + (rho_v - 2 rho_l) rho^2 - 3 sqrt(rho_v) rho^2.5
 *                              + 2 sqrt(rho_v) rho_l rho^1.5 + sqrt(rho_v) rho_l^2 rho^0.5] */
static double paper_pressure(const orc_params *P, double rho) {
    double rv = P->pe_rho_v, rl = P->pe_rho_l, sv = sqrt(rv), sr = sqrt(rho);
    double bracket = 2.0 * rho * rho * rho + (rv - 2.0 * rl) * rho * rho - 3.0 * sv * rho * rho * sr
                   + 2.0 * sv * rl * rho * sr + sv * rl * rl * sr;
    return P->pe_P * bracket;
}

double orc_pressure(const orc_params *P, double rho) {
    double p = P->eos_kind == 0 ? pr_pressure(P, rho) : paper_pressure(P, rho);
    return P->p_scale * p;
}

/* Eq. Interaction_Potential: psi = sqrt(2 (p - rho/3) / G); p already carries Delta t^2/Delta x^2. */
static int psi_of_rho(const orc_params *P, double rho, double *psi) {
    if (!(rho > 0.0) || !isfinite(rho)) return ORC_ENONFINITE;
    double arg = (ORC_MUTANT == 8 ? 1.0 : 2.0) * (orc_pressure(P, rho) - rho / 3.0) / P->G;
    if (!(arg >= 0.0)) return ORC_EPSI_DOMAIN;
    *psi = sqrt(arg);
    return ORC_OK;
}

/* ------------------------------------------------------- local collision parts */

/* Eq. Single_Phase_EDF. */
void orc_feq(int lattice, double rho, const double *u, double *feq) {
    int q = lat_q(lattice);
    for (int i = 0; i < q; ++i) {
        const int *c = lat_c(lattice)[i];
        double cu = 0.0, quad = 0.0;
        for (int a = 0; a < 3; ++a) cu += c[a] * u[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                quad += (c[a] * c[b] - CS2 * (a == b)) * u[a] * u[b];
#if ORC_MUTANT == 1
        feq[i] = lat_w(lattice, i) * rho * (1.0 + cu * INV_CS2 - quad * (0.5 * INV_CS4));
#else
        feq[i] = lat_w(lattice, i) * rho * (1.0 + cu * INV_CS2 + quad * (0.5 * INV_CS4));
#endif
    }
}

/* The bracket of Eq. Guo_Forcing_Scheme without the (1 - 1/(2 tau)) factor. */
static void guo_bracket(int lattice, const double *F, const double *u, double *out) {
    int q = lat_q(lattice);
    for (int i = 0; i < q; ++i) {
        const int *c = lat_c(lattice)[i];
        double cF = 0.0, quad = 0.0;
        for (int a = 0; a < 3; ++a) cF += c[a] * F[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                quad += (c[a] * c[b] - CS2 * (a == b)) * F[a] * u[b];
#if ORC_MUTANT == 2
        out[i] = lat_w(lattice, i) * (cF * INV_CS2 + 0.0 * quad);
#else
        out[i] = lat_w(lattice, i) * (cF * INV_CS2 + quad * INV_CS4);
#endif
    }
}

/* Eq. Guo_Forcing_Scheme. */
void orc_guo(int lattice, double tau, const double *F, const double *u, double *Fi) {
    int q = lat_q(lattice);
    guo_bracket(lattice, F, u, Fi);
    for (int i = 0; i < q; ++i) Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * Fi[i];
}

/* tau(rho) of Sec. VI, interpolation weight clamped to [0, 1]. */
static double tau_of_rho(const orc_params *P, double rho) {
    if (P->tau_v == P->tau_l) return P->tau_l;
    double wgt = (rho - P->tau_rho_v) / (P->tau_rho_l - P->tau_rho_v);
    if (wgt < 0.0) wgt = 0.0;
    if (wgt > 1.0 && ORC_MUTANT != 9) wgt = 1.0;
    return P->tau_v + wgt * (P->tau_l - P->tau_v);
}

/* ---------------------------------------------------------------- MRT bases */

/* Moment polynomials of the orthogonal bases, evaluated at velocity c.
 * D2Q9 (Lallemand & Luo 2000): rho, e, eps, jx, qx, jy, qy, pxx, pxy.
 * D3Q19 (d'Humieres et al. 2002): rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx,
 *   pww, piww, pxy, pyz, pxz, mx, my, mz. */
static double mrt_row(int lattice, int k, const int *c) {
    double x = c[0], y = c[1], z = c[2];
    double c2 = x * x + y * y + z * z;
    if (lattice == 0) {
        switch (k) {
            case 0: return 1.0;
            case 1: return -4.0 + 3.0 * c2;
            case 2: return 4.0 - 10.5 * c2 + 4.5 * c2 * c2;
            case 3: return x;
            case 4: return (-5.0 + 3.0 * c2) * x;
            case 5: return y;
            case 6: return (-5.0 + 3.0 * c2) * y;
            case 7: return x * x - y * y;
            case 8: return x * y;
        }
        return 0.0;
    }
    switch (k) {
        case 0: return 1.0;
        case 1: return 19.0 * c2 - 30.0;
        case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
        case 3: return x;
        case 4: return (5.0 * c2 - 9.0) * x;
        case 5: return y;
        case 6: return (5.0 * c2 - 9.0) * y;
        case 7: return z;
        case 8: return (5.0 * c2 - 9.0) * z;
        case 9: return 3.0 * x * x - c2;
        case 10: return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
        case 11: return y * y - z * z;
        case 12: return (3.0 * c2 - 5.0) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        case 18: return (x * x - y * y) * z;
    }
    return 0.0;
}

/* Relaxation rate of moment k; the stress moments relax with 1/tau. */
static double mrt_rate(const orc_params *P, int k, double tau) {
    if (P->lattice == 0) {
        switch (k) {
            case 1: return P->s_e;
            case 2: return P->s_eps;
            case 4: case 6: return P->s_q;
            case 7: case 8: return 1.0 / tau;
            default: return 1.0 / tau;  /* conserved: rho, jx, jy */
        }
    }
    switch (k) {
        case 1: return P->s_e;
        case 2: return P->s_eps;
        case 4: case 6: case 8: return ORC_MUTANT == 5 ? P->s_m : P->s_q;
        case 10: case 12: return P->s_pi;
        case 16: case 17: case 18: return ORC_MUTANT == 5 ? P->s_q : P->s_m;
        case 9: case 11: case 13: case 14: case 15: return 1.0 / tau;
        default: return 1.0 / tau;  /* conserved: rho, jx, jy, jz */
    }
}

/* Fills M (q x q, row-major) and its inverse M^-1 = M^T diag(1 / |row_k|^2). */
static void mrt_matrices(int lattice, double *M, double *Minv) {
    int q = lat_q(lattice);
    for (int k = 0; k < q; ++k)
        for (int i = 0; i < q; ++i) M[k * q + i] = mrt_row(lattice, k, lat_c(lattice)[i]);
    for (int k = 0; k < q; ++k) {
        double n2 = 0.0;
        for (int i = 0; i < q; ++i) n2 += M[k * q + i] * M[k * q + i];
        for (int i = 0; i < q; ++i) Minv[i * q + k] = M[k * q + i] / n2;
    }
}

int orc_mrt_matrix(int lattice, double *M, double *Minv) {
    if (lattice != 0 && lattice != 1) return -1;
    mrt_matrices(lattice, M, Minv);
    return lat_q(lattice);
}

/* ------------------------------------------------------------- grid helpers */

static long cell_index(const orc_params *P, int x, int y, int z) {
    return (long)x + (long)P->nx * ((long)y + (long)P->ny * (long)z);
}

static int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

/* psi at x + c (periodic wrap; walls mirror psi of the adjacent fluid row, or carry
   psi(wall_rho) when a wall density is prescribed). */
static double psi_neighbour(const orc_params *P, const double *psi, int x, int y, int z, const int *c) {
    int xn = wrap(x + c[0], P->nx);
    int zn = wrap(z + c[2], P->nz);
    int yn = y + c[1];
    if (P->wall_y && P->wall_rho > 0.0 && (yn < 0 || yn >= P->ny)) {
        double pw = 0.0;
        psi_of_rho(P, P->wall_rho, &pw);     /* validated in check_params */
        return pw;
    }
    if (P->wall_y) {
        if (yn < 0) yn = -1 - yn;
        if (yn >= P->ny) yn = 2 * P->ny - 1 - yn;
    } else {
        yn = wrap(yn, P->ny);
    }
    return psi[cell_index(P, xn, yn, zn)];
}

static int check_params(const orc_params *P) {
    if (P->lattice != 0 && P->lattice != 1) return ORC_EINVAL;
    if (P->nx < 1 || P->ny < 1 || P->nz < 1) return ORC_EINVAL;
    if (P->lattice == 0 && P->nz != 1) return ORC_EINVAL;
    if (!(P->G < 0.0)) return ORC_EINVAL;
    if (!(P->tau_l > 0.5) || !(P->tau_v > 0.5)) return ORC_EINVAL;
    if (P->wall_rho > 0.0) {
        double pw;
        if (psi_of_rho(P, P->wall_rho, &pw) != ORC_OK) return ORC_EINVAL;
    }
    return ORC_OK;
}

/* rho and psi on every cell. */
static int density_and_psi(const orc_params *P, const double *f, double *rho, double *psi) {
    int q = lat_q(P->lattice);
    long n = (long)P->nx * P->ny * P->nz;
    int status = ORC_OK;
    for (long s = 0; s < n; ++s) {
        double r = 0.0;
        for (int i = 0; i < q; ++i) r += f[s * q + i];                    /* Eq. Density */
        rho[s] = r;
        int st = psi_of_rho(P, r, &psi[s]);
        if (st != ORC_OK && status == ORC_OK) status = st;
    }
    return status;
}

/* M^(1), M^(2) and the total force on one cell (Eq. interactionForce + external). */
static void cell_force(const orc_params *P, const double *psi, int x, int y, int z,
                       double *M1, double *M2, double *F) {
    int q = lat_q(P->lattice);
    const int (*c)[3] = lat_c(P->lattice);
    double sc[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        M1[a] = 0.0;
        for (int b = 0; b < 3; ++b) M2[3 * a + b] = 0.0;
    }
    for (int i = 0; i < q; ++i) {
        double pn = psi_neighbour(P, psi, x, y, z, c[i]);
        double w = lat_w(P->lattice, i);
        for (int a = 0; a < 3; ++a) {
#if ORC_MUTANT == 4
            M1[a] += w * pn * c[i][a];
#else
            M1[a] += w * pn * c[i][a] * INV_CS2;
#endif
            for (int b = 0; b < 3; ++b)
                M2[3 * a + b] += w * pn * (c[i][a] * c[i][b] - CS2 * (a == b)) * INV_CS4;
        }
        if (i > 0)
            for (int a = 0; a < 3; ++a) sc[a] += lat_omega(P->lattice, i) * pn * c[i][a];
    }
    int d = lat_d(P->lattice);
    double psi0 = psi[cell_index(P, x, y, z)];
    double trM2 = 0.0;
    for (int b = 0; b < d; ++b) trM2 += M2[3 * b + b];
    for (int a = 0; a < 3; ++a) {
        double Fsc = -P->G * psi0 * sc[a];
        double M1M2 = 0.0;
        for (int b = 0; b < d; ++b) M1M2 += M1[b] * M2[3 * a + b];
        double eps_term = P->eps_printed ? 1.5 * P->eps : -3.0 * P->eps;
#if ORC_MUTANT == 3
        double Fint = Fsc - (P->G / 12.0) * (eps_term + 2.0 * P->kappa - 2.0) * M1M2
                          - (P->G / 6.0) * (P->kappa - 1.0) * M1[a] * trM2;
#else
        double Fint = Fsc - (P->G / 12.0) * (eps_term + 2.0 * P->kappa - 2.0) * M1M2
                          + (P->G / 6.0) * (P->kappa - 1.0) * M1[a] * trM2;
#endif
        F[a] = a < d ? Fint + P->fext[a] : 0.0;
    }
}

/* ------------------------------------------------------------------ exports */

int orc_force_field(const orc_params *P, const double *f, double *M1, double *M2, double *F) {
    int st = check_params(P);
    if (st) return st;
    long n = (long)P->nx * P->ny * P->nz;
    double *rho = malloc(sizeof(double) * n), *psi = malloc(sizeof(double) * n);
    st = density_and_psi(P, f, rho, psi);
    if (st == ORC_OK)
        for (int z = 0; z < P->nz; ++z)
            for (int y = 0; y < P->ny; ++y)
                for (int x = 0; x < P->nx; ++x) {
                    long s = cell_index(P, x, y, z);
                    cell_force(P, psi, x, y, z, M1 + 3 * s, M2 + 9 * s, F + 3 * s);
                }
    free(rho);
    free(psi);
    return st;
}

/* Moments of a psi field given directly (used to pin the stencils). */
int orc_psi_moments(const orc_params *P, const double *psi, double *M1, double *M2, double *F) {
    int st = check_params(P);
    if (st) return st;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long s = cell_index(P, x, y, z);
                cell_force(P, psi, x, y, z, M1 + 3 * s, M2 + 9 * s, F + 3 * s);
            }
    return ORC_OK;
}

int orc_psi_field(const orc_params *P, const double *f, double *psi) {
    int st = check_params(P);
    if (st) return st;
    long n = (long)P->nx * P->ny * P->nz;
    double *rho = malloc(sizeof(double) * n);
    st = density_and_psi(P, f, rho, psi);
    free(rho);
    return st;
}

/* Initial populations f_i = f_i^eq(rho0, u0). */
int orc_init(const orc_params *P, const double *rho0, const double *u0, double *f) {
    int st = check_params(P);
    if (st) return st;
    int q = lat_q(P->lattice), d = lat_d(P->lattice);
    long n = (long)P->nx * P->ny * P->nz;
    for (long s = 0; s < n; ++s) {
        double u[3] = {0.0, 0.0, 0.0};
        if (u0)
            for (int a = 0; a < d; ++a) u[a] = u0[(long)a * n + s];
        orc_feq(P->lattice, rho0[s], u, f + s * q);
    }
    return ORC_OK;
}

/* One collision of a single cell: BGK (Eq. LBE) or MRT with Guo forcing. */
static void collide_cell(const orc_params *P, const double *fc, const double *F, double *fpost,
                         const double *M, const double *Minv) {
    int q = lat_q(P->lattice);
    const int (*c)[3] = lat_c(P->lattice);
    double rho = 0.0, u[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < q; ++i) rho += fc[i];
    for (int a = 0; a < 3; ++a) {
        double m = 0.0;
        for (int i = 0; i < q; ++i) m += fc[i] * c[i][a];
        u[a] = (m + F[a] / 2.0) / rho;                                      /* Eq. Momentum */
    }
    double tau = tau_of_rho(P, rho);
    double feq[19], Fi[19];
    orc_feq(P->lattice, rho, u, feq);
    if (!P->mrt) {
        orc_guo(P->lattice, tau, F, u, Fi);
        for (int i = 0; i < q; ++i) fpost[i] = fc[i] - (fc[i] - feq[i]) / tau + Fi[i];
        return;
    }
    double Ft[19], fneq[19], dm[19], mF[19];
    guo_bracket(P->lattice, F, u, Ft);
    for (int i = 0; i < q; ++i) fneq[i] = fc[i] - feq[i];
    for (int k = 0; k < q; ++k) {
        /* m - m^eq = M (f - f^eq): the same quantity by linearity of M, without
           subtracting two large moments that nearly cancel */
        double mneq = 0.0, mf = 0.0;
        for (int i = 0; i < q; ++i) {
            mneq += M[k * q + i] * fneq[i];
            mf += M[k * q + i] * Ft[i];
        }
        double s = mrt_rate(P, k, tau);
        dm[k] = s * mneq;
        mF[k] = (ORC_MUTANT == 6 ? 1.0 - s : 1.0 - s / 2.0) * mf;
    }
    for (int i = 0; i < q; ++i) {
        double corr = 0.0;
        for (int k = 0; k < q; ++k) corr += Minv[i * q + k] * (mF[k] - dm[k]);
        fpost[i] = fc[i] + corr;
    }
}

/* nsteps full time steps, in place on f (Eq. LBE with push streaming). */
int orc_run(const orc_params *P, double *f, int nsteps) {
    int st = check_params(P);
    if (st) return st;
    int q = lat_q(P->lattice);
    const int (*c)[3] = lat_c(P->lattice);
    long n = (long)P->nx * P->ny * P->nz;
    double *rho = malloc(sizeof(double) * n), *psi = malloc(sizeof(double) * n);
    double *fnew = malloc(sizeof(double) * n * q);
    double M[361], Minv[361];
    int opp[19];
    for (int i = 0; i < q; ++i) opp[i] = lat_opposite(P->lattice, i);
    if (P->mrt) mrt_matrices(P->lattice, M, Minv);
    for (int step = 0; step < nsteps && st == ORC_OK; ++step) {
        st = density_and_psi(P, f, rho, psi);
        if (st != ORC_OK) break;
        int nz = P->nz, ny = P->ny, nx = P->nx;
#pragma omp parallel for collapse(2) schedule(static) if (n >= 32768)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    long s = cell_index(P, x, y, z);
                    double M1[3], M2[9], F[3], fpost[19];
                    cell_force(P, psi, x, y, z, M1, M2, F);
                    collide_cell(P, f + s * q, F, fpost, M, Minv);
                    for (int i = 0; i < q; ++i) {
                        int yn = y + c[i][1];
                        if (P->wall_y && (yn < 0 || (ORC_MUTANT == 7 ? yn > ny : yn >= ny))) {
                            fnew[s * q + opp[i]] = fpost[i];              /* halfway bounce-back */
                        } else {
                            long t = cell_index(P, wrap(x + c[i][0], nx), wrap(yn, ny), wrap(z + c[i][2], nz));
                            fnew[t * q + i] = fpost[i];
                        }
                    }
                }
        memcpy(f, fnew, sizeof(double) * n * q);
        for (long k = 0; k < n * q; ++k)
            if (!isfinite(f[k])) { st = ORC_ENONFINITE; break; }
    }
    free(rho);
    free(psi);
    free(fnew);
    return st;
}

/* Macroscopic fields: rho (Eq. Density), u (Eq. Momentum, with the force of the
 * current populations), p = p_scale p_EOS(rho). */
int orc_moments(const orc_params *P, const double *f, double *rho, double *u, double *p) {
    int st = check_params(P);
    if (st) return st;
    int q = lat_q(P->lattice), d = lat_d(P->lattice);
    const int (*c)[3] = lat_c(P->lattice);
    long n = (long)P->nx * P->ny * P->nz;
    double *psi = malloc(sizeof(double) * n);
    double *r = malloc(sizeof(double) * n);
    st = density_and_psi(P, f, r, psi);
    for (int z = 0; z < P->nz && st == ORC_OK; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long s = cell_index(P, x, y, z);
                double M1[3], M2[9], F[3];
                cell_force(P, psi, x, y, z, M1, M2, F);
                if (rho) rho[s] = r[s];
                if (p) p[s] = orc_pressure(P, r[s]);
                if (u)
                    for (int a = 0; a < d; ++a) {
                        double m = 0.0;
                        for (int i = 0; i < q; ++i) m += f[s * q + i] * c[i][a];
                        u[(long)a * n + s] = (m + F[a] / 2.0) / r[s];
                    }
            }
    free(psi);
    free(r);
    return st;
}
