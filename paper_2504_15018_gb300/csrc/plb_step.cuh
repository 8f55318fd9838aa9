// The two hot kernels of a time step, written for instruction economy:
//  - 3-D launch (x fastest in a warp), no division to recover coordinates;
//  - one base pointer per population plane, 32-bit cell offsets when the lattice
//    has fewer than 2^31 cells;
//  - AA parity and the wall rows are compile-time branches (the wall test only runs
//    on the first and last rows, and is warp-uniform there);
//  - the collision in fused multiply-add form, and the MRT non-hydrodynamic moments
//    computed from the symmetric / antisymmetric parts of opposite-direction pairs.
#pragma once
#include "plb_device.cuh"
#include "plb_plain.cuh"

namespace plb {

template <class S> struct Planes {
    S *p[19];
};

// Per-thread lattice geometry: the cell, and the offsets of its +-1 neighbours along
// each axis including the periodic wrap.
template <class I> struct Geo {
    int x, y, z;
    I s;
    I ox[3], oy[3], oz[3];   // [0]: -1, [1]: 0, [2]: +1
    __device__ __forceinline__ I nb(int cx, int cy, int cz) const { return ox[cx + 1] + oy[cy + 1] + oz[cz + 1]; }
};

template <class I> __device__ __forceinline__ void geo_at(const KParams &p, int x, int y, int z, Geo<I> &g) {
    g.x = x;
    g.y = y;
    g.z = z;
    const I row = (I)p.nx, plane = (I)p.nx * (I)p.ny;
    g.s = (I)g.x + row * ((I)g.y + (I)p.ny * (I)g.z);
    g.ox[1] = g.oy[1] = g.oz[1] = 0;
    g.ox[0] = g.x > 0 ? (I)-1 : (I)(p.nx - 1);
    g.ox[2] = g.x < p.nx - 1 ? (I)1 : (I)(1 - p.nx);
    g.oy[0] = g.y > 0 ? -row : row * (I)(p.ny - 1);
    g.oy[2] = g.y < p.ny - 1 ? row : -row * (I)(p.ny - 1);
    g.oz[0] = g.z > 0 ? -plane : plane * (I)(p.nz - 1);
    g.oz[2] = g.z < p.nz - 1 ? plane : -plane * (I)(p.nz - 1);
}

template <class I> __device__ __forceinline__ bool make_geo(const KParams &p, Geo<I> &g) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return false;
    geo_at<I>(p, x, y, blockIdx.z + p.z0, g);
    return true;
}

// Stored values of the pre-collision populations for parity ODD (for FP16 storage the
// deviations f_i - w_i rho_ref).  WALL: this row touches a bounce-back wall.
template <class L, class S, bool ODD, bool WALL, class Pol = LdStream, class I>
__device__ __forceinline__ void load_fast(const KParams &p, const Planes<S> &A, const Geo<I> &g,
                                          typename Store<S>::T *f) {
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = opp(i);
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        if (!ODD) {
            f[i] = Store<S>::template ld<Pol>(A.p[i] + g.s);
        } else {
            bool from_wall = false;
            if (WALL && cy != 0) from_wall = (g.y - cy < 0) || (g.y - cy >= p.ny);
            if (from_wall)
                f[i] = Store<S>::template ld<Pol>(A.p[i] + g.s);
            else
                f[i] = Store<S>::template ld<Pol>(A.p[o] + (g.s + g.nb(-cx, -cy, -cz)));
        }
    });
}

// SR: FP16 stores with stochastic rounding, random bits from cell_hash(cell, salt).
template <class L, class S, bool ODD, bool WALL, bool SR = false, class I>
__device__ __forceinline__ void store_fast(const KParams &p, const Planes<S> &A, const Geo<I> &g,
                                           const typename Store<S>::T *f, unsigned salt = 0) {
    unsigned hsh = 0;
    if constexpr (SR) hsh = cell_hash((unsigned)g.s + p.cell_base, salt);
    auto st = [&](S *a, typename Store<S>::T v, int i) {
        if constexpr (SR) Store<S>::st_sr(a, v, dir_bits(hsh, i));
        else Store<S>::st(a, v);
    };
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = opp(i);
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        if (!ODD) {
            st(A.p[o] + g.s, f[i], i);
        } else {
            bool to_wall = false;
            if (WALL && cy != 0) to_wall = (g.y + cy < 0) || (g.y + cy >= p.ny);
            if (to_wall)
                st(A.p[o] + g.s, f[i], i);
            else
                st(A.p[i] + (g.s + g.nb(cx, cy, cz)), f[i], i);
        }
    });
}

// Total force density from the padded psi field (pc points at the cell's psi).
template <class L, class T, class Pol = LdStream, class PsiT>
__device__ __forceinline__ void force_fast(const KParams &p, const PsiT *__restrict__ pc, T F[3]) {
    const T psi0 = (T)Pol::ro(pc);
    T m1[3] = {0, 0, 0};
    T m2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const int sy = p.px, sz = p.px * p.py;
    Unroll<0, (L::Q - 1) / 2>::run([&](auto kc) {
        constexpr int i = 2 * decltype(kc)::value + 1;
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const int off = cx + cy * sy + cz * sz;
        const T pa = (T)Pol::ro(pc + off), pb = (T)Pol::ro(pc - off);
        const T dif = pa - pb;
        const T sym = (pa + pb) - (T)2 * psi0;
        constexpr double w3 = 3.0 * L::w(i), w9 = 9.0 * L::w(i);
        constexpr int c[3] = {cx, cy, cz};
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
            if (c[a] != 0) m1[a] = mad((T)(w3 * c[a]), dif, m1[a]);
#pragma unroll
            for (int b = a; b < L::D; ++b) {
                const double coef = w9 * (c[a] * c[b] - (a == b ? 1.0 / 3.0 : 0.0));
                if (coef != 0.0) m2[a][b] = mad((T)coef, sym, m2[a][b]);
            }
        }
    });
    T tr = 0;
#pragma unroll
    for (int a = 0; a < L::D; ++a) tr += m2[a][a];
    const Phys<T> &q = phys<T>(p);
    const T mG = -q.G * psi0, Ac = q.A_m1m2, Bt = q.B_m1tr * tr;
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
        T m21 = 0;
#pragma unroll
        for (int b = 0; b < L::D; ++b) m21 = mad(a <= b ? m2[a][b] : m2[b][a], m1[b], m21);
        F[a] = mad(mG + Bt, m1[a], mad(Ac, m21, q.fext[a]));
    }
    if (L::D == 2) F[2] = 0;
}

template <class L> struct RowParity {
    // true when row k is even under c -> -c (it then depends on the symmetric pair sums only)
    __host__ __device__ static constexpr bool even(int k) {
        bool e = true;
        for (int q = 0; q < (L::Q - 1) / 2; ++q) e = e && (Ghosts<L>::row(k, 2 * q + 1) == Ghosts<L>::row(k, 2 * q + 2));
        return e;
    }
};

// acc += c v for c in {-1, 0, 1} known at compile time (no multiplication).
template <int C, class T> __device__ __forceinline__ void add_c(T &acc, const T &v) {
    if (C > 0) acc += v;
    if (C < 0) acc -= v;
}
template <int CX, int CY, int CZ, class T> __device__ __forceinline__ T dot_c(const T *v) {
    T r = T(0);
    bool first = true;
    auto term = [&](int c, const T &x) {
        if (c == 0) return;
        if (first) {
            r = c > 0 ? x : -x;
            first = false;
        } else {
            r = c > 0 ? r + x : r - x;
        }
    };
    term(CX, v[0]);
    term(CY, v[1]);
    term(CZ, v[2]);
    return r;
}

// MRT ghost-moment part of the collision, generic over the lattice: m_k = sum_i M_ki g_i for
// the non-hydrodynamic rows, A_k = (s_k - omega) m_k / |M_k|^2, f_i -= sum_k M_ki A_k.
// g0 = g_0; gs[r] / ga[r] = g_i +- g_{i+1} of the opposite pair r (i = 2 r + 1); the pair's
// populations are held as fs[r] / fa[r] = f_i +- f_{i+1}, so f_i -= E + O, f_{i+1} -= E - O
// becomes fs -= 2 E, fa -= 2 O.
template <class L, class T, class R>
__device__ __forceinline__ void ghosts_generic(const Phys<R> &q, const T &om, const T &g0, const T *gs,
                                               const T *ga, T &f0, T *fs, T *fa) {
    constexpr int NP = (L::Q - 1) / 2;
    T Ak[Ghosts<L>::K];
    Unroll<0, Ghosts<L>::K>::run([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr bool ev = RowParity<L>::even(k);
        T m = ev ? T(Ghosts<L>::row(k, 0)) * g0 : T(0);
        Unroll<0, NP>::run([&](auto qc) {
            constexpr int r = decltype(qc)::value;
            constexpr double c = Ghosts<L>::row(k, 2 * r + 1);
            if (c != 0.0) m = mad(T(c), ev ? gs[r] : ga[r], m);
        });
        Ak[k] = (T(q.s_rate[Ghosts<L>::kind(k)]) - om) * (T(1.0 / row_norm2<L>(k)) * m);
    });
    T e0 = T(0);
    Unroll<0, Ghosts<L>::K>::run([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        if (RowParity<L>::even(k) && Ghosts<L>::row(k, 0) != 0.0) e0 = mad(T(Ghosts<L>::row(k, 0)), Ak[k], e0);
    });
    f0 -= e0;
    Unroll<0, NP>::run([&](auto qc) {
        constexpr int r = decltype(qc)::value;
        T E = T(0), O = T(0);
        Unroll<0, Ghosts<L>::K>::run([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            constexpr double c = Ghosts<L>::row(k, 2 * r + 1);
            if (c != 0.0) {
                if (RowParity<L>::even(k)) E = mad(T(c), Ak[k], E);
                else O = mad(T(c), Ak[k], O);
            }
        });
        fs[r] = mad(T(-2), E, fs[r]);
        fa[r] = mad(T(-2), O, fa[r]);
    });
}

// The same for D3Q19 with the rows of the d'Humieres et al. (2002) basis grouped by velocity
// class: the energy rows see only |c|^2, the pi rows only the axis or plane of c, and every
// plane's two pairs share their q / m coefficients up to signs, so sums over classes are
// formed once (pairs: 0-2 axes x, y, z; 3, 4: (1, +-1, 0); 5, 6: (1, 0, +-1); 7, 8: (0, 1, +-1)).
template <class T, class R>
__device__ __forceinline__ void ghosts_d3q19(const Phys<R> &q, const T &om, const T &g0, const T *gs,
                                             const T *ga, T &f0, T *fs, T *fa) {
    using G = Ghosts<D3Q19>;
    static_assert(D3Q19::cx(1) == 1 && D3Q19::cy(3) == 1 && D3Q19::cz(5) == 1 &&
                  D3Q19::cx(7) == 1 && D3Q19::cy(7) == 1 && D3Q19::cx(9) == 1 && D3Q19::cy(9) == -1 &&
                  D3Q19::cx(11) == 1 && D3Q19::cz(11) == 1 && D3Q19::cx(13) == 1 && D3Q19::cz(13) == -1 &&
                  D3Q19::cy(15) == 1 && D3Q19::cz(15) == 1 && D3Q19::cy(17) == 1 && D3Q19::cz(17) == -1,
                  "pair order assumed by the grouped projection");
    // even rows from the symmetric sums
    const T sx = gs[0], sy = gs[1], sz = gs[2];
    const T Dxy = gs[3] + gs[4], Dxz = gs[5] + gs[6], Dyz = gs[7] + gs[8];
    const T syz = sy + sz;
    const T S1 = sx + syz, S2 = Dxy + Dxz + Dyz;
    const T m_e = mad(T(-30), g0, mad(T(-11), S1, T(8) * S2));
    const T m_eps = mad(T(12), g0, mad(T(-4), S1, S2));
    const T m_pxx = mad(T(-4), sx, mad(T(2), syz, mad(T(-2), Dyz, Dxy + Dxz)));
    const T m_pww = mad(T(2), sz - sy, Dxy - Dxz);
    // odd rows from the antisymmetric sums
    const T Pxy = ga[3] + ga[4], Qxy = ga[3] - ga[4];
    const T Pxz = ga[5] + ga[6], Qxz = ga[5] - ga[6];
    const T Pyz = ga[7] + ga[8], Qyz = ga[7] - ga[8];
    const T m_qx = mad(T(-4), ga[0], Pxy + Pxz), m_mx = Pxy - Pxz;
    const T m_qy = mad(T(-4), ga[1], Qxy + Pyz), m_my = Pyz - Qxy;
    const T m_qz = mad(T(-4), ga[2], Qxz + Qyz), m_mz = Qxz - Qyz;
    auto A = [&](int k, const T &m) { return (T(q.s_rate[G::kind(k)]) - om) * (T(1.0 / row_norm2<D3Q19>(k)) * m); };
    const T Ae = A(0, m_e), Aeps = A(1, m_eps), Aqx = A(2, m_qx), Aqy = A(3, m_qy), Aqz = A(4, m_qz);
    const T Apxx = A(5, m_pxx), Apww = A(6, m_pww), Amx = A(7, m_mx), Amy = A(8, m_my), Amz = A(9, m_mz);
    // back-projection: f_i -= sum_k M_ki A_k, by class
    f0 -= mad(T(-30), Ae, T(12) * Aeps);
    const T C1 = mad(T(-11), Ae, T(-4) * Aeps), C2 = mad(T(8), Ae, Aeps);
    auto pair = [&](int r, const T &E, const T &O) {
        fs[r] = mad(T(-2), E, fs[r]);
        fa[r] = mad(T(-2), O, fa[r]);
    };
    pair(0, mad(T(-4), Apxx, C1), T(-4) * Aqx);
    const T Cy = mad(T(2), Apxx, C1);
    pair(1, mad(T(-2), Apww, Cy), T(-4) * Aqy);
    pair(2, mad(T(2), Apww, Cy), T(-4) * Aqz);
    {
        const T E = C2 + Apxx + Apww, a = Aqx + Amx, b = Aqy - Amy;
        pair(3, E, a + b);
        pair(4, E, a - b);
    }
    {
        const T E = C2 + Apxx - Apww, a = Aqx - Amx, b = Aqz + Amz;
        pair(5, E, a + b);
        pair(6, E, a - b);
    }
    {
        const T E = mad(T(-2), Apxx, C2), a = Aqy + Amy, b = Aqz - Amz;
        pair(7, E, a + b);
        pair(8, E, a - b);
    }
}

// In place: stored values h -> post-collision stored values.  SHIFT: h_i = f_i - w_i rho_ref
// (FP16 storage); then rho = sum h + rho_ref (sum_i w_i = 1), j = sum c_i h_i
// (sum_i w_i c_i = 0), and the update adds to h.
// feq_i = w_i rho (1 + delta_i), delta_i = 3 c.u + 4.5 (c.u)^2 - 1.5 u^2 is kept without the 1,
// so that the u^2 terms are not lost to rounding against 1 (sum_i w_i delta_i = 0 in exact
// arithmetic; rounding 1 + ... biases the mass at small u).  An opposite pair (c, -c) is
// updated through its sum and difference: with S = 4.5 (c.u)^2 - 1.5 u^2 and the Guo term
// Ft_+- = w (Gs +- 3 c.F), Gs = 9 (c.u)(c.F) - 3 u.F, the sum of f - feq is
// f_+ + f_- - 2 w rho - 2 w rho S and the difference f_+ - f_- - 6 w rho c.u.
// T is double, float, or f2 (two cells at once).
template <class L, int MRT, bool SHIFT, class T>
__device__ __forceinline__ void collide_fast(const KParams &p, T *f, const T F[3]) {
    using R = typename ScalarOf<T>::type;
    const Phys<R> &q = phys<R>(p);
    constexpr int NP = (L::Q - 1) / 2;
    // the pairs as sums and differences from here on
    T fs[NP], fa[NP];
    T rho = f[0], j[3] = {T(0), T(0), T(0)};
    Unroll<0, NP>::run([&](auto kc) {
        constexpr int r = decltype(kc)::value;
        constexpr int i = 2 * r + 1;
        fs[r] = f[i] + f[i + 1];
        fa[r] = f[i] - f[i + 1];
        rho += fs[r];
        add_c<L::cx(i)>(j[0], fa[r]);
        add_c<L::cy(i)>(j[1], fa[r]);
        add_c<L::cz(i)>(j[2], fa[r]);
    });
    if (SHIFT) rho += T(q.rho_ref);
    const T irho = fdiv(T(1), rho);
    const T u[3] = {mad(T(0.5), F[0], j[0]) * irho, mad(T(0.5), F[1], j[1]) * irho, mad(T(0.5), F[2], j[2]) * irho};
    const T om = omega_of<T>(p, rho);
    const T nom = -om;
    const T Bq = T(-1.5) * mad(u[0], u[0], mad(u[1], u[1], u[2] * u[2]));
    const T nuF3 = T(-3) * mad(u[0], F[0], mad(u[1], F[1], u[2] * F[2]));
    const T kguo = mad(T(-0.5), om, T(1));
    const T drho = SHIFT ? rho - T(q.rho_ref) : rho;     // rho minus the stored shift
    // rest population
    T g0;
    {
        constexpr double w = wcol<L, R>(0);
        const T dn = mad(-(T(w) * rho), Bq, f[0] - T(w) * drho);   // f - feq
        if (!MRT) {
            f[0] = mad(kguo * T(w), nuF3, mad(nom, dn, f[0]));
        } else {
            g0 = mad(T(0.5 * w), nuF3, dn);                        // f - feq + Ft/2
            f[0] = mad(nom, g0, mad(T(w), nuF3, f[0]));             // BGK part with Ft
        }
    }
    T gs[NP], ga[NP];
    // opposite pair r = (i, i + 1): c_{i+1} = -c_i, the first non-zero component of c_i is +1
    Unroll<0, NP>::run([&](auto kc) {
        constexpr int r = decltype(kc)::value;
        constexpr int i = 2 * r + 1;
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        constexpr double w = wcol<L, R>(i);
        const T cu = dot_c<cx, cy, cz>(u);
        const T cF = dot_c<cx, cy, cz>(F);
        const T S = mad(T(4.5) * cu, cu, Bq);
        const T Gs = mad(T(9) * cu, cF, nuF3);
        const T dns = mad(-(T(2 * w) * rho), S, fs[r] - T(2 * w) * drho);   // sum of f - feq
        const T dna = mad(-(T(6 * w) * rho), cu, fa[r]);                     // difference
        if (!MRT) {
            fs[r] += mad(nom, dns, (kguo * T(2 * w)) * Gs);
            fa[r] += mad(nom, dna, (kguo * T(6 * w)) * cF);
        } else {
            gs[r] = mad(T(w), Gs, dns);                  // sums of g = f - feq + Ft/2
            ga[r] = mad(T(3 * w), cF, dna);
            fs[r] += mad(nom, gs[r], T(2 * w) * Gs);     // BGK part with Ft
            fa[r] += mad(nom, ga[r], T(6 * w) * cF);
        }
    });
    if (MRT) {
        if constexpr (std::is_same<L, D3Q19>::value) ghosts_d3q19<T, R>(q, om, g0, gs, ga, f[0], fs, fa);
        else ghosts_generic<L, T, R>(q, om, g0, gs, ga, f[0], fs, fa);
    }
    Unroll<0, NP>::run([&](auto kc) {
        constexpr int r = decltype(kc)::value;
        const T h = T(0.5) * fa[r];
        f[2 * r + 1] = mad(T(0.5), fs[r], h);
        f[2 * r + 2] = mad(T(0.5), fs[r], -h);
    });
}

// The collision of collide_fast with its output streamed: emit(ic, v) receives the new stored
// value of population decltype(ic)::value as soon as it is final, so that a pair's registers
// are free once it is stored.  Equal to collide_fast in exact arithmetic (rounding differs).
// D3Q19 (BGK and MRT), whose pair kernels are bound by registers, takes the streamed form;
// D2Q9 runs collide_fast and then emits.  For D3Q19 MRT the ghost moments of
// g = f - feq + Ft/2 come first, from the pair sums of the stored values and closed forms for
// the moments of feq and Ft, so no per-population g is kept.  With v = j - F/2 (= rho u - F) and P_a = u_a v_a, the rows of the
// d'Humieres et al. (2002) basis applied to the equilibrium and the Guo term of Sec. II give
// (sums over the D3Q19 velocities):
//   m_e(g)   = m_e(h)   + 11 drho - 19 u.v        m_eps(g) = m_eps(h) - 3 drho + 5.5 u.v
//   m_pxx(g) = m_pxx(h) + P_x - (P_y + P_z) / 2   m_pww(g) = m_pww(h) + (P_y - P_z) / 2
//   (m_pxx, m_pww: the fourth-order 3 pi_xx and pi_ww rows, as in ghosts_d3q19)
//   m_q(g)   = m_q(h)   + (2/3) j                 m_m(g)   = m_m(h)
// where h is the stored value (f, or f - w rho_ref with the shift) and drho = sum_i h_i.
template <class L, int MRT, bool SHIFT, class T, class Emit>
__device__ __forceinline__ void collide_emit(const KParams &p, T *f, const T F[3], Emit &&emit) {
    if constexpr (!std::is_same<L, D3Q19>::value) {
        collide_fast<L, MRT, SHIFT, T>(p, f, F);
        Unroll<0, L::Q>::run([&](auto ic) { emit(ic, f[decltype(ic)::value]); });
    } else {
        using R = typename ScalarOf<T>::type;
        const Phys<R> &q = phys<R>(p);
        constexpr int NP = (L::Q - 1) / 2;
        T fs[NP], fa[NP];
        T rho = f[0], j[3] = {T(0), T(0), T(0)};
        Unroll<0, NP>::run([&](auto kc) {
            constexpr int r = decltype(kc)::value;
            constexpr int i = 2 * r + 1;
            fs[r] = f[i] + f[i + 1];
            fa[r] = f[i] - f[i + 1];
            rho += fs[r];
            add_c<L::cx(i)>(j[0], fa[r]);
            add_c<L::cy(i)>(j[1], fa[r]);
            add_c<L::cz(i)>(j[2], fa[r]);
        });
        const T drho = rho;                                // sum of the stored values
        if (SHIFT) rho += T(q.rho_ref);
        const T irho = fdiv(T(1), rho);
        const T u[3] = {mad(T(0.5), F[0], j[0]) * irho, mad(T(0.5), F[1], j[1]) * irho,
                        mad(T(0.5), F[2], j[2]) * irho};
        const T om = omega_of<T>(p, rho);
        const T nom = -om;
        const T Bq = T(-1.5) * mad(u[0], u[0], mad(u[1], u[1], u[2] * u[2]));
        const T nuF3 = T(-3) * mad(u[0], F[0], mad(u[1], F[1], u[2] * F[2]));
        const T kguo = mad(T(-0.5), om, T(1));
        // relaxation amplitudes A_k = (s_k - omega) m_k(g) / |M_k|^2 of the ghost rows (MRT)
        T Ae, Aeps, Aqx, Aqy, Aqz, Apxx, Apww, Amx, Amy, Amz;
        if constexpr (MRT) {
            using G = Ghosts<D3Q19>;
            const T sx = fs[0], sy = fs[1], sz = fs[2];
            const T Dxy = fs[3] + fs[4], Dxz = fs[5] + fs[6], Dyz = fs[7] + fs[8];
            const T syz = sy + sz;
            const T S1 = sx + syz, S2 = Dxy + Dxz + Dyz;
            const T Px = u[0] * mad(T(-0.5), F[0], j[0]), Py = u[1] * mad(T(-0.5), F[1], j[1]),
                    Pz = u[2] * mad(T(-0.5), F[2], j[2]);
            const T uv = Px + Py + Pz;
            const T m_e = mad(T(-30), f[0], mad(T(-11), S1, mad(T(8), S2, mad(T(11), drho, T(-19) * uv))));
            const T m_eps = mad(T(12), f[0], mad(T(-4), S1, S2 + mad(T(-3), drho, T(5.5) * uv)));
            const T m_pxx = mad(T(-4), sx, mad(T(2), syz, mad(T(-2), Dyz, (Dxy + Dxz) + mad(T(-0.5), Py + Pz, Px))));
            const T m_pww = mad(T(2), sz - sy, (Dxy - Dxz) + T(0.5) * (Py - Pz));
            const T Pxy = fa[3] + fa[4], Qxy = fa[3] - fa[4];
            const T Pxz = fa[5] + fa[6], Qxz = fa[5] - fa[6];
            const T Pyz = fa[7] + fa[8], Qyz = fa[7] - fa[8];
            const T m_qx = mad(T(-4), fa[0], mad(T(2.0 / 3.0), j[0], Pxy + Pxz)), m_mx = Pxy - Pxz;
            const T m_qy = mad(T(-4), fa[1], mad(T(2.0 / 3.0), j[1], Qxy + Pyz)), m_my = Pyz - Qxy;
            const T m_qz = mad(T(-4), fa[2], mad(T(2.0 / 3.0), j[2], Qxz + Qyz)), m_mz = Qxz - Qyz;
            auto A = [&](int k, const T &m) {
                return (T(q.s_rate[G::kind(k)]) - om) * (T(1.0 / row_norm2<D3Q19>(k)) * m);
            };
            Ae = A(0, m_e), Aeps = A(1, m_eps), Aqx = A(2, m_qx), Aqy = A(3, m_qy), Aqz = A(4, m_qz);
            Apxx = A(5, m_pxx), Apww = A(6, m_pww), Amx = A(7, m_mx), Amy = A(8, m_my), Amz = A(9, m_mz);
        }
        // rest population
        {
            constexpr double w = wcol<L, R>(0);
            const T dn = mad(T(-w) * rho, Bq, mad(T(-w), drho, f[0]));       // f - feq
            T v = mad(kguo * T(w), nuF3, mad(nom, dn, f[0]));
            if constexpr (MRT) v -= mad(T(-30), Ae, T(12) * Aeps);
            emit(std::integral_constant<int, 0>{}, v);
        }
        // opposite pair r = (i, i + 1): c_{i+1} = -c_i, the first non-zero component of c_i is +1
        Unroll<0, NP>::run([&](auto kc) {
            constexpr int r = decltype(kc)::value;
            constexpr int i = 2 * r + 1;
            constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            constexpr double w = wcol<L, R>(i);
            const T cu = dot_c<cx, cy, cz>(u);
            const T cF = dot_c<cx, cy, cz>(F);
            const T S = mad(T(4.5) * cu, cu, Bq);
            const T Gs = mad(T(9) * cu, cF, nuF3);
            const T dns = mad(T(-2 * w) * rho, S, mad(T(-2 * w), drho, fs[r]));   // sum of f - feq
            const T dna = mad(T(-6 * w) * rho, cu, fa[r]);                        // difference
            T vs = mad(kguo * T(2 * w), Gs, mad(nom, dns, fs[r]));
            T va = mad(kguo * T(6 * w), cF, mad(nom, dna, fa[r]));
            if constexpr (MRT) {
                // back-projection f_i -= sum_k M_ki A_k by velocity class (pairs: 0-2 axes x, y,
                // z; 3, 4: (1, +-1, 0); 5, 6: (1, 0, +-1); 7, 8: (0, 1, +-1))
                const T C1 = mad(T(-11), Ae, T(-4) * Aeps), C2 = mad(T(8), Ae, Aeps);
                T E, O;
                if constexpr (r == 0) { E = mad(T(-4), Apxx, C1); O = T(-4) * Aqx; }
                if constexpr (r == 1) { E = mad(T(-2), Apww, mad(T(2), Apxx, C1)); O = T(-4) * Aqy; }
                if constexpr (r == 2) { E = mad(T(2), Apww, mad(T(2), Apxx, C1)); O = T(-4) * Aqz; }
                if constexpr (r == 3 || r == 4) {
                    E = (C2 + Apxx) + Apww;
                    const T a = Aqx + Amx, b = Aqy - Amy;
                    O = r == 3 ? a + b : a - b;
                }
                if constexpr (r == 5 || r == 6) {
                    E = (C2 + Apxx) - Apww;
                    const T a = Aqx - Amx, b = Aqz + Amz;
                    O = r == 5 ? a + b : a - b;
                }
                if constexpr (r == 7 || r == 8) {
                    E = mad(T(-2), Apxx, C2);
                    const T a = Aqy + Amy, b = Aqz - Amz;
                    O = r == 7 ? a + b : a - b;
                }
                vs = mad(T(-2), E, vs);
                va = mad(T(-2), O, va);
            }
            const T hs = T(0.5) * vs;
            emit(std::integral_constant<int, i>{}, mad(T(0.5), va, hs));
            emit(std::integral_constant<int, i + 1>{}, mad(T(-0.5), va, hs));
        });
    }
}

// ------------------------------------------------------------------ kernels
// Minimum resident 256-thread blocks per SM requested from the register allocator.
#ifndef PLB_COLLIDE_MINB
#define PLB_COLLIDE_MINB 3
#endif

template <class L, class S, bool ODD, bool WALL, class Pol = LdStream, class I>
__device__ __forceinline__ void psi_body(const KParams &p, const Planes<S> &A, typename Store<S>::PsiT *psi,
                                         const Geo<I> &g) {
    using T = typename Store<S>::T;
    using PsiT = typename Store<S>::PsiT;
    T f[L::Q];
    load_fast<L, S, ODD, WALL, Pol>(p, A, g, f);
    PsiT v;
    if constexpr (std::is_same<S, double>::value) {
        v = plain::psi(p, plain::density<L>(f));                // FP64: the plain evaluation
    } else {
        T rho = f[0];
#pragma unroll
        for (int i = 1; i < L::Q; ++i) rho += f[i];
        if (Store<S>::SHIFT) rho += phys<T>(p).rho_ref;      // sum_i w_i rho_ref = rho_ref
        v = (PsiT)psi_of<T>(p, rho);
    }
    psi[psi_index(p, g.x, g.y, g.z)] = v;
    // periodic images / wall mirrors in the ghost layer (boundary cells only)
    const bool bx = g.x == 0 || g.x == p.nx - 1, by = g.y == 0 || g.y == p.ny - 1;
    const bool bz = L::D == 3 && (g.z == 0 || g.z == p.nz - 1);
    if (bx || by || bz) {
        int xs[3], ys[3], zs[3];
        int nxs = 1, nys = 1, nzs = 1;
        xs[0] = g.x;
        if (g.x == p.nx - 1) xs[nxs++] = -1;
        if (g.x == 0) xs[nxs++] = p.nx;
        ys[0] = g.y;
        if (p.wall_y) {
            // mirror rule; wetting walls keep the constant psi_wall written at creation
            if (g.y == 0 && !p.wall_fixed) ys[nys++] = -1;
            if (g.y == p.ny - 1 && !p.wall_fixed) ys[nys++] = p.ny;
        } else {
            if (g.y == p.ny - 1) ys[nys++] = -1;
            if (g.y == 0) ys[nys++] = p.ny;
        }
        zs[0] = g.z;
        if (L::D == 3) {
            if (g.z == p.nz - 1) zs[nzs++] = -1;
            if (g.z == 0) zs[nzs++] = p.nz;
        }
        for (int c = 0; c < nzs; ++c)
            for (int b = 0; b < nys; ++b)
                for (int a = (c == 0 && b == 0) ? 1 : 0; a < nxs; ++a) psi[psi_index(p, xs[a], ys[b], zs[c])] = v;
    }
}

template <class L, class S, bool ODD, class I>
__global__ void __launch_bounds__(256) k_psi_fast(KParams p, Planes<S> A, typename Store<S>::PsiT *__restrict__ psi) {
    Geo<I> g;
    if (!make_geo<I>(p, g)) return;
    if (ODD && p.wall_y && (g.y == 0 || g.y == p.ny - 1))
        psi_body<L, S, ODD, true>(p, A, psi, g);
    else
        psi_body<L, S, ODD, false>(p, A, psi, g);
}

template <class L, class S, int MRT, bool ODD, bool WALL, class Pol = LdStream, bool SR = false, class I>
__device__ __forceinline__ void collide_body(const KParams &p, const Planes<S> &A,
                                             const typename Store<S>::PsiT *__restrict__ psi, const Geo<I> &g,
                                             unsigned salt = 0) {
    using T = typename Store<S>::T;
    T f[L::Q];
    load_fast<L, S, ODD, WALL, Pol>(p, A, g, f);
    T F[3];
    if constexpr (std::is_same<S, double>::value) {
        // FP64: the plain evaluation, term by term in the equations' order
        plain::force<L, Pol>(p, psi + psi_index(p, g.x, g.y, g.z), F);
        plain::collide<L, MRT>(p, f, F);
    } else {
        force_fast<L, T, Pol>(p, psi + psi_index(p, g.x, g.y, g.z), F);
        collide_fast<L, MRT, Store<S>::SHIFT, T>(p, f, F);
    }
    store_fast<L, S, ODD, WALL, SR>(p, A, g, f, salt);
}

// FP64 storage: the plain evaluation holds f, f - f^eq, the Guo bracket and the moment
// corrections at once (about 60 doubles for D3Q19 MRT), so it runs in 128-thread blocks
// without a residency floor on the register allocation.
template <class L, int MRT, bool ODD, class I>
__global__ void __launch_bounds__(128) k_collide_plain(KParams p, Planes<double> A, const double *__restrict__ psi) {
    Geo<I> g;
    if (!make_geo<I>(p, g)) return;
    if (ODD && p.wall_y && (g.y == 0 || g.y == p.ny - 1))
        collide_body<L, double, MRT, ODD, true>(p, A, psi, g);
    else
        collide_body<L, double, MRT, ODD, false>(p, A, psi, g);
}

template <class L, class S, int MRT, bool ODD, class I>
__global__ void __launch_bounds__(256, PLB_COLLIDE_MINB) k_collide_fast(KParams p, Planes<S> A,
                                                      const typename Store<S>::PsiT *__restrict__ psi) {
    Geo<I> g;
    if (!make_geo<I>(p, g)) return;
    const bool wall = ODD && p.wall_y && (g.y == 0 || g.y == p.ny - 1);
    if constexpr (Store<S>::SHIFT) {
        if (p.stochastic) {
            if (wall) collide_body<L, S, MRT, ODD, true, LdStream, true>(p, A, psi, g, p.salt);
            else collide_body<L, S, MRT, ODD, false, LdStream, true>(p, A, psi, g, p.salt);
            return;
        }
    }
    if (wall)
        collide_body<L, S, MRT, ODD, true>(p, A, psi, g);
    else
        collide_body<L, S, MRT, ODD, false>(p, A, psi, g);
}

}  // namespace plb
