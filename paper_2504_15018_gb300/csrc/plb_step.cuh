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
    geo_at<I>(p, x, y, blockIdx.z, g);
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
    if constexpr (SR) hsh = cell_hash((unsigned)g.s, salt);
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

// In place: stored values h -> post-collision stored values.  SHIFT: h_i = f_i - w_i rho_ref
// (FP16 storage); then rho = sum h + rho_ref (sum_i w_i = 1), j = sum c_i h_i
// (sum_i w_i c_i = 0), f_i - feq_i = h_i - w_i (rho - rho_ref) - w_i rho delta_i, and the
// update adds to h.
// T is double, float, or f2 (two cells at once).
template <class L, int MRT, bool SHIFT, class T>
__device__ __forceinline__ void collide_fast(const KParams &p, T *f, const T F[3]) {
    using R = typename ScalarOf<T>::type;
    const Phys<R> &q = phys<R>(p);
    T rho = f[0], j[3] = {T(0), T(0), T(0)};
    Unroll<0, (L::Q - 1) / 2>::run([&](auto kc) {
        constexpr int i = 2 * decltype(kc)::value + 1;
        const T a = f[i] - f[i + 1];
        rho += f[i] + f[i + 1];
        add_c<L::cx(i)>(j[0], a);
        add_c<L::cy(i)>(j[1], a);
        add_c<L::cz(i)>(j[2], a);
    });
    if (SHIFT) rho += T(q.rho_ref);
    const T irho = fdiv(T(1), rho);
    const T u[3] = {mad(T(0.5), F[0], j[0]) * irho, mad(T(0.5), F[1], j[1]) * irho, mad(T(0.5), F[2], j[2]) * irho};
    const T om = omega_of<T>(p, rho);
    const T nom = -om;
    // feq_i = w_i rho (1 + delta_i), delta_i = 3 c.u + 4.5 (c.u)^2 - 1.5 u^2, kept without the 1 so
    // that the u^2 terms are not lost to rounding against 1 (sum_i w_i delta_i = 0 exactly in
    // exact arithmetic; rounding the 1 + ... away biases the mass at small u).
    const T Bq = T(-1.5) * mad(u[0], u[0], mad(u[1], u[1], u[2] * u[2]));
    const T nuF3 = T(-3) * mad(u[0], F[0], mad(u[1], F[1], u[2] * F[2]));
    const T kguo = mad(T(-0.5), om, T(1));
    const T drho = SHIFT ? rho - T(q.rho_ref) : rho;     // rho minus the stored shift
    T g[L::Q];
    // one direction: delta = feq / (w rho) - 1, t4 = Ft / w
    auto update = [&](int i, double w, const T &delta, const T &t4) {
        const T wrho = T(w) * rho;
        const T dn = mad(-wrho, delta, f[i] - T(w) * drho);          // f - feq
        if (!MRT) {
            f[i] = mad(kguo * T(w), t4, mad(nom, dn, f[i]));
        } else {
            g[i] = mad(T(0.5 * w), t4, dn);                      // f - feq + Ft/2
            f[i] = mad(nom, g[i], mad(T(w), t4, f[i]));           // BGK part with Ft
        }
    };
    update(0, wcol<L, R>(0), Bq, nuF3);
    // opposite pair (i, i + 1): c_{i+1} = -c_i, the first non-zero component of c_i is +1
    Unroll<0, (L::Q - 1) / 2>::run([&](auto kc) {
        constexpr int i = 2 * decltype(kc)::value + 1;
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const T cu = dot_c<cx, cy, cz>(u);
        const T cF = dot_c<cx, cy, cz>(F);
        constexpr double w = wcol<L, R>(i);
        update(i, w, mad(cu, mad(T(4.5), cu, T(3)), Bq), mad(cF, mad(T(9), cu, T(3)), nuF3));
        update(i + 1, w, mad(cu, mad(T(4.5), cu, T(-3)), Bq), mad(cF, mad(T(9), cu, T(-3)), nuF3));
    });
    if (MRT) {
        constexpr int NP = (L::Q - 1) / 2;
        T gs[NP], ga[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            gs[k] = g[2 * k + 1] + g[2 * k + 2];
            ga[k] = g[2 * k + 1] - g[2 * k + 2];
        }
        T Ak[Ghosts<L>::K];
        Unroll<0, Ghosts<L>::K>::run([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            constexpr bool ev = RowParity<L>::even(k);
            T m = ev ? T(Ghosts<L>::row(k, 0)) * g[0] : T(0);
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
        f[0] -= e0;
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
            f[2 * r + 1] -= E + O;
            f[2 * r + 2] -= E - O;
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
    T rho = f[0];
#pragma unroll
    for (int i = 1; i < L::Q; ++i) rho += f[i];
    if (Store<S>::SHIFT) rho += phys<T>(p).rho_ref;          // sum_i w_i rho_ref = rho_ref
    const PsiT v = (PsiT)psi_of<T>(p, rho);
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
            if (g.y == 0) ys[nys++] = -1;
            if (g.y == p.ny - 1) ys[nys++] = p.ny;
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
    force_fast<L, T, Pol>(p, psi + psi_index(p, g.x, g.y, g.z), F);
    collide_fast<L, MRT, Store<S>::SHIFT, T>(p, f, F);
    store_fast<L, S, ODD, WALL, SR>(p, A, g, f, salt);
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
