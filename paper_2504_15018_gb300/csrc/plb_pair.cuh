// Two-cell variants of the step kernels for FP32 arithmetic (FP32 and FP16-shifted storage).
//
// Each thread updates the x-adjacent cells (x0, x0 + 1), x0 even, with packed FP32
// arithmetic (plb_f2.cuh).  nx must be even.  Population I/O per direction:
//  - aligned pairs (every even-parity access; odd-parity accesses with c_x = 0, whose
//    row offsets are multiples of nx) move as one 8-byte (FP32) or 4-byte (FP16) access;
//  - odd-parity accesses with c_x != 0 are shifted by one element and move as two
//    scalar accesses (per-cell x offsets carry the periodic wrap).
// The psi stencil of the two cells is read as float2 vectors: 3 per row where the
// stencil spans x0 - 1 .. x0 + 2, 1 where it spans x0 .. x0 + 1.
#pragma once
#include "plb_moment.cuh"
#include "plb_step.cuh"

// D3Q19 collision of the pair kernels: 0 = the per-pair BGK update with the ghost-moment
// correction (collide_emit) for every storage; 1 = the moment-space collision
// (collide_moments_d3q19) for FP16-shifted storage, collide_emit for FP32; 2 = the moment-space
// collision for both.
#ifndef PLB_MOMENT_COLLIDE
#define PLB_MOMENT_COLLIDE 1
#endif

namespace plb {

// Element idx >= 0 of a population plane, addressed as the plane base plus a 32-bit unsigned
// byte offset (PLB_U32_ADDR; planes hold fewer than 2^31 elements on the pair paths, at most
// 2^31 x 4 bytes), which the compiler can fold into the memory instruction's addressing, else as
// plain pointer arithmetic.  Measured: FP32 step 27.0 -> 27.8 GLUPS, FP16S 41.1 -> 41.8.
#ifndef PLB_U32_ADDR
#define PLB_U32_ADDR 1
#endif
template <class S> __device__ __forceinline__ S *elem(S *base, int idx) {
#if PLB_U32_ADDR
    return reinterpret_cast<S *>(reinterpret_cast<char *>(base) + (unsigned)idx * (unsigned)sizeof(S));
#else
    return base + idx;
#endif
}

template <class S> struct PairIO;
template <> struct PairIO<float> {
    template <class Pol> __device__ static f2 ld2(const float *a) {
        return f2(Pol::ld(reinterpret_cast<const float2 *>(a)));
    }
    template <class Pol> __device__ static f2 ld11(const float *a0, const float *a1) {
        return f2(Pol::ld(a0), Pol::ld(a1));
    }
    __device__ static void st2(float *a, f2 v) { __stcs(reinterpret_cast<float2 *>(a), v.v); }
    __device__ static void st11(float *a0, float *a1, f2 v) {
        __stcs(a0, v.v.x);
        __stcs(a1, v.v.y);
    }
};
template <> struct PairIO<__half> {
    template <class Pol> __device__ static f2 ld2(const __half *a) {
        const unsigned int b = Pol::ld(reinterpret_cast<const unsigned int *>(a));
        __half2 h;
        *reinterpret_cast<unsigned int *>(&h) = b;
        return f2(__half22float2(h));
    }
    template <class Pol> __device__ static f2 ld11(const __half *a0, const __half *a1) {
        return f2(Store<__half>::ld<Pol>(a0), Store<__half>::ld<Pol>(a1));
    }
    __device__ static void st2(__half *a, f2 v) {
        const __half2 h = __floats2half2_rn(v.v.x, v.v.y);
        __stcs(reinterpret_cast<unsigned int *>(a), *reinterpret_cast<const unsigned int *>(&h));
    }
    __device__ static void st11(__half *a0, __half *a1, f2 v) {
        Store<__half>::st(a0, v.v.x);
        Store<__half>::st(a1, v.v.y);
    }
    // stochastic rounding, 16 random bits per cell from r
    __device__ static f2 dither(f2 v, unsigned r) {
        return f2(Store<__half>::sr_dither(v.v.x, r), Store<__half>::sr_dither(v.v.y, r >> 16));
    }
};

// Geometry of the cell pair: shared row offsets, per-cell x offsets with the wrap.
struct GeoPair {
    int x0, y, z;
    int s0;                      // cell index of x0 (lattices below 2^31 cells)
    int ox0[3], ox1[3], oy[3], oz[3];
};

__device__ __forceinline__ void geo_pair_at(const KParams &p, int x0, int y, int z, GeoPair &g) {
    g.x0 = x0;
    g.y = y;
    g.z = z;
    const int row = p.nx, plane = p.nx * p.ny;
    g.s0 = g.x0 + row * (g.y + p.ny * g.z);
    g.ox0[0] = g.x0 > 0 ? -1 : p.nx - 1;
    g.ox0[1] = 0;
    g.ox0[2] = 1;
    g.ox1[0] = -1;
    g.ox1[1] = 0;
    g.ox1[2] = g.x0 + 1 < p.nx - 1 ? 1 : 1 - p.nx;
    g.oy[0] = g.y > 0 ? -row : row * (p.ny - 1);
    g.oy[1] = 0;
    g.oy[2] = g.y < p.ny - 1 ? row : -row * (p.ny - 1);
    g.oz[0] = g.z > 0 ? -plane : plane * (p.nz - 1);
    g.oz[1] = 0;
    g.oz[2] = g.z < p.nz - 1 ? plane : -plane * (p.nz - 1);
}

__device__ __forceinline__ bool make_geo_pair(const KParams &p, GeoPair &g) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x), y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return false;
    geo_pair_at(p, x0, y, blockIdx.z + p.z0, g);
    return true;
}

template <class L, class S, bool ODD, bool WALL, class Pol = LdStream>
__device__ __forceinline__ void load_pair(const KParams &p, const Planes<S> &A, const GeoPair &g, f2 *f) {
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = opp(i);
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        if (!ODD) {
            f[i] = PairIO<S>::template ld2<Pol>(elem(A.p[i], g.s0));
        } else {
            bool from_wall = false;
            if (WALL && cy != 0) from_wall = (g.y - cy < 0) || (g.y - cy >= p.ny);
            if (from_wall) {
                f[i] = PairIO<S>::template ld2<Pol>(elem(A.p[i], g.s0));
            } else {
                const int r = g.s0 + g.oy[1 - cy] + g.oz[1 - cz];
                if (cx == 0)
                    f[i] = PairIO<S>::template ld2<Pol>(elem(A.p[o], r));
                else
                    f[i] = PairIO<S>::template ld11<Pol>(elem(A.p[o], r + g.ox0[1 - cx]),
                                                        elem(A.p[o], r + 1 + g.ox1[1 - cx]));
            }
        }
    });
}

// Population I of the pair to its place: the aligned slot of the opposite direction on even
// steps; on odd steps the neighbour in direction c_I, or, across a wall, the opposite slot of
// the cell itself (halfway bounce-back).  hsh: the pair's random bits (SR).
template <class L, class S, bool ODD, bool WALL, bool SR, int I>
__device__ __forceinline__ void store_dir(const KParams &p, const Planes<S> &A, const GeoPair &g, f2 v,
                                          unsigned hsh) {
    constexpr int o = opp(I);
    constexpr int cx = L::cx(I), cy = L::cy(I), cz = L::cz(I);
    if constexpr (SR) v = PairIO<S>::dither(v, dir_bits(hsh, I));
    if (!ODD) {
        PairIO<S>::st2(elem(A.p[o], g.s0), v);
    } else {
        bool to_wall = false;
        if (WALL && cy != 0) to_wall = (g.y + cy < 0) || (g.y + cy >= p.ny);
        if (to_wall) {
            PairIO<S>::st2(elem(A.p[o], g.s0), v);
        } else {
            const int r = g.s0 + g.oy[1 + cy] + g.oz[1 + cz];
            if (cx == 0)
                PairIO<S>::st2(elem(A.p[I], r), v);
            else
                PairIO<S>::st11(elem(A.p[I], r + g.ox0[1 + cx]), elem(A.p[I], r + 1 + g.ox1[1 + cx]), v);
        }
    }
}

// Collision of the pair with each population stored as soon as it is final (collide_emit).
template <class L, class S> struct UseMomentCollide {
    static constexpr bool value =
        std::is_same<L, D3Q19>::value && (PLB_MOMENT_COLLIDE == 2 || (PLB_MOMENT_COLLIDE == 1 && Store<S>::SHIFT));
};

// MOM: -1 the collision form of UseMomentCollide, 0 per pair, 1 moment space (D3Q19).
template <class L, class S, int MRT, bool ODD, bool WALL, bool SR, int MOM = -1>
__device__ __forceinline__ void collide_store_pair(const KParams &p, const Planes<S> &A, const GeoPair &g, f2 *f,
                                                   const f2 F[3], unsigned salt) {
    const unsigned hsh = SR ? cell_hash((unsigned)g.s0 + p.cell_base, salt) : 0u;
    auto emit = [&](auto ic, const f2 &v) { store_dir<L, S, ODD, WALL, SR, decltype(ic)::value>(p, A, g, v, hsh); };
    constexpr bool moment = MOM < 0 ? UseMomentCollide<L, S>::value : (MOM > 0 && std::is_same<L, D3Q19>::value);
    if constexpr (moment)
        collide_moments_d3q19<MRT, Store<S>::SHIFT, f2>(p, f, F, emit);
    else
        collide_emit<L, MRT, Store<S>::SHIFT, f2>(p, f, F, emit);
}

// Force densities of the two cells from their psi stencil; at(cx, cy, cz) returns psi of both
// cells at offset (cx, cy, cz) (the global or the shared-memory psi field).
// D3Q19 force stencil summed by velocity class (1) or direction by direction (0).
#ifndef PLB_GROUPED_FORCE
#define PLB_GROUPED_FORCE 1
#endif

// D3Q19: the moments summed by velocity class.  With dif_r / sum_r = psi(x + c_r) -+ psi(x - c_r)
// for the pairs r (axes x, y, z; (1, +-1, 0); (1, 0, +-1); (0, 1, +-1)), 3 w = 1/6 (axes) and
// 1/12 (edges), 9 w = 1/2 and 1/4, and 9 w_0 (0 - 1/3) = -1 at the rest velocity:
//   M1_x = dif_x / 6 + (dif_xy+ + dif_xy- + dif_xz+ + dif_xz-) / 12        (and y, z)
//   M2_xx = K + sum_x / 2 - S_yz / 4,   K = (S_edges - S_axes) / 6 - psi0    (and yy, zz)
//   M2_xy = (sum_xy+ - sum_xy-) / 4                                          (and xz, yz)
//   tr M2 = S_edges / 4 - 3 psi0
// where S_ab = sum_ab+ + sum_ab-, S_edges = S_xy + S_xz + S_yz, S_axes = sum_x + sum_y + sum_z.
template <class At>
__device__ __forceinline__ void force_pair_d3q19(const KParams &p, At &&at, f2 F[3]) {
    using L = D3Q19;
    const f2 psi0 = at(0, 0, 0);
    f2 dif[9], sum[9];
    Unroll<0, 9>::run([&](auto kc) {
        constexpr int i = 2 * decltype(kc)::value + 1;
        const f2 pa = at(L::cx(i), L::cy(i), L::cz(i)), pb = at(-L::cx(i), -L::cy(i), -L::cz(i));
        dif[decltype(kc)::value] = pa - pb;
        sum[decltype(kc)::value] = pa + pb;
    });
    const f2 m1[3] = {mad(f2(1.0f / 6.0f), dif[0], f2(1.0f / 12.0f) * ((dif[3] + dif[4]) + (dif[5] + dif[6]))),
                      mad(f2(1.0f / 6.0f), dif[1], f2(1.0f / 12.0f) * ((dif[3] - dif[4]) + (dif[7] + dif[8]))),
                      mad(f2(1.0f / 6.0f), dif[2], f2(1.0f / 12.0f) * ((dif[5] - dif[6]) + (dif[7] - dif[8])))};
    const f2 Sxy = sum[3] + sum[4], Sxz = sum[5] + sum[6], Syz = sum[7] + sum[8];
    const f2 Se = (Sxy + Sxz) + Syz, Sa = (sum[0] + sum[1]) + sum[2];
    const f2 K = mad(f2(1.0f / 6.0f), Se - Sa, -psi0);
    const f2 m2d[3] = {mad(f2(0.5f), sum[0], mad(f2(-0.25f), Syz, K)), mad(f2(0.5f), sum[1], mad(f2(-0.25f), Sxz, K)),
                       mad(f2(0.5f), sum[2], mad(f2(-0.25f), Sxy, K))};
    const f2 m2xy = f2(0.25f) * (sum[3] - sum[4]), m2xz = f2(0.25f) * (sum[5] - sum[6]),
             m2yz = f2(0.25f) * (sum[7] - sum[8]);
    const f2 tr = mad(f2(0.25f), Se, f2(-3.0f) * psi0);
    const Phys<float> &q = p.f;
    const f2 cA = f2(q.A_m1m2), cM = mad(f2(-q.G), psi0, f2(q.B_m1tr) * tr);
    const f2 m21[3] = {mad(m2d[0], m1[0], mad(m2xy, m1[1], m2xz * m1[2])),
                       mad(m2xy, m1[0], mad(m2d[1], m1[1], m2yz * m1[2])),
                       mad(m2xz, m1[0], mad(m2yz, m1[1], m2d[2] * m1[2]))};
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] = mad(cM, m1[a], mad(cA, m21[a], f2(q.fext[a])));
}

template <class L, class At>
__device__ __forceinline__ void force_pair_from(const KParams &p, At &&at, f2 F[3]) {
    if constexpr (std::is_same<L, D3Q19>::value && PLB_GROUPED_FORCE) {
        force_pair_d3q19(p, at, F);
        return;
    }
    const f2 psi0 = at(0, 0, 0);
    const f2 two_psi0 = psi0 + psi0;
    f2 m1[3] = {f2(0), f2(0), f2(0)};
    f2 m2[3][3] = {{f2(0), f2(0), f2(0)}, {f2(0), f2(0), f2(0)}, {f2(0), f2(0), f2(0)}};
    Unroll<0, (L::Q - 1) / 2>::run([&](auto kc) {
        constexpr int i = 2 * decltype(kc)::value + 1;
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const f2 pa = at(cx, cy, cz), pb = at(-cx, -cy, -cz);
        const f2 dif = pa - pb;
        const f2 sym = (pa + pb) - two_psi0;
        constexpr double w3 = 3.0 * L::w(i), w9 = 9.0 * L::w(i);
        constexpr int c[3] = {cx, cy, cz};
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
            if (c[a] != 0) m1[a] = mad(f2(w3 * c[a]), dif, m1[a]);
#pragma unroll
            for (int b = a; b < L::D; ++b) {
                const double coef = w9 * (c[a] * c[b] - (a == b ? 1.0 / 3.0 : 0.0));
                if (coef != 0.0) m2[a][b] = mad(f2(coef), sym, m2[a][b]);
            }
        }
    });
    f2 tr = m2[0][0] + m2[1][1];
    if (L::D == 3) tr += m2[2][2];
    const Phys<float> &q = p.f;
    const f2 cA = f2(q.A_m1m2), cM = mad(f2(-q.G), psi0, f2(q.B_m1tr) * tr);
#pragma unroll
    for (int a = 0; a < L::D; ++a) {
        f2 m21 = f2(0);
#pragma unroll
        for (int b = 0; b < L::D; ++b) m21 = mad(a <= b ? m2[a][b] : m2[b][a], m1[b], m21);
        F[a] = mad(cM, m1[a], mad(cA, m21, f2(q.fext[a])));
    }
    if (L::D == 2) F[2] = f2(0);
}

// Force densities of the two cells; pc points at psi of cell x0 (an even padded index).
template <class L, class Pol = LdStream>
__device__ __forceinline__ void force_pair(const KParams &p, const float *__restrict__ pc, f2 F[3]) {
    auto ldg2 = [](const float *a) { return Pol::ro(reinterpret_cast<const float2 *>(a)); };
    const int sy = p.px, sz = p.px * p.py;
    // psi of both cells at offset (cx, cy, cz), from three float2 per row
    auto at = [&](int cx, int cy, int cz) -> f2 {
        const float *r = pc + cy * sy + cz * sz;
        const float2 c = ldg2(r);
        if (cx == 0) return f2(c);
        if (cx < 0) return f2(ldg2(r - 2).y, c.x);
        return f2(c.y, ldg2(r + 2).x);
    };
    force_pair_from<L>(p, at, F);
}

// psi of one cell into the ghost layer (boundary cells only).
template <class L>
__device__ __forceinline__ void psi_ghosts(const KParams &p, float *psi, int x, int y, int z, float v) {
    int xs[3], ys[3], zs[3];
    int nxs = 1, nys = 1, nzs = 1;
    xs[0] = x;
    if (x == p.nx - 1) xs[nxs++] = -1;
    if (x == 0) xs[nxs++] = p.nx;
    ys[0] = y;
    if (p.wall_y) {
        // mirror rule; wetting walls keep the constant psi_wall written at creation
        if (y == 0 && !p.wall_fixed) ys[nys++] = -1;
        if (y == p.ny - 1 && !p.wall_fixed) ys[nys++] = p.ny;
    } else {
        if (y == p.ny - 1) ys[nys++] = -1;
        if (y == 0) ys[nys++] = p.ny;
    }
    zs[0] = z;
    if (L::D == 3) {
        if (z == p.nz - 1) zs[nzs++] = -1;
        if (z == 0) zs[nzs++] = p.nz;
    }
    for (int c = 0; c < nzs; ++c)
        for (int b = 0; b < nys; ++b)
            for (int a = (c == 0 && b == 0) ? 1 : 0; a < nxs; ++a) psi[psi_index(p, xs[a], ys[b], zs[c])] = v;
}

// psi of Eq. Interaction_Potential for two cells; raises the device flags on domain errors.
__device__ __forceinline__ f2 psi_pair_of(const KParams &p, f2 rho) {
    const Phys<float> &q = p.f;
    f2 pr;
    if (p.eos_kind == 0) {
        const f2 br = f2(q.pr_b) * rho;
        const f2 d1 = f2(1.0f) - br, d2 = mad(br, f2(2.0f) - br, f2(1.0f));
        pr = fdiv(rho * mad(f2(q.pr_RT), d2, f2(-q.pr_aalpha) * rho * d1), d1 * d2);
    } else {
        const f2 sr = f2(sqrtf(rho.v.x), sqrtf(rho.v.y));
        const f2 r2 = rho * rho;
        const float rv = q.pe_rv, rl = q.pe_rl, sv = q.pe_sv;
        // 2 r^3 + (rv - 2 rl) r^2 - 3 sv r^2.5 + 2 sv rl r^1.5 + sv rl^2 r^0.5
        f2 poly = mad(f2(2.0f), rho, f2(rv - 2.0f * rl)) * r2;
        poly = mad(mad(f2(-3.0f * sv), r2, mad(f2(2.0f * sv * rl), rho, f2(sv * rl * rl))), sr, poly);
        pr = f2(q.pe_P) * poly;
    }
    const f2 arg = f2(2.0f * q.inv_G) * mad(f2(q.p_scale), pr, f2(-1.0f / 3.0f) * rho);
    float out[2];
    const float rr[2] = {rho.v.x, rho.v.y}, aa[2] = {arg.v.x, arg.v.y};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(rr[c] > 0.0f) || !(rr[c] < INFINITY)) {
            atomicOr(p.flags, FLAG_NONFINITE);
            out[c] = 0.0f;
        } else if (!(aa[c] >= 0.0f)) {
            atomicOr(p.flags, FLAG_PSI_DOMAIN);
            out[c] = 0.0f;
        } else {
            out[c] = sqrtf(aa[c]);
        }
    }
    return f2(out[0], out[1]);
}

template <class L, class S, bool ODD, bool WALL, class Pol = LdStream>
__device__ __forceinline__ void psi_pair_body(const KParams &p, const Planes<S> &A, float *psi, const GeoPair &g) {
    f2 f[L::Q];
    load_pair<L, S, ODD, WALL, Pol>(p, A, g, f);
    f2 rho = f[0];
#pragma unroll
    for (int i = 1; i < L::Q; ++i) rho += f[i];
    if (Store<S>::SHIFT) rho += f2(p.f.rho_ref);   // sum_i w_i rho_ref = rho_ref
    const f2 v = psi_pair_of(p, rho);
    float *dst = psi + psi_index(p, g.x0, g.y, g.z);
    *reinterpret_cast<float2 *>(dst) = v.v;
    const bool by = g.y == 0 || g.y == p.ny - 1, bz = L::D == 3 && (g.z == 0 || g.z == p.nz - 1);
    if (by || bz || g.x0 == 0) psi_ghosts<L>(p, psi, g.x0, g.y, g.z, v.v.x);
    if (by || bz || g.x0 + 1 == p.nx - 1) psi_ghosts<L>(p, psi, g.x0 + 1, g.y, g.z, v.v.y);
}

template <class L, class S, bool ODD>
__global__ void __launch_bounds__(256) k_psi_pair(KParams p, Planes<S> A, float *__restrict__ psi) {
    GeoPair g;
    if (!make_geo_pair(p, g)) return;
    if (ODD && p.wall_y && (g.y == 0 || g.y == p.ny - 1))
        psi_pair_body<L, S, ODD, true>(p, A, psi, g);
    else
        psi_pair_body<L, S, ODD, false>(p, A, psi, g);
}

// psi pass over four cells per thread for FP16-shifted storage (x0 = 4 t, nx a multiple of 4):
// each direction is one aligned 8-byte load of the four cells' values, plus, for the x-shifted
// reads of odd steps, one 2-byte load of the element beyond the word (periodic wrap included).
template <class L, bool ODD, bool WALL>
__device__ __forceinline__ void psi_quad_body(const KParams &p, const Planes<__half> &A, float *psi, int x0, int y,
                                              int z) {
    GeoPair g;                                  // geometry of the pair (x0, x0 + 1): rows and planes
    geo_pair_at(p, x0, y, z, g);
    f2 r01 = f2(0.0f), r23 = f2(0.0f);
    auto h2f = [](unsigned w) {
        __half2 h;
        *reinterpret_cast<unsigned *>(&h) = w;
        return f2(__half22float2(h));
    };
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = opp(i);
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        bool from_wall = false;
        if (ODD && WALL && cy != 0) from_wall = (y - cy < 0) || (y - cy >= p.ny);
        const __half *base;
        int r;
        if (!ODD || from_wall) {
            base = A.p[i];
            r = g.s0;
        } else {
            base = A.p[o];
            r = g.s0 + g.oy[1 - cy] + g.oz[1 - cz];
        }
        const uint2 w = __ldcs(reinterpret_cast<const uint2 *>(base + r));     // elements x0 .. x0 + 3
        if (!ODD || cx == 0 || from_wall) {
            r01 += h2f(w.x);
            r23 += h2f(w.y);
        } else if (cx > 0) {
            // elements x0 - 1 .. x0 + 2
            const int xl = x0 > 0 ? -1 : p.nx - 1;
            const unsigned e = __ldcs(reinterpret_cast<const unsigned short *>(base + r + xl));
            r01 += h2f(__byte_perm(e, w.x, 0x5410));
            r23 += h2f(__byte_perm(w.x, w.y, 0x5432));
        } else {
            // elements x0 + 1 .. x0 + 4
            const int xr = x0 + 4 < p.nx ? 4 : 4 - p.nx;
            const unsigned e = __ldcs(reinterpret_cast<const unsigned short *>(base + r + xr));
            r01 += h2f(__byte_perm(w.x, w.y, 0x5432));
            r23 += h2f(__byte_perm(w.y, e, 0x5432));
        }
    });
    r01 += f2(p.f.rho_ref);                        // sum_i w_i rho_ref = rho_ref
    r23 += f2(p.f.rho_ref);
    const f2 v01 = psi_pair_of(p, r01), v23 = psi_pair_of(p, r23);
    float *dst = psi + psi_index(p, x0, y, z);
    *reinterpret_cast<float4 *>(dst) = make_float4(v01.v.x, v01.v.y, v23.v.x, v23.v.y);
    const bool by = y == 0 || y == p.ny - 1, bz = L::D == 3 && (z == 0 || z == p.nz - 1);
    if (by || bz || x0 == 0) psi_ghosts<L>(p, psi, x0, y, z, v01.v.x);
    if (by || bz) {
        psi_ghosts<L>(p, psi, x0 + 1, y, z, v01.v.y);
        psi_ghosts<L>(p, psi, x0 + 2, y, z, v23.v.x);
    }
    if (by || bz || x0 + 3 == p.nx - 1) psi_ghosts<L>(p, psi, x0 + 3, y, z, v23.v.y);
}

// Blocks of 256 threads with an explicit minimum of one resident block per SM: the register
// allocator then keeps more loads in flight per thread (54 / 72 registers for even / odd steps
// against 32 / 44 with the thread count alone), measured 92.9 -> 94.2 % of the copy bandwidth.
template <class L, bool ODD>
__global__ void __launch_bounds__(256, 1) k_psi_quad(KParams p, Planes<__half> A, float *__restrict__ psi) {
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x), y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return;
    const int z = blockIdx.z + p.z0;
    if (ODD && p.wall_y && (y == 0 || y == p.ny - 1))
        psi_quad_body<L, ODD, true>(p, A, psi, x0, y, z);
    else
        psi_quad_body<L, ODD, false>(p, A, psi, x0, y, z);
}

// Threads per block and register cap of the pair collide kernel: 64 threads and 112
// registers leave 18 warps resident per SM (measured best for FP32 and FP16 storage against
// 256 x 128, 128 x 96, 128 x 80 and 64 x 88).
#ifndef PLB_PAIR_THREADS
#define PLB_PAIR_THREADS 64
#endif
#ifndef PLB_PAIR_MAXREG
#define PLB_PAIR_MAXREG 112
#endif

template <class L, class S, int MRT, bool ODD, bool WALL, class Pol = LdStream, bool SR = false>
__device__ __forceinline__ void collide_pair_body(const KParams &p, const Planes<S> &A, const float *__restrict__ psi,
                                                  const GeoPair &g, unsigned salt = 0) {
    f2 f[L::Q];
    load_pair<L, S, ODD, WALL, Pol>(p, A, g, f);
    f2 F[3];
    force_pair<L, Pol>(p, psi + psi_index(p, g.x0, g.y, g.z), F);
    collide_store_pair<L, S, MRT, ODD, WALL, SR>(p, A, g, f, F, salt);
}

// L2 prefetch of the populations of the cell pair that the same thread of the block
// `ahead` launch slots later will update (blocks start roughly in linear order), so that one
// wave of blocks has the next wave's loads in flight without holding them in registers.
template <class L, class S>
__device__ __forceinline__ void prefetch_ahead_pair(const KParams &p, const Planes<S> &A) {
    // block index + prefetch_ahead in linear launch order, from its per-axis parts with carries
    int bx = blockIdx.x + p.pf_step[0], by = blockIdx.y + p.pf_step[1], bz = blockIdx.z + p.pf_step[2];
    if (bx >= (int)gridDim.x) { bx -= gridDim.x; ++by; }
    if (by >= (int)gridDim.y) { by -= gridDim.y; ++bz; }
    if (bz >= (int)gridDim.z) return;
    const int x0 = 2 * (bx * blockDim.x + threadIdx.x), y = by * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return;
    const int s0 = x0 + p.nx * (y + p.ny * (bz + p.z0));
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(A.p[i] + s0));
    });
}

// SR: stochastic rounding of the FP16 stores, a compile-time choice so that the
// round-to-nearest kernel is register-allocated for its own path.
template <class L, class S, int MRT, bool ODD, bool SR>
__global__ void __maxnreg__(PLB_PAIR_MAXREG) k_collide_pair(KParams p, Planes<S> A, const float *__restrict__ psi) {
    if (p.prefetch_ahead > 0) prefetch_ahead_pair<L, S>(p, A);
    GeoPair g;
    if (!make_geo_pair(p, g)) return;
    const bool wall = ODD && p.wall_y && (g.y == 0 || g.y == p.ny - 1);
    if (wall)
        collide_pair_body<L, S, MRT, ODD, true, LdStream, SR>(p, A, psi, g, p.salt);
    else
        collide_pair_body<L, S, MRT, ODD, false, LdStream, SR>(p, A, psi, g, p.salt);
}

}  // namespace plb
