// Single-pass time step: psi, force, collision and streaming in one kernel (FP32 arithmetic,
// FP32 or FP16-shifted storage, even nx).
//
// The two-pass step reads every population twice per step (psi pass, fused pass).  Here each
// block owns a tile of TX x TY cells in x-y and walks along z through a chunk of ZC planes.
// For plane z + 1 it computes psi of the tile plus a one-cell halo (two cells in x, so that
// psi is formed for aligned cell pairs exactly as in the psi pass) into a three-plane ring in
// shared memory; then it collides plane z, whose psi stencil (planes z - 1, z, z + 1) is now
// in shared memory, reading the plane's populations a second time (from L2: they were read
// one plane earlier for psi).  Halo psi values are recomputed by every block that needs them.
//
// Populations live in two copies: the kernel reads A (natural layout, f_i(x) at A[i][x]) and
// pushes the post-collision populations into B (B[i][x + c_i], halfway bounce-back at the y
// walls), so no block can read a population another block has already overwritten.  The
// per-cell arithmetic (psi_pair_of, force_pair_from, collide_store_pair) is the code of the
// two-pass kernels; with the same collision form (always for D2Q9 and FP16 storage) both give
// the same populations bit for bit.
#pragma once
#include "plb_pair.cuh"

#ifndef PLB_FUSED_PSI_POL
#define PLB_FUSED_PSI_POL LdKeep
#endif

// Collision form of the single pass: 1 the moment-space D3Q19 collision for every storage
// precision (FP32 single pass on the D3Q19 plates workload: 27.3 -> 29.1 GLUPS; its populations
// then differ from the two-pass FP32 kernels, which keep the per-pair form, by rounding), -1 the
// form of the two-pass kernels (bit-identical to them).
#ifndef PLB_FUSED_MOMENT
#define PLB_FUSED_MOMENT 1
#endif

namespace plb {

// v in [-n, 2n) wrapped into [0, n); any v for lattices narrower than a tile.
__device__ __forceinline__ int wrap_near(int v, int n) {
    if (v < 0) v += n;
    else if (v >= n) v -= n;
    if ((unsigned)v >= (unsigned)n) v = ((v % n) + n) % n;
    return v;
}

// Tile rows (FP32 and FP16 storage) and threads per block of the single pass (two blocks of 256
// threads per SM at the 128-register cap).  D3Q19 plates workload, GLUPS with 8 / 16 / 32 rows:
// FP32 27.9 / 29.0 / 26.6, FP16S 31.7 / 34.3 / 36.2.
#ifndef PLB_FUSED_TY
#define PLB_FUSED_TY 16
#endif
#ifndef PLB_FUSED_TY_HALF
#define PLB_FUSED_TY_HALF 32
#endif
#ifndef PLB_FUSED_THREADS
#define PLB_FUSED_THREADS 256
#endif

template <class L, class S> struct FusedTile {
    static constexpr int TX = 64;                      // cells in x (32 pairs)
    static constexpr int TY = sizeof(S) == 2 ? PLB_FUSED_TY_HALF : PLB_FUSED_TY;   // rows
    static constexpr int HP = TX / 2 + 2;              // pairs per shared row: one halo pair each side
    static constexpr int RY = TY + 2;                  // rows with the halo
    static constexpr int NPL = L::D == 3 ? 3 : 1;      // psi planes in the ring
    static constexpr int THREADS = PLB_FUSED_THREADS;
};

// psi of the halo-extended tile of plane zg (any integer: wrapped) into ring plane `plane`.
// Shared element (ly, 2 hp + c) holds psi of x = x0 - 2 + 2 hp + c, y = y0 - 1 + ly.
template <class L, class S>
__device__ __forceinline__ void fused_psi_plane(const KParams &p, const Planes<S> &A, float *plane, int x0, int y0,
                                                int zg) {
    using Tl = FusedTile<L, S>;
    const int z = wrap_near(zg, p.nz);
    for (int k = threadIdx.x; k < Tl::RY * Tl::HP; k += Tl::THREADS) {
        const int ly = k / Tl::HP, hp = k - ly * Tl::HP;
        int y = y0 - 1 + ly;
        float *dst = plane + ly * (2 * Tl::HP) + 2 * hp;
        if (p.wall_fixed && (y < 0 || y >= p.ny)) {
            // wetting walls: the nodes beyond the walls carry psi_wall
            *reinterpret_cast<float2 *>(dst) = make_float2(p.f.psi_wall, p.f.psi_wall);
            continue;
        }
        if (p.wall_y) {
            // the ghost rows beyond the walls mirror the first and last fluid rows; rows past
            // the halo of a ragged tile are clamped (computed, never read)
            y = y < 0 ? 0 : (y >= p.ny ? p.ny - 1 : y);
        } else {
            y = wrap_near(y, p.ny);
        }
        const int x = wrap_near(x0 - 2 + 2 * hp, p.nx);     // even: nx is even
        const int s0 = x + p.nx * (y + p.ny * z);
        f2 f[L::Q];
        Unroll<0, L::Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            f[i] = PairIO<S>::template ld2<PLB_FUSED_PSI_POL>(A.p[i] + s0);
        });
        f2 rho = f[0];
#pragma unroll
        for (int i = 1; i < L::Q; ++i) rho += f[i];
        if (Store<S>::SHIFT) rho += f2(p.f.rho_ref);   // sum_i w_i rho_ref = rho_ref
        const f2 v = psi_pair_of(p, rho);
        *reinterpret_cast<float2 *>(dst) = v.v;
    }
}

template <class L, class S, int MRT, bool SR>
__device__ __forceinline__ void fused_collide_plane(const KParams &p, const Planes<S> &A, const Planes<S> &B,
                                                    const float *pm, const float *pc, const float *pp, int x0,
                                                    int y0, int z, unsigned salt) {
    using Tl = FusedTile<L, S>;
    constexpr int NP = Tl::TX / 2;
    constexpr int row = 2 * Tl::HP;
    for (int k = threadIdx.x; k < Tl::TY * NP; k += Tl::THREADS) {
        const int ly = k / NP, lp = k - ly * NP;
        const int x = x0 + 2 * lp, y = y0 + ly;
        if (x >= p.nx || y >= p.ny) continue;
        GeoPair g;
        geo_pair_at(p, x, y, z, g);
        f2 f[L::Q];
        load_pair<L, S, false, false>(p, A, g, f);
        // psi of both cells at offset (cx, cy, cz) from the shared ring
        const int e = (ly + 1) * row + 2 * (lp + 1);
        auto at = [&](int cx, int cy, int cz) -> f2 {
            const float *r = (cz < 0 ? pm : (cz > 0 ? pp : pc)) + e + cy * row;
            const float2 c = *reinterpret_cast<const float2 *>(r);
            if (cx == 0) return f2(c);
            if (cx < 0) return f2(reinterpret_cast<const float2 *>(r - 2)->y, c.x);
            return f2(c.y, reinterpret_cast<const float2 *>(r + 2)->x);
        };
        f2 F[3];
        force_pair_from<L>(p, at, F);
        // push streaming into B: the odd-parity store of the two-pass kernels
        if (p.wall_y && (y == 0 || y == p.ny - 1))
            collide_store_pair<L, S, MRT, true, true, SR, PLB_FUSED_MOMENT>(p, B, g, f, F, salt);
        else
            collide_store_pair<L, S, MRT, true, false, SR, PLB_FUSED_MOMENT>(p, B, g, f, F, salt);
    }
}

// Grid: (ceil(nx / TX), ceil(ny / TY), ceil(nz / zc)); block: THREADS threads.
template <class L, class S, int MRT, bool SR>
__global__ void __launch_bounds__(PLB_FUSED_THREADS, 512 / PLB_FUSED_THREADS) k_fused_pair(KParams p, Planes<S> A, Planes<S> B, int zc) {
    using Tl = FusedTile<L, S>;
    constexpr int PLANE = Tl::RY * 2 * Tl::HP;
    __shared__ __align__(16) float ring[Tl::NPL * PLANE];
    const int x0 = blockIdx.x * Tl::TX, y0 = blockIdx.y * Tl::TY;
    const int zb = blockIdx.z * zc;
    const int ze = min(zb + zc, p.nz);
    const unsigned salt = p.salt;
    if (L::D == 2) {
        fused_psi_plane<L, S>(p, A, ring, x0, y0, 0);
        __syncthreads();
        fused_collide_plane<L, S, MRT, SR>(p, A, B, ring, ring, ring, x0, y0, 0, salt);
        return;
    }
    // ring slot of plane zz: (zz - zb + 1) mod 3
    fused_psi_plane<L, S>(p, A, ring, x0, y0, zb - 1);
    fused_psi_plane<L, S>(p, A, ring + PLANE, x0, y0, zb);
    for (int z = zb; z < ze; ++z) {
        const int r = z - zb;
        fused_psi_plane<L, S>(p, A, ring + ((r + 2) % 3) * PLANE, x0, y0, z + 1);
        __syncthreads();
        fused_collide_plane<L, S, MRT, SR>(p, A, B, ring + (r % 3) * PLANE, ring + ((r + 1) % 3) * PLANE,
                                           ring + ((r + 2) % 3) * PLANE, x0, y0, z, salt);
        __syncthreads();
    }
}

}  // namespace plb
