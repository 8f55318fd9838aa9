// Fused force / collide / stream pass of the two-cell kernels with the populations of the
// next plane staged in shared memory (cp.async) while the current plane is computed.
//
// A block of 64 threads owns a row segment of 128 cells (one cell pair per thread) and walks a
// chunk of z planes.  For every plane it copies, per direction, the 64 aligned two-cell words
// the threads read (plus one word on each side of the segment for the x-shifted reads of odd
// steps, periodic wrap included, copied by ten lanes of the first warp, one x-shifted direction
// each) from global memory into one of two shared-memory buffers with asynchronous 4-byte
// (FP16) or 8-byte (FP32) copies, one plane ahead of the computation, so the loads of plane
// z + 1 are in flight while plane z is collided, without holding them in registers.  One
// barrier per plane: after it, every thread's copies of plane z are visible and every thread
// has finished reading plane z - 1, whose buffer then receives plane z + 1.  The arithmetic and
// the stores are those of k_collide_pair (the same functions), so the populations are the same
// bit for bit.
//
// In the AA pattern every population slot is read and written by one cell only (the reading
// cell's own write), so loading a plane ahead of the previous plane's stores reads nothing that
// those stores change.
#pragma once
#include "plb_pair.cuh"

// z planes walked by one block of the staged kernel (D3Q19 FP16S plates workload, GLUPS of the
// step: 4 planes 42.5, 6 42.6, 8 42.6, 12 42.7, 16 42.3, 32 41.7).
#ifndef PLB_STAGED_ZC
#define PLB_STAGED_ZC 8
#endif
// Plane buffers in shared memory: NB - 1 planes are loaded ahead of the one computed (three
// buffers measured 0.5 % slower than two: the larger shared-memory share leaves less L1 for the
// psi stencil).
#ifndef PLB_STAGED_BUFS
#define PLB_STAGED_BUFS 2
#endif

namespace plb {

template <class S> struct StageWord;
template <> struct StageWord<__half> {
    using W = unsigned;                                   // two FP16 values
    __device__ static void copy(W *dst, const __half *src) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                     "l"(src));
    }
    __device__ static f2 value(W w) {
        __half2 h;
        *reinterpret_cast<unsigned *>(&h) = w;
        return f2(__half22float2(h));
    }
    // elements (hi of a, lo of b)
    __device__ static W straddle(W a, W b) { return __byte_perm(a, b, 0x5432); }
};
template <> struct StageWord<float> {
    using W = float2;
    __device__ static void copy(W *dst, const float *src) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                     "l"(src));
    }
    __device__ static f2 value(W w) { return f2(w); }
    __device__ static W straddle(W a, W b) { return make_float2(a.y, b.x); }
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Cell pairs of a row segment (threads of a block).
#ifndef PLB_STAGED_THREADS
#define PLB_STAGED_THREADS 64
#endif

template <class L> struct StagedShape {
    static constexpr int THREADS = PLB_STAGED_THREADS;
    static constexpr int WORDS = THREADS + 2;       // words staged per direction and plane
};

// Odd steps, D3Q19: the outer neighbour word of the segment for the k-th of the ten directions
// with c_x != 0 (k < 10): x = X0 - 2 for c_x = +1, X0 + 2 nw for c_x = -1, periodic, from the
// source row of the direction (y - c_y, z - c_z).  Directions 1, 2 (x axis), 7-10 (x-y edges),
// 11-14 (x-z edges); odd i has c_x = +1, and c_y (7-10) or c_z (11-14) is +1, -1, -1, +1.
template <class S, bool WALL>
__device__ __forceinline__ void stage_halo_d3q19(const KParams &p, const Planes<S> &A, typename StageWord<S>::W *buf,
                                                 int X0, int nw, int k, int y, int z) {
    using SW = StageWord<S>;
    constexpr int NW = StagedShape<D3Q19>::WORDS;
    const int i = k < 2 ? 1 + k : 5 + k;
    const int o = (i & 1) ? i + 1 : i - 1;
    const int m = (i - 7) & 3;
    const int sign = (m == 0 || m == 3) ? 1 : -1;
    const int cy = (i >= 7 && i <= 10) ? sign : 0, cz = i >= 11 ? sign : 0;
    if (WALL && cy != 0 && (y - cy < 0 || y - cy >= p.ny)) return;      // bounced: no shifted read
    GeoPair g;
    geo_pair_at(p, X0, y, z, g);
    const int oyv = cy > 0 ? g.oy[0] : (cy < 0 ? g.oy[2] : 0);
    const int ozv = cz > 0 ? g.oz[0] : (cz < 0 ? g.oz[2] : 0);
    const int r = g.s0 - X0 + oyv + ozv;                                  // x = 0 of the source row
    if (i & 1)
        SW::copy(buf + i * NW, elem(A.p[o], r + (X0 >= 2 ? X0 - 2 : p.nx - 2)));
    else
        SW::copy(buf + i * NW + nw + 1, elem(A.p[o], r + (X0 + 2 * nw < p.nx ? X0 + 2 * nw : 0)));
}

// Copies plane z's words of every direction into buf.  x0 = X0 + 2 t; nw: active threads of
// the segment; active: this thread's pair lies in the lattice.
template <class L, class S, bool ODD, bool WALL>
__device__ __forceinline__ void stage_plane(const KParams &p, const Planes<S> &A, typename StageWord<S>::W *buf,
                                            int X0, int nw, int t, int y, int z) {
    using SW = StageWord<S>;
    constexpr int NW = StagedShape<L>::WORDS;
    // the segment's outer words of the ten x-shifted directions, one lane each
    static_assert(std::is_same<L, D3Q19>::value, "staged kernel: D3Q19 directions");
    if (ODD && t < 10) stage_halo_d3q19<S, WALL>(p, A, buf, X0, nw, t, y, z);
    if (t >= nw) return;
    GeoPair g;
    geo_pair_at(p, X0 + 2 * t, y, z, g);
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = opp(i);
        constexpr int cy = L::cy(i), cz = L::cz(i);
        typename SW::W *row = buf + i * NW;
        bool from_wall = false;
        if (ODD && WALL && cy != 0) from_wall = (y - cy < 0) || (y - cy >= p.ny);
        if (!ODD || from_wall) {
            SW::copy(row + 1 + t, elem(A.p[i], g.s0));
        } else {
            const int r = g.s0 + g.oy[1 - cy] + g.oz[1 - cz];      // the pair's own x in the source row
            SW::copy(row + 1 + t, elem(A.p[o], r));
        }
    });
}

// The two cells' pre-collision populations from the staged buffer.
template <class L, class S, bool ODD, bool WALL>
__device__ __forceinline__ void read_staged(const KParams &p, const typename StageWord<S>::W *buf, int t, int y,
                                            f2 *f) {
    using SW = StageWord<S>;
    constexpr int NW = StagedShape<L>::WORDS;
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int cx = L::cx(i), cy = L::cy(i);
        const typename SW::W *row = buf + i * NW;
        bool from_wall = false;
        if (ODD && WALL && cy != 0) from_wall = (y - cy < 0) || (y - cy >= p.ny);
        if (!ODD || cx == 0 || from_wall) {
            f[i] = SW::value(row[1 + t]);
        } else if (cx > 0) {
            f[i] = SW::value(SW::straddle(row[t], row[1 + t]));             // x0 - 1, x0
        } else {
            f[i] = SW::value(SW::straddle(row[1 + t], row[2 + t]));         // x0 + 1, x0 + 2
        }
    });
}

template <class L, class S, int MRT, bool ODD, bool WALL, bool SR>
__device__ __forceinline__ void staged_walk(const KParams &p, const Planes<S> &A, const float *__restrict__ psi,
                                            typename StageWord<S>::W (*stage)[L::Q * StagedShape<L>::WORDS]) {
    const int t = threadIdx.x, X0 = blockIdx.x * (2 * StagedShape<L>::THREADS), y = blockIdx.y;
    const int rem = (p.nx - X0) / 2;
    const int nw = rem < StagedShape<L>::THREADS ? rem : StagedShape<L>::THREADS;
    const int zb = p.z0 + blockIdx.z * PLB_STAGED_ZC;
    const int zlim = p.z0 + p.nzl;
    const int ze = zb + PLB_STAGED_ZC < zlim ? zb + PLB_STAGED_ZC : zlim;
    // planes zb .. zb + NB - 2 in flight before the first is computed
    constexpr int NB = PLB_STAGED_BUFS;
#pragma unroll
    for (int j = 0; j < NB - 1; ++j) {
        if (zb + j < ze) stage_plane<L, S, ODD, WALL>(p, A, stage[j], X0, nw, t, y, zb + j);
        cp_async_commit();
    }
    int cur = 0;                                   // buffer of plane z
    for (int z = zb; z < ze; ++z) {
        // this thread's copies of plane z are done once at most NB - 2 later groups are pending;
        // the barrier makes every thread's copies visible and ends the reads of plane z - 1
        cp_async_wait<NB - 2>();
        __syncthreads();
        const int nxt = cur == 0 ? NB - 1 : cur - 1;   // (cur + NB - 1) mod NB: plane z - 1's buffer
        if (z + NB - 1 < ze) stage_plane<L, S, ODD, WALL>(p, A, stage[nxt], X0, nw, t, y, z + NB - 1);
        cp_async_commit();
        if (t < nw) {
            f2 f[L::Q];
            read_staged<L, S, ODD, WALL>(p, stage[cur], t, y, f);
            GeoPair g;
            geo_pair_at(p, X0 + 2 * t, y, z, g);
            f2 F[3];
            force_pair<L>(p, psi + psi_index(p, g.x0, g.y, g.z), F);
            collide_store_pair<L, S, MRT, ODD, WALL, SR>(p, A, g, f, F, p.salt);
        }
        cur = cur + 1 == NB ? 0 : cur + 1;
    }
}

// Register caps of the staged kernel without and with stochastic rounding.  Uncapped, the
// stochastic-rounding kernels take 106 (even) and 118 (odd) registers; at 84 they fit 11 blocks
// per SM instead of 8-9 without spilling, measured +3 % for the FP16S step with stochastic
// rounding.  The round-to-nearest kernels take 94 / 100 registers uncapped and 86 / 92 at 96
// (no spills; +0.4 %); at 84 they measured the same as uncapped.
#ifndef PLB_STAGED_MAXREG
#define PLB_STAGED_MAXREG 96
#endif
#ifndef PLB_STAGED_MAXREG_SR
#define PLB_STAGED_MAXREG_SR 84
#endif

template <class L, class S, int MRT, bool ODD, bool SR>
__global__ void __maxnreg__(SR ? PLB_STAGED_MAXREG_SR : PLB_STAGED_MAXREG) k_collide_staged(KParams p, Planes<S> A, const float *__restrict__ psi) {
    __shared__ __align__(16) typename StageWord<S>::W stage[PLB_STAGED_BUFS][L::Q * StagedShape<L>::WORDS];
    const int y = blockIdx.y;
    if (ODD && p.wall_y && (y == 0 || y == p.ny - 1))
        staged_walk<L, S, MRT, ODD, true, SR>(p, A, psi, stage);
    else
        staged_walk<L, S, MRT, ODD, false, SR>(p, A, psi, stage);
}

}  // namespace plb
