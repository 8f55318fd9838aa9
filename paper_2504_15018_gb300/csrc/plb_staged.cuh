// Fused force / collide / stream pass of the two-cell kernels with the populations of the
// next plane staged in shared memory (cp.async) while the current plane is computed.
//
// A block of 64 threads owns a row segment of 128 cells (one cell pair per thread) and walks a
// chunk of z planes.  For every plane it copies, per direction, the 64 aligned two-cell words
// the threads read (plus one word on each side of the segment for the x-shifted reads of odd
// steps, periodic wrap included) from global memory into one of two shared-memory buffers with
// asynchronous 4-byte (FP16) or 8-byte (FP32) copies, one plane ahead of the computation, so the
// loads of plane z + 1 are in flight while plane z is collided, without holding them in
// registers.  The arithmetic and the stores are those of k_collide_pair (the same functions),
// so the populations are the same bit for bit.
//
// In the AA pattern every population slot is read and written by one cell only (the reading
// cell's own write), so loading a plane ahead of the previous plane's stores reads nothing that
// those stores change.
#pragma once
#include "plb_pair.cuh"

// z planes walked by one block of the staged kernel.
#ifndef PLB_STAGED_ZC
#define PLB_STAGED_ZC 16
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

template <class L> struct StagedShape {
    static constexpr int THREADS = 64;              // cell pairs of a row segment
    static constexpr int WORDS = THREADS + 2;       // words staged per direction and plane
};

// Copies plane z's words of every direction into buf.  x0 = X0 + 2 t; nw: active threads of
// the segment; active: this thread's pair lies in the lattice.
template <class L, class S, bool ODD, bool WALL>
__device__ __forceinline__ void stage_plane(const KParams &p, const Planes<S> &A, typename StageWord<S>::W *buf,
                                            int X0, int nw, int t, int y, int z) {
    using SW = StageWord<S>;
    constexpr int NW = StagedShape<L>::WORDS;
    if (t >= nw) return;
    GeoPair g;
    geo_pair_at(p, X0 + 2 * t, y, z, g);
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int o = opp(i);
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        typename SW::W *row = buf + i * NW;
        bool from_wall = false;
        if (ODD && WALL && cy != 0) from_wall = (y - cy < 0) || (y - cy >= p.ny);
        if (!ODD || from_wall) {
            SW::copy(row + 1 + t, elem(A.p[i], g.s0));
        } else {
            const int r = g.s0 + g.oy[1 - cy] + g.oz[1 - cz];      // the pair's own x in the source row
            const S *src = elem(A.p[o], r);
            SW::copy(row + 1 + t, src);
            if (cx != 0) {
                // the segment's outer neighbours, x = X0 - 2 and X0 + 2 nw (periodic)
                const int xs = X0 + 2 * t;
                if (cx > 0 && t == 0) SW::copy(row, src - xs + (X0 >= 2 ? X0 - 2 : p.nx - 2));
                if (cx < 0 && t == nw - 1) SW::copy(row + nw + 1, src - xs + (X0 + 2 * nw < p.nx ? X0 + 2 * nw : 0));
            }
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
    stage_plane<L, S, ODD, WALL>(p, A, stage[0], X0, nw, t, y, zb);
    cp_async_commit();
    for (int z = zb, k = 0; z < ze; ++z, ++k) {
        if (z + 1 < ze) {
            stage_plane<L, S, ODD, WALL>(p, A, stage[(k + 1) & 1], X0, nw, t, y, z + 1);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (t < nw) {
            f2 f[L::Q];
            read_staged<L, S, ODD, WALL>(p, stage[k & 1], t, y, f);
            GeoPair g;
            geo_pair_at(p, X0 + 2 * t, y, z, g);
            f2 F[3];
            force_pair<L>(p, psi + psi_index(p, g.x0, g.y, g.z), F);
            collide_store_pair<L, S, MRT, ODD, WALL, SR>(p, A, g, f, F, p.salt);
        }
        __syncthreads();
    }
}

#ifndef PLB_STAGED_MAXREG
#define PLB_STAGED_MAXREG 128
#endif

template <class L, class S, int MRT, bool ODD, bool SR>
__global__ void __maxnreg__(PLB_STAGED_MAXREG) k_collide_staged(KParams p, Planes<S> A, const float *__restrict__ psi) {
    __shared__ __align__(16) typename StageWord<S>::W stage[2][L::Q * StagedShape<L>::WORDS];
    const int y = blockIdx.y;
    if (ODD && p.wall_y && (y == 0 || y == p.ny - 1))
        staged_walk<L, S, MRT, ODD, true, SR>(p, A, psi, stage);
    else
        staged_walk<L, S, MRT, ODD, false, SR>(p, A, psi, stage);
}

}  // namespace plb
