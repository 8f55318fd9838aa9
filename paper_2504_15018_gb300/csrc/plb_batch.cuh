// Persistent kernel of a batch of independent lattices: every step runs the psi pass over
// all tiles of all instances, a grid barrier, the fused force/collide/stream pass, and a
// second barrier, for nsteps steps in one launch.  Loads follow LdBatch (populations through
// L2 only, the psi stencil through L1 after the barrier's acquire):
// blocks read, across barriers, what other SMs wrote in the same launch.
#pragma once
#include "plb_pair.cuh"

namespace plb {

// Minimum resident 256-thread blocks per SM requested from the register allocator: the
// most that fit without spilling (D2Q9: 80 registers, 3 blocks; D3Q19 MRT: 128, 2 blocks).
template <class L> struct BatchMinBlocks { static constexpr int value = L::Q == 9 ? 3 : 2; };

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of the block) when
// any block gave up waiting, after which the kernel returns.
__device__ __forceinline__ bool grid_sync(GridBar *bar, unsigned expected, unsigned spin_limit) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned *vgen = &bar->gen;
        volatile unsigned *verr = &bar->err;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&bar->count, 1u);
        if (arrived == expected - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            unsigned spins = 0;
            while (*vgen == gen) {
                if (*verr) break;
                if (++spins > spin_limit) {
                    atomicOr(&bar->err, 1u);
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        s_ok = *verr == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class L, class S, int MRT, bool PSI, bool SR>
__device__ __forceinline__ void batch_tile(const BatchInst &in, const BatchTile &tl, int odd, unsigned salt) {
    const KParams &p = in.kp;
    const Planes<S> &A = *reinterpret_cast<const Planes<S> *>(in.pl);
    using PsiT = typename Store<S>::PsiT;
    const int units = (tl.y1 - tl.y0) * in.upr;
    for (int j = threadIdx.x; j < units; j += blockDim.x) {
        const int r = j / in.upr;
        const int y = tl.y0 + r, xu = j - r * in.upr;
        const bool wall = odd && p.wall_y && (y == 0 || y == p.ny - 1);
        bool done = false;
        if constexpr (!std::is_same<S, double>::value) {
            if (in.pair) {
                GeoPair g;
                geo_pair_at(p, 2 * xu, y, tl.z, g);
                float *psi = static_cast<float *>(in.psi);
                if (PSI) {
                    if (!odd) psi_pair_body<L, S, false, false, LdBatch>(p, A, psi, g);
                    else if (wall) psi_pair_body<L, S, true, true, LdBatch>(p, A, psi, g);
                    else psi_pair_body<L, S, true, false, LdBatch>(p, A, psi, g);
                } else {
                    if (!odd) collide_pair_body<L, S, MRT, false, false, LdBatch, SR>(p, A, psi, g, salt);
                    else if (wall) collide_pair_body<L, S, MRT, true, true, LdBatch, SR>(p, A, psi, g, salt);
                    else collide_pair_body<L, S, MRT, true, false, LdBatch, SR>(p, A, psi, g, salt);
                }
                done = true;
            }
        }
        if (!done) {
            Geo<int> g;
            geo_at<int>(p, xu, y, tl.z, g);
            PsiT *psi = static_cast<PsiT *>(in.psi);
            if (PSI) {
                if (!odd) psi_body<L, S, false, false, LdBatch>(p, A, psi, g);
                else if (wall) psi_body<L, S, true, true, LdBatch>(p, A, psi, g);
                else psi_body<L, S, true, false, LdBatch>(p, A, psi, g);
            } else {
                if (!odd) collide_body<L, S, MRT, false, false, LdBatch, SR>(p, A, psi, g, salt);
                else if (wall) collide_body<L, S, MRT, true, true, LdBatch, SR>(p, A, psi, g, salt);
                else collide_body<L, S, MRT, true, false, LdBatch, SR>(p, A, psi, g, salt);
            }
        }
    }
}

template <class L, class S, int MRT>
__global__ void __launch_bounds__(256, BatchMinBlocks<L>::value) k_batch(BatchLaunch b) {
    const unsigned salt0 = *reinterpret_cast<volatile unsigned *>(&b.bar->salt);
    for (int step = 0; step < b.nsteps; ++step) {
        for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
            const BatchTile tl = b.tiles[t];
            const BatchInst &in = b.insts[tl.inst];
            batch_tile<L, S, MRT, true, false>(in, tl, (in.odd + step) & 1, 0);
        }
        if (!grid_sync(b.bar, b.expected, b.spin_limit)) return;
        for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
            const BatchTile tl = b.tiles[t];
            const BatchInst &in = b.insts[tl.inst];
            const int odd = (in.odd + step) & 1;
            if constexpr (Store<S>::SHIFT) {
                if (in.kp.stochastic) {
                    batch_tile<L, S, MRT, false, true>(in, tl, odd, salt0 + step);
                    continue;
                }
            }
            batch_tile<L, S, MRT, false, false>(in, tl, odd, 0);
        }
        if (!grid_sync(b.bar, b.expected, b.spin_limit)) return;
    }
    // every block has passed the last barrier: advance the stored parities and the step salt
    if (blockIdx.x == 0) {
        if (b.nsteps & 1)
            for (int k = threadIdx.x; k < b.ninst; k += blockDim.x) b.insts[k].odd ^= 1;
        if (threadIdx.x == 0) b.bar->salt = salt0 + b.nsteps;
    }
}

}  // namespace plb
