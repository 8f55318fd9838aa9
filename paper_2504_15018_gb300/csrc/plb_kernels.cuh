// Readout kernels (init, moments, population exchange, reductions) and the launcher
// table of the step kernels (plb_step.cuh), templated over lattice and storage.
// Instantiated once per storage precision (plb_kern_*.cu).
#pragma once
#include <cuda_runtime.h>

#include "plb_device.cuh"
#include "plb_launch.h"
#include "plb_batch.cuh"
#include "plb_fused.cuh"
#include "plb_pair.cuh"
#include "plb_staged.cuh"
#include "plb_step.cuh"

// L2 prefetch one wave ahead in the FP32 fused pass (1) or not (0).
#ifndef PLB_L2_PREFETCH
#define PLB_L2_PREFETCH 1
#endif
// The same for FP16-shifted storage.
#ifndef PLB_L2_PREFETCH_HALF
#define PLB_L2_PREFETCH_HALF 0
#endif
// L2 prefetch distance of the fused pass in waves of resident blocks.
#ifndef PLB_PF_WAVES
#define PLB_PF_WAVES 1
#endif
// D3Q19 fused pass with the next plane staged in shared memory (plb_staged.cuh): FP16S storage
// (PLB_STAGED_HALF) and FP32 storage (PLB_STAGED_FLOAT).
#ifndef PLB_STAGED_HALF
#define PLB_STAGED_HALF 1
#endif
#ifndef PLB_STAGED_FLOAT
#define PLB_STAGED_FLOAT 0
#endif
// psi pass of FP16S storage over four cells per thread where nx is a multiple of 4.
#ifndef PLB_PSI_QUAD
#define PLB_PSI_QUAD 1
#endif
// Two cells per thread for FP16 storage (1) or one (0).
#ifndef PLB_HALF_PAIR
#define PLB_HALF_PAIR 1
#endif

namespace plb {

// Linear thread -> cell mapping (x fastest) for the readout kernels.
__device__ __forceinline__ bool cell_coords(const KParams &p, long long s, int &x, int &y, int &z) {
    if (s >= p.n) return false;
    const long long plane = (long long)p.nx * p.ny;
    z = (int)(s / plane);
    const long long r = s - (long long)z * plane;
    y = (int)(r / p.nx);
    x = (int)(r - (long long)y * p.nx);
    return true;
}

// ------------------------------------------------------------ init (a1)
// Records an invalid initial value: FLAG_BAD_INPUT and the smallest such index in `slot`.
__device__ __forceinline__ void bad_input(const KParams &p, int slot, long long idx) {
    atomicOr(p.flags, FLAG_BAD_INPUT);
    atomicMin(reinterpret_cast<unsigned long long *>(p.flags + slot), (unsigned long long)idx);
}

// f_i = f_i^eq(rho0, u0) in natural layout, for cells [c0, c0 + cn).  A rho0 that is not a
// positive finite number, or a non-finite u0 component, is recorded (bad_input).
template <class L, class S>
__global__ void k_init(KParams p, S *__restrict__ A, const double *__restrict__ rho0, const double *__restrict__ u0,
                       long long c0, long long cn, int has_u) {
    using T = typename Store<S>::T;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cn) return;
    const long long s = c0 + k;
    const double r0 = rho0[k];
    if (!(r0 > 0.0) || !(r0 < INFINITY)) bad_input(p, FLAG_SLOT_RHO, s);
    const T rho = (T)r0;
    T u[3] = {0, 0, 0};
    if (has_u)
        for (int a = 0; a < L::D; ++a) {
            const double ua = u0[a * cn + k];
            if (!(fabs(ua) < INFINITY)) bad_input(p, FLAG_SLOT_U, a * p.n + s);
            u[a] = (T)ua;
        }
    if constexpr (std::is_same<S, double>::value) {
        // FP64: Eq. Single_Phase_EDF evaluated as the plain collision does
        double f[L::Q];
        plain::equilibrium<L>(r0, u, f);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) Store<S>::st(A + (long long)i * p.pstride + s, f[i]);
        return;
    }
    const T usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T rref = phys<T>(p).rho_ref;
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const T cu = (T)L::cx(i) * u[0] + (T)L::cy(i) * u[1] + (T)L::cz(i) * u[2];
        const T feq = (T)L::w(i) * rho * ((T)1 - (T)1.5 * usq + (T)3 * cu + (T)4.5 * cu * cu);
        Store<S>::st(A + (long long)i * p.pstride + s, Store<S>::SHIFT ? feq - (T)L::w(i) * rref : feq);
    });
}

// -------------------------------------------------------------- moments (a6)
template <class L, class S>
__global__ void k_moments(KParams p, const S *__restrict__ A, const typename Store<S>::PsiT *__restrict__ psi, int odd,
                          double *__restrict__ rho_out, double *__restrict__ u_out, double *__restrict__ p_out,
                          long long c0, long long cn) {
    using T = typename Store<S>::T;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cn) return;
    const long long s = c0 + k;
    int x, y, z;
    cell_coords(p, s, x, y, z);
    const Nbr nb = neighbours(p, x, y, z);
    T f[L::Q];
    load_pops<L, S>(p, A, x, y, z, nb, s, odd != 0, f);
    T rho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        rho += f[i];
        j[0] += (T)L::cx(i) * f[i];
        j[1] += (T)L::cy(i) * f[i];
        j[2] += (T)L::cz(i) * f[i];
    }
    T F[3];
    cell_force<L, T>(p, psi, psi_index(p, x, y, z), F);
    if (rho_out) rho_out[k] = (double)rho;
    if (u_out)
        for (int a = 0; a < L::D; ++a) u_out[a * cn + k] = (double)((j[a] + (T)0.5 * F[a]) / rho);
    if (p_out) p_out[k] = (double)eos_pressure<T>(p, rho);
}

// ------------------------------------------------- balanced start (plb_init_physical)
// At t = 0 (even parity, natural layout) the populations are f^eq(rho, u0), so sum f c = rho u0.
// Rewrites them as f^eq(rho, u0 - F / (2 rho)), F the force of the initial density (psi pass
// already run), so that the velocity of Eq. Momentum, (sum f c + F/2) / rho, is u0.  Each
// thread reads and writes its own cell only.
template <class L, class S>
__global__ void k_rebalance(KParams p, S *__restrict__ A, const typename Store<S>::PsiT *__restrict__ psi) {
    using T = typename Store<S>::T;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    if (!cell_coords(p, s, x, y, z)) return;
    const Nbr nb = neighbours(p, x, y, z);
    T f[L::Q];
    load_pops<L, S>(p, A, x, y, z, nb, s, false, f);
    T rho = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        rho += f[i];
        j[0] += (T)L::cx(i) * f[i];
        j[1] += (T)L::cy(i) * f[i];
        j[2] += (T)L::cz(i) * f[i];
    }
    T F[3];
    cell_force<L, T>(p, psi, psi_index(p, x, y, z), F);
    T u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] - (T)0.5 * F[a]) / rho;
    const T usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T rref = phys<T>(p).rho_ref;
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const T cu = (T)L::cx(i) * u[0] + (T)L::cy(i) * u[1] + (T)L::cz(i) * u[2];
        const T feq = (T)L::w(i) * rho * ((T)1 - (T)1.5 * usq + (T)3 * cu + (T)4.5 * cu * cu);
        Store<S>::st(A + (long long)i * p.pstride + s, Store<S>::SHIFT ? feq - (T)L::w(i) * rref : feq);
    });
}

// ------------------------------------------------------------- wetting walls
// psi_wall into the ghost rows y = -1 and y = ny of the padded psi field, over the ghost columns
// and planes too (every node beyond a wall).  Nothing else writes these rows when the walls
// are wetting (psi_ghosts skips them), so this runs once, when the lattice is created.
template <class L, class S>
__global__ void k_wall_fill(KParams p, typename Store<S>::PsiT *__restrict__ psi) {
    using T = typename Store<S>::T;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cols = (long long)p.nx + 2, planes = L::D == 3 ? p.nz + 2 : 1;
    if (k >= cols * planes) return;
    const int x = (int)(k % cols) - 1;
    const int z = L::D == 3 ? (int)(k / cols) - 1 : 0;
    const typename Store<S>::PsiT v = (typename Store<S>::PsiT)phys<T>(p).psi_wall;
    psi[psi_index(p, x, -1, z)] = v;
    psi[psi_index(p, x, p.ny, z)] = v;
}

// ------------------------------------------------------ population exchange
template <class L, class S>
__global__ void k_get_pops(KParams p, const S *__restrict__ A, int odd, double *__restrict__ out, long long c0,
                           long long cn) {
    using T = typename Store<S>::T;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cn) return;
    const long long s = c0 + k;
    int x, y, z;
    cell_coords(p, s, x, y, z);
    const Nbr nb = neighbours(p, x, y, z);
    T f[L::Q];
    load_pops<L, S>(p, A, x, y, z, nb, s, odd != 0, f);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) out[i * cn + k] = (double)f[i];
}

template <class L, class S>
__global__ void k_set_pops(KParams p, S *__restrict__ A, const double *__restrict__ in, long long c0, long long cn) {
    using T = typename Store<S>::T;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cn) return;
    const long long s = c0 + k;
    const T rref = phys<T>(p).rho_ref;
    Unroll<0, L::Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const T v = (T)in[i * cn + k];
        Store<S>::st(A + (long long)i * p.pstride + s, Store<S>::SHIFT ? v - (T)L::w(i) * rref : v);
    });
}

// ----------------------------------------------------------- reductions (a4)
// Per-thread FP64 accumulation over a grid-stride loop, warp-shuffle tree, one
// partial per block (4 doubles); plb_reduce_final sums the partials in block order.
template <class L, class S>
__global__ void __launch_bounds__(256) k_reduce(KParams p, const S *__restrict__ A,
                                                const typename Store<S>::PsiT *__restrict__ psi, int odd, int what,
                                                int lox, int loy, int loz, int hix, int hiy, int hiz,
                                                double *__restrict__ partials) {
    using T = typename Store<S>::T;
    double acc[4] = {0, 0, 0, 0};
    const bool is_max = (what == 2);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < p.n; s += stride) {
        int x, y, z;
        cell_coords(p, s, x, y, z);
        if (x < lox || x >= hix || y < loy || y >= hiy || z < loz || z >= hiz) continue;
        const Nbr nb = neighbours(p, x, y, z);
        T f[L::Q];
        load_pops<L, S>(p, A, x, y, z, nb, s, odd != 0, f);
        double rho = 0, j[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < L::Q; ++i) rho += (double)f[i];
        if (what >= 1 && what <= 4) {
            // momentum only where it is used (GB300's FP64 rate is low); terms with a
            // zero velocity component add exactly 0 and are skipped
            Unroll<0, L::Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                if (L::cx(i) != 0) j[0] += (double)(L::cx(i) * f[i]);
                if (L::cy(i) != 0) j[1] += (double)(L::cy(i) * f[i]);
                if (L::cz(i) != 0) j[2] += (double)(L::cz(i) * f[i]);
            });
        }
        if (what == 0 || what == 5) {
            acc[0] += rho;
        } else if (what == 6) {
            acc[0] += (double)eos_pressure<T>(p, (T)rho);
        } else {
            T F[3];
            cell_force<L, T>(p, psi, psi_index(p, x, y, z), F);
            const double m[3] = {j[0] + 0.5 * (double)F[0], j[1] + 0.5 * (double)F[1], j[2] + 0.5 * (double)F[2]};
            if (what == 1) {
                acc[0] += m[0];
                acc[1] += m[1];
                acc[2] += m[2];
            } else {
                const double u2 = (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / (rho * rho);
                if (what == 2) acc[0] = fmax(acc[0], sqrt(u2));
                else if (what == 3) acc[0] += sqrt(u2);
                else acc[0] += u2;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = is_max ? fmax(v, w) : v + w;
        }
        acc[c] = v;
    }
    __shared__ double red[8][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int c = 0; c < 4; ++c) red[warp][c] = acc[c];
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = is_max ? 0.0 : 0.0;
        const int nw = blockDim.x >> 5;
        for (int w = 0; w < nw; ++w) v = is_max ? fmax(v, red[w][threadIdx.x]) : v + red[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = v;
    }
}

// Total mass of the whole lattice.  In either AA layout every population of every cell sits in
// exactly one slot of the store, so the mass is the sum of the Q planes over the N cells (plus
// N rho_ref with the FP16 shift): no coordinates, no neighbour addressing, coalesced loads.
// FP32 arithmetic: each cell's Q values are summed with an error-free compensated sum (TwoSum),
// the cell's sum and correction then added in FP64 per thread; FP64 storage sums in FP64.
// One partial per block in partials[4 * block] (the final pass sums them in block order).
template <class L, class S>
__global__ void __launch_bounds__(256) k_mass_flat(KParams p, const S *__restrict__ A, double *__restrict__ partials) {
    using T = typename Store<S>::T;
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < p.n; s += stride) {
        if constexpr (std::is_same<T, double>::value) {
            double r = 0.0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) r += Store<S>::ld(A + i * p.pstride + s);
            acc += r;
        } else {
            float sum = 0.0f, cor = 0.0f;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const float x = Store<S>::ld(A + i * p.pstride + s);
                const float t = sum + x, bb = t - sum;
                cor += (sum - (t - bb)) + (x - bb);
                sum = t;
            }
            acc += (double)sum + (double)cor;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        if (Store<S>::SHIFT && blockIdx.x == 0) v += (double)p.n * p.d.rho_ref;
        partials[blockIdx.x * 4] = v;
        partials[blockIdx.x * 4 + 1] = partials[blockIdx.x * 4 + 2] = partials[blockIdx.x * 4 + 3] = 0.0;
    }
}

// ----------------------------------------------------------------- launchers
template <class L, class S> struct Launch {
    using PsiT = typename Store<S>::PsiT;
    static unsigned blocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }
    // SMs of the current device (queried once per device, up to 64 devices)
    static int sm_count() {
        static int cache[64] = {0};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64) return 152;
        if (cache[dev] == 0) {
            int n = 0;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
            cache[dev] = n;
        }
        return cache[dev];
    }

    static void init(const KParams &p, void *A, const double *rho0, const double *u0, long long c0, long long cn,
                     cudaStream_t st) {
        k_init<L, S><<<blocks(cn, 256), 256, 0, st>>>(p, (S *)A, rho0, u0, c0, cn, u0 != nullptr);
    }
    static Planes<S> planes(const KParams &p, const void *A) {
        Planes<S> pl;
        for (int i = 0; i < 19; ++i) pl.p[i] = (S *)A + (i < L::Q ? (long long)i * p.pstride : 0);
        return pl;
    }
    static void dims3(const KParams &p, dim3 &grid, dim3 &block, int threads = 256) {
        int bx = p.nx >= threads ? threads : (p.nx + 31) / 32 * 32;
        int by = threads / bx;
        if (by > p.ny) by = p.ny;
        block = dim3(bx, by, 1);
        grid = dim3((p.nx + bx - 1) / bx, (p.ny + by - 1) / by, p.nzl);
    }
    // Two cells per thread with packed FP32 arithmetic where it applies (FP32 arithmetic,
    // even nx, fewer than 2^31 cells); one cell per thread otherwise.
    static bool use_pair(const KParams &p) {
        if (std::is_same<S, __half>::value && !PLB_HALF_PAIR) return false;
        // one population plane addressable with 32-bit cell indices and byte offsets
        return !std::is_same<S, double>::value && (p.nx % 2 == 0) && p.n * (long long)sizeof(S) < (1LL << 32);
    }
    static void dims_pair(const KParams &p, dim3 &grid, dim3 &block, int threads = 256) {
        const int npx = p.nx / 2;
        int bx = npx >= threads ? threads : (npx + 31) / 32 * 32;
        if (threads & (threads - 1)) bx = npx >= 64 ? 64 : (npx + 31) / 32 * 32;   // 64 wide
        int by = threads / bx;
        if (by > p.ny) by = p.ny;
        block = dim3(bx, by, 1);
        grid = dim3((npx + bx - 1) / bx, (p.ny + by - 1) / by, p.nzl);
    }
    template <bool ODD> static void psi_t(const KParams &p, const void *A, void *psi, cudaStream_t st) {
        dim3 grid, block;
        if constexpr (std::is_same<S, __half>::value) {
            if (PLB_PSI_QUAD && p.nx % 4 == 0 && p.n < (1LL << 31)) {
                const int nq = p.nx / 4;
                const int bx = nq >= 64 ? 64 : (nq + 31) / 32 * 32;
                int by = 256 / bx;
                if (by > p.ny) by = p.ny;
                k_psi_quad<L, ODD><<<dim3((nq + bx - 1) / bx, (p.ny + by - 1) / by, p.nzl), dim3(bx, by), 0, st>>>(
                    p, planes(p, A), (float *)psi);
                return;
            }
        }
        if constexpr (!std::is_same<S, double>::value) {
            if (use_pair(p)) {
                dims_pair(p, grid, block);
                k_psi_pair<L, S, ODD><<<grid, block, 0, st>>>(p, planes(p, A), (float *)psi);
                return;
            }
        }
        dims3(p, grid, block);
        if (p.n < (1LL << 31))
            k_psi_fast<L, S, ODD, int><<<grid, block, 0, st>>>(p, planes(p, A), (PsiT *)psi);
        else
            k_psi_fast<L, S, ODD, long long><<<grid, block, 0, st>>>(p, planes(p, A), (PsiT *)psi);
    }
    static void psi(const KParams &p, const void *A, void *psi, int odd, cudaStream_t st) {
        if (odd) psi_t<true>(p, A, psi, st);
        else psi_t<false>(p, A, psi, st);
    }
    // resident blocks per SM of the pair collide kernel (one wave = this x SM count)
    template <int MRT, bool ODD> static int pair_blocks_per_sm() {
        static int nb = 0;
        if (nb == 0) {
            int v = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_collide_pair<L, S, MRT, ODD, false>,
                                                              PLB_PAIR_THREADS, 0) != cudaSuccess || v < 1)
                v = 1;
            nb = v;
        }
        return nb;
    }
    template <int MRT, bool ODD> static void collide_t(const KParams &p, void *A, const void *psi, cudaStream_t st) {
        dim3 grid, block;
        if constexpr (!std::is_same<S, double>::value) {
            if constexpr (std::is_same<L, D3Q19>::value) {
                if (use_pair(p) && (std::is_same<S, __half>::value ? PLB_STAGED_HALF : PLB_STAGED_FLOAT) != 0) {
                    constexpr int per = 2 * StagedShape<L>::THREADS;
                    const dim3 sgrid((p.nx + per - 1) / per, p.ny, (p.nzl + PLB_STAGED_ZC - 1) / PLB_STAGED_ZC);
                    const dim3 sblock(StagedShape<L>::THREADS);
                    if constexpr (Store<S>::SHIFT) {
                        if (p.stochastic) {
                            k_collide_staged<L, S, MRT, ODD, true><<<sgrid, sblock, 0, st>>>(p, planes(p, A),
                                                                                             (const float *)psi);
                            return;
                        }
                    }
                    k_collide_staged<L, S, MRT, ODD, false><<<sgrid, sblock, 0, st>>>(p, planes(p, A), (const float *)psi);
                    return;
                }
            }
            if (use_pair(p)) {
                dims_pair(p, grid, block, PLB_PAIR_THREADS);
                // FP32 storage: prefetch into L2 for the block one wave (the resident blocks of
                // every SM) later; FP16S is bound by arithmetic and loses more to the extra
                // instructions than it gains
                KParams q = p;
                if ((std::is_same<S, float>::value ? PLB_L2_PREFETCH : PLB_L2_PREFETCH_HALF) != 0) {
                    const int ahead = PLB_PF_WAVES * pair_blocks_per_sm<MRT, ODD>() * sm_count();
                    q.prefetch_ahead = ahead;
                    q.pf_step[0] = ahead % (int)grid.x;
                    q.pf_step[1] = (ahead / (int)grid.x) % (int)grid.y;
                    q.pf_step[2] = ahead / ((int)grid.x * (int)grid.y);
                }
                if constexpr (Store<S>::SHIFT) {
                    if (p.stochastic) {
                        k_collide_pair<L, S, MRT, ODD, true><<<grid, block, 0, st>>>(q, planes(p, A),
                                                                                    (const float *)psi);
                        return;
                    }
                }
                k_collide_pair<L, S, MRT, ODD, false><<<grid, block, 0, st>>>(q, planes(p, A), (const float *)psi);
                return;
            }
        }
        if constexpr (std::is_same<S, double>::value) {
            dims3(p, grid, block, 128);
            if (p.n < (1LL << 31))
                k_collide_plain<L, MRT, ODD, int><<<grid, block, 0, st>>>(p, planes(p, A), (const double *)psi);
            else
                k_collide_plain<L, MRT, ODD, long long><<<grid, block, 0, st>>>(p, planes(p, A), (const double *)psi);
            return;
        }
        dims3(p, grid, block);
        if (p.n < (1LL << 31))
            k_collide_fast<L, S, MRT, ODD, int><<<grid, block, 0, st>>>(p, planes(p, A), (const PsiT *)psi);
        else
            k_collide_fast<L, S, MRT, ODD, long long><<<grid, block, 0, st>>>(p, planes(p, A), (const PsiT *)psi);
    }
    static void collide_bgk(const KParams &p, void *A, const void *psi, int odd, cudaStream_t st) {
        if (odd) collide_t<0, true>(p, A, psi, st);
        else collide_t<0, false>(p, A, psi, st);
    }
    static void collide_mrt(const KParams &p, void *A, const void *psi, int odd, cudaStream_t st) {
        if (odd) collide_t<1, true>(p, A, psi, st);
        else collide_t<1, false>(p, A, psi, st);
    }
    static void moments(const KParams &p, const void *A, const void *psi, int odd, double *r, double *u, double *pr,
                        long long c0, long long cn, cudaStream_t st) {
        k_moments<L, S><<<blocks(cn, 256), 256, 0, st>>>(p, (const S *)A, (const PsiT *)psi, odd, r, u, pr, c0, cn);
    }
    static void get_pops(const KParams &p, const void *A, int odd, double *out, long long c0, long long cn,
                         cudaStream_t st) {
        k_get_pops<L, S><<<blocks(cn, 256), 256, 0, st>>>(p, (const S *)A, odd, out, c0, cn);
    }
    static void set_pops(const KParams &p, void *A, const double *in, long long c0, long long cn, cudaStream_t st) {
        k_set_pops<L, S><<<blocks(cn, 256), 256, 0, st>>>(p, (S *)A, in, c0, cn);
    }
    static void reduce(const KParams &p, const void *A, const void *psi, int odd, int what, const int lo[3],
                       const int hi[3], double *partials, int nblocks, cudaStream_t st) {
        k_reduce<L, S><<<nblocks, 256, 0, st>>>(p, (const S *)A, (const PsiT *)psi, odd, what, lo[0], lo[1], lo[2],
                                                hi[0], hi[1], hi[2], partials);
    }
    static void mass(const KParams &p, const void *A, double *partials, int nblocks, cudaStream_t st) {
        k_mass_flat<L, S><<<nblocks, 256, 0, st>>>(p, (const S *)A, partials);
    }
    static void wall_fill(const KParams &p, void *psi, cudaStream_t st) {
        const long long n = ((long long)p.nx + 2) * (L::D == 3 ? p.nz + 2 : 1);
        k_wall_fill<L, S><<<blocks(n, 256), 256, 0, st>>>(p, (PsiT *)psi);
    }
    static void rebalance(const KParams &p, void *A, const void *psi, cudaStream_t st) {
        k_rebalance<L, S><<<blocks(p.n, 256), 256, 0, st>>>(p, (S *)A, (const PsiT *)psi);
    }
    // resident blocks per SM of the single-pass kernel
    template <int MRT> static int fused_blocks_per_sm() {
        static int nb = 0;
        if (nb == 0) {
            int v = 0;
            if constexpr (!std::is_same<S, double>::value) {
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_fused_pair<L, S, MRT, false>,
                                                                  FusedTile<L, S>::THREADS, 0) != cudaSuccess || v < 1)
                    v = 1;
            }
            nb = v < 1 ? 1 : v;
        }
        return nb;
    }
    // single pass: tiles of 64 x 16 (FP32) or 64 x 32 (FP16) cells, each block walking a chunk
    // of zc planes.  The chunk
    // count minimises (waves of resident blocks) x (planes per chunk + 0.5): a block also forms
    // psi of the two planes before its chunk, at about a third of a collided plane's cost each,
    // and the last wave of a grid that is not a multiple of the resident blocks runs partly idle.
    template <int MRT> static void fused_t(const KParams &p, const void *A, void *B, cudaStream_t st) {
        if constexpr (!std::is_same<S, double>::value) {
            using Tl = FusedTile<L, S>;
            const int gx = (p.nx + Tl::TX - 1) / Tl::TX, gy = (p.ny + Tl::TY - 1) / Tl::TY;
            int zc = 1, gz = 1;
            if (L::D == 3) {
                const long long tiles = (long long)gx * gy;
                const long long resident = (long long)fused_blocks_per_sm<MRT>() * sm_count();
                // the last search's result (one lattice stepped many times asks the same again)
                static thread_local long long key[3] = {-1, -1, -1};
                static thread_local int last[2] = {1, 1};
                if (key[0] != tiles || key[1] != resident || key[2] != p.nz) {
                    double best = 0.0;
                    const int gmax = p.nz < 4096 ? p.nz : 4096;
                    for (int g = 1; g <= gmax; ++g) {
                        const int zcg = (p.nz + g - 1) / g;
                        const int gzg = (p.nz + zcg - 1) / zcg;
                        if (gzg != g) continue;                       // the same chunking as a smaller g
                        const long long waves = (tiles * gzg + resident - 1) / resident;
                        const double cost = (double)waves * (zcg + 0.5);
                        if (g == 1 || cost < best) {
                            best = cost;
                            last[0] = zcg;
                            last[1] = gzg;
                        }
                    }
                    key[0] = tiles;
                    key[1] = resident;
                    key[2] = p.nz;
                }
                zc = last[0];
                gz = last[1];
            }
            const dim3 grid(gx, gy, gz), block(Tl::THREADS);
            if constexpr (Store<S>::SHIFT) {
                if (p.stochastic) {
                    k_fused_pair<L, S, MRT, true><<<grid, block, 0, st>>>(p, planes(p, A), planes(p, B), zc);
                    return;
                }
            }
            k_fused_pair<L, S, MRT, false><<<grid, block, 0, st>>>(p, planes(p, A), planes(p, B), zc);
        }
    }
    static void fused_bgk(const KParams &p, const void *A, void *B, cudaStream_t st) { fused_t<0>(p, A, B, st); }
    static void fused_mrt(const KParams &p, const void *A, void *B, cudaStream_t st) { fused_t<1>(p, A, B, st); }
    static const void *batch_bgk() { return reinterpret_cast<const void *>(&k_batch<L, S, 0>); }
    static const void *batch_mrt() { return reinterpret_cast<const void *>(&k_batch<L, S, 1>); }
    static constexpr Launchers table() {
        return Launchers{&init,     &psi,    {&collide_bgk, &collide_mrt}, &moments, &get_pops, &set_pops, &reduce,
                         {&batch_bgk, &batch_mrt}, &rebalance, &wall_fill,
                         {std::is_same<S, double>::value ? nullptr : &fused_bgk,
                          std::is_same<S, double>::value ? nullptr : &fused_mrt},
                         &mass};
    }
};

}  // namespace plb
