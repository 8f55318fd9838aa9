// Host-visible kernel parameter block and launcher table (one table per
// lattice x storage precision, defined in plb_kern_*.cu).
#pragma once
#include <cuda_runtime.h>

namespace plb {

enum : unsigned { FLAG_PSI_DOMAIN = 1u, FLAG_NONFINITE = 2u, FLAG_BAD_INPUT = 4u };
// Device flag area of a lattice (64 bytes): word 0 holds the FLAG_* bits; the 8-byte slots
// at words 2 and 4 hold the first invalid rho0 and u0 index k_init met (all ones if none).
enum : int { FLAG_SLOT_RHO = 2, FLAG_SLOT_U = 4 };

// Physical parameters in the arithmetic precision of a kernel (FP64 and FP32 copies are
// both filled on the host, so no kernel converts a double per thread).
template <class T> struct Phys {
    T G, A_m1m2, B_m1tr;      // F = -G psi M1 + A (M2 . M1) + B M1 tr(M2) + fext
    T inv_G;                  // 1 / G
    T tau_l, tau_v, tau_rho_v, inv_drho_tau;
    T om_const;               // 1 / tau_l (constant-tau case)
    T s_rate[6];              // MRT rate by Ghosts::kind (1..5)
    T fext[3];
    T rho_ref;                // FP16S shift
    T pr_RT, pr_b, pr_aalpha;
    T pe_P, pe_rv, pe_rl, pe_sv;
    T p_scale;
    T psi_wall;               // psi on wetting walls (used when KParams::wall_fixed)
};

// Constants of the plain FP64 evaluation (plb_plain.cuh), each formed on the host the way
// the equations write it.
struct PlainPhys {
    double R, T, b, a_alpha;                   // Peng-Robinson: R, absolute T, b, a alpha(T)
    double P, rv_2rl, sv3, sv2rl, svrlrl;      // Eq. EOS: p_c/rho_c^3, rho_v - 2 rho_l, 3 sqrt(rho_v),
                                               //   2 sqrt(rho_v) rho_l, sqrt(rho_v) rho_l rho_l
    double p_scale, G;
    double K1, K2;                             // G/12 (2 kappa - 2 - 3 eps), G/6 (kappa - 1)
    double tau_l, tau_v, tau_rho_v, d_rho, d_tau;   // tau(rho): rho_l - rho_v, tau_l - tau_v
    double s_rate[6];                          // MRT rates by kind (1..5)
    double fext[3];
};

struct KParams {
    int nx, ny, nz;
    int z0, nzl;          // the step kernels update planes z0 <= z < z0 + nzl (a slab: the planes between
                          // its two ghost planes; else 0 and nz)
    long long n;          // cells
    long long pstride;    // elements between population planes
    int wall_y;
    int wall_fixed;       // walls carry the constant psi_wall (ghost rows filled once), not a mirror
    // padded psi array: ghost layer of 1 in y (and z for 3-D), gx in x
    int px;               // row pitch in elements
    int py;               // rows per plane (ny + 2)
    long long psi_origin; // element offset of interior cell (0, 0, 0)
    int var_tau;
    int eos_kind;         // 0 PR, 1 paper
    int stochastic;       // FP16 stores with stochastic rounding
    int prefetch_ahead;   // k_collide_pair: prefetch into L2 for the block this many launch slots later (0: off)
    int pf_step[3];       // that offset split along the grid axes (x, y, z), for carry propagation
    unsigned salt;        // step counter mixed into the rounding noise
    unsigned cell_base;   // added to the cell index hashed for the rounding noise (a slab: its offset)
    Phys<double> d;
    Phys<float> f;
    PlainPhys pl;
    unsigned *flags;
};

// One instance of a batch, as the persistent kernel sees it (device memory).
struct BatchInst {
    KParams kp;            // kp.flags points at the instance's flags
    void *pl[19];          // population planes
    void *psi;             // padded psi field
    int odd;               // AA parity at the start of the launch (the kernel flips it at the end)
    int pair;              // 1: two cells per thread
    int upr;               // work units per row: nx / 2 (pair) or nx
    int pad;
};
// A tile: rows y0 <= y < y1 of plane z of one instance.
struct BatchTile {
    int inst, z, y0, y1;
};
// Grid barrier state (device memory, zeroed at creation).
struct GridBar {
    unsigned count, gen, err, salt;   // salt: steps taken, for the stochastic rounding noise
};
// Launch parameters of the persistent kernel.
struct BatchLaunch {
    BatchInst *insts;
    const BatchTile *tiles;
    int ninst, ntiles, nsteps;
    GridBar *bar;
    unsigned spin_limit;     // bounded wait: polls of the barrier before giving up
    unsigned expected;       // blocks the barrier waits for (gridDim.x unless testing a timeout)
};

struct Launchers {
    void (*init)(const KParams &, void *A, const double *rho0, const double *u0, long long c0, long long cn,
                 cudaStream_t);
    void (*psi)(const KParams &, const void *A, void *psi, int odd, cudaStream_t);
    void (*collide[2])(const KParams &, void *A, const void *psi, int odd, cudaStream_t);   // [BGK, MRT]
    void (*moments)(const KParams &, const void *A, const void *psi, int odd, double *rho, double *u, double *p,
                    long long c0, long long cn, cudaStream_t);
    void (*get_pops)(const KParams &, const void *A, int odd, double *out, long long c0, long long cn, cudaStream_t);
    void (*set_pops)(const KParams &, void *A, const double *in, long long c0, long long cn, cudaStream_t);
    void (*reduce)(const KParams &, const void *A, const void *psi, int odd, int what, const int lo[3],
                   const int hi[3], double *partials, int nblocks, cudaStream_t);
    // persistent batch kernel [BGK, MRT]: returns its entry point for launch / occupancy queries
    const void *(*batch_kernel[2])();
    // balanced start: f^eq(rho, u0) -> f^eq(rho, u0 - F / (2 rho)) at even parity (psi of rho given)
    void (*rebalance)(const KParams &, void *A, const void *psi, cudaStream_t);
    // wetting walls: psi_wall into the ghost rows y = -1 and y = ny of the padded psi field
    void (*wall_fill)(const KParams &, void *psi, cudaStream_t);
    // single-pass step [BGK, MRT]: reads A (natural layout), pushes into B; NULL for FP64
    void (*fused[2])(const KParams &, const void *A, void *B, cudaStream_t);
    // total mass of the whole lattice, one partial per block (slot 0 of 4)
    void (*mass)(const KParams &, const void *A, double *partials, int nblocks, cudaStream_t);
};

// Defined in plb_kern_fp64.cu / plb_kern_fp32.cu / plb_kern_fp16.cu; lattice 0 = D2Q9, 1 = D3Q19.
const Launchers *launchers_fp64(int lattice);
const Launchers *launchers_fp32(int lattice);
const Launchers *launchers_fp16(int lattice);

}  // namespace plb
