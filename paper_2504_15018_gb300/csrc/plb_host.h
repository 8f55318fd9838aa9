// Internal host-side declarations shared by the runtime and the parameter solve.
#pragma once
#include <cstddef>

#include "plb.h"

namespace plb {

struct PrConstants {
    double Tc, alpha, RT, aalpha;
};

PrConstants pr_constants(const plb_eos_params &e);
double eos_pressure_host(const plb_eos_params &e, double rho);
int solve_coexistence(const plb_eos_params &e, double &rho_v, double &rho_l, double &p0);
int si_convert(const double si[6], const double lat[3], double xi, double out[11]);

// Byte layout of the caller's device workspace (every region 256-byte aligned).
struct Layout {
    int Q, D;
    long long n;            // cells
    long long pstride;      // elements per population plane
    int s_pop, s_psi;       // bytes per stored population / psi value
    int gx, px, py, pz;     // psi padding and padded extents
    long long psi_elems;
    long long chunk;        // cells per staging chunk
    int max_blocks;         // reduction partial blocks
    size_t off_pops, off_pops2, off_psi, off_partials, off_out, off_staging, off_flags, total;
};

// streaming = PLB_STREAM_FUSED adds the second population copy (off_pops2; else off_pops2 = off_pops).
bool make_layout(int lattice, const int dims[3], int precision, Layout &L, int streaming = PLB_STREAM_AA);

struct KParams;
struct Launchers;

// Records the message of a failure for plb_last_error() and returns code.
int set_error(int code, const char *fmt, ...);
// Validation shared by the lattice constructors; o receives the options in effect.
int check_create_args(int lattice, const int dims[3], const plb_eos_params *eos, double tau, double G, double eps,
                      const plb_opts *opts, plb_opts &o, Layout &lay);
// Kernel parameter block of a lattice (everything but the device pointers).
int fill_kparams(const int dims[3], const plb_eos_params &eos, double tau, double G, double eps, const plb_opts &o,
                 const Layout &lay, double rho_v, double rho_l, KParams &k);
const Launchers *launchers_for_precision(int lattice, int precision);

}  // namespace plb

#include "plb_launch.h"

// A lattice handle: its parameters and the device regions it works on.  plb_create points
// the regions into the caller's workspace; a batch points them into its arena.
struct plb_state {
    int lattice;
    int dims[3];
    plb_opts opts;
    plb_eos_params eos;
    double tau, G, eps;
    double rho_v, rho_l, p0;   // coexistence densities of the EOS (p_scale = 1)
    plb::Layout lay;
    plb::KParams kp;
    const plb::Launchers *L;
    char *ws;
    char *pops, *psi;          // population store (the current copy), padded psi field
    char *pops2;               // PLB_STREAM_FUSED: the copy the next step writes (else NULL)
    double *partials, *out;    // reduction partials (lay.max_blocks x 4), final values (4)
    double *staging;           // host<->device staging (lay.chunk cells)
    cudaStream_t stream;
    long long t;
    int odd;
    int view;                  // 1: an instance of a batch (stepped only by plb_batch_step)
    int slab;                  // 1: a z-slab whose first and last planes are ghost planes (plb_slab_*)
    int slab_stage;            // slab: 0 = the next pass is the psi pass, 1 = the collide pass
};

namespace plb {
// f = f^eq(rho0, u0) on every cell of h (the body of plb_init).
int init_state(plb_state *h, const double *rho0, const double *u0);
// After init_state: psi pass and k_rebalance, so the physical velocity at t = 0 is u0.
int rebalance_state(plb_state *h);
}  // namespace plb
