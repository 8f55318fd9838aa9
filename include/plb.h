/*
 * plb.h -- C ABI of a GB300 (sm_103a) implementation of the per-time-step update
 * of the pseudo-potential lattice Boltzmann method (P-LBM) of
 * "On the consistency of pseudo-potential lattice Boltzmann methods"
 * (Czelusniak, Bingert, Krause, Simonis; arXiv 2504.15018).
 *
 * One time step (Sec. II, Eq. LBE) on a D2Q9 or D3Q19 lattice, lattice units
 * Delta x = Delta t = 1:
 *   rho = sum_i f_i                                   (Eq. Density)
 *   psi = sqrt(2 (p_EOS(rho) - rho/3) / G)            (Eq. Interaction_Potential)
 *   M1_a = sum_i w_i psi(x+c_i) c_ia / c_s^2,
 *   M2_ab = sum_i w_i psi(x+c_i) (c_ia c_ib - c_s^2 d_ab) / c_s^4   (Sec. II)
 *   F = -G psi M1 + eps/kappa terms + F_ext            (Eqs. Shan_Chen_Force, interactionForce)
 *   u = (sum_i f_i c_i + F/2) / rho                    (Eq. Momentum)
 *   f_i* = f_i - (f_i - f_i^eq)/tau + F_i'             (Eqs. LBE, Single_Phase_EDF, Guo_Forcing_Scheme)
 *          or the MRT generalisation (same Guo term in moment space)
 *   f_i(x + c_i, t + 1) = f_i*(x, t)                   (streaming; halfway bounce-back at walls)
 *
 * eps term: Eq. interactionForce as printed contradicts Eq. New_Pressure_Tensor and the
 * Maxwell rule at eps = 2 (Sec. IV); this library uses the coefficient that realises the
 * printed pressure tensor: -G/12 (2 kappa - 2 - 3 eps) M1_b M2_ab + G/6 (kappa - 1) M1_a M2_bb.
 *
 * Conventions (all entry points):
 *   - Cell index s = x + nx * (y + ny * z), x fastest.  D2Q9 uses nz = 1.
 *   - Host arrays are FP64 whatever the storage precision.  Velocity fields are
 *     stored component-major: u[a * N + s].  Population arrays exchanged with the
 *     host are FP64, direction-major: f[i * N + s], directions in the order
 *     reported by plb_velocity_set().
 *   - Every function returns a PLB_* status; no exception crosses the ABI.
 *     plb_last_error() gives a message for the last failure on the calling thread.
 *     A NULL handle gives PLB_EINVAL before any device work (the few functions that
 *     return a value instead say what they return for it; the destroy calls ignore it).
 *   - The caller owns the device workspace and the CUDA stream; the library never
 *     allocates device memory.  A handle is not thread-safe; use one stream per handle.
 *   - Device work is enqueued on the handle's stream.  Functions that return host
 *     data (plb_moments, plb_reduce, plb_get_*, plb_status) synchronise that stream.
 */
#ifndef PLB_H
#define PLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum {
    PLB_OK = 0,
    PLB_EINVAL = 1,        /* invalid argument */
    PLB_ENOMEM = 2,        /* workspace or host buffer too small */
    PLB_ECUDA = 3,         /* CUDA runtime error (message in plb_last_error) */
    PLB_ENONFINITE = 4,    /* a density became non-positive or non-finite */
    PLB_EPSI_DOMAIN = 5,   /* 2 (p_EOS - rho/3) / G < 0 somewhere: psi undefined */
    PLB_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
    PLB_EUNSUPPORTED = 7   /* combination not built */
};

enum { PLB_D2Q9 = 0, PLB_D3Q19 = 1 };
enum { PLB_EOS_PR = 0, PLB_EOS_PAPER = 1 };
enum { PLB_FP64 = 0, PLB_FP32 = 1, PLB_FP16S = 2 };
enum { PLB_BGK = 0, PLB_MRT = 1 };

/* quantities of plb_reduce */
enum {
    PLB_MASS = 0,       /* sum rho                                  -> out[0]     */
    PLB_MOMENTUM = 1,   /* sum rho u (u with the F/2 shift)         -> out[0..2]  */
    PLB_UMAX = 2,       /* max |u|            (L_inf of Eq. norms)  -> out[0]     */
    PLB_UL1 = 3,        /* sum |u|            (L_1 of Eq. norms)    -> out[0]     */
    PLB_UL2 = 4,        /* sqrt(sum |u|^2)    (L_2 of Eq. norms)    -> out[0]     */
    PLB_MEAN_RHO = 5,   /* mean rho over the box                    -> out[0]     */
    PLB_MEAN_P = 6      /* mean p_scale p_EOS(rho) over the box     -> out[0]     */
};

/* Equation of state.
 * PLB_EOS_PR: Peng-Robinson in lattice units (not in the paper; the usual choice of
 *   pseudo-potential benchmarks): p = rho R T/(1 - b rho) - a alpha(T) rho^2/(1 + 2 b rho - b^2 rho^2),
 *   alpha = [1 + (0.37464 + 1.54226 w - 0.26992 w^2)(1 - sqrt(T/Tc))]^2, Tc = 0.0778 a/(0.45724 b R).
 * PLB_EOS_PAPER: Eq. EOS of Sec. IV with rho_v, rho_l and P = p_c / rho_c^3.
 * p_scale multiplies p_EOS (the Delta t^2/Delta x^2 factor of Eq. Interaction_Potential;
 *   1 in lattice units at r = 1). */
typedef struct plb_eos_params {
    int kind;
    double a, b, R, omega, T_over_Tc;
    double rho_v, rho_l, pc_over_rhoc3;
    double p_scale;
} plb_eos_params;

/* Per-lattice options.  plb_default_opts() fills the defaults given in brackets. */
typedef struct plb_opts {
    double kappa;            /* surface-tension parameter of Eq. interactionForce [1] */
    double tau_v;            /* <= 0: constant tau; else tau(rho) = tau_v + w (tau_l - tau_v),
                                w = clamp((rho - tau_rho_v)/(tau_rho_l - tau_rho_v), 0, 1) (Sec. VI) [0] */
    double tau_rho_v, tau_rho_l;   /* densities of the tau interpolation [coexistence densities] */
    int collision;           /* PLB_BGK or PLB_MRT [PLB_BGK] */
    double s_e, s_eps, s_q, s_pi, s_m;  /* MRT rates of the energy, energy-square, heat-flux,
                                           and (D3Q19) pi and m moments; stress moments use 1/tau [1] */
    int precision;           /* storage precision of the populations [PLB_FP32] */
    double rho_ref;          /* PLB_FP16S stores f_i - w_i rho_ref; <= 0 picks the vapour
                                coexistence density of the EOS [0] */
    int wall_y;              /* 1: halfway bounce-back walls at y = -1/2 and y = ny - 1/2;
                                psi on the wall equals psi of the adjacent fluid row [0 = periodic] */
    double body_force[3];    /* external force density F_ext added to F (Sec. II) [0] */
    int fp16_rounding;       /* PLB_FP16S stores: 0 round to nearest even; 1 stochastic rounding
                                (unbiased: no drift from repeated rounding, no stagnation) [0] */
    int streaming;           /* PLB_STREAM_AA: two kernels per step (psi pass, fused force/collide/
                                stream) on one in-place population copy (AA pattern).
                                PLB_STREAM_FUSED: one kernel per step that forms psi of each tile and
                                its halo in shared memory, collides and pushes into a second copy of
                                the populations (twice the population memory, about 30 % fewer DRAM
                                bytes per step); PLB_FP32 / PLB_FP16S with even nx and population
                                planes below 4 GiB (fewer than 2^30 / 2^31 cells) only, not in
                                batches [PLB_STREAM_AA].  Both give the same populations bit for
                                bit, except D3Q19 with PLB_FP32 storage, where the single pass
                                collides in moment space and the two-pass kernels population pair
                                by population pair: there they agree to FP32 rounding. */
    double wall_rho;         /* wall_y = 1 only: > 0 makes the walls wetting walls, whose nodes carry
                                the pseudo-potential psi(wall_rho) of a prescribed wall density
                                instead of mirroring the adjacent fluid row; wall_rho near rho_l
                                wets, near rho_v does not (not in the paper, which has neutral
                                walls only); <= 0: mirror rule [0] */
} plb_opts;

enum { PLB_STREAM_AA = 0, PLB_STREAM_FUSED = 1 };

typedef struct plb_state plb_t;

/* Fills *opts with the defaults listed above. */
void plb_default_opts(plb_opts *opts);

/* Directions of the lattice in the library's order: c[3*i + a] and w[i]
 * (Eq. VelocitySet for D2Q9; standard D3Q19).  Opposite directions are adjacent:
 * opp(i) = i + 1 for odd i.  Returns Q (9 or 19), or -1 for an unknown lattice. */
int plb_velocity_set(int lattice, int *c, double *w);

/* Bytes of device workspace plb_create needs for this lattice, size and options
 * (populations in one copy, padded psi field, reduction partials, staging, flags).
 * Returns 0 on invalid arguments. */
size_t plb_workspace_bytes(int lattice, const int dims[3], const plb_opts *opts);

/* Creates a lattice.  dims = {nx, ny, nz} (nz = 1 for D2Q9).  tau = tau_l (> 1/2);
 * G < 0 (any negative value gives the same dynamics, Eq. Interaction_Potential);
 * eps: mechanical-stability exponent of Sec. IV (2 = Maxwell rule).
 * dev_workspace: caller-owned device memory of at least plb_workspace_bytes(...) bytes,
 * 256-byte aligned; it must outlive the handle.  cuda_stream: a cudaStream_t (NULL = default).
 * opts may be NULL (defaults).  Errors: PLB_EINVAL, PLB_ENOMEM (workspace too small),
 * PLB_EUNSUPPORTED, PLB_ECUDA. */
int plb_create(int lattice, const int dims[3], const plb_eos_params *eos, double tau, double G, double eps,
               const plb_opts *opts, void *dev_workspace, size_t ws_bytes, void *cuda_stream, plb_t **out);

/* Frees the handle (host memory only). */
void plb_destroy(plb_t *h);

/* f_i = f_i^eq(rho0, u0) (Eq. Single_Phase_EDF) on every cell; time reset to 0.
 * rho0: host FP64 [N]; u0: host FP64 [d * N] or NULL (u = 0).  Pinned host memory makes
 * the uploads asynchronous; the call synchronises the stream once at the end, because the
 * values are checked on the device as they are read.  Errors: PLB_EINVAL (a non-positive or
 * non-finite rho0, or a non-finite u0; the message names the first such index, and the
 * populations are undefined until the next successful plb_init), PLB_ECUDA. */
int plb_init(plb_t *h, const double *rho0, const double *u0);

/* As plb_init, then the populations become f^eq(rho0, u0 - F/(2 rho0)) (Eq. Single_Phase_EDF),
 * F the total force of Eqs. interactionForce and F_ext on the initial density, so that the
 * velocity of Eq. Momentum, (sum f c + F/2)/rho, equals u0 from the first step.  plb_init
 * leaves interfaces with the velocity F/(2 rho), which launches sound waves; the Sec. VI
 * benchmarks (the planar interface set in motion in Sec. VI.C) need the balanced start to
 * converge at second order.  Arguments and errors as plb_init; a density outside the psi
 * domain is reported by plb_status. */
int plb_init_physical(plb_t *h, const double *rho0, const double *u0);

/* Advances n time steps (two kernels per step: psi pass, then the fused force +
 * collide + stream pass).  Asynchronous; returns launch errors only.  Device-side
 * faults of the method (psi domain, non-finite density) are recorded in a device flag
 * and reported by plb_status / plb_moments / plb_reduce. */
int plb_step(plb_t *h, int n);

/* Same as plb_step(h, n), with CUDA events recorded on the handle's stream around every
 * launch; ms[0] receives the summed duration of the n psi passes, ms[1] of the n fused
 * force + collide + stream passes (milliseconds).  Synchronises.  For measurement. */
int plb_step_timed(plb_t *h, int n, double ms[2]);

/* Synchronises the stream and returns PLB_EPSI_DOMAIN / PLB_ENONFINITE if a kernel
 * met such a cell since creation or the last plb_init, else PLB_OK. */
int plb_status(plb_t *h);

/* Number of steps since plb_init; -1 for a NULL handle. */
long long plb_time(const plb_t *h);

/* Macroscopic fields of the current state: rho (Eq. Density), u with the F/2 shift
 * (Eq. Momentum), p = p_scale p_EOS(rho).  Host FP64 outputs, each may be NULL:
 * rho [N], u [d * N], p [N].  Synchronises.  Errors: PLB_EINVAL (NULL handle),
 * PLB_EPSI_DOMAIN / PLB_ENONFINITE (as plb_status), PLB_ECUDA. */
int plb_moments(plb_t *h, double *rho, double *u, double *p);

/* A reduction over the box lo <= (x, y, z) < hi (clipped to the lattice; NULL = whole), summed in
 * FP64 in a fixed order (deterministic).  out receives 1 value (3 for PLB_MOMENTUM).
 * Synchronises.  Errors: PLB_EINVAL (NULL handle or out, unknown reduction, empty box),
 * PLB_EPSI_DOMAIN / PLB_ENONFINITE (as plb_status), PLB_ECUDA. */
int plb_reduce(plb_t *h, int what, const int lo[3], const int hi[3], double *out);

/* Current populations f_i(x, t) (pre-collision) as host FP64 [Q * N], direction-major.
 * Errors: PLB_EINVAL (NULL argument), PLB_ECUDA. */
int plb_get_populations(plb_t *h, double *f);

/* Replaces the populations (host FP64 [Q * N]); keeps the step counter.  Errors:
 * PLB_EINVAL (NULL argument, or a batch instance view), PLB_ECUDA. */
int plb_set_populations(plb_t *h, const double *f);

/* Raw checkpoint of the population store and the step counter (bit-exact restart).
 * plb_state_bytes gives the size (0 for a NULL handle); get/set return PLB_ENOMEM if bytes
 * is too small, PLB_EINVAL for a NULL argument (set also for a batch instance view or a
 * state taken from another lattice), PLB_ECUDA. */
size_t plb_state_bytes(const plb_t *h);
int plb_get_state(plb_t *h, void *host_buf, size_t bytes);
int plb_set_state(plb_t *h, const void *host_buf, size_t bytes);

/* Host FP64 parameter solve (Sec. IV): coexistence densities of the EOS by the
 * equal-area (Maxwell) rule, and the coexistence pressure p0 (p_scale = 1).
 * For PLB_EOS_PAPER these are rho_v, rho_l by construction. */
int plb_solve_params(const plb_eos_params *eos, double *rho_v, double *rho_l, double *p0);

/* Multiphase SI unit converter of Sec. V (Eqs. unit, unit2) plus the parameter
 * formulas of Sec. IV (Eqs. thickness, surface_tension, r = 1).
 * si = {rho_v, rho_l, nu_v, nu_l, gamma, L} (kg/m^3, m^2/s, N/m, m);
 * lat = {L, tau_l, rho_l}; xi = interface width in lattice units.
 * out = {C_L, C_T, C_M, C_U, C_VF, C_gamma, rho_v, tau_v, gamma_lat, pc_over_rhoc3, kappa}. */
int plb_si_convert(const double si[6], const double lat[3], double xi, double out[11]);

/* ------------------------------------------------------------------ batches
 * Many independent lattices of one lattice type, storage precision and collision (sizes,
 * EOS, tau, eps, kappa, walls and forces may differ per instance) advanced together by one
 * persistent kernel launch per plb_batch_step call: every step is a psi pass over all
 * instances, a grid barrier, the fused force/collide/stream pass, and another barrier
 * (the same per-cell update as plb_step, Sec. II of the paper).  Work is split into tiles of
 * whole rows; the tile size and resident blocks per SM are set by plb_batch_autotune or
 * plb_batch_configure.  The grid barrier waits a bounded time: a wait that runs out sets a
 * device error word, the kernel returns, and plb_batch_status reports PLB_ETIMEOUT. */
typedef struct plb_batch_state plb_batch_t;

typedef struct plb_instance {
    int dims[3];
    plb_eos_params eos;
    double tau, G, eps;
    plb_opts opts;         /* precision and collision must match across a batch */
} plb_instance;

/* Bytes of device workspace for a batch (0 on invalid arguments). */
size_t plb_batch_workspace_bytes(int lattice, int n, const plb_instance *inst);

/* Creates a batch of n instances over a caller-owned, 256-byte aligned device workspace and
 * stream.  On a non-default stream each step count is captured once as a CUDA graph and
 * replayed.  Errors: PLB_EINVAL, PLB_ENOMEM, PLB_EUNSUPPORTED, PLB_ECUDA. */
int plb_batch_create(int lattice, int n, const plb_instance *inst, void *dev_workspace, size_t ws_bytes,
                     void *cuda_stream, plb_batch_t **out);
void plb_batch_destroy(plb_batch_t *b);

/* Instance k as a read-only lattice handle for plb_moments, plb_reduce, plb_get_populations,
 * plb_get_state, plb_status and plb_time (plb_step / plb_init / plb_set_* refuse it; do not
 * destroy it).  NULL for a NULL batch or a bad index. */
plb_t *plb_batch_instance(plb_batch_t *b, int k);

/* f = f^eq(rho0, u0) on instance k (as plb_init); plb_batch_init_physical as plb_init_physical. */
int plb_batch_init(plb_batch_t *b, int k, const double *rho0, const double *u0);
int plb_batch_init_physical(plb_batch_t *b, int k, const double *rho0, const double *u0);

/* Advances every instance by nsteps steps in one persistent launch.  Asynchronous. */
int plb_batch_step(plb_batch_t *b, int nsteps);

/* Synchronises; PLB_ETIMEOUT if a grid barrier gave up, else the first instance's
 * PLB_EPSI_DOMAIN / PLB_ENONFINITE, else PLB_OK. */
int plb_batch_status(plb_batch_t *b);

/* Clears a recorded barrier timeout. */
int plb_batch_reset_error(plb_batch_t *b);

/* Tile size in cells (rows of a tile = tile_cells / nx, at least 1), resident 256-thread
 * blocks per SM, and the barrier's polling limit (0 keeps the default, about a second or more).
 * A non-positive tile_cells or blocks_per_sm keeps the current value. */
int plb_batch_configure(plb_batch_t *b, int tile_cells, int blocks_per_sm, unsigned spin_limit);

/* Times steps_per_candidate steps for every tile size in {512, ..., 16384} cells and every
 * resident count from 1 block per SM to the kernel's occupancy limit (at most 4; the kernel
 * is compiled for 3 D2Q9 / 2 D3Q19 blocks per SM without spilling), keeps the fastest, and reports it (any output may be NULL; best_ms is per
 * step).  The timed steps advance the batch. */
int plb_batch_autotune(plb_batch_t *b, int steps_per_candidate, int *tile_cells, int *blocks_per_sm, double *best_ms);

/* Test hook for failure detection: the next plb_batch_step launch's barriers wait for count
 * blocks more than are launched, so every wait runs out (bounded by the polling limit) and
 * plb_batch_status reports PLB_ETIMEOUT.  Nothing faults or hangs. */
int plb_batch_withhold_arrivals(plb_batch_t *b, unsigned count);

/* Steps taken by the batch; -1 for a NULL batch. */
long long plb_batch_time(const plb_batch_t *b);

/* How plb_batch_step calls were launched since the batch was created: counts[0] = CUDA graphs
 * captured and instantiated (one per distinct nsteps on a non-default stream, captured again
 * after plb_batch_configure), counts[1] = calls served by a graph launch, counts[2] = calls
 * launched directly (the default stream, a withheld-arrival test launch, or a stream whose
 * capture failed).  PLB_EINVAL for NULL arguments. */
int plb_batch_launch_counts(const plb_batch_t *b, long long counts[3]);

/* ---------------------------------------------------------------- slab decomposition
 * One D3Q19 lattice of nx x ny x NZ cells, periodic in z, split along z into slabs (one per
 * GPU, or several on one GPU).  The force of Eq. interactionForce reaches the nearest
 * neighbours only (Sec. IV), so each step exchanges a one-plane psi halo after the psi pass and
 * five population planes per face after the collide pass.  A slab owning the global planes
 * z_first .. z_first + m - 1 is an ordinary handle (plb_create) of dims (nx, ny, m + 2) whose
 * local planes 0 and m + 1 are ghost planes (copies of global planes z_first - 1 and z_first + m,
 * wrapped periodically); plb_init is given the m + 2 planes.  After plb_slab_bind, plb_step
 * refuses the handle: a step is
 *     plb_slab_pass(h, 0) on every slab;  the pass-0 exchange across every face;
 *     plb_slab_pass(h, 1) on every slab;  the pass-1 exchange across every face,
 * and the owned planes then equal the same planes of the whole lattice stepped by plb_step, bit
 * for bit (same kernels; stochastic rounding hashes the whole lattice's cell index).  Readouts
 * of a slab handle cover its m + 2 planes; the ghost planes' moments are not meaningful.
 * D3Q19 only, in place (AA) streaming only; walls in y allowed. */

/* One transfer of the exchange plan: bytes from send_off on this slab to recv_off on the
 * neighbour across `face` (0: toward lower z, 1: toward higher z), offsets in bytes from the
 * start of the population store (region 0) or of the padded psi field (region 1), as returned
 * by plb_slab_regions.  Entry k of face f on one slab pairs with entry k of face 1 - f on the
 * neighbour: that entry's send range arrives in this entry's receive range and vice versa. */
typedef struct {
    long long send_off, recv_off, bytes;
    int face, region;
} plb_xfer;

/* The exchange plan after pass `pass` (0: psi pass, 1: collide pass) of a step of AA parity
 * `odd` (the parity the step had when its passes ran), for a slab of local dims (nx, ny, m + 2),
 * storage `precision`, walls in y or not.  Host-only (no device work): pass 0 lists two psi
 * planes, pass 1 ten population planes (after an even step the slots that the neighbour's odd
 * step reads; after an odd step the slots this slab's boundary cells streamed into its ghost
 * planes, less the wall row of the slots whose upstream cell is beyond a wall).  out[max]:
 * caller's array; *count receives the number of entries.  PLB_EUNSUPPORTED for D2Q9,
 * PLB_EINVAL for bad arguments or max too small. */
int plb_slab_plan(int lattice, const int dims[3], int precision, int wall_y, int pass, int odd, plb_xfer *out,
                  int max, int *count);

/* Makes h (D3Q19, in-place streaming, at an even step) a slab owning global planes from
 * z_first on: its first and last local planes become ghost planes. */
int plb_slab_bind(plb_t *h, int z_first);

/* Pass 0 (psi pass) or 1 (collide pass; advances the step) over the owned planes, in the order
 * 0, 1, 0, 1, ...  Asynchronous on the handle's stream. */
int plb_slab_pass(plb_t *h, int pass);

/* Device base addresses of the population store and of the padded psi field (the offsets of
 * plb_slab_plan are relative to them). */
int plb_slab_regions(plb_t *h, void **pops, void **psi);

/* Carries out the exchange after pass `pass` across the face between two slabs, `lower` owning
 * the planes just below `upper`'s (periodic: the last slab is below the first), with
 * cudaMemcpyAsync on lower's stream (device memory of any GPUs the runtime can copy between).
 * The caller orders the two handles' streams around it.  PLB_EINVAL unless both handles are
 * slabs of the same cross-section, precision and walls, just after that pass of the same step. */
int plb_slab_exchange(plb_t *lower, plb_t *upper, int pass);

/* Allocation-free stepping, for callers that cannot allocate device memory: a plugin
 * that lives inside another framework's memory arena and only receives the buffers it
 * works on, or a real-time loop in which cudaMalloc (which may synchronise the device) is
 * not allowed.  The paper has no counterpart to this entry point; it is part of this
 * library's interface only.
 *
 * Advances the populations in dev_pops by 2 * npairs time steps with the same kernels as
 * plb_step.  dev_pops: caller-owned device array of Q * N stored populations, direction-major
 * f[i * N + s] in the plb_velocity_set() order, element type double (PLB_FP64), float
 * (PLB_FP32) or half holding f_i - w_i rho_ref (PLB_FP16S); 256-byte aligned; updated in place
 * and, after an even number of steps, again in this natural layout.  t0 >= 0: the time step
 * the populations are at (what plb_time would report for a lattice in this state); step
 * t0 + m draws its stochastic-rounding noise (PLB_FP16S with fp16_rounding = 1) from the
 * counter t0 + m, as plb_step does, so the result equals plb_step's bit for bit.  The other
 * arguments are those of plb_create.
 *
 * Scratch: the padded psi field and the error flags live in one file-scope device array of
 * 8 MiB that every GPU loading this library holds until the process exits.  The padded psi
 * field must fit in 8 MiB - 256 bytes (padded extents (nx + 2g rounded up to 32) x (ny + 2)
 * [x (nz + 2)], 4 bytes per value, 8 for PLB_FP64; e.g. a 120^3 D3Q19 lattice in FP32); larger
 * lattices are rejected with PLB_ENOMEM and a message.  The function calls no cudaMalloc,
 * cudaFree or other allocating routine.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) for that device and keeps it for the life of the
 * process; make that first call before any stream capture.  After cudaDeviceReset (or anything
 * else that tears down the device's primary context) the kept address is stale: do not call
 * this entry point again in that process.  Every call shares the array and leaves its contents
 * behind; the flags are cleared at the start of each call.  Calls whose work overlaps on the
 * GPU (different streams, or without an ordering between them) race on the array.
 *
 * Returns after the steps have finished (the call waits for its stream while it reads the
 * flags back), with PLB_EPSI_DOMAIN or PLB_ENONFINITE if a kernel met such a cell, PLB_EINVAL /
 * PLB_ENOMEM on bad arguments, and PLB_ECUDA without launching anything if a CUDA error from
 * earlier work is still pending on the calling thread. */
int plb_step_pairs_static(int lattice, const int dims[3], const plb_eos_params *eos, double tau, double G,
                          double eps, const plb_opts *opts, void *dev_pops, int npairs, long long t0,
                          void *cuda_stream);

/* Message of the last failure on this thread ("" if none). */
const char *plb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PLB_H */
