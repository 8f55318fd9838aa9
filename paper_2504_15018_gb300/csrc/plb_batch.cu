// Batched lattices in one persistent launch (include/plb.h, plb_batch_*).
//
// One device arena holds, for every instance, its populations, padded psi field and flags,
// plus one staging / reduction area shared by all instances, the instance descriptors, the
// tile table and the grid-barrier state.  plb_batch_step launches k_batch once for all the
// requested steps (a cooperative launch, so all blocks are co-resident) and, on a non-default
// stream, captures that launch in a CUDA graph the first time a step count is used and
// replays the graph afterwards.  Each instance is also exposed as a plb_t view for the
// readout entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include "plb.h"
#include "plb_host.h"
#include "plb_launch.h"

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

constexpr unsigned kDefaultSpinLimit = 1u << 22;   // ~ 1-4 s of polling with 256 ns sleeps

struct InstLayout {
    plb::Layout lay;
    size_t off_pops, off_psi, off_flags;
};

struct ArenaLayout {
    int Q;
    std::vector<InstLayout> inst;
    size_t off_bar, off_insts, off_tiles, off_partials, off_out, off_staging, total;
    long long max_tiles, chunk;
};

bool arena_layout(int lattice, int n, const plb_instance *d, ArenaLayout &A) {
    if (n < 1 || !d) return false;
    size_t off = 0;
    A.off_bar = off;
    off = align256(off + sizeof(plb::GridBar));
    A.off_insts = off;
    off = align256(off + (size_t)n * sizeof(plb::BatchInst));
    A.inst.resize(n);
    long long cells = 0, rows = 0, maxn = 0;
    for (int k = 0; k < n; ++k) {
        plb::Layout L;
        if (!plb::make_layout(lattice, d[k].dims, d[k].opts.precision, L)) return false;
        cells += L.n;
        rows += (long long)d[k].dims[1] * d[k].dims[2];
        maxn = std::max(maxn, L.n);
        A.inst[k].lay = L;
    }
    // the tile table is sized for the finest tiling (one row per tile)
    A.max_tiles = rows;
    A.off_tiles = off;
    off = align256(off + (size_t)A.max_tiles * sizeof(plb::BatchTile));
    for (int k = 0; k < n; ++k) {
        const plb::Layout &L = A.inst[k].lay;
        A.inst[k].off_pops = off;
        off = align256(off + (size_t)L.Q * L.pstride * L.s_pop);
        A.inst[k].off_psi = off;
        off = align256(off + (size_t)L.psi_elems * L.s_psi);
        A.inst[k].off_flags = off;
        off = align256(off + 64);
    }
    A.Q = A.inst[0].lay.Q;
    A.chunk = maxn < (1LL << 18) ? maxn : (1LL << 18);
    A.off_partials = off;
    off = align256(off + (size_t)1024 * 4 * sizeof(double));
    A.off_out = off;
    off = align256(off + 4 * sizeof(double));
    A.off_staging = off;
    const int per_cell = A.Q > A.inst[0].lay.D + 2 ? A.Q : A.inst[0].lay.D + 2;
    off = align256(off + (size_t)A.chunk * per_cell * sizeof(double));
    A.total = off;
    (void)cells;
    return true;
}

}  // namespace

struct plb_batch_state {
    int lattice, n, precision, collision;
    ArenaLayout A;
    std::vector<plb_state *> views;
    std::vector<plb::BatchInst> host_insts;
    char *ws;
    cudaStream_t stream;
    const plb::Launchers *L;
    int nsm;
    int tile_cells;        // target cells per tile
    int blocks_per_sm;     // resident blocks requested per SM
    int max_blocks_per_sm; // occupancy limit of the kernel
    int ntiles;
    unsigned spin_limit;
    unsigned missing_arrivals;   // test hook: barrier waits for this many extra blocks once
    std::map<int, cudaGraphExec_t> graphs;
    bool graph_ok;         // false once a capture failed: launch directly
    long long t;
    long long graph_captures;   // graphs captured and instantiated
    long long graph_launches;   // plb_batch_step calls served by a graph launch
    long long direct_launches;  // plb_batch_step calls launched without a graph
};

namespace {

int build_tiles(plb_batch_t *b) {
    std::vector<plb::BatchTile> tiles;
    for (int k = 0; k < b->n; ++k) {
        const int nx = b->views[k]->dims[0], ny = b->views[k]->dims[1], nz = b->views[k]->dims[2];
        int rows = b->tile_cells / nx;
        if (rows < 1) rows = 1;
        if (rows > ny) rows = ny;
        for (int z = 0; z < nz; ++z)
            for (int y0 = 0; y0 < ny; y0 += rows) tiles.push_back({k, z, y0, std::min(ny, y0 + rows)});
    }
    // interleave the instances so that consecutive tiles (taken by neighbouring blocks) mix sizes
    std::stable_sort(tiles.begin(), tiles.end(), [&](const plb::BatchTile &a, const plb::BatchTile &c) {
        const long long ia = (long long)a.y0 * 1000003LL + a.z, ic = (long long)c.y0 * 1000003LL + c.z;
        return ia < ic;
    });
    if ((long long)tiles.size() > b->A.max_tiles) return plb::set_error(PLB_EINVAL, "tile table overflow");
    b->ntiles = (int)tiles.size();
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    cudaError_t e = cudaMemcpyAsync(b->ws + b->A.off_tiles, tiles.data(), tiles.size() * sizeof(plb::BatchTile),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "tile upload: %s", cudaGetErrorString(e));
    return PLB_OK;
}

const void *batch_kernel(plb_batch_t *b) { return b->L->batch_kernel[b->collision == PLB_MRT ? 1 : 0](); }

cudaError_t launch_persistent(plb_batch_t *b, int nsteps, unsigned expected_extra) {
    plb::BatchLaunch bl;
    bl.insts = reinterpret_cast<plb::BatchInst *>(b->ws + b->A.off_insts);
    bl.tiles = reinterpret_cast<const plb::BatchTile *>(b->ws + b->A.off_tiles);
    bl.ninst = b->n;
    bl.ntiles = b->ntiles;
    bl.nsteps = nsteps;
    bl.bar = reinterpret_cast<plb::GridBar *>(b->ws + b->A.off_bar);
    bl.spin_limit = b->spin_limit;
    const unsigned grid = (unsigned)(b->nsm * b->blocks_per_sm);
    bl.expected = grid + expected_extra;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&bl};
    return cudaLaunchKernelExC(&cfg, batch_kernel(b), args);
}


}  // namespace

extern "C" {

size_t plb_batch_workspace_bytes(int lattice, int n, const plb_instance *inst) {
    ArenaLayout A;
    if (!arena_layout(lattice, n, inst, A)) return 0;
    return A.total;
}

int plb_batch_create(int lattice, int n, const plb_instance *inst, void *dev_workspace, size_t ws_bytes,
                     void *cuda_stream, plb_batch_t **out) {
    if (!out) return plb::set_error(PLB_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !inst) return plb::set_error(PLB_EINVAL, "need at least one instance");
    for (int k = 1; k < n; ++k)
        if (inst[k].opts.precision != inst[0].opts.precision || inst[k].opts.collision != inst[0].opts.collision)
            return plb::set_error(PLB_EINVAL, "all instances of a batch need the same precision and collision");
    for (int k = 0; k < n; ++k)
        if (inst[k].opts.streaming != PLB_STREAM_AA)
            return plb::set_error(PLB_EINVAL, "batches step in place (PLB_STREAM_AA)");
    ArenaLayout A;
    if (!arena_layout(lattice, n, inst, A)) return plb::set_error(PLB_EINVAL, "bad lattice, dims or precision");
    if (!dev_workspace || reinterpret_cast<uintptr_t>(dev_workspace) % 256 != 0)
        return plb::set_error(PLB_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    if (ws_bytes < A.total) return plb::set_error(PLB_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, A.total);
    // validate every instance before allocating host state
    for (int k = 0; k < n; ++k) {
        plb_opts o;
        plb::Layout lay;
        int st = plb::check_create_args(lattice, inst[k].dims, &inst[k].eos, inst[k].tau, inst[k].G, inst[k].eps,
                                        &inst[k].opts, o, lay);
        if (st != PLB_OK) return st;
    }
    plb_batch_t *b = new plb_batch_state();
    b->lattice = lattice;
    b->n = n;
    b->precision = inst[0].opts.precision;
    b->collision = inst[0].opts.collision;
    b->A = A;
    b->ws = static_cast<char *>(dev_workspace);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->L = plb::launchers_for_precision(lattice, b->precision);
    b->spin_limit = kDefaultSpinLimit;
    b->missing_arrivals = 0;
    b->t = 0;
    b->ntiles = 0;
    b->graph_ok = true;
    auto fail_destroy = [&](int code) {
        plb_batch_destroy(b);
        return code;
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel(b), 256, 0);
    if (e != cudaSuccess) return fail_destroy(plb::set_error(PLB_ECUDA, "device query: %s", cudaGetErrorString(e)));
    if (occ < 1) return fail_destroy(plb::set_error(PLB_EUNSUPPORTED, "batch kernel does not fit on an SM"));
    b->max_blocks_per_sm = occ;
    b->blocks_per_sm = occ;
    b->tile_cells = 4096;
    b->views.resize(n, nullptr);
    b->host_insts.resize(n);
    for (int k = 0; k < n; ++k) {
        plb_opts o;
        plb::Layout lay;
        plb::check_create_args(lattice, inst[k].dims, &inst[k].eos, inst[k].tau, inst[k].G, inst[k].eps,
                               &inst[k].opts, o, lay);
        plb_state *h = new plb_state();
        b->views[k] = h;
        h->view = 1;
        h->lattice = lattice;
        std::memcpy(h->dims, inst[k].dims, sizeof(h->dims));
        h->opts = o;
        h->eos = inst[k].eos;
        h->tau = inst[k].tau;
        h->G = inst[k].G;
        h->eps = inst[k].eps;
        h->lay = lay;
        h->ws = b->ws;
        h->pops = b->ws + A.inst[k].off_pops;
        h->psi = b->ws + A.inst[k].off_psi;
        h->partials = reinterpret_cast<double *>(b->ws + A.off_partials);
        h->out = reinterpret_cast<double *>(b->ws + A.off_out);
        h->staging = reinterpret_cast<double *>(b->ws + A.off_staging);
        h->lay.chunk = A.chunk;
        h->stream = b->stream;
        h->t = 0;
        h->odd = 0;
        h->L = b->L;
        double rv = 0, rl = 0, pp = 0;
        if (plb::solve_coexistence(inst[k].eos, rv, rl, pp) != PLB_OK) rv = rl = pp = 0;
        h->rho_v = rv;
        h->rho_l = rl;
        h->p0 = pp;
        int st = plb::fill_kparams(inst[k].dims, inst[k].eos, inst[k].tau, inst[k].G, inst[k].eps, o, lay, rv, rl,
                                   h->kp);
        if (st != PLB_OK) return fail_destroy(st);
        h->opts.rho_ref = h->kp.d.rho_ref;
        h->kp.flags = reinterpret_cast<unsigned *>(b->ws + A.inst[k].off_flags);
        plb::BatchInst &bi = b->host_insts[k];
        std::memset(&bi, 0, sizeof(bi));
        bi.kp = h->kp;
        for (int i = 0; i < 19; ++i)
            bi.pl[i] = i < lay.Q ? static_cast<void *>(h->pops + (size_t)i * lay.pstride * lay.s_pop) : nullptr;
        bi.psi = h->psi;
        bi.odd = 0;
        // two cells per thread: FP32 arithmetic, even nx, population planes below 4 GiB
        const long long ncell = (long long)inst[k].dims[0] * inst[k].dims[1] * inst[k].dims[2];
        bi.pair = (b->precision != PLB_FP64 && inst[k].dims[0] % 2 == 0 &&
                   ncell * (b->precision == PLB_FP32 ? 4 : 2) < (1LL << 32)) ? 1 : 0;
        bi.upr = bi.pair ? inst[k].dims[0] / 2 : inst[k].dims[0];
        e = cudaMemsetAsync(h->psi, 0, (size_t)lay.psi_elems * lay.s_psi, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->kp.flags, 0, 64, b->stream);
        if (e == cudaSuccess && h->kp.wall_fixed) {
            b->L->wall_fill(h->kp, h->psi, b->stream);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return fail_destroy(plb::set_error(PLB_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e)));
    }
    e = cudaMemsetAsync(b->ws + A.off_bar, 0, sizeof(plb::GridBar), b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ws + A.off_insts, b->host_insts.data(), n * sizeof(plb::BatchInst),
                            cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return fail_destroy(plb::set_error(PLB_ECUDA, "descriptor upload: %s", cudaGetErrorString(e)));
    int st = build_tiles(b);
    if (st != PLB_OK) return fail_destroy(st);
    *out = b;
    return PLB_OK;
}

void plb_batch_destroy(plb_batch_t *b) {
    if (!b) return;
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    for (plb_state *h : b->views) delete h;
    delete b;
}

plb_t *plb_batch_instance(plb_batch_t *b, int k) {
    if (!b || k < 0 || k >= b->n) return nullptr;
    return b->views[k];
}

static int batch_init(plb_batch_t *b, int k, const double *rho0, const double *u0, bool physical) {
    if (!b || k < 0 || k >= b->n) return plb::set_error(PLB_EINVAL, "bad batch or instance index");
    int st = plb::init_state(b->views[k], rho0, u0);
    if (st == PLB_OK && physical) st = plb::rebalance_state(b->views[k]);
    if (st != PLB_OK) return st;
    // the instance restarts at even parity; the device descriptor must say so
    b->host_insts[k].odd = 0;
    cudaError_t e = cudaMemcpyAsync(b->ws + b->A.off_insts + k * sizeof(plb::BatchInst) + offsetof(plb::BatchInst, odd),
                                    &b->host_insts[k].odd, sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "parity upload: %s", cudaGetErrorString(e));
    return PLB_OK;
}

int plb_batch_init(plb_batch_t *b, int k, const double *rho0, const double *u0) {
    return batch_init(b, k, rho0, u0, false);
}

int plb_batch_init_physical(plb_batch_t *b, int k, const double *rho0, const double *u0) {
    return batch_init(b, k, rho0, u0, true);
}

int plb_batch_configure(plb_batch_t *b, int tile_cells, int blocks_per_sm, unsigned spin_limit) {
    if (!b) return plb::set_error(PLB_EINVAL, "NULL batch");
    if (tile_cells > 0) b->tile_cells = tile_cells;
    if (blocks_per_sm > 0) {
        if (blocks_per_sm > b->max_blocks_per_sm)
            return plb::set_error(PLB_EINVAL, "at most %d resident blocks per SM", b->max_blocks_per_sm);
        b->blocks_per_sm = blocks_per_sm;
    }
    b->spin_limit = spin_limit > 0 ? spin_limit : kDefaultSpinLimit;
    return build_tiles(b);
}

int plb_batch_step(plb_batch_t *b, int nsteps) {
    if (!b || nsteps < 0) return plb::set_error(PLB_EINVAL, "bad argument");
    if (nsteps == 0) return PLB_OK;
    cudaError_t e = cudaSuccess;
    const unsigned extra = b->missing_arrivals;
    b->missing_arrivals = 0;
    const bool graphable = b->stream != nullptr && extra == 0 && b->graph_ok;
    if (graphable) {
        auto it = b->graphs.find(nsteps);
        if (it == b->graphs.end()) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = launch_persistent(b, nsteps, 0);
                e = cudaStreamEndCapture(b->stream, &g);
                if (le != cudaSuccess) e = le;
            }
            cudaGraphExec_t ex = nullptr;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                // the runtime cannot capture this launch: launch it directly from now on
                cudaGetLastError();
                b->graph_ok = false;
                e = launch_persistent(b, nsteps, 0);
                ++b->direct_launches;
            } else {
                it = b->graphs.emplace(nsteps, ex).first;
                ++b->graph_captures;
                e = cudaGraphLaunch(it->second, b->stream);
                ++b->graph_launches;
            }
        } else {
            e = cudaGraphLaunch(it->second, b->stream);
            ++b->graph_launches;
        }
    } else {
        e = launch_persistent(b, nsteps, extra);
        ++b->direct_launches;
    }
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "batch launch: %s", cudaGetErrorString(e));
    b->t += nsteps;
    for (int k = 0; k < b->n; ++k) {
        b->views[k]->t += nsteps;
        b->views[k]->odd ^= (nsteps & 1);
        b->host_insts[k].odd = b->views[k]->odd;
    }
    return PLB_OK;
}

int plb_batch_status(plb_batch_t *b) {
    if (!b) return plb::set_error(PLB_EINVAL, "NULL batch");
    plb::GridBar bar;
    cudaError_t e = cudaMemcpyAsync(&bar, b->ws + b->A.off_bar, sizeof(bar), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "reading the barrier state: %s", cudaGetErrorString(e));
    if (bar.err) return plb::set_error(PLB_ETIMEOUT, "a grid barrier of the batch kernel gave up waiting");
    for (int k = 0; k < b->n; ++k) {
        int st = plb_status(b->views[k]);
        if (st != PLB_OK) return st;
    }
    return PLB_OK;
}

int plb_batch_reset_error(plb_batch_t *b) {
    if (!b) return plb::set_error(PLB_EINVAL, "NULL batch");
    cudaError_t e = cudaMemsetAsync(b->ws + b->A.off_bar, 0, sizeof(plb::GridBar), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return PLB_OK;
}

int plb_batch_withhold_arrivals(plb_batch_t *b, unsigned count) {
    if (!b) return plb::set_error(PLB_EINVAL, "NULL batch");
    b->missing_arrivals = count;
    return PLB_OK;
}

int plb_batch_autotune(plb_batch_t *b, int steps_per_candidate, int *tile_cells, int *blocks_per_sm, double *best_ms) {
    if (!b || steps_per_candidate < 1) return plb::set_error(PLB_EINVAL, "bad argument");
    const int cand_tiles[] = {512, 1024, 2048, 4096, 8192, 16384};
    float best = 1e30f;
    int bt = b->tile_cells, bb = b->blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return plb::set_error(PLB_ECUDA, "cudaEventCreate failed");
    int st = PLB_OK;
    for (int bps = 1; bps <= std::min(b->max_blocks_per_sm, 4) && st == PLB_OK; ++bps) {
        for (int tc : cand_tiles) {
            st = plb_batch_configure(b, tc, bps, b->spin_limit);
            if (st != PLB_OK) break;
            st = plb_batch_step(b, 2);   // warm-up (graph capture)
            if (st != PLB_OK) break;
            cudaEventRecord(e0, b->stream);
            st = plb_batch_step(b, steps_per_candidate);
            cudaEventRecord(e1, b->stream);
            if (st != PLB_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bt = tc;
                bb = bps;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PLB_OK) return st;
    st = plb_batch_configure(b, bt, bb, b->spin_limit);
    if (tile_cells) *tile_cells = bt;
    if (blocks_per_sm) *blocks_per_sm = bb;
    if (best_ms) *best_ms = best / steps_per_candidate;
    if (st != PLB_OK) return st;
    return plb_batch_status(b);
}

long long plb_batch_time(const plb_batch_t *b) { return b ? b->t : -1; }

int plb_batch_launch_counts(const plb_batch_t *b, long long counts[3]) {
    if (!b || !counts) return plb::set_error(PLB_EINVAL, "NULL argument");
    counts[0] = b->graph_captures;
    counts[1] = b->graph_launches;
    counts[2] = b->direct_launches;
    return PLB_OK;
}

}  // extern "C"
