// Slab decomposition of one D3Q19 lattice along z (include/plb.h, plb_slab_*).
//
// The force of Eq. interactionForce reaches the nearest neighbours only (Sec. IV), so a
// lattice split into z-slabs exchanges two thin layers per step and face.  A slab is an
// ordinary lattice handle of nz_own + 2 planes whose first and last planes are ghost planes
// (copies of the neighbouring slabs' boundary planes); the step kernels update only the
// owned planes 1 .. nz_own.  With the in-place AA pattern each step is
//   psi pass (owned planes)  ->  psi halo: each boundary psi plane into the neighbour's ghost plane
//   collide pass (owned)     ->  populations:
//       after an even step (pull): the five slots of a boundary plane that the neighbour's
//           cells read in the odd step (those of the velocities pointing at the neighbour) are
//           copied into the neighbour's ghost plane;
//       after an odd step (push): the five slots the boundary cells streamed into a ghost plane
//           are copied into the neighbour's owned boundary plane.
// Even steps read and write each cell's own slots, so the ghost planes matter only to odd
// steps (reads) and after them (writes).  The plan below lists every transfer as byte ranges
// of the population store and of the padded psi field; plb_slab_exchange carries it out with
// cudaMemcpyAsync between two handles, and a multi-process caller can carry out the same plan
// with its own transport (each entry of face f on one slab pairs with the same entry of face
// 1 - f on its neighbour: send range here -> receive range there).
#include <cuda_runtime.h>

#include <cstring>

#include "plb.h"
#include "plb_device.cuh"
#include "plb_host.h"
#include "plb_launch.h"

namespace {

using plb::D3Q19;

// D3Q19 slots with c_z = +1 and, in the same order, their opposites (c_z = -1).
constexpr int kUp[5] = {5, 11, 14, 15, 18};
constexpr int kDown[5] = {6, 12, 13, 16, 17};

int plan(int lattice, const int dims[3], int precision, int wall_y, int pass, int odd, plb_xfer *out, int max,
         int *count) {
    if (!count) return plb::set_error(PLB_EINVAL, "count is NULL");
    *count = 0;
    if (lattice != PLB_D3Q19) return plb::set_error(PLB_EUNSUPPORTED, "slabs split D3Q19 lattices along z");
    if (!dims || dims[2] < 3) return plb::set_error(PLB_EINVAL, "a slab needs two ghost planes and one owned plane");
    if (pass != 0 && pass != 1) return plb::set_error(PLB_EINVAL, "pass must be 0 (psi) or 1 (collide)");
    plb::Layout L;
    if (!plb::make_layout(lattice, dims, precision, L)) return plb::set_error(PLB_EINVAL, "bad dims or precision");
    const int nz = dims[2];
    const long long plane = (long long)dims[0] * dims[1];
    const int n = pass == 0 ? 2 : 10;
    if (max < n || !out) return plb::set_error(PLB_EINVAL, "the plan has %d transfers", n);
    int k = 0;
    if (pass == 0) {
        // padded psi plane of local plane z is z + 1; the psi plane holds px x py values
        const long long pp = (long long)L.px * L.py * L.s_psi;
        out[k++] = {2 * pp, 1 * pp, pp, 0, 1};                              // plane 1 -> below; ghost 0 <- below
        out[k++] = {(long long)(nz - 1) * pp, (long long)nz * pp, pp, 1, 1};  // plane nz-2 -> above; ghost nz-1 <- above
    } else {
        auto off = [&](int slot, int z) { return ((long long)slot * L.pstride + plane * z) * L.s_pop; };
        const long long full = plane * L.s_pop;
        for (int f = 0; f < 2; ++f) {
            for (int m = 0; m < 5; ++m) {
                plb_xfer x;
                x.face = f;
                x.region = 0;
                if (!odd) {
                    // pull, for the odd step: face 0 sends plane 1's c_z = +1 slots (read by the
                    // cells below) and receives the cells below's c_z = -1 slots into ghost plane 0;
                    // face 1 the mirror image
                    const int snd = f == 0 ? kUp[m] : kDown[m], rcv = f == 0 ? kDown[m] : kUp[m];
                    x.send_off = off(snd, f == 0 ? 1 : nz - 2);
                    x.recv_off = off(rcv, f == 0 ? 0 : nz - 1);
                    x.bytes = full;
                } else {
                    // push, after the odd step: face 0 sends the c_z = -1 slots its plane-1 cells
                    // streamed into ghost plane 0 and receives into plane 1 the c_z = +1 slots the
                    // cells below streamed into their upper ghost plane.  A slot whose upstream
                    // cell lies beyond a y wall is written by its own cell (halfway bounce-back),
                    // so that row is left out: rows 1 .. ny-1 (c_y = +1) or 0 .. ny-2 (c_y = -1).
                    const int snd = f == 0 ? kDown[m] : kUp[m], rcv = f == 0 ? kUp[m] : kDown[m];
                    x.send_off = off(snd, f == 0 ? 0 : nz - 1);
                    x.recv_off = off(rcv, f == 0 ? 1 : nz - 2);
                    x.bytes = full;
                    // snd and rcv are opposite slots: their c_y are both zero or of opposite signs
                    if (wall_y && D3Q19::cy(snd) != 0) {
                        const long long row = (long long)dims[0] * L.s_pop;
                        x.bytes = full - row;
                        if (D3Q19::cy(snd) > 0) x.send_off += row;
                        if (D3Q19::cy(rcv) > 0) x.recv_off += row;
                    }
                }
                out[k++] = x;
            }
        }
    }
    *count = k;
    return PLB_OK;
}

}  // namespace

extern "C" {

int plb_slab_plan(int lattice, const int dims[3], int precision, int wall_y, int pass, int odd, plb_xfer *out,
                  int max, int *count) {
    return plan(lattice, dims, precision, wall_y, pass, odd != 0, out, max, count);
}

int plb_slab_bind(plb_t *h, int z_first) {
    if (!h) return plb::set_error(PLB_EINVAL, "NULL handle");
    if (h->view) return plb::set_error(PLB_EINVAL, "a batch instance cannot be a slab");
    if (h->lattice != PLB_D3Q19) return plb::set_error(PLB_EUNSUPPORTED, "slabs split D3Q19 lattices along z");
    if (h->pops2) return plb::set_error(PLB_EUNSUPPORTED, "slabs step in place (AA streaming)");
    if (h->dims[2] < 3) return plb::set_error(PLB_EINVAL, "a slab needs two ghost planes and one owned plane");
    if (h->odd) return plb::set_error(PLB_EINVAL, "bind the slab at an even step (natural layout)");
    if (z_first < 0) return plb::set_error(PLB_EINVAL, "z_first must be >= 0");
    h->slab = 1;
    // stochastic rounding draws its noise from the cell index of the whole lattice
    h->kp.cell_base = (unsigned)((long long)(z_first - 1) * h->dims[0] * h->dims[1]);
    h->slab_stage = 0;
    h->kp.z0 = 1;
    h->kp.nzl = h->dims[2] - 2;
    return PLB_OK;
}

int plb_slab_pass(plb_t *h, int pass) {
    if (!h) return plb::set_error(PLB_EINVAL, "NULL handle");
    if (!h->slab) return plb::set_error(PLB_EINVAL, "not a slab (plb_slab_bind)");
    if (pass != h->slab_stage)
        return plb::set_error(PLB_EINVAL, "pass %d out of order: the next pass is %d", pass, h->slab_stage);
    if (pass == 0) {
        h->kp.salt = (unsigned)h->t;
        h->L->psi(h->kp, h->pops, h->psi, h->odd, h->stream);
        h->slab_stage = 1;
    } else {
        const int coll = h->opts.collision == PLB_MRT ? 1 : 0;
        h->kp.salt = (unsigned)h->t;
        h->L->collide[coll](h->kp, h->pops, h->psi, h->odd, h->stream);
        h->odd ^= 1;
        h->t += 1;
        h->slab_stage = 0;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return PLB_OK;
}

int plb_slab_regions(plb_t *h, void **pops, void **psi) {
    if (!h || !pops || !psi) return plb::set_error(PLB_EINVAL, "NULL argument");
    *pops = h->pops;
    *psi = h->psi;
    return PLB_OK;
}

int plb_slab_exchange(plb_t *lower, plb_t *upper, int pass) {
    if (!lower || !upper) return plb::set_error(PLB_EINVAL, "NULL handle");
    if (!lower->slab || !upper->slab) return plb::set_error(PLB_EINVAL, "not a slab (plb_slab_bind)");
    if (lower->dims[0] != upper->dims[0] || lower->dims[1] != upper->dims[1] ||
        lower->opts.precision != upper->opts.precision || lower->opts.wall_y != upper->opts.wall_y)
        return plb::set_error(PLB_EINVAL, "slabs of different cross-sections, precisions or walls");
    // after the psi pass the next pass is the collide pass; after the collide pass it is the psi
    // pass again and odd has flipped
    const int want_stage = pass == 0 ? 1 : 0;
    if (lower->slab_stage != want_stage || upper->slab_stage != want_stage || lower->t != upper->t)
        return plb::set_error(PLB_EINVAL, "the slabs are not both just after pass %d of the same step", pass);
    const int odd = pass == 0 ? lower->odd : lower->odd ^ 1;   // parity of the step that ran
    plb_xfer lo[10], up[10];
    int nlo = 0, nup = 0;
    int st = plan(PLB_D3Q19, lower->dims, lower->opts.precision, lower->opts.wall_y, pass, odd, lo, 10, &nlo);
    if (st != PLB_OK) return st;
    st = plan(PLB_D3Q19, upper->dims, upper->opts.precision, upper->opts.wall_y, pass, odd, up, 10, &nup);
    if (st != PLB_OK) return st;
    auto base = [](plb_t *h, int region) { return region == 0 ? h->pops : h->psi; };
    // lower's face 1 <-> upper's face 0, entry by entry
    const int per_face = nlo / 2;
    for (int m = 0; m < per_face; ++m) {
        const plb_xfer &a = lo[per_face + m];   // lower, face 1
        const plb_xfer &b = up[m];              // upper, face 0
        cudaError_t e = cudaMemcpyAsync(base(upper, b.region) + b.recv_off, base(lower, a.region) + a.send_off,
                                        (size_t)a.bytes, cudaMemcpyDefault, lower->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base(lower, a.region) + a.recv_off, base(upper, b.region) + b.send_off,
                                (size_t)b.bytes, cudaMemcpyDefault, lower->stream);
        if (e != cudaSuccess) return plb::set_error(PLB_ECUDA, "slab exchange: %s", cudaGetErrorString(e));
    }
    return PLB_OK;
}

}  // extern "C"
