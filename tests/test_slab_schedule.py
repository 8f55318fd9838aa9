"""The exchange schedule of the slab decomposition (plb_slab_plan), run by two gloo ranks on
the CPU.  Each rank holds one slab of a small D3Q19 lattice (walls in y, periodic in x and z)
in the library's storage layout (structure of arrays with the plane stride of the workspace,
FP64, in-place AA pattern, padded psi field) and steps it with a NumPy stand-in for the two
kernels: a psi pass (psi of each owned cell from the sum of its populations) and a collide
pass (a local mix of the populations driven by the psi of the 18 neighbours), both with the
library's AA addressing and halfway bounce-back.  After each pass the ranks exchange exactly
the byte ranges the plan lists (torch.distributed isend / irecv); the owned planes must then
equal a single NumPy lattice stepped the same way, bit for bit.  The stand-in is data movement
and a made-up local update, not the method: what is checked is the plan (which planes and
slots move where, including the wall rows left out after odd steps)."""
import os
import socket

import numpy as np
import pytest

C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
              [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
OPP = np.array([0] + [i + 1 if i % 2 else i - 1 for i in range(1, 19)])
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


class Store:
    """A local lattice of (nx, ny, nz) cells in the library's byte layout (FP64)."""

    def __init__(self, nx, ny, nz):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        self.pstride = (self.n + 127) // 128 * 128
        self.gx = 2
        self.px = (nx + 2 * self.gx + 31) // 32 * 32
        self.py = ny + 2
        self.pops = np.zeros(19 * self.pstride)
        self.psi = np.zeros((nz + 2) * self.py * self.px)

    def A(self):
        return self.pops.reshape(19, self.pstride)[:, :self.n].reshape(19, self.nz, self.ny, self.nx)

    def P(self):
        return self.psi.reshape(self.nz + 2, self.py, self.px)


def _read(st, odd, zr, periodic_z):
    """Pre-collision populations of the cells of planes zr (AA addressing, bounce-back)."""
    A = st.A()
    z, y, x = np.meshgrid(zr, np.arange(st.ny), np.arange(st.nx), indexing="ij")
    f = np.empty((19,) + z.shape)
    for i in range(19):
        if not odd:
            f[i] = A[i, z, y, x]
            continue
        xs, ys, zs = (x - C[i, 0]) % st.nx, y - C[i, 1], z - C[i, 2]
        if periodic_z:
            zs = zs % st.nz
        wall = (ys < 0) | (ys >= st.ny)
        own = A[i, z, y, x]
        src = A[OPP[i], zs, np.clip(ys, 0, st.ny - 1), xs]
        f[i] = np.where(wall, own, src)
    return f, (z, y, x)


def _write(st, odd, cells, f, periodic_z):
    A = st.A()
    z, y, x = cells
    for i in range(19):
        if not odd:
            A[OPP[i], z, y, x] = f[i]
            continue
        xt, yt, zt = (x + C[i, 0]) % st.nx, y + C[i, 1], z + C[i, 2]
        if periodic_z:
            zt = zt % st.nz
        wall = (yt < 0) | (yt >= st.ny)
        A[OPP[i], z[wall], y[wall], x[wall]] = f[i][wall]
        A[i, zt[~wall], yt[~wall], xt[~wall]] = f[i][~wall]


def psi_pass(st, odd, zr, periodic_z):
    f, (z, y, x) = _read(st, odd, zr, periodic_z)
    st.P()[z + 1, y + 1, x + st.gx] = np.sqrt(f.sum(axis=0))


def collide_pass(st, odd, zr, periodic_z):
    f, (z, y, x) = _read(st, odd, zr, periodic_z)
    P = st.P()
    F = np.zeros((3,) + z.shape)
    for i in range(1, 19):
        xn, yn, zn = (x + C[i, 0]) % st.nx, np.clip(y + C[i, 1], 0, st.ny - 1), z + C[i, 2]
        if periodic_z:
            zn = zn % st.nz
        pn = P[zn + 1, yn + 1, xn + st.gx]
        for a in range(3):
            F[a] += W[i] * pn * C[i, a]
    mean = f.mean(axis=0)
    post = np.empty_like(f)
    for i in range(19):
        post[i] = f[i] + 0.3 * (mean - f[i]) + 0.01 * (C[i] @ F.reshape(3, -1)).reshape(z.shape)
    _write(st, odd, (z, y, x), post, periodic_z)


def _exchange(st, plan, rank, world):
    import torch
    import torch.distributed as dist
    regions = {0: st.pops.view(np.uint8), 1: st.psi.view(np.uint8)}
    nb = {0: (rank - 1) % world, 1: (rank + 1) % world}
    per_face = len(plan) // 2
    reqs, inbox = [], []
    for k, x in enumerate(plan):
        m = k % per_face
        send = torch.from_numpy(regions[x["region"]][x["send_off"]:x["send_off"] + x["bytes"]].copy())
        reqs.append(dist.isend(send, nb[x["face"]], tag=10 * x["face"] + m))
        recv = torch.empty(x["bytes"], dtype=torch.uint8)
        reqs.append(dist.irecv(recv, nb[x["face"]], tag=10 * (1 - x["face"]) + m))
        inbox.append((x, recv))
    for r in reqs:
        r.wait()
    for x, recv in inbox:
        regions[x["region"]][x["recv_off"]:x["recv_off"] + x["bytes"]] = recv.numpy()


def _initial(nx, ny, nz):
    rng = np.random.default_rng(17)
    return W[:, None, None, None] * rng.uniform(0.5, 1.5, (1, nz, ny, nx)) * (1 + 0.05 * rng.standard_normal(
        (19, nz, ny, nx)))


def _worker(rank, world, port, dims, cuts, steps, out):
    import torch.distributed as dist
    import paper_2504_15018_gb300 as plb
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny, nz = dims
        f0 = _initial(nx, ny, nz)
        z0, z1 = cuts[rank], cuts[rank + 1]
        m = z1 - z0
        st = Store(nx, ny, m + 2)
        st.A()[:] = f0[:, np.arange(z0 - 1, z1 + 1) % nz]
        owned = np.arange(1, m + 1)
        for t in range(steps):
            odd = t % 2
            psi_pass(st, odd, owned, False)
            _exchange(st, plb.plb_slab_plan(plb.PLB_D3Q19, (nx, ny, m + 2), plb.PLB_FP64, 1, 0, odd), rank, world)
            collide_pass(st, odd, owned, False)
            _exchange(st, plb.plb_slab_plan(plb.PLB_D3Q19, (nx, ny, m + 2), plb.PLB_FP64, 1, 1, odd), rank, world)
        np.save(out, st.A()[:, 1:m + 1])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("cuts", [(0, 5, 11), (0, 3, 11)])
def test_two_rank_slab_exchange_matches_the_whole_lattice(tmp_path, cuts):
    import multiprocessing as mp
    dims, steps = (10, 7, 11), 6
    nx, ny, nz = dims
    whole = Store(nx, ny, nz)
    whole.A()[:] = _initial(nx, ny, nz)
    allz = np.arange(nz)
    for t in range(steps):
        psi_pass(whole, t % 2, allz, True)
        collide_pass(whole, t % 2, allz, True)
    ctx = mp.get_context("spawn")
    port = _free_port()
    outs = [str(tmp_path / f"r{r}.npy") for r in range(2)]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, dims, cuts, steps, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        got = np.load(outs[r])
        assert np.array_equal(got, whole.A()[:, cuts[r]:cuts[r + 1]]), r


def _swap_in_process(slabs, plans):
    """Carries out the plans between two slabs of one process (each is above and below the other)."""
    reg = lambda st, r: (st.pops if r == 0 else st.psi).view(np.uint8)
    for k in range(2):
        lo, up = slabs[k], slabs[(k + 1) % 2]
        pl_lo, pl_up = plans[k], plans[(k + 1) % 2]
        per = len(pl_lo) // 2
        for m in range(per):
            a, b = pl_lo[per + m], pl_up[m]          # lower slab's face 1 <-> upper slab's face 0
            sa, sb = reg(lo, a["region"]), reg(up, b["region"])
            sb[b["recv_off"]:b["recv_off"] + a["bytes"]] = sa[a["send_off"]:a["send_off"] + a["bytes"]]
            sa[a["recv_off"]:a["recv_off"] + b["bytes"]] = sb[b["send_off"]:b["send_off"] + b["bytes"]]


@pytest.mark.parametrize("wall_rule", [True, False])
def test_the_wall_rows_of_the_push_matter(wall_rule):
    """The check is sharp: with the plan of a lattice without walls (whole planes pushed after
    odd steps, overwriting the slots that the receiving cells' own bounce-back wrote) the slabs
    of a walled lattice no longer equal the whole lattice; with the walled plan they do."""
    import paper_2504_15018_gb300 as plb
    dims, steps, cuts = (10, 7, 11), 4, (0, 5, 11)
    nx, ny, nz = dims
    whole = Store(nx, ny, nz)
    whole.A()[:] = _initial(nx, ny, nz)
    for t in range(steps):
        psi_pass(whole, t % 2, np.arange(nz), True)
        collide_pass(whole, t % 2, np.arange(nz), True)
    f0 = _initial(nx, ny, nz)
    slabs = []
    for z0, z1 in zip(cuts[:-1], cuts[1:]):
        st = Store(nx, ny, z1 - z0 + 2)
        st.A()[:] = f0[:, np.arange(z0 - 1, z1 + 1) % nz]
        slabs.append(st)
    for t in range(steps):
        odd = t % 2
        for pass_ in (0, 1):
            for st in slabs:
                (psi_pass if pass_ == 0 else collide_pass)(st, odd, np.arange(1, st.nz - 1), False)
            _swap_in_process(slabs, [plb.plb_slab_plan(plb.PLB_D3Q19, (nx, ny, st.nz), plb.PLB_FP64,
                                                       int(wall_rule), pass_, odd) for st in slabs])
    same = all(np.array_equal(st.A()[:, 1:-1], whole.A()[:, z0:z1])
               for st, (z0, z1) in zip(slabs, zip(cuts[:-1], cuts[1:])))
    assert same == wall_rule


def test_plan_sizes_and_pairing():
    """Pass 0: two padded psi planes; pass 1: five population planes per face, equal sizes on
    paired entries; without walls every plane is whole."""
    import paper_2504_15018_gb300 as plb
    nx, ny, nz = 12, 9, 6
    for prec, sp in ((plb.PLB_FP64, 8), (plb.PLB_FP32, 4), (plb.PLB_FP16S, 2)):
        p0 = plb.plb_slab_plan(plb.PLB_D3Q19, (nx, ny, nz), prec, 1, 0, 0)
        assert len(p0) == 2 and all(x["region"] == 1 for x in p0)
        for odd in (0, 1):
            for wall in (0, 1):
                p1 = plb.plb_slab_plan(plb.PLB_D3Q19, (nx, ny, nz), prec, wall, 1, odd)
                assert len(p1) == 10 and [x["face"] for x in p1] == [0] * 5 + [1] * 5
                for m in range(5):
                    assert p1[m]["bytes"] == p1[5 + m]["bytes"]
                sizes = sorted({x["bytes"] for x in p1})
                if wall and odd:
                    assert sizes == [(ny - 1) * nx * sp, ny * nx * sp]
                else:
                    assert sizes == [ny * nx * sp]
    with pytest.raises(plb.PlbError) as e:
        plb.plb_slab_plan(plb.PLB_D2Q9, (nx, ny, 1), plb.PLB_FP32, 0, 0, 0)
    assert e.value.code == plb.PLB_EUNSUPPORTED
