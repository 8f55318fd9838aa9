"""Oracle parity in the launch geometry of the benchmark workload.

The small parity cases of test_gpu_parity.py fit one thread block along x.  Here:
  - a D3Q19 MRT lattice between walls (liquid layer, droplet, body force, noise) of
    256 x 64 x 32 cells: two 64-thread blocks of cell pairs along x, 4096 blocks, several
    resident waves of the pair collide kernel, so its one-wave-ahead L2 prefetch (FP32) runs,
    compared with the oracle element by element after 100 (FP32) or 50 (FP16S) steps;
  - the benchmark workload itself (512 x 256 x 256, the configuration bench.py times, with
    seeded noise so that no two columns are alike): its stored state after 2 steps is run
    through the oracle for 2 more steps on windows of 16 x 256 x 16 cells (periodic x and z
    wrap included), and the inner 8 x 256 x 8 cells of each window (beyond the 2-step
    dependency radius of 4 cells from the window's edges) are compared with the library's
    state after those 2 steps."""
import numpy as np
import pytest

import oracle
from gpu_cases import direction_map, make_lattice, max_rel_err, maxwell, oracle_params
from paper_2504_15018_gb300 import inputs

pytestmark = pytest.mark.gpu

RATES = dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.3, s_m=1.5)


def _slab_droplet(dims, rv, rl):
    nx, ny, nz = dims
    # liquid on the lower wall (the layer's other edge lies outside the lattice), interface at y = ny/4 - 1/2
    layer = inputs.slab(dims, 1, -ny, ny // 4, rl, rv, 4.0, periodic=False)
    drop = inputs.droplet(dims, (nx / 2 - 0.3, 0.62 * ny, nz / 2 + 0.1), ny / 6, rv, rl, 4.0, periodic=False)
    return inputs.add_noise(np.maximum(layer, drop), inputs.MASTER_SEED + 300, 1e-4)


def _run(precision, steps, fp16_rounding=0):
    dims = (256, 64, 32)
    rv, rl, _ = maxwell(0.8)
    rho = _slab_droplet(dims, rv, rl)
    case = dict(lattice=1, dims=dims, wall=True, mrt=True, rates=RATES, fext=(2e-6, 0.0, 1e-6),
                precision=precision, fp16_rounding=fp16_rounding)
    P = oracle_params(case, rv, rl)
    fo = oracle.run(P, oracle.init(P, rho), steps)[:, direction_map(1)].T
    lat = make_lattice(case, rv, rl)
    lat.init(rho)
    lat.step(steps)
    lat.status()
    return fo, lat.populations()


def test_fp32_pair_kernels_at_production_geometry():
    """FP32: each step rounds a population through about 8 FP32 operations, so 100 steps
    stay within 100 * 8 * 2^-24 relative of the FP64 oracle."""
    ref, got = _run(1, 100)
    err = max_rel_err(ref, got)
    print(f"fp32 256x64x32, 100 steps: max rel err {err:.3e}")
    assert err <= 100 * 8 * 2.0 ** -24


@pytest.mark.parametrize("sr", [0, 1])
def test_fp16s_pair_kernels_at_production_geometry(sr):
    """FP16S: each store rounds the deviation from w_i rho_ref by at most half an ulp (one ulp
    with stochastic rounding), <= 2^-11 (2^-10) of w_i rho_l; over n steps a random walk:
    sqrt(n) times that, relative to w_i rho_l."""
    steps = 50
    ref, got = _run(2, steps, sr)
    c_w = np.abs(ref).max(axis=1, keepdims=True)
    err = float(np.max(np.abs(got - ref) / c_w))
    print(f"fp16s (sr={sr}) 256x64x32, {steps} steps: max err / (w_i rho_l) {err:.3e}")
    assert err <= np.sqrt(steps) * 2.0 ** (-10 if sr else -11)


def _state_view(lat, buf, dtype):
    """(Q, nz, ny, nx) view, in the storage type, of the stored populations of a raw state
    taken at even parity (natural layout)."""
    raw = np.frombuffer(buf, dtype=dtype, offset=64)
    pstride = raw.size // lat.Q
    nx, ny, nz = lat.dims
    return raw.reshape(lat.Q, pstride)[:, :lat.n].reshape(lat.Q, nz, ny, nx)


def _window(view, xs, zs, shift):
    """Populations f_i (FP64) of the cells (xs, all y, zs); shift: w_i rho_ref per direction
    (FP16S stores f_i - w_i rho_ref), else zeros."""
    return view[:, zs][:, :, :, xs].astype(np.float64) + shift[:, None, None, None]


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_benchmark_workload_sampled_windows_against_oracle(precision):
    import bench
    import paper_2504_15018_gb300 as plb

    dims = (512, 256, 256)
    rv, rl, _ = plb.plb_solve_params(plb.pr_eos(bench.T_RATIO))
    rho = inputs.add_noise(bench.initial_density(dims, rv, rl), inputs.MASTER_SEED + 301, 1e-4)
    lat = bench.make_lattice(dims, precision, "mrt")
    lat.init(rho)
    del rho
    lat.step(2)
    lat.status()
    dtype = np.float32 if precision == "fp32" else np.float16
    _, w = plb.plb_velocity_set(plb.PLB_D3Q19)
    # FP16S stores f_i - w_i rho_ref with rho_ref the vapour density of the EOS (the default)
    shift = w * rv if precision == "fp16s" else np.zeros(19)
    nx, ny, nz = dims
    W, M = 16, 4                                      # window width in x and z, margin (2 steps x radius 2)
    corners = [(0, 0), (120, 64), (248, 128), (nx - 8, nz - 8), (300, nz - 4), (500, 200)]
    wins = []
    buf = lat.get_state()
    view = _state_view(lat, buf, dtype)
    for (x0, z0) in corners:
        xs = (np.arange(W) + x0 - M) % nx
        zs = (np.arange(W) + z0 - M) % nz
        wins.append((xs, zs, _window(view, xs, zs, shift)))
    del view, buf
    lat.step(2)
    lat.status()
    buf = lat.get_state()
    view = _state_view(lat, buf, dtype)
    perm = direction_map(1)
    inv = np.argsort(perm)
    worst = 0.0
    for (xs, zs, fw) in wins:
        case = dict(lattice=1, dims=(W, ny, W), wall=True, mrt=True, rates=bench.MRT_RATES,
                    fext=(bench.BODY_FORCE, 0.0, 0.0))
        P = oracle_params(case, rv, rl)
        fo_in = np.ascontiguousarray(fw.reshape(19, -1).T[:, inv])
        fo = oracle.run(P, fo_in, 2)[:, perm].T.reshape(19, W, ny, W)
        want = fo[:, M:W - M, :, M:W - M].reshape(19, -1)
        got = _window(view, xs[M:W - M], zs[M:W - M], shift).reshape(19, -1)
        # error relative to the largest population of each direction in the window (~ w_i rho_l):
        # FP32, about 8 roundings of 2^-24 per step; FP16S, one rounding of the stored deviation
        # per step, at most 2^-11 of w_i rho_l
        c_w = np.abs(want).max(axis=1, keepdims=True)
        err = float(np.max(np.abs(got - want) / c_w))
        assert err <= 2 * (8 * 2.0 ** -24 if precision == "fp32" else 2.0 ** -11), err
        worst = max(worst, err)
    print(f"{precision} 512x256x256, {len(wins)} windows of {W}x{ny}x{W}, 2 steps: worst error {worst:.3e}")
