"""Seeded synthetic inputs for the P-LBM workloads.

This module only shapes initial fields (tanh slabs, droplets, seeded noise) and
names workloads; it holds none of the method's arithmetic.  Coexistence
densities, EOS constants and relaxation times are passed in by the caller, so
the same arrays can be fed to the CUDA library and to an independent checker.

Noise: SplitMix64 (Steele, Lea & Flood 2014) of ``seed ^ (index * 0x9E3779B97F4A7C15)``,
top 53 bits mapped to U[-1, 1), scaled by the amplitude.  Master seed 250415018;
workload k uses seed + k.

Field layout: cell index ``x + nx * (y + ny * z)``; velocity arrays are (d, N).
"""
from __future__ import annotations

import numpy as np

MASTER_SEED = 250415018
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_pm1(n: int, seed: int) -> np.ndarray:
    """n values in U[-1, 1) from the counter-based SplitMix64 stream."""
    idx = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        bits = splitmix64(np.uint64(seed) ^ (idx * _GOLDEN))
    return (bits >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def grid_coords(dims):
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1).astype(np.float64), y.reshape(-1).astype(np.float64), z.reshape(-1).astype(np.float64)


def tanh_blend(d, rho_v: float, rho_l: float, width: float):
    """rho(d) = rho_v + (rho_l - rho_v) (1 - tanh(2 d / W)) / 2; d > 0 toward the vapour."""
    return rho_v + (rho_l - rho_v) * 0.5 * (1.0 - np.tanh(2.0 * d / width))


def slab(dims, axis: int, lo: float, hi: float, rho_in: float, rho_out: float, width: float = 4.0,
         periodic: bool = True):
    """Layer of density rho_in for coordinate in [lo, hi) (interfaces at lo - 1/2 and hi - 1/2),
    rho_out elsewhere.  Distances wrap when periodic."""
    coords = grid_coords(dims)
    n_ax = (list(dims) + [1, 1])[axis]
    s = coords[axis]
    a, b = lo - 0.5, hi - 0.5
    d = np.maximum(a - s, s - b)          # signed distance, > 0 outside the layer
    if periodic:
        outside = d > 0
        d_wrap = np.minimum(np.mod(a - s, n_ax), np.mod(s - b, n_ax))
        d = np.where(outside, d_wrap, d)
    return rho_out + (rho_in - rho_out) * 0.5 * (1.0 - np.tanh(2.0 * d / width))


def droplet(dims, center, radius: float, rho_v: float, rho_l: float, width: float = 4.0, periodic: bool = True):
    """Liquid disc / sphere of the given radius in vapour (minimum-image distance when periodic)."""
    coords = grid_coords(dims)
    nd = len(center)
    r2 = np.zeros_like(coords[0])
    for a in range(nd):
        n_ax = (list(dims) + [1, 1])[a]
        dx = coords[a] - center[a]
        if periodic:
            dx = (dx + n_ax / 2) % n_ax - n_ax / 2
        r2 += dx * dx
    return tanh_blend(np.sqrt(r2) - radius, rho_v, rho_l, width)


def add_noise(rho: np.ndarray, seed: int, amplitude: float) -> np.ndarray:
    if amplitude == 0.0:
        return rho.copy()
    return rho + amplitude * uniform_pm1(rho.size, seed)


# ------------------------------------------------------------------ workloads
#
# Peng-Robinson constants in lattice units (a = 2/49, b = 2/21, R = 1,
# acentric factor 0.327) shared by all named workloads.
PR_CONSTANTS = dict(a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.327)


def planar_d2q9_8x256(rho_v: float, rho_l: float, seed: int = MASTER_SEED + 1):
    """D2Q9 planar interface: 8 x 256 periodic, liquid for y in [64, 192), W = 4, noise 1e-4."""
    dims = (8, 256, 1)
    rho = slab(dims, 1, 64, 192, rho_l, rho_v, 4.0)
    return dims, add_noise(rho, seed, 1e-4)


def laplace_d2q9_256(rho_v: float, rho_l: float, radius: float):
    """D2Q9 static droplet: 256 x 256 periodic, centre (128, 128), tanh width 4, no noise."""
    dims = (256, 256, 1)
    return dims, droplet(dims, (128.0, 128.0), radius, rho_v, rho_l, 4.0)


def droplet_d3q19(n: int, rho_v: float, rho_l: float, width: float = 4.0):
    """D3Q19 static droplet: n^3 periodic, radius n/4 at the centre."""
    dims = (n, n, n)
    return dims, droplet(dims, (n / 2, n / 2, n / 2), n / 4, rho_v, rho_l, width)


def plates_d3q19(dims, rho_v: float, rho_l: float, y_lo: int | None = None, y_hi: int | None = None,
                 width: float = 4.0):
    """D3Q19 two-phase flow between plates: walls bound y, liquid next to both walls,
    vapour core for y in [y_lo, y_hi) (default [ny/4, 3 ny/4), i.e. [64, 192) at ny = 256)."""
    ny = dims[1]
    y_lo = ny // 4 if y_lo is None else y_lo
    y_hi = 3 * ny // 4 if y_hi is None else y_hi
    rho = slab(dims, 1, y_lo, y_hi, rho_v, rho_l, width, periodic=False)
    return dims, rho


def batched_d2q9_instances(count: int = 96, seed: int = MASTER_SEED + 4):
    """Descriptors of the uneven batched D2Q9 workload: side in {64, ..., 512}, kind in
    {static droplet, translating droplet, planar}, T/Tc in [0.7, 0.9]; drawn from the seed."""
    sides = np.array([64, 96, 128, 192, 256, 384, 512])
    u = (uniform_pm1(6 * count, seed) + 1.0) / 2.0     # U[0, 1)
    out = []
    for k in range(count):
        side = int(sides[min(int(u[6 * k] * len(sides)), len(sides) - 1)])
        kind = ["static", "translating", "planar"][min(int(u[6 * k + 1] * 3), 2)]
        t_ratio = 0.7 + 0.2 * u[6 * k + 2]
        rfrac = 0.1 + 0.2 * u[6 * k + 3]
        angle = 2.0 * np.pi * u[6 * k + 4]
        speed = 0.01 + 0.04 * u[6 * k + 5]
        out.append(dict(side=side, kind=kind, T_over_Tc=float(t_ratio), radius=float(rfrac * side),
                        velocity=(float(speed * np.cos(angle)), float(speed * np.sin(angle)))
                        if kind == "translating" else (0.0, 0.0)))
    return out
