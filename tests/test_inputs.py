"""The seeded input generators shared by the CUDA tests and the oracle: the noise stream is
SplitMix64 as published, the fields have the stated geometry, and the batched workload's
descriptors stay in their stated ranges."""
import math

import numpy as np

from paper_2504_15018_gb300 import inputs

GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def test_splitmix64_matches_the_published_sequence():
    # the generator seeded with state 0 (Steele, Lea & Flood 2014; public reference outputs)
    with np.errstate(over="ignore"):
        got = inputs.splitmix64(np.arange(3, dtype=np.uint64) * GOLDEN)
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_stream_range_moments_and_determinism():
    a = inputs.uniform_pm1(200_000, 7)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 4 * math.sqrt(1 / 3 / a.size)
    assert abs(a.var() - 1 / 3) < 0.01
    assert np.array_equal(a, inputs.uniform_pm1(200_000, 7))
    assert np.array_equal(a[:1000], inputs.uniform_pm1(1000, 7))      # counter-based: prefix-stable
    assert not np.array_equal(a[:1000], inputs.uniform_pm1(1000, 8))


def test_slab_interfaces_are_odd_about_the_half_cells():
    dims = (2, 256, 1)
    rho = inputs.slab(dims, 1, 64, 192, 7.0, 0.3, 4.0).reshape(256, 2)[:, 0]
    mid = (7.0 + 0.3) / 2
    for lo, inside in ((64, 64), (192, 191)):                       # interfaces at 63.5 and 191.5
        outside = 2 * lo - 1 - inside
        assert abs((rho[inside] - mid) + (rho[outside] - mid)) < 1e-12
    assert rho[128] > 7.0 - 1e-6 and rho[0] < 0.3 + 1e-6
    full = inputs.slab(dims, 1, 64, 192, 7.0, 0.3, 4.0).reshape(256, 2)
    assert np.array_equal(full[:, 0], full[:, 1])


def test_droplet_area_and_minimum_image():
    n, R, rv, rl = 128, 20.0, 0.3, 7.0
    rho = inputs.droplet((n, n, 1), (64.0, 64.0), R, rv, rl, 4.0)
    area = ((rho - rv) / (rl - rv)).sum()
    assert abs(area / (math.pi * R * R) - 1) < 0.01
    corner = inputs.droplet((n, n, 1), (0.0, 0.0), R, rv, rl, 4.0).reshape(n, n)
    assert corner[0, 0] > rl - 1e-3 and corner[-1, -1] > rl - 0.2     # wraps across the corner
    assert np.allclose(corner[1:, 1:], corner[1:, 1:][::-1, ::-1])   # symmetric about (0, 0)


def test_plates_geometry():
    dims = (4, 256, 3)
    _, rho = inputs.plates_d3q19(dims, 0.25, 7.2)
    r = rho.reshape(3, 256, 4)
    assert np.array_equal(r[0], r[2]) and np.array_equal(r[:, :, 0], r[:, :, 3])   # x- and z-invariant
    col = r[0, :, 0]
    assert col[0] > 7.19 and col[255] > 7.19 and col[128] < 0.26                    # liquid at walls, vapour core
    assert abs(col[63] + col[64] - (0.25 + 7.2)) < 1e-12                             # interface at y = 63.5


def test_batched_descriptors_stay_in_range():
    insts = inputs.batched_d2q9_instances()
    assert len(insts) == 96
    assert insts == inputs.batched_d2q9_instances()
    assert {d["kind"] for d in insts} == {"static", "translating", "planar"}
    for d in insts:
        assert d["side"] in (64, 96, 128, 192, 256, 384, 512)
        assert 0.7 <= d["T_over_Tc"] < 0.9
        assert 0.1 * d["side"] <= d["radius"] < 0.3 * d["side"]
        speed = math.hypot(*d["velocity"])
        if d["kind"] == "translating":
            assert 0.01 - 1e-12 <= speed < 0.05
        else:
            assert speed == 0.0
