"""The seeded input generators shared by the oracle tests, the GPU tests and
the bench: the counter-based generator and the Section 3 initial conditions."""
import math

import numpy as np

from paper_2306_04322_gb300 import inputs as I


def test_splitmix64_known_values():
    # splitmix64 with state 0: the first outputs of the published generator
    v = I.splitmix64(0, 3)
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_offset():
    u = I.uniform_pm1(7, 1000)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert np.array_equal(I.uniform_pm1(7, 10, offset=5), u[5:15])


def test_benchmark_ic_at_origin():
    """At x = y = 0 every cosine is 1 except cos(-4) in eta_i's first term:
    c = c0 + 3 eps, eta_i = eta_nu (cos 4 + 1 + psi)^2."""
    pr = I.Problem(n=(16, 16), p=3)
    f = I.benchmark_ic_fields(pr)
    assert abs(f[0, 0, 0] - 0.65) < 1e-15
    for i in range(1, 4):
        assert abs(f[i, 0, 0] - 0.1 * (math.cos(4.0) + 2.5) ** 2) < 1e-14


def test_benchmark_ic_axes_and_index():
    """eta_i depends on i through the wavenumbers, and x runs along the last axis."""
    pr = I.Problem(n=(32, 64), p=2, dx=(0.5, 2.0))
    f = I.benchmark_ic_fields(pr)
    assert f.shape == (3, 64, 32)
    x, y = 3 * 0.5, 5 * 2.0
    want = 0.5 + 0.05 * (math.cos(0.105 * x) * math.cos(0.11 * y) + (math.cos(0.13 * x) * math.cos(0.087 * y)) ** 2
                         + math.cos(0.025 * x - 0.15 * y) * math.cos(0.07 * x - 0.02 * y))
    assert abs(f[0, 5, 3] - want) < 1e-15
    assert not np.allclose(f[1], f[2])


def test_extrusion_plane_and_symmetry():
    """At z = lz/2 the extruded field equals the 2D one; it is even about that
    plane and falls towards 0 away from it; c is uniform."""
    pr = I.Problem(n=(32, 32), p=2)
    f2 = I.benchmark_ic_fields(pr)
    f2[1:] = np.clip(f2[1:], 0.0, 1.0)
    g = I.extrude_3d(f2, 64)
    assert g.shape == (3, 64, 32, 32)
    inside = (f2[1] > 1e-6) & (f2[1] < 1 - 1e-6)
    assert np.allclose(g[1, 32][inside], f2[1][inside], rtol=0, atol=1e-12)
    assert np.allclose(g[1, 32 - 3], g[1, 32 + 3], rtol=0, atol=1e-15)
    assert np.all(g[1, 32 + 4] <= g[1, 32] + 1e-15)
    assert np.all(g[1, 0] < 1e-6)
    assert np.all(g[0] == 0.5)
