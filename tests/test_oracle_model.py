"""Pins for the oracle's model terms: the free-energy density and its
derivatives (Section 2.1), the frequency norms (Eqs. Gamma_fft, Gamma_fft-fdO2,
Gamma_fft-fdO4 and their 3D forms) and the free energy, Eq. (fe)."""
import math

import numpy as np
import pytest

from paper_2306_04322_gb300 import inputs as I


def test_fchem_values_from_definition(O):
    """f_chem in the pure phases: alpha matrix (all eta = 0) gives rho^2 (c-c_a)^2;
    a beta grain (eta_i = 1, others 0) gives rho^2 (c_b - c)^2 (h = 1, g = 0)."""
    pr = I.Problem(p=3)
    for c in (0.1, 0.5, 0.83):
        assert O.fchem_point(pr, c, [0, 0, 0]) == pytest.approx(2.0 * (c - 0.3) ** 2, abs=1e-15)
        for i in range(3):
            e = [0.0, 0.0, 0.0]
            e[i] = 1.0
            assert O.fchem_point(pr, c, e) == pytest.approx(2.0 * (0.7 - c) ** 2, abs=1e-15)
    # eta_1 = eta_2 = 1: h = 2, and the alpha double sum over ordered pairs
    # (i, j), j != i, counts eta_1^2 eta_2^2 twice: g = 2 alpha.
    c = 0.4
    fa, fb = 2.0 * (c - 0.3) ** 2, 2.0 * (0.7 - c) ** 2
    assert O.fchem_point(pr, c, [1.0, 1.0, 0.0]) == pytest.approx(fa * (1 - 2) + fb * 2 + 1.0 * 2 * 5.0,
                                                                  abs=1e-14)
    # single eta = 1/2: h = 1/2, g = 1/16
    assert O.fchem_point(I.Problem(p=1), c, [0.5]) == pytest.approx(0.5 * fa + 0.5 * fb + 1 / 16, abs=1e-15)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_derivatives_match_central_differences(O, p):
    pr = I.Problem(p=p)
    rng = np.random.default_rng(p)
    for _ in range(5):
        c = rng.uniform(-0.2, 1.2)
        eta = rng.uniform(-0.2, 1.2, size=p)
        d = O.dfchem_point(pr, c, eta)
        H = O.d2fchem_point(pr, c, eta)
        h = 1e-5
        x0 = np.concatenate([[c], eta])
        for k in range(1 + p):
            xp, xm = x0.copy(), x0.copy()
            xp[k] += h
            xm[k] -= h
            fd = (O.fchem_point(pr, xp[0], xp[1:]) - O.fchem_point(pr, xm[0], xm[1:])) / (2 * h)
            assert d[k] == pytest.approx(fd, rel=1e-8, abs=1e-8)
            dd = (O.dfchem_point(pr, xp[0], xp[1:]) - O.dfchem_point(pr, xm[0], xm[1:])) / (2 * h)
            assert np.allclose(H[:, k], dd, rtol=1e-7, atol=1e-7)
        assert np.allclose(H, H.T, atol=1e-14)


def test_derivative_fields_layout(O):
    pr = I.Problem(n=(8, 16), p=2)
    f = I.noise_fields(pr, seed=3, amp=0.3)
    d = O.derivatives(pr, f)
    for (y, x) in [(0, 0), (5, 3), (15, 7)]:
        ref = O.dfchem_point(pr, f[0, y, x], f[1:, y, x])
        assert np.allclose(d[:, y, x], ref, atol=1e-15)


def _apply_symbol(O, field, sym):
    F = O.fft(field.astype(complex), -1)
    return (O.fft(F * sym, 1) / field.size).real


@pytest.mark.parametrize("n,dx", [((16, 8), (1.0, 1.0)), ((8, 8, 16), (0.5, 1.0, 2.0)), ((32, 16), (0.7, 1.3))])
def test_k2_spectral_is_minus_laplacian_of_trig_polynomial(O, n, dx):
    """For a trigonometric polynomial below the Nyquist band, F^-1(-|xi|^2 F phi)
    equals the analytic Laplacian."""
    pr = I.Problem(n=n, dx=dx, p=1, lap=0)
    coords = I.grid_coords(pr)
    lens = [a * b for a, b in zip(n, dx)]
    phi = np.zeros(pr.shape)
    lap = np.zeros(pr.shape)
    rng = np.random.default_rng(0)
    for _ in range(4):
        ks = [rng.integers(-(m // 2) + 1, m // 2) for m in n]
        amp, ph = rng.standard_normal(), rng.uniform(0, 2 * math.pi)
        arg = sum(2 * math.pi * k * x / l for k, x, l in zip(ks, coords, lens)) + ph
        xi2 = sum((2 * math.pi * k / l) ** 2 for k, l in zip(ks, lens))
        phi += amp * np.cos(arg)
        lap += -xi2 * amp * np.cos(arg)
    got = _apply_symbol(O, phi, -O.k2(pr))
    assert np.max(np.abs(got - lap)) < 1e-11 * max(1.0, np.max(np.abs(lap)))


def _stencil_lap(phi, dx, order):
    out = np.zeros_like(phi)
    nd = phi.ndim
    for d in range(len(dx)):
        ax = nd - 1 - d  # x is the last numpy axis
        h2 = dx[d] ** 2
        if order == 2:
            out += (np.roll(phi, 1, ax) - 2 * phi + np.roll(phi, -1, ax)) / h2
        else:
            out += (-np.roll(phi, 2, ax) + 16 * np.roll(phi, 1, ax) - 30 * phi
                    + 16 * np.roll(phi, -1, ax) - np.roll(phi, -2, ax)) / (12 * h2)
    return out


@pytest.mark.parametrize("lap,order", [(1, 2), (2, 4)])
@pytest.mark.parametrize("n,dx", [((16, 8), (1.0, 0.5)), ((8, 16, 8), (1.0, 2.0, 0.25))])
def test_k2_fd_variants_equal_stencils(O, lap, order, n, dx):
    """The FS-FD |xi_c2|^2 / |xi_c4|^2 symbols reproduce the centred 3-point and
    5-point-per-axis finite-difference Laplacians exactly (up to rounding)."""
    pr = I.Problem(n=n, dx=dx, p=1, lap=lap)
    rng = np.random.default_rng(5)
    phi = rng.standard_normal(pr.shape)
    got = _apply_symbol(O, phi, -O.k2(pr))
    ref = _stencil_lap(phi, dx, order)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_k2_frequency_vector_order(O):
    """Index k maps to n_k = [0..n/2, -(n/2-1)..-1]: |xi|^2 is even in k and the
    Nyquist bin carries (pi/dx)^2."""
    pr = I.Problem(n=(8, 4), dx=(0.5, 1.0), p=1)
    K = O.k2(pr)
    assert K[0, 0] == 0.0
    assert K[0, 4] == pytest.approx((math.pi / 0.5) ** 2, rel=1e-15)
    assert K[2, 0] == pytest.approx(math.pi ** 2, rel=1e-15)
    for x in range(1, 8):
        assert K[0, x] == pytest.approx(K[0, 8 - x], rel=1e-15)


def test_free_energy_closed_forms(O):
    pr = I.Problem(n=(32, 16), dx=(0.5, 2.0), p=2)
    V = 32 * 0.5 * 16 * 2.0
    # uniform fields: F = f_chem * V
    f = np.empty((3,) + pr.shape)
    f[0], f[1], f[2] = 0.45, 0.2, 0.6
    F = O.free_energy(pr, f)
    assert F == pytest.approx(O.fchem_point(pr, 0.45, [0.2, 0.6]) * V, rel=1e-13)
    # one cosine mode in c, eta = 0: chemical rho2 V ((cbar-ca)^2 + eps^2/2),
    # gradient kappa_c/2 eps^2 xi^2 V / 2
    eps, cbar = 0.05, 0.5
    g = I.cosine_mode_fields(pr, (3, 2), cbar, eps, eta_val=0.0)
    F, parts = O.free_energy(pr, g, parts=True)
    xi2 = (2 * math.pi * 3 / 16) ** 2 + (2 * math.pi * 2 / 32) ** 2
    assert parts[0] == pytest.approx(2.0 * V * ((cbar - 0.3) ** 2 + eps ** 2 / 2), rel=1e-12)
    assert parts[1] == pytest.approx(1.5 * eps ** 2 * xi2 * V / 2, rel=1e-12)
    assert abs(parts[2]) < 1e-20 and abs(parts[3]) < 1e-20


def test_free_energy_closed_forms_3d(O):
    """The same closed forms on an anisotropic 3D grid (Eq. fe with the 3D
    frequency vector): uniform fields give f_chem V; one cosine mode in c
    (eta = 0) gives rho2 V ((cbar - ca)^2 + eps^2 / 2) and kappa_c eps^2 xi^2 V / 4;
    one cosine mode in eta_1 gives kappa_eta eps^2 xi^2 V / 4 as its gradient part."""
    pr = I.Problem(n=(8, 16, 4), dx=(1.0, 0.5, 2.0), p=1)
    V = 8 * 1.0 * 16 * 0.5 * 4 * 2.0
    f = np.empty((2,) + pr.shape)
    f[0], f[1] = 0.62, 0.35
    assert O.free_energy(pr, f) == pytest.approx(O.fchem_point(pr, 0.62, [0.35]) * V, rel=1e-13)
    eps, cbar = 0.04, 0.55
    k = (1, 3, 1)
    xi2 = sum((2 * math.pi * ki / (ni * di)) ** 2 for ki, ni, di in zip(k, pr.n, pr.dx))
    g = I.cosine_mode_fields(pr, k, cbar, eps, eta_val=0.0)
    _, parts = O.free_energy(pr, g, parts=True)
    assert parts[0] == pytest.approx(2.0 * V * ((cbar - 0.3) ** 2 + eps ** 2 / 2), rel=1e-12)
    assert parts[1] == pytest.approx(3.0 * eps ** 2 * xi2 * V / 4, rel=1e-12)
    assert abs(parts[2]) < 1e-20
    h = I.cosine_mode_fields(pr, k, cbar, eps, eta_val=0.5, which=1)
    _, parts = O.free_energy(pr, h, parts=True)
    assert abs(parts[1]) < 1e-20
    assert parts[2] == pytest.approx(3.0 * eps ** 2 * xi2 * V / 4, rel=1e-12)


def test_paper_fd_dt_tables_below_von_neumann_bound():
    """Every explicit-FD dt the paper ran (Tables 1 and 2) lies below the
    linearised von Neumann bound used here for 'the FD stable dt'."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_fd_dt.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 10
    for dim, n, length, dt in rows:
        dim, n = int(dim), int(n)
        pr = I.Problem(n=(n,) * dim, dx=(float(length) / n,) * dim, p=4)
        bound = I.fd_stable_dt(pr)
        assert float(dt) <= bound, (dim, n, dt, bound)
        assert float(dt) >= 0.1 * bound  # same order as the bound
