"""Pins for the oracle's time step (Algorithm 1; Eqs. C-H_discrete_fft,
A-C_discrete_fft, C-H_fft_b, A-C_fft_b, A-C_discrete_fft_c/eta), the explicit
FD comparison scheme (Section 2.2) and the adjoint of one step."""
import math

import numpy as np
import pytest

from paper_2306_04322_gb300 import inputs as I


def config1():
    pr = I.Problem(n=(64, 64), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    return pr


def test_config1_dt_value():
    assert config1().dt == pytest.approx(5 * 2 / 1120, rel=1e-15)


@pytest.mark.parametrize("n,p", [((64, 64), 1), ((32, 16), 2), ((8, 16, 8), 2)])
def test_mean_c_conserved(O, n, p):
    """The k = 0 row of the c update is the identity (|xi|^2 = 0)."""
    pr = I.Problem(n=n, p=p)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f = I.noise_fields(pr, seed=1)
    g, worst = O.step(pr, f, 50)
    assert abs(g[0].mean() - f[0].mean()) <= 1e-14 * 50 * abs(f[0].mean())
    assert worst < 1e-13


@pytest.mark.parametrize("n,k", [((16, 16), (1, 2)), ((32, 8), (5, 3)), ((8, 8, 8), (1, 2, 3)),
                                 ((2048, 4), (37, 1)), ((4, 2048), (1, 611))])
@pytest.mark.parametrize("lap", [0, 1, 2])
def test_linear_c_mode_closed_form(O, n, k, lap):
    """eta = 0 is a fixed point (h' = g' = 0) and df/dc = 2 rho^2 (c - c_alpha)
    is then linear, so a cosine mode of c is multiplied each step by exactly
    G = (1 - 2 rho^2 M dt K2) / (1 + kappa_c M dt K2^2)."""
    pr = I.Problem(n=n, p=2, dt=2e-2, lap=lap)
    eps, cbar = 0.1, 0.5
    f = I.cosine_mode_fields(pr, k, cbar, eps)
    # K2 of the mode from the paper's definitions for each variant
    xi = [2 * math.pi * kk / (nn * 1.0) for kk, nn in zip(k, n)]
    if lap == 0:
        K2 = sum(x * x for x in xi)
    elif lap == 1:
        K2 = sum(-2 * (math.cos(x) - 1) for x in xi)
    else:
        K2 = sum(-(16 * math.cos(x) - math.cos(2 * x) - 15) / 6 for x in xi)
    G = (1 - 2 * 2.0 * 5.0 * pr.dt * K2) / (1 + 3.0 * 5.0 * pr.dt * K2 * K2)
    g, _ = O.step(pr, f, 1)
    assert np.max(np.abs((g[0] - cbar) - G * (f[0] - cbar))) <= 1e-14
    assert np.max(np.abs(g[1:])) == 0.0
    g10, _ = O.step(pr, f, 10)
    assert np.max(np.abs((g10[0] - cbar) - G ** 10 * (f[0] - cbar))) <= 1e-13
    # continuous decay rate sigma = -M K2 (2 rho^2 + kappa_c K2), matched to O(dt)
    if lap == 0:
        sigma = -5.0 * K2 * (4.0 + 3.0 * K2)
        assert abs(math.log(abs(G)) / pr.dt - sigma) < 0.5 * abs(sigma) * abs(sigma) * pr.dt + 1e-12


@pytest.mark.parametrize("eta_bar,gain", [(0.5, lambda w, L, dt: 1 + w * L * dt),
                                          (0.0, lambda w, L, dt: 1 - 2 * w * L * dt)])
def test_linear_eta_mode_growth(O, eta_bar, gain):
    """p = 1, c = 0.5 (so f_beta = f_alpha), M = 0.  Around eta = 1/2,
    df/deta ~ w g''(1/2) d = -w d; around eta = 0, df/deta ~ 2 w d.  A small
    cosine mode is multiplied by G = gain / (1 + kappa_eta L dt K2)."""
    pr = I.Problem(n=(32, 16), p=1, M=0.0, dt=1e-2)
    eps = 1e-8
    for k in [(1, 0), (2, 3), (0, 1)]:
        f = I.cosine_mode_fields(pr, k, 0.5, eps, eta_val=eta_bar, which=1)
        K2 = (2 * math.pi * k[0] / 32) ** 2 + (2 * math.pi * k[1] / 16) ** 2
        G = gain(1.0, 5.0, pr.dt) / (1 + 3.0 * 5.0 * pr.dt * K2)
        g, _ = O.step(pr, f, 1)
        delta = g[1] - eta_bar
        want = G * (f[1] - eta_bar)
        # remaining terms are O(eps^2) relative to the mode
        assert np.max(np.abs(delta - want)) <= 10 * eps * eps + 4e-17
        assert np.max(np.abs(g[0] - 0.5)) == 0.0
        if eta_bar == 0.5 and K2 < 1.0 / 3.0:
            assert G > 1.0  # growth for K2 < w / kappa_eta


def test_stationary_flat_allen_cahn_interface(O):
    """p = 1, c = 0.5, M = 0: the slab eta = (tanh((x-a)/l) - tanh((x-b)/l))/2 with
    l = sqrt(2 kappa_eta / w) solves kappa_eta eta'' = w g'(eta); interfaces
    64 apart interact at ~exp(-52).  The scheme's fixed point is the spectral
    equilibrium, so eta must stay within the spectral resolution error."""
    pr = I.Problem(n=(512, 8), dx=(0.5, 0.5), p=1, M=0.0, dt=0.05)
    width = math.sqrt(2 * 3.0 / 1.0)
    f = I.tanh_slab_fields(pr, 64.0, 192.0, width)
    g, _ = O.step(pr, f, 1000)
    assert np.max(np.abs(g[1] - f[1])) < 1e-8
    # a wrong interface width is not stationary
    f2 = I.tanh_slab_fields(pr, 64.0, 192.0, 1.5 * width)
    g2, _ = O.step(pr, f2, 20)
    assert np.max(np.abs(g2[1] - f2[1])) > 1e-3


def test_free_energy_decreases_config1(O):
    """Eq. (fe) decreases monotonically along config 1's 200 steps (the paper
    observes monotone decrease, Section 3.1)."""
    pr = config1()
    f = I.noise_fields(pr, seed=0)
    E = [O.free_energy(pr, f)]
    for _ in range(20):
        f, _ = O.step(pr, f, 10)
        E.append(O.free_energy(pr, f))
    assert all(b < a for a, b in zip(E, E[1:])), E


def test_brute_force_step_dense_dft(O):
    """One step on 4 x 4 (and 4 x 4 x 4) with dense DFT matrices, written from
    the paper's Fourier-space equations, equals the oracle's FFT step."""
    for shape_n in [(4, 4), (4, 4, 4)]:
        pr = I.Problem(n=shape_n, p=2, dt=0.03)
        f = I.noise_fields(pr, seed=7, amp=0.2)
        d = O.derivatives(pr, f)
        K2 = O.k2(pr)
        shape = pr.shape
        N = pr.npoints
        # dense DFT matrix over the flattened multi-index
        idx = np.array(np.unravel_index(np.arange(N), shape)).T
        ph = np.zeros((N, N))
        for ax, n in enumerate(shape):
            ph += np.outer(idx[:, ax], idx[:, ax]) / n
        W = np.exp(-2j * np.pi * ph)
        Winv = np.conj(W) / N
        k2 = K2.ravel()
        out = np.empty_like(f)
        for fi in range(pr.nf):
            uh = W @ f[fi].ravel()
            fh = W @ d[fi].ravel()
            if fi == 0:
                b = uh - pr.M * pr.dt * k2 * fh
                new = b / (1 + pr.M * pr.dt * pr.kappa_c * k2 ** 2)
            else:
                b = uh - pr.L * pr.dt * fh
                new = b / (1 + pr.L * pr.dt * pr.kappa_eta * k2)
            out[fi] = (Winv @ new).real.reshape(shape)
        g, _ = O.step(pr, f, 1)
        assert np.max(np.abs(g - out)) < 1e-14


def test_fd_scheme_linear_mode_closed_form(O):
    """Explicit FD (Section 2.2) with eta = 0: a cosine c-mode is multiplied by
    1 - dt M lam (2 rho^2 + kappa_c lam), lam = sum_d 4 sin^2(pi k_d / n_d)/dx^2;
    an eta mode about 0 by 1 - dt L (2 w + kappa_eta lam); mean c conserved."""
    pr = I.Problem(n=(16, 32), dx=(1.0, 0.5), p=1, dt=1e-3)
    k = (3, 5)
    lam = 4 * math.sin(math.pi * 3 / 16) ** 2 / 1.0 + 4 * math.sin(math.pi * 5 / 32) ** 2 / 0.25
    f = I.cosine_mode_fields(pr, k, 0.5, 0.1)
    g = O.fd_step(pr, f, 3)
    G = 1 - pr.dt * 5.0 * lam * (4.0 + 3.0 * lam)
    assert np.max(np.abs((g[0] - 0.5) - G ** 3 * (f[0] - 0.5))) < 1e-13
    f = I.cosine_mode_fields(pr, k, 0.5, 1e-9, eta_val=0.0, which=1)
    g = O.fd_step(pr, f, 1)
    G = 1 - pr.dt * 5.0 * (2.0 + 3.0 * lam)
    assert np.max(np.abs(g[1] - G * f[1])) < 1e-15 + 10 * 1e-18
    pr = pr.replace(dt=0.9 * I.fd_stable_dt(pr))
    f = I.noise_fields(pr, seed=2)
    g = O.fd_step(pr, f, 20)
    assert np.all(np.isfinite(g))
    assert abs(g[0].mean() - f[0].mean()) < 1e-15 * 20


def test_fd_3d_matches_stencil(O):
    pr = I.Problem(n=(8, 8, 16), p=1, dt=1e-4)
    f = I.noise_fields(pr, seed=4, amp=0.2)
    d = O.derivatives(pr, f)

    def lap(a):
        return sum(np.roll(a, s, ax) for ax in range(3) for s in (1, -1)) - 6 * a

    mu = d[0] - 3.0 * lap(f[0])
    c = f[0] + pr.dt * 5.0 * lap(mu)
    e = f[1] - pr.dt * 5.0 * (d[1] - 3.0 * lap(f[1]))
    g = O.fd_step(pr, f, 1)
    assert np.max(np.abs(g[0] - c)) < 1e-15 and np.max(np.abs(g[1] - e)) < 1e-15


@pytest.mark.parametrize("n,p", [((16, 8), 2), ((8, 8, 4), 1)])
def test_adjoint_matches_central_differences(O, n, p):
    """<lam, (S(u + h v) - S(u - h v)) / 2h> = <J^T lam, v> and the parameter
    sensitivities equal central differences of <lam, S(u; theta)>."""
    pr = I.Problem(n=n, p=p, dt=0.02)
    rng = np.random.default_rng(11)
    u = I.noise_fields(pr, seed=5, amp=0.3)
    lam = rng.standard_normal(u.shape)
    v = rng.standard_normal(u.shape)
    lam_out, grad = O.adjoint_step(pr, u, lam)
    h = 1e-6
    sp, _ = O.step(pr, u + h * v, 1)
    sm, _ = O.step(pr, u - h * v, 1)
    fd = np.sum(lam * (sp - sm)) / (2 * h)
    assert np.sum(lam_out * v) == pytest.approx(fd, rel=1e-7)
    for t, name in enumerate(["M", "L", "kappa_c", "kappa_eta"]):
        th = getattr(pr, name)
        hp = h * th
        sp, _ = O.step(pr.replace(**{name: th + hp}), u, 1)
        sm, _ = O.step(pr.replace(**{name: th - hp}), u, 1)
        fd = np.sum(lam * (sp - sm)) / (2 * hp)
        assert grad[t] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.sum(np.abs(lam)))
