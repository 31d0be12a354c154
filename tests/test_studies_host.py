"""Host-side input preparation of the studies: Fourier resampling of the
t = 1 state between the grids of the Table 1 study."""
import math

import numpy as np

from paper_2306_04322_gb300 import experiments as X


def _modes(n, l=200.0):
    x = np.arange(n) * (l / n)
    X_, Y_ = np.meshgrid(x, x, indexing="xy")
    k = 2 * math.pi / l
    f = np.empty((2, n, n))
    f[0] = 0.5 + 0.1 * np.cos(3 * k * X_ - 5 * k * Y_) + 0.02 * np.sin(7 * k * Y_)
    f[1] = 0.3 * np.cos(k * X_) * np.cos(11 * k * Y_) + 0.05 * np.sin(13 * k * X_ + 2 * k * Y_)
    return f


def test_upsampling_a_band_limited_field_is_exact():
    """Modes below both Nyquist limits: the 32^2 samples resampled to 128^2
    equal the same closed form sampled on 128^2, and the coarse points are
    unchanged."""
    f32, f128 = _modes(32), _modes(128)
    g = X.spectral_resample(f32, 128)
    assert g.dtype == np.float64 and g.shape == (2, 128, 128)
    assert np.max(np.abs(g - f128)) < 1e-13
    assert np.max(np.abs(g[:, ::4, ::4] - f32)) < 1e-13


def test_down_then_identity_and_truncation():
    """128 -> 32 of a field whose modes fit the coarse grid returns its
    samples; a mode above the coarse Nyquist is removed, not aliased."""
    f = _modes(128)
    assert np.max(np.abs(X.spectral_resample(f, 32) - _modes(32))) < 1e-13
    x = np.arange(128) * (200.0 / 128)
    hi = 0.2 * np.cos(2 * math.pi * 20 * x / 200.0)[None, None, :] * np.ones((1, 128, 1))
    g = X.spectral_resample(f[:1] + hi, 32)
    assert np.max(np.abs(g - _modes(32)[:1])) < 1e-13


def test_table1_constants_match_the_paper():
    """The study's grids and FD time steps against the Table 1 fixture (the
    2D rows of tests/golden/paper_fd_dt.txt); FS time steps as printed."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_fd_dt.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    fd2 = {int(r[1]): float(r[3]) for r in rows if r[0] == "2"}
    assert all(float(r[2]) == 200.0 for r in rows if r[0] == "2")
    assert tuple(sorted(fd2)) == X.TABLE1_GRIDS
    assert X.TABLE1_FD_DT == fd2
    assert X.TABLE1_FS_DTS == (1e-4, 1e-3, 5e-3)


def test_table2_constants_match_the_paper():
    """The 3D study's grids and FD time steps against the Table 2 fixture (the
    3D rows of tests/golden/paper_fd_dt.txt, cube of edge 100)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_fd_dt.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    fd3 = {int(r[1]): float(r[3]) for r in rows if r[0] == "3"}
    assert all(float(r[2]) == 100.0 for r in rows if r[0] == "3")
    assert tuple(sorted(fd3)) == X.TABLE2_GRIDS
    assert X.TABLE2_FD_DT == fd3
