"""Pins for the oracle's FFT: brute-force DFT from its definition, numpy's FFT
(an independent library routine), round trip and Parseval's identity."""
import itertools

import numpy as np
import pytest


def brute_dft(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """O(N^2) multi-dimensional DFT written from the definition
    X[k] = sum_j x[j] exp(sign 2 pi i sum_d j_d k_d / n_d)."""
    shape = a.shape
    out = np.zeros(shape, dtype=np.complex128)
    idx = list(itertools.product(*[range(n) for n in shape]))
    for k in idx:
        acc = 0j
        for j in idx:
            ph = sum(jd * kd / nd for jd, kd, nd in zip(j, k, shape))
            acc += a[j] * np.exp(sign * 2j * np.pi * ph)
        out[k] = acc
    return out


@pytest.mark.parametrize("shape", [(4, 4), (8, 8), (16, 16), (16, 8, 4), (2, 8), (32,)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_brute_force(O, shape, sign):
    rng = np.random.default_rng(1)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    got = O.fft(a, sign)
    ref = brute_dft(a, sign)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(64, 64), (8, 32, 16), (1024,), (4, 256), (2048,), (2, 2048), (2048, 4)])
def test_fft_matches_numpy(O, shape):
    rng = np.random.default_rng(2)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    got = O.fft(a, -1)
    ref = np.fft.fftn(a)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref)) * np.log2(a.size)


def test_fft_round_trip_and_parseval(O):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((32, 64)) + 1j * rng.standard_normal((32, 64))
    A = O.fft(a, -1)
    back = O.fft(A, 1) / a.size
    assert np.max(np.abs(back - a)) < 1e-14 * np.max(np.abs(a)) * 16
    assert abs(np.sum(np.abs(A) ** 2) / a.size - np.sum(np.abs(a) ** 2)) < 1e-12 * np.sum(np.abs(a) ** 2)


def test_fft_of_delta_and_constant(O):
    a = np.zeros((8, 16), dtype=complex)
    a[0, 0] = 1.0
    assert np.allclose(O.fft(a), 1.0, atol=1e-15)
    b = np.ones((8, 16), dtype=complex)
    B = O.fft(b)
    assert abs(B[0, 0] - 128) < 1e-12 and np.max(np.abs(B.ravel()[1:])) < 1e-12
