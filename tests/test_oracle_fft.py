"""Pins of the oracle's own discrete Fourier transform (oracle/fft.py).

The transform is checked against the definition X[k] = sum_j x[j] exp(-2 pi i jk/N) evaluated as a
plain sum, against transforms known in closed form (a shifted delta, a sampled complex exponential,
a sampled Gaussian), against Parseval's identity and the shift theorem, and, as an independent
cross-check only, against numpy's FFT.
"""
import math

import numpy as np
import pytest

from oracle import fft as of

LENGTHS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 14, 15, 16, 18, 20, 25, 27, 30, 32, 36, 45, 49, 64, 81, 97,
           100, 121, 128]


def naive_dft(x):
    """The definition as a double loop over (k, j) with exact integer reduction of jk mod N."""
    n = x.shape[-1]
    out = np.zeros(x.shape, dtype=np.complex128)
    for k in range(n):
        for j in range(n):
            out[..., k] += x[..., j] * complex(math.cos(-2 * math.pi * ((j * k) % n) / n),
                                               math.sin(-2 * math.pi * ((j * k) % n) / n))
    return out


@pytest.mark.parametrize("n", LENGTHS)
def test_dft_equals_definition(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    ref = naive_dft(x)
    err = np.abs(of.dft_last(x) - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert err < 1e-13, (n, err)


@pytest.mark.parametrize("n", [1, 2, 7, 12, 30, 64, 81])
def test_inverse_undoes_forward(n):
    rng = np.random.default_rng(7 * n)
    x = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    assert np.abs(of.idft(of.dft(x)) - x).max() < 1e-13


@pytest.mark.parametrize("n", [6, 16, 45, 97])
def test_closed_form_transforms(n):
    # shifted delta: X[k] = exp(-2 pi i j0 k / N)
    j0 = n // 3
    x = np.zeros(n)
    x[j0] = 1.0
    k = np.arange(n)
    assert np.abs(of.dft(x) - np.exp(-2j * math.pi * j0 * k / n)).max() < 1e-13
    # sampled exponential exp(2 pi i m j / N): N at index m, zero elsewhere
    m = (2 * n) // 5
    e = np.exp(2j * math.pi * m * np.arange(n) / n)
    want = np.zeros(n, dtype=complex)
    want[m] = n
    assert np.abs(of.dft(e) - want).max() < 1e-11 * n
    # constant: N at k = 0
    want = np.zeros(n, dtype=complex)
    want[0] = n
    assert np.abs(of.dft(np.ones(n)) - want).max() < 1e-12 * n


def test_periodic_gaussian_matches_poisson_sum():
    # a Gaussian summed over its periodic images and sampled on N points of [0, 2 pi): by Poisson
    # summation its DFT is the Gaussian's Fourier transform at the integer modes, divided by h
    n, s = 48, 0.4
    h = 2 * math.pi / n
    xj = np.arange(n) * h
    g = sum(np.exp(-((xj - 2 * math.pi * q) ** 2) / (2 * s * s)) for q in range(-3, 4))
    X = of.dft(g)
    k = of.mode_numbers(n)
    # Fourier coefficient of the periodised Gaussian on [0, 2 pi): sqrt(2 pi) s exp(-s^2 k^2 / 2) / h
    want = math.sqrt(2 * math.pi) * s * np.exp(-0.5 * (s * k) ** 2) / h
    # aliasing from |k| beyond N/2 is below exp(-s^2 (N/2)^2 / 2) ~ 1e-40
    assert np.abs(X - want).max() < 1e-11 * want.max()


@pytest.mark.parametrize("shape", [(8, 6, 10), (9, 5, 4), (16, 16, 16), (3, 7, 12)])
def test_dftn_parseval_shift_and_numpy(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal((3,) + shape)
    X = of.dftn(x)
    # Parseval: sum |x|^2 = sum |X|^2 / N
    ntot = int(np.prod(shape))
    assert abs(np.sum(np.abs(X[0]) ** 2) / ntot - np.sum(x[0] ** 2)) < 1e-12 * np.sum(x[0] ** 2)
    # shift theorem along the middle axis
    xs = np.roll(x, 1, axis=2)
    k = of.mode_numbers(shape[1])
    ph = np.exp(-2j * math.pi * k / shape[1])[None, None, :, None]
    assert np.abs(of.dftn(xs) - X * ph).max() < 1e-11 * np.abs(X).max()
    # real input: Hermitian symmetry X[-k] = conj X[k]
    Xr = X[1]
    idx = [(-np.arange(m)) % m for m in shape]
    assert np.abs(Xr[np.ix_(*idx)] - np.conj(Xr)).max() < 1e-11 * np.abs(Xr).max()
    # independent cross-check against numpy's FFT (tests only; the oracle does not call it)
    assert np.abs(X - np.fft.fftn(x, axes=(-3, -2, -1))).max() < 1e-12 * np.abs(X).max()
    assert np.abs(of.idftn(X).real - x).max() < 1e-13


def test_mode_numbers():
    assert list(of.mode_numbers(6)) == [0, 1, 2, 3, -2, -1]
    assert list(of.mode_numbers(5)) == [0, 1, 2, -2, -1]
    assert list(of.mode_numbers(1)) == [0]


def test_oracle_calls_no_library_fft():
    import pathlib
    root = pathlib.Path(__file__).resolve().parents[1] / "oracle"
    for p in root.glob("*.py"):
        assert "np.fft" not in p.read_text() and "scipy.fft" not in p.read_text(), p.name
