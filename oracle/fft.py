"""Discrete Fourier transforms of the oracle: mixed-radix Cooley-Tukey, FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The Stokes solve of Section 2.1 (step 2) takes the force density to Fourier
space, applies the projection and comes back. The transforms are the
unnormalised discrete Fourier transform and its inverse,

    X[k] = sum_{j=0}^{N-1} x[j] exp(-2 pi i j k / N),
    x[j] = (1/N) sum_{k=0}^{N-1} X[k] exp(+2 pi i j k / N),

taken along every axis of a 3-D grid. They are written out here from that
definition rather than taken from a library:

* a length N with smallest prime factor p < N is split by decimation in time:
  the p interleaved subsequences x[r], x[r + p], ... (r = 0 .. p-1) of length
  m = N / p are transformed (recursively), their k-th outputs are multiplied by
  the twiddle factors exp(-2 pi i r k / N), and output k = q m + s is the
  p-point transform over r of those products,
      X[q m + s] = sum_r exp(-2 pi i r q / p) exp(-2 pi i r s / N) Y_r[s];
* a prime length is the definition itself (an N x N matrix of roots of unity).

Every sub-problem of one level is handled in one vectorised numpy operation,
so the Python recursion depth is the number of prime factors of N.
"""
from __future__ import annotations

import math

import numpy as np


def smallest_factor(n: int) -> int:
    """Smallest prime factor of n >= 2 (n itself when n is prime)."""
    if n % 2 == 0:
        return 2
    f = 3
    while f * f <= n:
        if n % f == 0:
            return f
        f += 2
    return n


def _roots(num, den):
    """exp(-2 pi i num / den) for an integer array num (reduced mod den first, so the angle stays small)."""
    return np.exp(-2j * math.pi * (np.asarray(num) % den) / den)


def dft_last(x):
    """Unnormalised forward DFT along the last axis (any length >= 1)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    p = smallest_factor(n)
    if p == n:   # prime length: X[k] = sum_j x[j] w^(jk)
        j = np.arange(n)
        W = _roots(np.outer(j, j), n)
        return x @ W.T
    m = n // p
    # subsequence r holds x[r + p s], s = 0 .. m-1: reshape (.., m, p) and swap to (.., p, m)
    sub = dft_last(np.swapaxes(x.reshape(x.shape[:-1] + (m, p)), -1, -2))
    r = np.arange(p)
    sub = sub * _roots(np.outer(r, np.arange(m)), n)   # twiddles exp(-2 pi i r s / N)
    Wp = _roots(np.outer(r, r), p)                       # [q, r]: exp(-2 pi i r q / p)
    X = np.matmul(Wp, sub)                               # (.., q, s)
    return X.reshape(x.shape[:-1] + (n,))


def dft(x, axis=-1):
    """Unnormalised forward DFT along one axis."""
    return np.moveaxis(dft_last(np.moveaxis(np.asarray(x), axis, -1)), -1, axis)


def idft(X, axis=-1):
    """Inverse DFT along one axis, divided by the length: conj(DFT(conj X)) / N."""
    X = np.asarray(X, dtype=np.complex128)
    n = X.shape[axis]
    return np.conj(dft(np.conj(X), axis)) / n


def dftn(x, axes=(-3, -2, -1)):
    """Unnormalised forward DFT over the given axes (one axis after the other)."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in axes:
        out = dft(out, ax)
    return out


def idftn(X, axes=(-3, -2, -1)):
    """Inverse of dftn (divided by the product of the lengths)."""
    out = np.asarray(X, dtype=np.complex128)
    for ax in axes:
        out = idft(out, ax)
    return out


def mode_numbers(n: int):
    """Signed mode number of each DFT index: i for i <= n/2 (so +n/2 on an even length's Nyquist index),
    i - n above."""
    i = np.arange(n)
    return np.where(i <= n // 2, i, i - n)
