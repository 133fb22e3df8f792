"""Fourier transform on a pattern, F(M), for the oracle.

Test infrastructure only (see ``oracle/__init__``).

Sec. 2.2, Eq. (Fouriermatrix): F(M) = (1/m) (exp(-2 pi i h^T y)), rows
h in G(M^T), columns y in P(M).  The forward transform carries the 1/m, the
inverse (F(M)^{-1} = m F(M)^H) carries none.

Two evaluations:
  * ``dft_naive`` is the definition written out: an m x m sum with the exact
    integer phase index (h^T (m y)) mod m into a table of the m-th roots of
    unity.  O(m^2); used for m up to a few thousand.
  * ``dft_fast`` is the paper's statement that, with the lexicographic
    orderings of lambda and k, F(M) is an ordinary d_M-dimensional DFT over
    the elementary-divisor box (Sec. 2.2, last paragraph; Theorem 2 of the
    cited FFT paper).  It calls numpy.fft.fftn as a library step.
Both act on arrays whose first axis runs over the m points (plan order of
``oracle.lattice.Lattice``); trailing axes are batched.
"""
from __future__ import annotations

import numpy as np


def _roots(m):
    j = np.arange(m, dtype=np.float64)
    return np.exp(-2j * np.pi * j / m)


def phase_index(lat):
    """(m x m) integer matrix P[h, y] = (h^T (m y)) mod m."""
    H = np.asarray(lat.h, dtype=object)
    Pn = np.asarray(lat.p, dtype=object)
    P = (H @ Pn.T) % lat.m
    return P.astype(np.int64)


def dft_naive(lat, a, inverse=False):
    """F(M) a (forward, with 1/m) or F(M)^{-1} a (inverse), by the definition."""
    m = lat.m
    P = phase_index(lat)
    w = _roots(m)
    if inverse:
        W = np.conj(w[P]).T          # columns h, rows y: exp(+2 pi i h^T y)
        return np.tensordot(W, a, axes=(1, 0))
    W = w[P]                          # rows h, columns y
    return np.tensordot(W, a, axes=(1, 0)) / m


def dft_fast(lat, a, inverse=False):
    """Same transform as ``dft_naive`` through the d_M-dimensional FFT over the divisor box."""
    a = np.asarray(a)
    m = lat.m
    tail = a.shape[1:]
    if lat.d_M == 0:
        return a.astype(np.complex128).copy()
    box = a.reshape(lat.shape + tail)
    axes = tuple(range(lat.d_M))
    if inverse:
        out = np.fft.ifftn(box, axes=axes) * m
    else:
        out = np.fft.fftn(box, axes=axes) / m
    return out.reshape((m,) + tail)
