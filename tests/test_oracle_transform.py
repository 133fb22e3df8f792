"""Pins of oracle.transform: the Fourier matrix F(M) of Sec. 2.2."""
import numpy as np
import pytest

from oracle.lattice import Lattice
from oracle.transform import dft_fast, dft_naive

RNG = np.random.default_rng(11)
MATS = [[[8, -4], [2, 7]], [[4, 4], [-4, 4]], [[3, 0], [0, 4]], [[6, 2], [0, 10]], [[2, 1, 0], [0, 3, 1], [1, 0, 4]],
        [[4, 1, 0], [0, 4, 2], [2, 0, 4]], [[16, 0], [4, 8]], [[5, 0], [0, 5]]]


@pytest.mark.parametrize("M", MATS)
def test_naive_equals_separable(M):
    L = Lattice(M)
    a = RNG.standard_normal((L.m, 2)) + 1j * RNG.standard_normal((L.m, 2))
    ref = dft_naive(L, a)
    assert np.abs(dft_fast(L, a) - ref).max() < 1e-13 * max(1.0, np.abs(ref).max())
    inv = dft_naive(L, ref, inverse=True)
    assert np.abs(inv - a).max() < 1e-12                          # F^{-1} F = I
    # Parseval: ||a||^2 = m ||F a||^2
    assert abs(np.sum(abs(a) ** 2) - L.m * np.sum(abs(ref) ** 2)) < 1e-10 * np.sum(abs(a) ** 2)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_diagonal_is_usual_2d_dft(n):
    # Sec. 2.2: for M = diag(n, n) the transform is the usual 2-D DFT (1/m normalization)
    L = Lattice([[n, 0], [0, n]])
    grid = RNG.standard_normal((n, n)) + 1j * RNG.standard_normal((n, n))
    a = grid[L.p[:, 0] // n % n, L.p[:, 1] // n % n]          # y = p/m = (j1/n, j2/n)
    ah = dft_naive(L, a)
    ref = np.fft.fft2(grid) / n ** 2
    assert np.abs(ah - ref[L.h[:, 0] % n, L.h[:, 1] % n]).max() < 1e-13


@pytest.mark.parametrize("M", MATS)
def test_aliasing_lemma(M):
    # Lemma 2.1: sampling exp(i k^T x) at x = 2 pi y gives c^M_h = 1 iff h = k mod M^T, else 0
    L = Lattice(M)
    MT = np.array(M).T
    H = L.h
    for _ in range(5):
        k = RNG.integers(-20, 21, size=L.d)
        a = np.exp(2j * np.pi * (L.p @ k) / L.m)
        c = dft_naive(L, a)
        # which h is congruent to k modulo M^T Z^d: M^{-T}(h - k) integral
        diff = (H - k).astype(float) @ np.linalg.inv(MT).T
        cong = np.all(np.abs(diff - np.round(diff)) < 1e-9, axis=1)
        assert cong.sum() == 1
        assert abs(c[cong][0] - 1) < 1e-12 and np.abs(c[~cong]).max() < 1e-12


@pytest.mark.parametrize("M", MATS)
def test_phase_index_is_the_divisor_box_product(M):
    # Sec. 2.2: with y(lambda) = R^{-1} E^{-1} lambda and h(k) = R^T k (mod the lattices),
    # h(k)^T y(lambda) = sum_j k_j lambda_j / e_j (mod 1), so the exact phase index of F(M) is
    # m sum_j k_j lambda_j / e_j mod m; k and lambda run over the same box in the same order, so the
    # phase matrix is symmetric (F(M) of the plan orderings equals its transpose)
    from oracle.transform import phase_index
    L = Lattice(M)
    lam = np.asarray(L.lam, dtype=np.int64)
    scale = np.array([L.m // e for e in L.e], dtype=np.int64)
    ref = ((lam * scale) @ lam.T) % L.m
    P = phase_index(L)
    assert np.array_equal(P, ref)
    assert np.array_equal(P, P.T)
