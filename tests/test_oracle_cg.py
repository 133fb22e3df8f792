"""Pins of the oracle's conjugate-gradient scheme (Sec. 6 names accelerated schemes as carrying over to
patterns; conjugate gradients on the Lippmann-Schwinger equation in the reference medium's inner
product), against Algorithm 1 and against properties fixed by the mathematics of conjugate gradients:

- the converged solution is Algorithm 1's (boundary frequencies zeroed, where Gamma0 C0 is a projector
  at every frequency, so the discrete solution does not depend on C0) and does not depend on C0;
- finite termination: on a tiny lattice the compatible zero-mean fields have dimension d (m - 1), and
  the residual vanishes (to rounding) after at most that many steps;
- the recurred residual equals the true residual -Gamma0 : sigma(x) of the returned iterate;
- the strain energy 1/2 <C x, x> falls monotonically (the iterates minimise it over growing Krylov
  spaces);
- homogeneous media need one transform; the aligned laminate is exact; high contrast needs far fewer
  iterations than Algorithm 1;
- the iteration stops at the rounding floor instead of amplifying rounding noise.
"""
import numpy as np
import pytest

from oracle import analytic as an
from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme, boundary_mask, conjugate_gradient
from oracle.transform import dft_naive
from paper_1605_05712_gb300 import synth


def _setup(M, k, seed=3):
    L = Lattice(M)
    d = L.d
    ph = synth.inclusions_phase(L.p, L.m, synth.random_inclusions(seed, d, 3, 0.3))
    S = np.array([el.iso_tensor(1, 1, d), el.iso_tensor(k, 0.6 * k, d)])
    E = np.eye(d) * 0.5
    E[0, 1] = E[1, 0] = 0.2
    return L, ph, S, E


def _true_residual(L, ph, S, C0, x):
    """-Gamma0 : (C : x) with mean and boundary frequencies zeroed, written out independently of the
    scheme (naive transform, per-point loops)."""
    d, m = L.d, L.m
    sig = np.array([np.einsum('ijkl,kl->ij', S[ph[y]], x[y]) for y in range(m)])
    sh = dft_naive(L, sig, False)
    bm = boundary_mask(L)
    out = np.zeros_like(sh)
    for k in range(m):
        if np.all(L.h[k] == 0) or bm[k]:
            continue
        out[k] = -el.gamma_iso_apply(L.h[k:k + 1].astype(float), sh[k:k + 1], *C0)[0]
    return dft_naive(L, out, True).real


@pytest.mark.parametrize("M", [[[16, 4], [0, 8]], [[6, 1, 0], [0, 4, 2], [0, 0, 4]]])
def test_converges_to_algorithm_1(M):
    L, ph, S, E = _setup(M, 10.0)
    b = basic_scheme(L, ph, S, (5.5, 3.3), E, tol=1e-13, maxit=5000, boundary='zero')
    c = conjugate_gradient(L, ph, S, (5.5, 3.3), E, tol=1e-13, maxit=500, boundary='zero')
    assert np.abs(b["eps"] - c["eps"]).max() < 1e-11
    assert np.abs(b["sigma_bar"] - c["sigma_bar"]).max() < 1e-10
    assert c["iters"] < b["iters"]


def test_solution_does_not_depend_on_c0():
    L, ph, S, E = _setup([[12, 3], [0, 6]], 30.0)
    a = conjugate_gradient(L, ph, S, (5.0, 3.0), E, tol=1e-13, maxit=500, boundary='zero')
    b = conjugate_gradient(L, ph, S, (0.5, 40.0), E, tol=1e-13, maxit=500, boundary='zero')
    assert np.abs(a["eps"] - b["eps"]).max() < 1e-11


@pytest.mark.parametrize("M", [[[3, 1], [0, 3]], [[5, 2], [0, 1]]])
def test_finite_termination(M):
    # odd lattices: no boundary frequencies; dim of the compatible zero-mean fields = d (m - 1)
    L, ph, S, E = _setup(M, 50.0, seed=7)
    assert not boundary_mask(L).any()
    ph = np.arange(L.m) % 2                        # both phases present whatever the inclusions hit
    dim = L.d * (L.m - 1)
    c = conjugate_gradient(L, ph, S, (2.0, 1.5), E, tol=0.0, maxit=dim + 1)
    h = np.array(c["history"])
    assert h[0] > 1e-2
    assert h[:dim + 1].min() < 1e-12 * h[0]
    # the basic scheme at the same count is nowhere near
    b = basic_scheme(L, ph, S, (2.0, 1.5), E, tol=0.0, maxit=dim + 1)
    assert b["history"][-1] > 1e-6


@pytest.mark.parametrize("k", [1, 3, 6])
def test_recurred_residual_is_true_residual(k):
    L, ph, S, E = _setup([[8, 2], [0, 4]], 20.0)
    c = conjugate_gradient(L, ph, S, (4.0, 2.0), E, tol=0.0, maxit=k + 1, boundary='zero')
    r = _true_residual(L, ph, S, (4.0, 2.0), c["eps"])
    norm0 = np.sqrt(L.m * el.frob2(E))
    assert abs(np.sqrt(el.frob2(r).sum()) / norm0 - c["history"][-1]) < 1e-12


def test_energy_decreases():
    L, ph, S, E = _setup([[8, 2], [0, 4]], 20.0)
    w = []
    for k in range(1, 8):
        x = conjugate_gradient(L, ph, S, (4.0, 2.0), E, tol=0.0, maxit=k, boundary='zero')["eps"]
        w.append(0.5 * sum(np.einsum('ij,ijkl,kl->', x[y], S[ph[y]], x[y]) for y in range(L.m)))
    assert all(w[i + 1] <= w[i] + 1e-12 * abs(w[0]) for i in range(len(w) - 1))
    assert w[-1] < w[0] - 1e-6 * abs(w[0])


def test_homogeneous_one_transform():
    L = Lattice([[9, 3], [0, 3]])
    E = np.array([[0.3, 0.1], [0.1, -0.2]])
    C = el.iso_tensor(3.0, 2.0, 2)
    c = conjugate_gradient(L, np.zeros(L.m, int), np.array([C]), (1.0, 0.5), E, tol=1e-12, maxit=10)
    assert c["iters"] == 1 and c["history"][0] < 1e-14
    assert np.abs(c["eps"] - E).max() < 1e-15


def test_aligned_laminate_exact():
    L = Lattice([[64, 192], [0, 1]])
    ph = synth.laminate_phase(L.p, L.m, [1, 3])
    S = np.array([el.iso_tensor(1, 1, 2), el.iso_tensor(10, 10, 2)])
    E = np.array([[0.7, 0.2], [0.2, -0.3]])
    r = conjugate_gradient(L, ph, S, (5.5, 5.5), E, tol=1e-14, maxit=200, boundary='zero')
    e1, e2, sb = an.laminate_fields(S[0], S[1], 0.5, np.array([1.0, 3.0]), E)
    ex = np.where(ph[:, None, None] == 0, e1, e2)
    assert np.abs(r["eps"] - ex).max() < 1e-12
    assert np.abs(r["sigma_bar"] - sb).max() < 1e-12


def test_fewer_iterations_at_high_contrast():
    k = 100.0
    L, ph, S, E = _setup([[15, 2], [0, 5]], k)
    b = basic_scheme(L, ph, S, ((1 + k) / 2, (1 + 0.6 * k) / 2), E, tol=1e-8, maxit=20000, transform='fast')
    c = conjugate_gradient(L, ph, S, ((1 + k) / 2, (1 + 0.6 * k) / 2), E, tol=1e-8, maxit=2000, transform='fast')
    assert np.abs(b["eps"] - c["eps"]).max() < 1e-5 * np.abs(b["eps"]).max()
    assert c["iters"] < b["iters"] / 4


def test_refusals():
    L, ph, S, E = _setup([[8, 2], [0, 4]], 10.0)
    with pytest.raises(ValueError):
        conjugate_gradient(L, ph, S, (5.5, 5.5), E)                     # boundary frequencies, literal
    with pytest.raises(ValueError):
        conjugate_gradient(L, ph, S, (5.5, 5.5), E, boundary='zero', eps0=np.zeros((L.m, 2, 2)))
    assert basic_scheme(L, ph, S, (5.5, 5.5), E, tol=1e-6, scheme='cg', boundary='zero')["iters"] > 1


def test_stops_at_the_rounding_floor():
    # homogeneous medium, tol = 0: r_0 is rounding noise.  Past the floor the step lengths divide noise
    # by noise (A annihilates the incompatible rounding in r) and the iterate drifts by O(1); the
    # iteration must stop there and keep eps = E to rounding
    L = Lattice([[16, 4], [0, 8]])
    E = np.array([[1.1, 0.1], [0.1, 0.1]])
    S = np.array([el.iso_tensor(1, 1, 2), el.iso_tensor(10, 10, 2)])
    c = conjugate_gradient(L, np.zeros(L.m, int), S, (5.5, 5.5), E, tol=0.0, maxit=20, boundary='zero')
    assert c["iters"] <= 2
    assert np.abs(c["eps"] - E).max() < 1e-14
