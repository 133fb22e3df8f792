"""Pins of the oracle's Eyre-Milton iteration (an accelerated scheme of the kind Sec. 6 says carries
over to patterns), against Algorithm 1:

- with the same reference medium both converge to the same discrete solution, also on lattices with
  even divisors (where the averaged boundary Green operator makes the discrete solution depend on C0);
- on lattices without boundary frequencies the discrete solution does not depend on C0, so the
  Eyre-Milton iteration at its own reference (geometric mean of the extremes) reproduces Algorithm 1
  at the arithmetic mean;
- it needs far fewer iterations at high contrast (rate (sqrt(k) - 1) / (sqrt(k) + 1) against
  (k - 1) / (k + 1));
- the aligned laminate is exact, as for Algorithm 1.
"""
import numpy as np
import pytest

from oracle import analytic as an
from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme
from paper_1605_05712_gb300 import synth


def _setup(M, k):
    L = Lattice(M)
    d = L.d
    ph = synth.inclusions_phase(L.p, L.m, synth.random_inclusions(3, d, 3, 0.3))
    S = np.array([el.iso_tensor(1, 1, d), el.iso_tensor(k, k, d)])
    E = np.eye(d) * 0.5
    E[0, 1] = E[1, 0] = 0.2
    return L, ph, S, E


@pytest.mark.parametrize("M", [[[32, 4], [0, 16]], [[8, 1, 0], [0, 8, 1], [0, 0, 8]]])
def test_same_fixed_point_as_algorithm_1(M):
    L, ph, S, E = _setup(M, 10.0)
    b = basic_scheme(L, ph, S, (5.5, 5.5), E, tol=1e-13, maxit=5000, transform='fast')
    em = basic_scheme(L, ph, S, (5.5, 5.5), E, tol=1e-13, maxit=5000, scheme='eyre_milton', transform='fast')
    assert np.abs(b["eps"] - em["eps"]).max() < 1e-11
    assert np.abs(b["sigma_bar"] - em["sigma_bar"]).max() < 1e-10


@pytest.mark.parametrize("M", [[[15, 2], [0, 5]], [[5, 1, 0], [0, 5, 0], [0, 0, 5]]])
def test_fewer_iterations_at_high_contrast(M):
    k = 100.0
    L, ph, S, E = _setup(M, k)
    b = basic_scheme(L, ph, S, ((1 + k) / 2, (1 + k) / 2), E, tol=1e-9, maxit=20000, transform='fast')
    g = np.sqrt(k)
    em = basic_scheme(L, ph, S, (g, g), E, tol=1e-9, maxit=20000, scheme='eyre_milton', transform='fast')
    assert np.abs(b["eps"] - em["eps"]).max() < 1e-6 * np.abs(b["eps"]).max()   # C0-independent here
    assert em["iters"] < b["iters"] / 4


def test_aligned_laminate_exact():
    L = Lattice([[64, 192], [0, 1]])
    ph = synth.laminate_phase(L.p, L.m, [1, 3])
    S = np.array([el.iso_tensor(1, 1, 2), el.iso_tensor(10, 10, 2)])
    E = np.array([[0.7, 0.2], [0.2, -0.3]])
    r = basic_scheme(L, ph, S, (np.sqrt(10), np.sqrt(10)), E, tol=1e-15, maxit=500, scheme='eyre_milton')
    e1, e2, sb = an.laminate_fields(S[0], S[1], 0.5, np.array([1.0, 3.0]), E)
    ex = np.where(ph[:, None, None] == 0, e1, e2)
    assert np.abs(r["eps"] - ex).max() < 1e-12 * np.abs(ex).max()


def test_zero_boundary_is_refused():
    L, ph, S, E = _setup([[8, 2], [0, 8]], 10.0)
    with pytest.raises(ValueError):
        basic_scheme(L, ph, S, (5.5, 5.5), E, maxit=2, scheme='eyre_milton', boundary='zero')
