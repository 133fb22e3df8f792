"""Pin of the oracle's Cauchy residual (Sec. 5.2 stopping rule, Algorithm 1 of Sec. 3.2) by hand algebra.

The measure is r_n = ||eps^(n+1) - eps^(n)|| / (sqrt(m) ||E||_F): the l2 norm over the m pattern points of
the Frobenius norm of the full symmetric tensor (so every off-diagonal entry counts twice), normalised by
the norm of the cold start eps^(0) = E.  Nothing here calls the oracle's norm or Green-operator helpers:
the expected values come from the algebra of a two-point pattern, written out in scalars.

Two-point pattern.  M = diag(2, 1) in 2-D (diag(2, 1, 1) in 3-D) has the points y = 0 and y = (-1/2, 0[, 0])
and the frequencies h = 0 and h = (-1, 0[, 0]) (Sec. 2.1).  Put phase A at y = 0 and phase B at the other
point.  One iteration from eps^(0) = E:
  * the polarization difference is Delta = tau_0 - tau_1 = (C_A - C_B) : E (the C0 terms cancel);
  * F(M) gives tau_hat at h = (-1, 0) equal to Delta / 2 (the exponential is +1 at y = 0 and -1 at the
    other point);
  * along the unit direction e1 the Green operator of an isotropic C0 maps a symmetric tau to the strain
    with (11) = tau_11 / (lam0 + 2 mu0), (1j) = tau_1j / (2 mu0) for j != 1 and zero elsewhere (the
    laminate solution: a compatible strain varying along x1 only, whose traction C0 : eps e1 balances
    tau e1);
  * the inverse transform adds that spectral value with sign +1 at y = 0 and -1 at the other point.
So eps^(1) = E + s delta with s = +1, -1 at the two points and delta = -Gamma0(e1) : Delta / 2, hence
    r_0 = sqrt(2 |delta|_F^2) / (sqrt(2) |E|_F) = |delta|_F / |E|_F.
The second iteration is the same algebra with Delta' = (C_A - C_B) : E + (C_A + C_B - 2 C0) : delta, giving
delta' and r_1 = |delta' - delta|_F / |E|_F.  A dropped sqrt(m), a shear entry counted once, or a
transposed shear term changes these numbers, so the oracle's history must reproduce them exactly.
"""
import itertools

import numpy as np
import pytest

from oracle.lattice import Lattice
from oracle.scheme import basic_scheme


def iso_ddot(lam, mu, e):
    """(C : e) of an isotropic law on a full symmetric tensor, written out entry by entry."""
    d = e.shape[0]
    tr = sum(e[i, i] for i in range(d))
    out = np.zeros_like(e)
    for i, j in itertools.product(range(d), range(d)):
        out[i, j] = 2.0 * mu * e[i, j] + (lam * tr if i == j else 0.0)
    return out


def gamma_e1(tau, lam0, mu0):
    """Gamma0 at the direction e1 (the laminate closed form stated in the module docstring)."""
    d = tau.shape[0]
    out = np.zeros_like(tau)
    out[0, 0] = tau[0, 0] / (lam0 + 2.0 * mu0)
    for j in range(1, d):
        out[0, j] = out[j, 0] = tau[0, j] / (2.0 * mu0)
    return out


def frob_sq_by_entries(a):
    """Sum of the squares of all d*d entries (an off-diagonal value appears at (i, j) and (j, i))."""
    d = a.shape[0]
    return sum(a[i, j] ** 2 for i in range(d) for j in range(d))


def expected_two_point(E, A, B, C0):
    lam0, mu0 = C0
    CA = lambda e: iso_ddot(A[0], A[1], e)
    CB = lambda e: iso_ddot(B[0], B[1], e)
    C0m = lambda e: iso_ddot(lam0, mu0, e)
    nE = np.sqrt(frob_sq_by_entries(E))
    delta = -0.5 * gamma_e1(CA(E) - CB(E), lam0, mu0)
    r0 = np.sqrt(frob_sq_by_entries(delta)) / nE
    Delta2 = CA(E) - CB(E) + CA(delta) + CB(delta) - 2.0 * C0m(delta)
    delta2 = -0.5 * gamma_e1(Delta2, lam0, mu0)
    r1 = np.sqrt(frob_sq_by_entries(delta2 - delta)) / nE
    return r0, r1, delta, delta2


def stiff_iso(lam, mu, d):
    C = np.zeros((d, d, d, d))
    for i, j, k, l in itertools.product(range(d), repeat=4):
        C[i, j, k, l] = lam * (i == j) * (k == l) + mu * ((i == k) * (j == l) + (i == l) * (j == k))
    return C


LOADS2 = [np.array([[0.0, 0.5], [0.5, 0.0]]),          # pure shear: only the doubly counted entries
          np.array([[1.0, 0.0], [0.0, 0.0]]),
          np.array([[0.3, -0.7], [-0.7, 0.2]])]
LOADS3 = [np.array([[0.0, 0.5, 0.0], [0.5, 0.0, 0.0], [0.0, 0.0, 0.0]]),
          np.array([[0.0, 0.0, 0.25], [0.0, 0.0, 0.0], [0.25, 0.0, 0.0]]),
          np.array([[0.4, 0.1, -0.3], [0.1, -0.2, 0.6], [-0.3, 0.6, 0.5]])]


@pytest.mark.parametrize("d,E", [(2, E) for E in LOADS2] + [(3, E) for E in LOADS3])
def test_two_point_residuals_by_hand(d, E):
    M = np.diag([2] + [1] * (d - 1)).tolist()
    L = Lattice(M)
    assert L.m == 2
    # phase A (index 0) at y = 0, phase B (index 1) at y = (-1/2, 0, ...)
    phase = np.array([0 if not np.any(p) else 1 for p in L.p.tolist()])
    assert sorted(phase.tolist()) == [0, 1]
    A, B, C0 = (1.0, 1.0), (10.0, 7.0), (5.0, 5.0)
    stiff = np.array([stiff_iso(*A, d), stiff_iso(*B, d)])
    r = basic_scheme(L, phase, stiff, C0, E, tol=0.0, maxit=2)
    r0, r1, delta, delta2 = expected_two_point(E, A, B, C0)
    assert r0 > 1e-3 and r1 > 1e-4
    assert abs(r["history"][0] - r0) <= 1e-14 * r0
    assert abs(r["history"][1] - r1) <= 1e-13 * r1
    # the fields themselves: E + delta2 at y = 0, E - delta2 at the other point
    i0 = int(np.flatnonzero(phase == 0)[0])
    i1 = 1 - i0
    assert np.abs(r["eps"][i0] - (E + delta2)).max() <= 1e-14
    assert np.abs(r["eps"][i1] - (E - delta2)).max() <= 1e-14


def test_single_counted_shear_would_differ():
    # the pinned numbers separate the double-counted Frobenius norm from a once-counted one: for a load
    # with normal and shear parts the two readings differ by far more than the tolerances above
    E = LOADS2[2]
    r0, _, delta, _ = expected_two_point(E, (1.0, 1.0), (10.0, 7.0), (5.0, 5.0))
    once = np.sqrt(delta[0, 0] ** 2 + delta[0, 1] ** 2) / np.sqrt(E[0, 0] ** 2 + E[1, 1] ** 2 + E[0, 1] ** 2)
    assert abs(once - r0) > 1e-3 * r0
