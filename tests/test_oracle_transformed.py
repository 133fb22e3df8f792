"""Pins of the transformed pattern P_L(M) (Sec. 3.3, Def. 3.3) in the oracle: the pattern point y sits
at x = L y in the cell L [-1/2, 1/2)^d and the Fourier index h stands for the frequency L^{-T} h.

- a scalar cell s I is the unit cube (Gamma0 is homogeneous of degree 0);
- the coordinate transformation of Sec. 3.3 (Milton's Sec. 8.3) holds exactly for the discrete
  scheme: with C = T(C~), C0 = T(C~0) (T the transformation of fourth-order tensors by L^{-1}) and
  E = L^T E~ L, the untransformed scheme with the general-C0 Green operator gives eps = L^T eps~ L at
  every iterate; it shares no transformation code with the L path;
- a laminate on a lattice whose frequencies are all parallel to n is the analytic laminate with the
  physical normal L^{-T} n (its planes n . y = const are (L^{-T} n) . x = const).
"""
import numpy as np
import pytest

from oracle import analytic as an
from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme
from paper_1605_05712_gb300 import synth


def _T(C, Linv):
    """C_mnop = Linv_mi Linv_nj Linv_ok Linv_pl C~_ijkl."""
    return np.einsum('mi,nj,ok,pl,...ijkl->...mnop', Linv, Linv, Linv, Linv, C)


CELLS = {2: np.array([[1.3, 0.4], [-0.2, 0.9]]),
         3: np.array([[1.1, 0.3, -0.2], [0.0, 0.8, 0.25], [0.15, -0.1, 1.2]])}


@pytest.mark.parametrize("M", [[[16, 4], [0, 8]], [[4, 1, 0], [0, 4, 2], [0, 0, 4]]])
def test_scalar_cell_is_the_unit_cube(M):
    L = Lattice(M)
    d = L.d
    incl = synth.random_inclusions(2, d, 2, 0.3)
    ph = synth.inclusions_phase(L.p, L.m, incl)
    S = np.array([el.iso_tensor(1, 1, d), el.iso_tensor(10, 10, d)])
    E = np.eye(d) * 0.7
    E[0, 1] = E[1, 0] = 0.3
    a = basic_scheme(L, ph, S, (5.5, 5.5), E, tol=0.0, maxit=5)
    b = basic_scheme(L, ph, S, (5.5, 5.5), E, tol=0.0, maxit=5, L=3.7 * np.eye(d))
    assert np.abs(a["eps"] - b["eps"]).max() < 1e-13


@pytest.mark.parametrize("M", [[[16, 4], [0, 8]], [[32, 1], [0, 16]], [[4, 1, 0], [0, 4, 2], [0, 0, 4]]])
def test_coordinate_transformation_is_exact(M):
    L = Lattice(M)
    d = L.d
    A = CELLS[d]
    Ai = np.linalg.inv(A)
    incl = synth.random_inclusions(4, d, 3, 0.3)
    ph = synth.inclusions_phase(L.p, L.m, incl)
    St = np.array([el.iso_tensor(1, 1, d), el.iso_tensor(6, 4, d)])
    C0t = el.iso_tensor(3.5, 2.5, d)
    Et = np.eye(d) * 0.5
    Et[0, 1] = Et[1, 0] = 0.2
    tr = basic_scheme(L, ph, St, (3.5, 2.5), Et, tol=0.0, maxit=6, L=A)
    un = basic_scheme(L, ph, _T(St, Ai), None, A.T @ Et @ A, tol=0.0, maxit=6, C0_tensor=_T(C0t, Ai))
    mapped = np.einsum('ai,yab,bj->yij', Ai, un["eps"], Ai)          # L^{-T} eps L^{-1}
    assert np.abs(tr["eps"] - mapped).max() < 1e-12 * np.abs(tr["eps"]).max()
    # stresses transform contravariantly: sigma = L^{-1} sigma~ L^{-T}
    sb = Ai @ tr["sigma_bar"] @ Ai.T
    assert np.abs(un["sigma_bar"] - sb).max() < 1e-12 * np.abs(sb).max()


@pytest.mark.parametrize("M,n_int", [([[64, 192], [0, 1]], [1, 3]), ([[4096, 12288], [0, 1]], [1, 3]),
                                     ([[8, 0, 0], [0, 4, 0], [0, 0, 16]], [0, 0, 1])])
def test_aligned_laminate_in_a_transformed_cell(M, n_int):
    L = Lattice(M)
    d = L.d
    A = CELLS[d]
    ph = synth.laminate_phase(L.p, L.m, n_int)
    assert float(np.mean(ph == 0)) == 0.5
    S = np.array([el.iso_tensor(1, 1, d), el.iso_tensor(10, 10, d)])
    E = np.eye(d) * 0.6
    E[0, -1] = E[-1, 0] = 0.25
    r = basic_scheme(L, ph, S, (5.5, 5.5), E, tol=1e-15, maxit=300, L=A)
    n_phys = np.linalg.inv(A).T @ np.array(n_int, float)
    e1, e2, sb = an.laminate_fields(S[0], S[1], 0.5, n_phys, E)
    ex = np.where(ph[:, None, None] == 0, e1, e2)
    assert np.abs(r["eps"] - ex).max() < 1e-12 * np.abs(ex).max()
    assert np.abs(r["sigma_bar"] - sb).max() < 1e-12 * np.abs(sb).max()
    # the unit-cube normal gives a different laminate: the pin separates the two
    e1u, _, _ = an.laminate_fields(S[0], S[1], 0.5, np.array(n_int, float), E)
    assert np.abs(e1u - e1).max() > 1e-3
