"""Pins of the oracle's effective stiffness (Sec. 3.1: column a of C^eff is the mean stress of unit load
case a) by properties the variational structure of the discrete problem fixes.

Where Gamma0 C0 is a projector at every frequency (boundary frequencies zeroed, or a lattice without
them), the converged strain minimises the strain energy <eps : C : eps> over E + the discrete compatible
fields, which contain the constants.  Hence, to the solver tolerance:
- C^eff is symmetric (E_i : C^eff : E_j = <eps_i : C : eps_j>);
- Hill's bounds hold in the Loewner order: Reuss <C^-1>^-1 <= C^eff <= Voigt <C>, since eps = E is a
  trial field and the unconstrained minimum over all fields with mean E is the Reuss value;
- the same C^eff comes out of conjugate gradients, which minimise that energy directly.
A dropped engineering-shear factor, a transposed column or a wrong mean would break the first or the
second.
"""
import numpy as np
import pytest

from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import effective_voigt
from paper_1605_05712_gb300 import synth


def _voigt(C, d):
    pairs = el.voigt_pairs(d)
    return np.array([[C[i, j, k, l] for (k, l) in pairs] for (i, j) in pairs])


def _mandel(V, d):
    n_c = len(el.voigt_pairs(d))
    w = np.array([1.0] * d + [np.sqrt(2.0)] * (n_c - d))
    return V * np.outer(w, w)


@pytest.mark.parametrize("M,boundary", [([[16, 4], [0, 8]], "zero"), ([[5, 1], [0, 5]], "literal"),
                                        ([[4, 1, 0], [0, 4, 2], [0, 0, 4]], "zero")])
def test_effective_stiffness_symmetric_and_within_hill_bounds(M, boundary):
    L = Lattice(M)
    d = L.d
    ph = synth.inclusions_phase(L.p, L.m, synth.random_inclusions(11, d, 2, 0.35))
    if np.bincount(ph, minlength=2).min() == 0:
        ph = (np.arange(L.m) % 3 == 0).astype(np.int64)
    S = np.array([el.iso_tensor(1.0, 1.0, d), el.iso_tensor(20.0, 8.0, d)])
    C0 = (10.5, 4.5)
    Ce = effective_voigt(L, ph, S, C0, tol=1e-12, maxit=20000, boundary=boundary)
    assert np.abs(Ce - Ce.T).max() < 1e-9 * np.abs(Ce).max()
    f = np.bincount(ph, minlength=2) / L.m
    Vp = [_voigt(S[p], d) for p in range(2)]
    voigt = f[0] * Vp[0] + f[1] * Vp[1]
    reuss = np.linalg.inv(f[0] * np.linalg.inv(Vp[0]) + f[1] * np.linalg.inv(Vp[1]))
    Cs = 0.5 * (Ce + Ce.T)
    tol = 1e-8 * np.abs(Ce).max()
    assert np.linalg.eigvalsh(_mandel(voigt - Cs, d)).min() > -tol
    assert np.linalg.eigvalsh(_mandel(Cs - reuss, d)).min() > -tol
    # strictly inside for a genuinely heterogeneous medium
    assert np.linalg.eigvalsh(_mandel(voigt - Cs, d)).max() > 1e-3
    assert np.linalg.eigvalsh(_mandel(Cs - reuss, d)).max() > 1e-3
    if boundary == "zero" or d == 2:
        Cg = effective_voigt(L, ph, S, C0, tol=1e-12, maxit=2000, boundary=boundary, scheme="cg")
        assert np.abs(Cg - Ce).max() < 1e-9 * np.abs(Ce).max()
