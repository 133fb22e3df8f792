"""Closed-form solutions of Sec. 4 for the oracle's pins.

Test infrastructure only (see ``oracle/__init__``).

Laminate (Sec. 4.1).  Two isotropic layers with unit normal n and volume
fractions f1 + f2 = 1; the strain is constant in each layer.  The system the
paper prints for eps^1, eps^2 is degenerate (its second equation is C^eff
times the first), so the fields come from the interface conditions that
define a laminate: strain compatibility eps^2 - eps^1 = sym(a (x) n), traction
continuity (C^1 eps^1 - C^2 eps^2) n = 0, and the mean f1 eps^1 + f2 eps^2 = E.
With eps^1 = E - f2 sym(a (x) n), eps^2 = E + f1 sym(a (x) n):
    a = (f2 K^1(n) + f1 K^2(n))^{-1} ((C^1 - C^2) : E) n,   K^p_ik = C^p_ijkl n_j n_l.
C^eff : E = f1 C^1 eps^1 + f2 C^2 eps^2.  Milton's formula (Sec. 4.1),
    (S - T)^{-1} = <(S~(x) - T)^{-1}>,  S = s0 (s0 I - C^eff)^{-1},
    T_ijkl = 1/2 (n_i d_jk n_l + n_i d_jl n_k + n_j d_ik n_l + n_j d_il n_k) - n_i n_j n_k n_l,
gives C^eff independently; a test checks both agree.  Operators on symmetric
tensors are inverted in the orthonormal Mandel basis.
"""
from __future__ import annotations

import numpy as np

from . import elasticity as el


def _mandel_basis(d):
    pairs = el.voigt_pairs(d)
    B = []
    for (i, j) in pairs:
        b = np.zeros((d, d))
        if i == j:
            b[i, i] = 1.0
        else:
            b[i, j] = b[j, i] = 1.0 / np.sqrt(2.0)
        B.append(b)
    return np.array(B)


def to_mandel(C):
    """Matrix of a minor-symmetric fourth-order tensor in the orthonormal Mandel basis."""
    d = C.shape[0]
    B = _mandel_basis(d)
    return np.einsum('aij,ijkl,bkl->ab', B, C, B)


def from_mandel(A, d):
    B = _mandel_basis(d)
    return np.einsum('aij,ab,bkl->ijkl', B, A, B)


def laminate_fields(C1, C2, f1, n, E):
    """(eps1, eps2, sigma_bar) of the two-layer laminate by the interface conditions."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    f2 = 1.0 - f1
    K1 = el.acoustic(C1, n)
    K2 = el.acoustic(C2, n)
    rhs = el.ddot(C1 - C2, E) @ n
    a = np.linalg.solve(f2 * K1 + f1 * K2, rhs)
    S = 0.5 * (np.outer(a, n) + np.outer(n, a))
    eps1 = E - f2 * S
    eps2 = E + f1 * S
    sbar = f1 * el.ddot(C1, eps1) + f2 * el.ddot(C2, eps2)
    return eps1, eps2, sbar


def laminate_ceff_milton(C1, C2, f1, n, s0=None):
    """C^eff of the laminate from Milton's formula (Sec. 4.1), as a full tensor."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    d = len(n)
    I = np.eye(d)
    T = 0.5 * (np.einsum('i,jk,l->ijkl', n, I, n) + np.einsum('i,jl,k->ijkl', n, I, n)
               + np.einsum('j,ik,l->ijkl', n, I, n) + np.einsum('j,il,k->ijkl', n, I, n)) \
        - np.einsum('i,j,k,l->ijkl', n, n, n, n)
    A1, A2, Tm = to_mandel(C1), to_mandel(C2), to_mandel(T)
    nm = A1.shape[0]
    if s0 is None:
        s0 = 1.5 * max(np.linalg.eigvalsh(A1).max(), np.linalg.eigvalsh(A2).max())
    Id = np.eye(nm)
    St1 = s0 * np.linalg.inv(s0 * Id - A1)
    St2 = s0 * np.linalg.inv(s0 * Id - A2)
    avg = f1 * np.linalg.inv(St1 - Tm) + (1.0 - f1) * np.linalg.inv(St2 - Tm)
    S = np.linalg.inv(avg) + Tm
    # S = s0 (s0 I - C^eff)^{-1}  =>  C^eff = s0 I - s0 S^{-1}
    Ceff = s0 * Id - s0 * np.linalg.inv(S)
    return from_mandel(Ceff, d)
