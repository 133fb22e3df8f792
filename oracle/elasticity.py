"""Elasticity pieces of the oracle: stiffness tensors, double contraction, Green operator.

Test infrastructure only (see ``oracle/__init__``).  Full tensors, float64.

Sec. 3.1: isotropic stiffness C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)
with major and minor symmetries; the double contraction (A : a)_ij = A_ijkl a_kl;
the symmetric-gradient multiplier grad_sym_k u = (i/2)(k u^T + u k^T) and the
Green operator of the Fourier-form Lippmann-Schwinger equation,
    Gamma0(k) = grad_k (grad_k^H C0 grad_k)^{-1} grad_k^H .
Writing it out: grad_k^H sigma = -i sigma k, grad_k^H C0 grad_k u = K(k) u with
the acoustic tensor K_ik = C0_ijkl k_j k_l, hence
    Gamma0(k) : tau = sym(k (x) K(k)^{-1} tau k).
For isotropic C0 = (lam0, mu0) this has the closed form (xi = k / |k|,
v = tau xi, s = xi . v)
    (Gamma0 : tau)_ij = (xi_i v_j + xi_j v_i) / (2 mu0)
                        - s xi_i xi_j (lam0 + mu0) / (mu0 (lam0 + 2 mu0)).
Both forms are here; a test checks they agree.  In d = 2 everything is the
in-plane (plane strain) restriction of the same formulas.

Voigt convention used at the library boundary: components ordered
(11, 22, 33, 23, 13, 12) in 3-D and (11, 22, 12) in 2-D; stiffness matrices in
Voigt form act on engineering strain (shear entries 2 eps_ij).
"""
from __future__ import annotations

import numpy as np

VOIGT3 = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
VOIGT2 = [(0, 0), (1, 1), (0, 1)]
# rows/columns of the 3-D Voigt matrix that form the plane-strain block
PLANE_IDX = [0, 1, 5]


def voigt_pairs(d):
    return VOIGT3 if d == 3 else VOIGT2


def iso_tensor(lam, mu, d):
    """C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)  (Sec. 3.1)."""
    I = np.eye(d)
    return (lam * np.einsum('ij,kl->ijkl', I, I)
            + mu * (np.einsum('ik,jl->ijkl', I, I) + np.einsum('il,jk->ijkl', I, I)))


def iso_voigt6(lam, mu):
    """6x6 Voigt matrix of the isotropic law (engineering shear)."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2 * mu
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    return C


def voigt6_to_tensor(V, d):
    """Full C_ijkl (d in {2,3}) from a 6x6 Voigt matrix; d = 2 takes the plane-strain block."""
    V = np.asarray(V, dtype=np.float64)
    C = np.zeros((3, 3, 3, 3))
    for a, (i, j) in enumerate(VOIGT3):
        for b, (k, l) in enumerate(VOIGT3):
            for (p, q) in {(i, j), (j, i)}:
                for (r, s) in {(k, l), (l, k)}:
                    C[p, q, r, s] = V[a, b]
    return C[:d, :d, :d, :d].copy()


def tensor_to_voigt6(C):
    """6x6 Voigt matrix of a 3-D stiffness tensor (inverse of voigt6_to_tensor)."""
    V = np.zeros((6, 6))
    for a, (i, j) in enumerate(VOIGT3):
        for b, (k, l) in enumerate(VOIGT3):
            V[a, b] = C[i, j, k, l]
    return V


def ddot(C, eps):
    """(C : eps)_ij = C_ijkl eps_kl; C (..., d,d,d,d) or (d,d,d,d), eps (..., d, d)."""
    return np.einsum('...ijkl,...kl->...ij', C, eps)


def frob2(eps):
    """Squared Frobenius norm over the trailing (d, d) axes (off-diagonals counted twice)."""
    return np.einsum('...ij,...ij->...', eps, eps).real if not np.iscomplexobj(eps) else \
        np.einsum('...ij,...ij->...', eps, np.conj(eps)).real


def sym_to_comps(eps):
    """(..., d, d) symmetric tensors -> (..., n_c) components in Voigt order (tensor, not engineering)."""
    d = eps.shape[-1]
    return np.stack([eps[..., i, j] for (i, j) in voigt_pairs(d)], axis=-1)


def comps_to_sym(c, d):
    """(..., n_c) tensor components -> (..., d, d) symmetric tensors."""
    c = np.asarray(c)
    out = np.zeros(c.shape[:-1] + (d, d), dtype=c.dtype)
    for a, (i, j) in enumerate(voigt_pairs(d)):
        out[..., i, j] = c[..., a]
        out[..., j, i] = c[..., a]
    return out


# ---------------------------------------------------------------- Green operator
def gamma_iso_apply(k, tau, lam0, mu0):
    """Gamma0(k) : tau for isotropic C0, closed form; k (..., d) nonzero real, tau (..., d, d)."""
    k = np.asarray(k, dtype=np.float64)
    xi = k / np.linalg.norm(k, axis=-1, keepdims=True)
    v = np.einsum('...ij,...j->...i', tau, xi)
    s = np.einsum('...i,...i->...', xi, v)
    c = (lam0 + mu0) / (mu0 * (lam0 + 2 * mu0))
    out = (np.einsum('...i,...j->...ij', xi, v) + np.einsum('...j,...i->...ij', xi, v)) / (2 * mu0)
    out = out - c * s[..., None, None] * np.einsum('...i,...j->...ij', xi, xi)
    return out


def acoustic(C0, k):
    """K_ik = C0_ijkl k_j k_l."""
    return np.einsum('ijkl,...j,...l->...ik', C0, k, k)


def gamma_tensor(C0, k):
    """Full fourth-order Gamma0(k)_ijkl from the operator definition (any C0, one k).

    Gamma0 : tau = sym(k (x) K^{-1} tau k), i.e. Gamma_ijkl =
    1/4 (k_i G_jk k_l + k_i G_jl k_k + k_j G_ik k_l + k_j G_il k_k), G = K^{-1}.
    """
    k = np.asarray(k, dtype=np.float64)
    G = np.linalg.inv(acoustic(C0, k))
    return 0.25 * (np.einsum('i,jk,l->ijkl', k, G, k) + np.einsum('i,jl,k->ijkl', k, G, k)
                   + np.einsum('j,ik,l->ijkl', k, G, k) + np.einsum('j,il,k->ijkl', k, G, k))


def gamma_general_apply(C0, k, tau):
    """Gamma0(k) : tau = sym(k (x) K(k)^{-1} tau k) for a general C0 (batched over k)."""
    k = np.asarray(k, dtype=np.float64)
    K = acoustic(C0, k)
    w = np.linalg.solve(K, np.einsum('...ij,...j->...i', tau, k)[..., None])[..., 0]
    a = np.einsum('...i,...j->...ij', k, w)
    return 0.5 * (a + np.swapaxes(a, -1, -2))
