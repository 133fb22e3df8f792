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


# ------------------------------------------------------------------ generalized Hashin structure
"""Coated confocal ellipsoid (Sec. 4.2, after Milton's neutral coated ellipsoid).

Geometry: x~ = R^{-1} x; the ellipsoidal radius rho(x~) is the largest root of
sum_i x~_i^2 / (c_i^2 + rho) = 1; core rho <= rho_c, coating rho_c < rho <= rho_e,
matrix outside.  Semi-axes l_j(rho) = sqrt(c_j^2 + rho); c_3 = inf is the
elliptic cylinder (2-D problem run in 3-D).

Readings of garbled passages (listed in the design notes):
  * depolarization factors: the general ellipsoid uses the depolarization integral
        d_i(rho) = (l1 l2 l3 / 2) int_0^inf ds / ((l_i^2 + s) sqrt(prod_j (l_j^2 + s)))
    (sum_i d_i = 1); the paper's prolate/oblate formulas are special cases once the
    garbles are fixed (prolate d3 carries a "-1", d1 = d2 = (1 - d3)/2; oblate
    d2 = d3 = (1 - d1)/2); the cylinder formulas are used as printed;
  * grad rho: (grad rho)_i = (2 x~_i / (c_i^2 + rho)) / sum_j x~_j^2 / (c_j^2 + rho)^2,
    from implicit differentiation of the defining equation;
  * the rotation R takes e_1 to n (Rodrigues), or is given directly.
"""


def depolarization(c, rho):
    """d_i(rho) for semi-axes c (c_3 may be inf: elliptic cylinder)."""
    from scipy.integrate import quad
    c = np.asarray(c, dtype=np.float64)
    if not np.isfinite(c[2]):
        l1, l2 = np.sqrt(c[0] ** 2 + rho), np.sqrt(c[1] ** 2 + rho)
        return np.array([l2 / (l1 + l2), l1 / (l1 + l2), 0.0])
    l2 = c ** 2 + rho
    pref = np.sqrt(np.prod(l2)) / 2.0
    out = []
    for i in range(3):
        f = lambda s, i=i: 1.0 / ((l2[i] + s) * np.sqrt((l2[0] + s) * (l2[1] + s) * (l2[2] + s)))
        # substitute s = t / (1 - t) to map [0, inf) onto [0, 1)
        g = lambda t, f=f: f(t / (1.0 - t)) / (1.0 - t) ** 2
        val, _ = quad(g, 0.0, 1.0, epsabs=0.0, epsrel=1e-13, limit=400)
        out.append(pref * val)
    return np.array(out)


def g_of(c, rho):
    c = np.asarray(c, dtype=np.float64)
    fin = np.isfinite(c)
    return np.prod(c[fin] ** 2 + rho)


def ellipsoidal_radius(c, xt):
    """Largest root rho of sum_i xt_i^2 / (c_i^2 + rho) = 1 (rows of xt), bisection then Newton."""
    c = np.asarray(c, dtype=np.float64)
    xt = np.atleast_2d(np.asarray(xt, dtype=np.float64))
    fin = np.isfinite(c)
    cc = c[fin] ** 2
    x2 = xt[:, fin] ** 2
    F = lambda r: np.sum(x2 / (cc + r[:, None]), axis=1) - 1.0
    lo = np.full(len(xt), -cc.min() + 1e-300)
    hi = np.full(len(xt), 1.0)
    while np.any(F(hi) > 0):
        hi = np.where(F(hi) > 0, 2 * hi + 1.0, hi)
    for _ in range(200):      # F decreases on (-c_min^2, inf)
        mid = 0.5 * (lo + hi)
        pos = F(mid) > 0
        lo = np.where(pos, mid, lo)
        hi = np.where(pos, hi, mid)
    r = 0.5 * (lo + hi)
    for _ in range(3):
        dF = -np.sum(x2 / (cc + r[:, None]) ** 2, axis=1)
        r = r - F(r) / dF
    return r


def rotation_to(n):
    """Rotation taking e_1 to the unit vector n (Rodrigues form of the matrix of Sec. 4.2)."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    if np.allclose(n, [1, 0, 0]):
        return np.eye(3)
    if np.allclose(n, [-1, 0, 0]):
        return np.diag([-1.0, -1.0, 1.0])
    K = np.array([[0, -n[1], -n[2]], [n[1], 0, 0], [n[2], 0, 0]])
    return np.eye(3) + K + K @ K / (1.0 + n[0])


class Hashin:
    """Neutral coated ellipsoid: eps0, C^eff eps0 and the strain field (Sec. 4.2).

    c: (c1, c2, c3) with c3 = inf for the cylinder; rho_c < rho_e; core (lam_c, mu_c) and
    coating (lam_e, mu_e) isotropic; R rotation (x = R x~).
    """

    def __init__(self, c, rho_c, rho_e, lam_c, mu_c, lam_e, mu_e, R=None):
        self.c = np.asarray(c, dtype=np.float64)
        self.rho_c, self.rho_e = float(rho_c), float(rho_e)
        self.R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
        self.kc, self.ke = lam_c + 2.0 * mu_c / 3.0, lam_e + 2.0 * mu_e / 3.0
        self.mu_e = mu_e
        self.Cc = el.iso_tensor(lam_c, mu_c, 3)
        self.Ce = el.iso_tensor(lam_e, mu_e, 3)
        self.Dc = np.diag(depolarization(self.c, self.rho_c))
        self.fe = self.f(self.rho_e)
        self.alpha = (3 * self.ke + 4 * self.mu_e) / (9 * (self.kc - self.ke))
        Se = self.S(self.rho_e)
        R = self.R
        self.eps0 = R @ (self.alpha * np.eye(3) + (1 - self.fe) * Se) @ R.T
        a = self.ke / (self.kc - self.ke) * (self.kc + 4.0 / 3.0 * mu_e) + 4.0 / 3.0 * mu_e * self.fe
        self.ceff_eps0 = R @ (a * np.eye(3)) @ R.T + R @ (2.0 / 3.0 * mu_e * (1 - self.fe) * (3 * Se - np.eye(3))) @ R.T

    def f(self, rho):
        return np.sqrt(g_of(self.c, self.rho_c)) / np.sqrt(g_of(self.c, rho))

    def S(self, rho):
        f = self.f(rho)
        return (self.Dc - f * np.diag(depolarization(self.c, rho))) / (1.0 - f)

    def region(self, x):
        """0 core, 1 coating, 2 matrix for points x (rows, cell coordinates centred at the inclusion)."""
        xt = np.atleast_2d(x) @ self.R  # rows of R^T x
        rho = ellipsoidal_radius(self.c, xt)
        return np.where(rho <= self.rho_c, 0, np.where(rho <= self.rho_e, 1, 2)), rho, xt

    def strain(self, x):
        """Analytic strain field at points x (rows)."""
        reg, rho, xt = self.region(x)
        n = len(reg)
        out = np.empty((n, 3, 3))
        out[reg == 2] = self.eps0
        out[reg == 0] = self.R @ (self.alpha * np.eye(3)) @ self.R.T
        idx = np.nonzero(reg == 1)[0]
        c = self.c
        fin = np.isfinite(c)
        cc = np.where(fin, c, 0.0) ** 2
        sgc = np.sqrt(g_of(c, self.rho_c))
        for i in idx:
            r = rho[i]
            x_ = xt[i]
            den = cc + r
            q = np.where(fin, x_ / den, 0.0) / np.sqrt(g_of(c, r))
            grad = np.where(fin, 2 * x_ / den, 0.0) / np.sum(np.where(fin, x_ ** 2 / den ** 2, 0.0))
            Dr = np.diag(depolarization(c, r))
            loc = self.alpha * np.eye(3) + self.Dc - self.f(r) * Dr + 0.5 * sgc * np.outer(q, grad)
            out[i] = self.R @ loc @ self.R.T
        return out
