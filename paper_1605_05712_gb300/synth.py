"""Seeded synthetic inputs for the lattice Basic Scheme: geometries, phases, materials, lattices.

This module serves both the CUDA path and the CPU oracle and holds none of the
method's arithmetic (no transform, no Green operator, no iteration).  Phases
are decided from the exact integer numerators p = m y of the pattern points
that each side enumerates on its own, so both sides label every point alike.

Workloads (shaped like the paper's examples, Sec. 4 and 5):
  * laminate: two isotropic layers with rational normal n_int (Sec. 4.1),
    phase 0 where frac(n_int . y) < f1;
  * coated ellipsoid (Sec. 4.2): core / coating / matrix by the confocal
    ellipsoid inequalities, optionally rotated;
  * random ellipsoidal inclusions in a matrix, periodic, seeded.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

BASE_SEED = 20160621


def iso_voigt(lam, mu):
    """6x6 Voigt stiffness (engineering shear) of an isotropic material with Lame constants (lam, mu)."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] = lam + 2 * mu
        C[i + 3, i + 3] = mu
    return C


def c0_mean_extremes(lams, mus):
    """Reference medium: arithmetic mean of the extreme Lame constants of the phases."""
    return (0.5 * (min(lams) + max(lams)), 0.5 * (min(mus) + max(mus)))


def laminate_phase(p, m, n_int, f1=Fraction(1, 2)):
    """Phase 0 where frac(n_int . y) in [0, f1), else 1; y = p / m, exact integer test."""
    p = np.asarray(p, dtype=np.int64)
    f1 = Fraction(f1)
    t = (p @ np.asarray(n_int, dtype=np.int64)) % m
    return np.where(t * f1.denominator < f1.numerator * m, 0, 1).astype(np.uint8)


def euler_zyz(a, b, c):
    """Rotation matrix R = Rz(a) Ry(b) Rz(c)."""
    def rz(t):
        return np.array([[np.cos(t), -np.sin(t), 0], [np.sin(t), np.cos(t), 0], [0, 0, 1.0]])

    def ry(t):
        return np.array([[np.cos(t), 0, np.sin(t)], [0, 1.0, 0], [-np.sin(t), 0, np.cos(t)]])
    return rz(a) @ ry(b) @ rz(c)


def coated_ellipsoid_phase(p, m, c, rho_c, rho_e, R=None, center=None):
    """0 = core (rho <= rho_c), 1 = coating (rho_c < rho <= rho_e), 2 = matrix.

    rho(x) <= rho_0  iff  sum_i x~_i^2 / (c_i^2 + rho_0) <= 1 (the left side
    decreases in rho), x~ = R^T (y - center) taken with the minimum-image
    convention on the unit torus.  c_i = inf (2-D cylinder) drops the term.
    """
    p = np.asarray(p, dtype=np.int64)
    d = p.shape[1]
    y = p.astype(np.float64) / m
    if center is not None:
        y = y - np.asarray(center)[:d]
        y -= np.round(y)
    if d == 2:
        y = np.concatenate([y, np.zeros((y.shape[0], 1))], axis=1)
    R = np.eye(3) if R is None else np.asarray(R)
    xt = y @ R  # rows: (R^T y)^T
    c = np.asarray(c, dtype=np.float64)

    def inside(rho0):
        s = np.zeros(len(xt))
        for i in range(3):
            if np.isfinite(c[i]):
                s += xt[:, i] ** 2 / (c[i] ** 2 + rho0)
        return s <= 1.0
    ph = np.full(len(xt), 2, dtype=np.uint8)
    ph[inside(rho_e)] = 1
    ph[inside(rho_c)] = 0
    return ph


def random_inclusions(seed, d, n_incl, vol_frac):
    """Seeded ellipsoidal inclusions: centres, semi-axes, rotations (d = 2 or 3)."""
    rng = np.random.default_rng(seed)
    cen = rng.random((n_incl, d))
    aspect = rng.uniform(1.0, 3.0, size=(n_incl, d))
    if d == 2:
        unit_vol = np.pi * np.prod(aspect, axis=1)
    else:
        unit_vol = 4.0 / 3.0 * np.pi * np.prod(aspect, axis=1)
    scale = (vol_frac / unit_vol.sum()) ** (1.0 / d)
    axes = np.minimum(aspect * scale, 0.45)
    rots = []
    for _ in range(n_incl):
        if d == 2:
            t = rng.uniform(0, np.pi)
            rots.append(np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]]))
        else:
            rots.append(euler_zyz(*rng.uniform(0, 2 * np.pi, 3)))
    return dict(centers=cen, axes=axes, rots=np.array(rots))


def inclusions_phase(p, m, incl):
    """1 inside any inclusion (periodic minimum image), else 0."""
    p = np.asarray(p, dtype=np.int64)
    y = p.astype(np.float64) / m
    ph = np.zeros(len(y), dtype=np.uint8)
    for c, a, R in zip(incl["centers"], incl["axes"], incl["rots"]):
        z = y - c
        z -= np.round(z)
        zt = z @ R
        ph[np.sum((zt / a) ** 2, axis=1) <= 1.0] = 1
    return ph


# lattices of the paper's experiments and of the benchmark workloads
def shear_matrix(j, k, alpha):
    """M_{j,k,alpha} of Sec. 5.1 (Eq. M-shear), restricted to the first two axes."""
    return [[2 ** j, alpha * k], [(1 - alpha) * k, 2 ** (14 - j)]]


LATTICES = {
    # 2-D, m = 4096: aligned rank-1 lattice (every frequency parallel to (1,3)) and a spread one
    "laminate4096_aligned": [[4096, 12288], [0, 1]],
    "laminate4096_rank1": [[64, 1], [0, 64]],
    # 2-D, m = 262144: tensor grid, rank-1, sheared rank-2
    "grid512": [[512, 0], [0, 512]],
    "rank1_262144": [[512, 1], [0, 512]],
    "rank2_262144": [[512, 16], [0, 512]],
    # 3-D, m = 2^21
    "grid128": [[128, 0, 0], [0, 128, 0], [0, 0, 128]],
    "sheared128": [[128, 16, 0], [0, 128, 16], [0, 0, 128]],
    "rank1_2097152": [[128, 1, 0], [0, 128, 1], [0, 0, 128]],
}


# ------------------------------------------------------------------ coated-ellipsoid (Hashin) workload
def _depol_carlson(c, rho):
    """Depolarization factors of the ellipsoid with semi-axes sqrt(c_j^2 + rho) by Carlson's R_D
    (d_i = l1 l2 l3 / 3 * R_D(l_j^2, l_k^2, l_i^2)); c_3 = inf gives the elliptic-cylinder factors."""
    from scipy.special import elliprd
    c = np.asarray(c, dtype=np.float64)
    if not np.isfinite(c[2]):
        l1, l2 = np.sqrt(c[0] ** 2 + rho), np.sqrt(c[1] ** 2 + rho)
        return np.array([l2 / (l1 + l2), l1 / (l1 + l2), 0.0])
    q = c ** 2 + rho
    pref = np.sqrt(np.prod(q)) / 3.0
    return np.array([pref * elliprd(q[(i + 1) % 3], q[(i + 2) % 3], q[i]) for i in range(3)])


def iso_tensor3(lam, mu):
    I = np.eye(3)
    return (lam * np.einsum('ij,kl->ijkl', I, I)
            + mu * (np.einsum('ik,jl->ijkl', I, I) + np.einsum('il,jk->ijkl', I, I)))


def tensor_to_voigt(C):
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    V = np.zeros((6, 6))
    for a, (i, j) in enumerate(pairs):
        for b, (k, l) in enumerate(pairs):
            V[a, b] = C[i, j, k, l]
    return V


def iso_projection(V):
    """(lam, mu) of the isotropic projection of a 6x6 Voigt stiffness."""
    kappa = V[:3, :3].sum() / 9.0
    mu = (V[0, 0] + V[1, 1] + V[2, 2] - (V[0, 1] + V[0, 2] + V[1, 2]) + 3 * (V[3, 3] + V[4, 4] + V[5, 5])) / 15.0
    return kappa - 2.0 * mu / 3.0, mu


def hashin_workload(seed=BASE_SEED, c=(0.1, 0.15, 0.2), total_fraction=0.25, core=(10.0, 10.0),
                    coating=(1.0, 1.0), matrix_base=(1.0, 1.0), rho_e=None, R=None):
    """Coated ellipsoid of the generalized Hashin structure (Sec. 4.2) as a benchmark input.

    Core semi-axes c (rho_c = 0), a confocal coating to the given total inclusion volume fraction,
    rotated by seeded ZYZ Euler angles; isotropic core and coating; the matrix is isotropic
    matrix_base plus the rank-one correction u (x) u / (u : eps0), u = C^eff eps0 - C_base eps0,
    the smallest change that makes the inclusion neutral for eps0 (an isotropic matrix has two
    constants against three conditions for a triaxial ellipsoid).
    Returns dict(c, rho_c, rho_e, R, stiffness [core, coating, matrix] Voigt, eps0, ceff_eps0, C0).
    """
    from scipy.optimize import brentq
    c = np.asarray(c, dtype=np.float64)
    rng = np.random.default_rng(seed)
    if R is None:
        R = euler_zyz(*rng.uniform(0, 2 * np.pi, 3))
    if rho_e is None:
        vol = lambda r: 4.0 / 3.0 * np.pi * np.prod(np.sqrt(c ** 2 + r)) - total_fraction
        rho_e = brentq(vol, 0.0, 1.0, xtol=1e-15)
    rho_c = 0.0
    lc, mc = core
    le, me = coating
    kc, ke = lc + 2 * mc / 3, le + 2 * me / 3
    g = lambda r: np.prod([ci ** 2 + r for ci in c if np.isfinite(ci)])
    f = lambda r: np.sqrt(g(rho_c) / g(r))
    Dc = np.diag(_depol_carlson(c, rho_c))
    fe = f(rho_e)
    Se = (Dc - fe * np.diag(_depol_carlson(c, rho_e))) / (1 - fe)
    alpha = (3 * ke + 4 * me) / (9 * (kc - ke))
    eps0 = R @ (alpha * np.eye(3) + (1 - fe) * Se) @ R.T
    a = ke / (kc - ke) * (kc + 4.0 / 3.0 * me) + 4.0 / 3.0 * me * fe
    ceff_eps0 = R @ (a * np.eye(3) + 2.0 / 3.0 * me * (1 - fe) * (3 * Se - np.eye(3))) @ R.T
    Cb = iso_tensor3(*matrix_base)
    u = ceff_eps0 - np.einsum('ijkl,kl->ij', Cb, eps0)
    Cm = Cb + np.einsum('ij,kl->ijkl', u, u) / np.einsum('ij,ij', u, eps0)
    Vm = tensor_to_voigt(Cm)
    Vi = iso_voigt(*iso_projection(Vm))
    if np.abs(Vm - Vi).max() <= 1e-12 * np.abs(Vm).max():
        # u is a multiple of the identity when the coating and base shear moduli agree (the Se terms of u
        # cancel), so the matrix is isotropic: take its exact form, without the rotation's rounding
        Vm = Vi
    stiff = [iso_voigt(*core), iso_voigt(*coating), Vm]
    lams, mus = zip(*[iso_projection(V) for V in stiff])
    return dict(c=c, rho_c=rho_c, rho_e=rho_e, R=R, stiffness=stiff, eps0=eps0, ceff_eps0=ceff_eps0,
                C0=c0_mean_extremes(lams, mus))


# ------------------------------------------------------------------ serving sweep (uneven batch)
def _unimodular(rng, d, n_shears=3, amp=2):
    """Product of n_shears random elementary shears I + s e_i e_j^T (i != j, s in [-amp, amp])."""
    U = np.eye(d, dtype=np.int64)
    for _ in range(n_shears):
        i, j = rng.choice(d, size=2, replace=False)
        S = np.eye(d, dtype=np.int64)
        S[i, j] = int(rng.integers(-amp, amp + 1))
        U = U @ S
    return U


def sweep_matrix(rng, d, U_exp, kind):
    """Integer M with |det M| = 2^U_exp of the given kind:
    'rank1'  divisors (1, .., 1, m): M = [[m, 0(, 0)], [-z2, 1(, 0)](, [-z3, 0, 1])], z random;
    'rank2'  divisors (e1, m / e1) in 2-D or (1, e2, m / e2) in 3-D, e = 2^a, a in [1, U_exp / 2],
             wrapped in random unimodular shears: M = U1 diag(e) V1;
    'diag'   the tensor grid diag(2^a_1, .., 2^a_d), exponents a random composition of U_exp (each >= 1)."""
    m = 1 << U_exp
    if kind == "rank1":
        M = np.eye(d, dtype=np.int64)
        M[0, 0] = m
        for i in range(1, d):
            M[i, 0] = -int(rng.integers(1, m))
        return M.tolist()
    if kind == "rank2":
        a = int(rng.integers(1, U_exp // 2 + 1))
        e = [1 << a, m >> a] if d == 2 else [1, 1 << a, m >> a]
        return (_unimodular(rng, d) @ np.diag(e).astype(np.int64) @ _unimodular(rng, d)).tolist()
    cuts = np.sort(rng.choice(np.arange(1, U_exp), size=d - 1, replace=False))
    a = np.diff(np.concatenate([[0], cuts, [U_exp]]))
    return np.diag([1 << int(x) for x in a]).astype(np.int64).tolist()


def serving_sweep(n=256, seed=BASE_SEED, m_exp=(12, 21), contrast_log10=(-2.0, 2.0)):
    """Seeded uneven batch of independent problems (one dict per instance, seed + i):
    d in {2, 3}; m = 2^U, U uniform in m_exp (inclusive); kind uniform in rank1 / rank2 / diag; 1-8
    periodic ellipsoidal inclusions (ellipses in 2-D) at volume fraction U(0.05, 0.4); matrix (1, 1) and
    inclusion lam = mu = 10^U(contrast_log10); C0 the mean of the extremes; the n_c unit load cases."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        d = int(rng.integers(2, 4))
        U_exp = int(rng.integers(m_exp[0], m_exp[1] + 1))
        kind = ["rank1", "rank2", "diag"][int(rng.integers(0, 3))]
        M = sweep_matrix(rng, d, U_exp, kind)
        n_incl = int(rng.integers(1, 9))
        incl = random_inclusions(int(rng.integers(1 << 30)), d, n_incl, float(rng.uniform(0.05, 0.4)))
        k = float(10.0 ** rng.uniform(*contrast_log10))
        n_c = d * (d + 1) // 2
        E = np.zeros((n_c, n_c))
        for a in range(n_c):
            E[a, a] = 1.0 if a < d else 0.5
        out.append(dict(d=d, M=M, kind=kind, m=1 << U_exp, incl=incl, contrast=k,
                        stiffness=[iso_voigt(1.0, 1.0), iso_voigt(k, k)], C0=c0_mean_extremes([1.0, k], [1.0, k]),
                        E=E))
    return out


# ------------------------------------------------------------------ Sec. 5.1 shear sweep (Table 1)
def hashin2d_workload():
    """Example 4.1 as a two-dimensional problem (one point along x3): the coated ellipse c = (0.05,
    0.35, inf), rho_c = 0, rho_e = 0.09, rotated by 60 degrees about x3 (n = (1/2, sqrt(3)/2, 0), the
    reading of the printed n = (1/2, 1, 0)); core (10, 10), coating (1, 1), the neutral matrix
    (the Lame constants of the paper's experiment are not printed)."""
    t = np.pi / 3.0
    R = np.array([[np.cos(t), -np.sin(t), 0.0], [np.sin(t), np.cos(t), 0.0], [0.0, 0.0, 1.0]])
    return hashin_workload(c=(0.05, 0.35, np.inf), rho_e=0.09, R=R)


def shear_sweep_matrices():
    """The pattern matrices of Sec. 5.1 as (name, 3 x 3 list): M_{j,k,alpha} = [[2^j, alpha k, 0],
    [(1 - alpha) k, 2^(14-j), 0], [0, 0, 1]] for j in {7, 8, 9}, alpha in {0, 1}, k in 16 {-32, ..., 32}
    (390 matrices, det 2^14), and M~_j = 1/2 [[1, 1, 0], [-1, 1, 0], [0, 0, 2]] diag(2^j, 2^(14-j), 1)
    for j in {7, 8, 9} (det 2^13)."""
    out = []
    for j in (7, 8, 9):
        for alpha in (0, 1):
            for k in range(-32 * 16, 32 * 16 + 1, 16):
                out.append(("M_%d,%d,%d" % (j, k, alpha),
                            [[2 ** j, alpha * k, 0], [(1 - alpha) * k, 2 ** (14 - j), 0], [0, 0, 1]]))
    for j in (7, 8, 9):
        out.append(("M~_%d" % j, [[2 ** (j - 1), 2 ** (13 - j), 0], [-2 ** (j - 1), 2 ** (13 - j), 0], [0, 0, 1]]))
    return out
