"""Algorithm 1 (fixed-point algorithm on patterns) for the oracle.

Test infrastructure only (see ``oracle/__init__``).  float64 throughout.

Sec. 3.2, Algorithm 1 (collocation of the Lippmann-Schwinger equation at the
pattern points 2 pi y, y in P(M)):
    eps^(0)_y <- E for all y
    repeat
        tau_y      <- (C_y - C0) : eps^(n)_y                 (polarization)
        tau_hat    <- F(M) tau                                (forward, with 1/m)
        epshat_h   <- -Gamma0(h) : tau_hat_h,  h in G(M^T) \\ {0}
        epshat_0   <- E
        eps^(n+1)  <- F(M)^{-1} epshat                        (inverse, no 1/m)
    until converged
with the Cauchy criterion of Sec. 5.2,
    r_n = ||eps^(n+1) - eps^(n)|| / ||eps^(0)|| < tol,
the norm being the l2 norm over the pattern of the Frobenius norm.
Outputs also the stress sigma_y = C_y : eps_y and its mean, which is
C^eff : E (Sec. 3.1, definition of the effective matrix).

Readings where the paper is silent (each listed in the design notes):
  * Gamma0 is evaluated at the integer frequency h in G(M^T) itself: the
    Fourier multiplier of the symmetric gradient at coefficient index h.
  * The strain is real (Sec. 3.2 seeks real symmetric eps_y).  At boundary
    frequencies of the symmetric cell (even divisors) h(k) and h(-k) are not
    negatives of each other, so F^{-1} of the literal spectrum is complex;
    the iterate is its real part.  ``boundary='zero'`` instead sets those
    frequencies to zero (the usual Nyquist convention), as an option.
  * ||eps^(0)|| is sqrt(m) ||E||_F also for a warm start (1 if E = 0), so cold
    and warm runs share one threshold.
"""
from __future__ import annotations

import numpy as np

from . import elasticity as el
from .lattice import Lattice
from .transform import dft_fast, dft_naive


def _phase_ddot(C, phase, eps):
    """(C_{phase(y)} : eps_y)_y, one phase at a time (no (m, d, d, d, d) temporary)."""
    out = np.zeros_like(eps)
    for p in np.unique(phase):
        sel = phase == p
        out[sel] = el.ddot(C[p], eps[sel])
    return out


def _transform(lat, a, inverse, mode):
    if mode == 'naive' or (mode == 'auto' and lat.m <= 1024):
        return dft_naive(lat, a, inverse)
    return dft_fast(lat, a, inverse)


def boundary_mask(lat):
    """True at k where h(-k) != -h(k) (frequencies on the boundary of the symmetric cell)."""
    m = lat.m
    e = np.array(lat.e, dtype=np.int64)
    neg = (-lat.lam) % e
    flat = np.zeros(m, dtype=np.int64)
    for j in range(lat.d):
        flat = flat * e[j] + neg[:, j]
    return np.any(lat.h[flat] != -lat.h, axis=1)


def basic_scheme(M, phase, stiff, C0, E, tol=1e-8, maxit=1000, eps0=None,
                 transform='auto', boundary='literal', L=None, C0_tensor=None, scheme='basic'):
    """Run Algorithm 1.

    M        integer matrix (d x d) or an ``oracle.lattice.Lattice``
    phase    (m,) int phase index per pattern point, in lattice (lambda) order
    stiff    (n_phases, d, d, d, d) stiffness tensors C_p
    C0       (lam0, mu0) isotropic reference medium
    E        (d, d) macroscopic strain (tensor components)
    tol      Cauchy threshold; maxit caps the iteration count
    eps0     optional (m, d, d) warm start
    L        optional regular real (d x d) cell matrix: the transformed pattern P_L(M) = L Lambda(M) cap
             L [-1/2, 1/2)^d of Sec. 3.3 (Def. 3.3).  The point y of P(M) sits at x = L y in the cell
             L [-1/2, 1/2)^d, whose dual lattice is L^{-T} Z^d, so the Fourier index h stands for the
             physical frequency L^{-T} h: Gamma0 is evaluated there.  The DFT over the index sets is
             unchanged.  None = the unit cube (L = I).
    C0_tensor  optional (d, d, d, d) general reference medium (replaces C0); Gamma0 then comes from
             the acoustic tensor K(xi) = C0 xi xi (the operator form of Sec. 3.1)
    scheme   'basic' (Algorithm 1) or 'eyre_milton', an accelerated scheme of the kind the paper names
             as carrying over to patterns (Sec. 6), written from the projector identities: with
             u = (C + C0) eps, v = (C - C0) eps and Pi = C0 Gamma0 (the projector onto C0 times
             compatible fields), compatibility of eps and equilibrium of C eps read u = (I - 2 Pi) v at
             h != 0 and <u> = <v> + 2 C0 E; the iteration u <- (I - 2 Pi) v(u) contracts at
             max |c - c0| / (c + c0).  Each step: v = (C - C0) eps, u_hat = v_hat - 2 C0 Gamma0 v_hat
             (h != 0), u_hat_0 = v_hat_0 + 2 C0 E, u = Re F^{-1} u_hat, eps <- (C + C0)^{-1} u.  Its
             fixed point is Algorithm 1's.
             'cg': conjugate gradients on the same discrete equation (``conjugate_gradient``).
    Returns dict(eps, sigma, sigma_bar, iters, history).
    """
    lat = M if isinstance(M, Lattice) else Lattice(M)
    d, m = lat.d, lat.m
    phase = np.asarray(phase, dtype=np.int64)
    stiff = np.asarray(stiff, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    if C0_tensor is None:
        lam0, mu0 = C0
        C0t = el.iso_tensor(lam0, mu0, d)
    else:
        C0t = np.asarray(C0_tensor, dtype=np.float64)
    dC = stiff - C0t                                   # (C_p - C0)
    h = lat.h.astype(np.float64)
    if L is not None:
        h = h @ np.linalg.inv(np.asarray(L, dtype=np.float64))      # rows: (L^{-T} h)^T = h^T L^{-1}
    nz = np.any(lat.h != 0, axis=1)
    assert nz.sum() == m - 1 and not nz[0], "h = 0 must be exactly k = 0"
    bmask = boundary_mask(lat) if boundary == 'zero' else None

    eps = np.broadcast_to(E, (m, d, d)).copy() if eps0 is None else np.array(eps0, dtype=np.float64)
    nE = np.sqrt(el.frob2(E))
    norm0 = np.sqrt(m) * nE if nE > 0 else 1.0
    history = []
    it = 0
    if scheme == 'eyre_milton':
        # (C_p + C0)^{-1} per phase, as the inverse of the linear map on symmetric tensors
        Wp = np.array([_inverse_on_sym(stiff[q] + C0t) for q in range(len(stiff))])
        if boundary == 'zero':
            # zeroing eps_hat at the boundary frequencies has no counterpart in the u iteration
            raise ValueError("the Eyre-Milton scheme takes the literal (averaged) boundary treatment")
    elif scheme == 'cg':
        return conjugate_gradient(lat, phase, stiff, C0, E, tol, maxit, eps0=eps0, transform=transform,
                                  boundary=boundary, L=L, C0_tensor=C0_tensor)
    elif scheme != 'basic':
        raise ValueError("scheme must be 'basic', 'eyre_milton' or 'cg'")
    while it < maxit:
        tau = _phase_ddot(dC, phase, eps)                              # polarization (v for Eyre-Milton)
        tau_hat = _transform(lat, tau, False, transform)               # F(M) tau
        eps_hat = np.zeros_like(tau_hat)
        if C0_tensor is None:
            g = el.gamma_iso_apply(h[nz], tau_hat[nz], lam0, mu0)
        else:
            g = el.gamma_general_apply(C0t, h[nz], tau_hat[nz])
        if scheme == 'basic':
            eps_hat[nz] = -g
            if bmask is not None:
                eps_hat[bmask] = 0.0
            eps_hat[~nz] = E                                           # mean strain
            eps_new = _transform(lat, eps_hat, True, transform).real   # F(M)^{-1}
        else:
            eps_hat[nz] = tau_hat[nz] - 2.0 * el.ddot(C0t, g)         # u_hat = (I - 2 C0 Gamma0) v_hat
            if bmask is not None:
                eps_hat[bmask] = 0.0
            eps_hat[~nz] = tau_hat[~nz] + 2.0 * el.ddot(C0t, E)       # <u> = <v> + 2 C0 E
            u = _transform(lat, eps_hat, True, transform).real
            eps_new = _phase_ddot(Wp, phase, u)                        # eps = (C + C0)^{-1} u
        r = np.sqrt(el.frob2(eps_new - eps).sum()) / norm0
        eps = eps_new
        it += 1
        history.append(float(r))
        if r < tol:
            break
    sigma = _phase_ddot(stiff, phase, eps)
    return dict(eps=eps, sigma=sigma, sigma_bar=sigma.mean(axis=0), iters=it, history=history)


def conjugate_gradient(M, phase, stiff, C0, E, tol=1e-8, maxit=1000, eps0=None, transform='auto',
                       boundary='literal', L=None, C0_tensor=None):
    """Conjugate gradients on the discrete Lippmann-Schwinger equation (an accelerated scheme of the
    kind Sec. 6 says carries over to patterns; the paper cites Zeman et al. 2010 for it).

    With eps = E + e and e compatible with zero mean, Algorithm 1's fixed point solves
    A e = b,  A = Gamma0 C,  b = -Gamma0 C E.
    On the compatible zero-mean fields Gamma0 C0 is the identity, so <C0 A a, c> = <C a, c>: A is
    self-adjoint and positive in the inner product <a, c>_C0 = sum_y a_y : C0 : c_y, and plain
    (Hestenes-Stiefel) conjugate gradients apply in that inner product:
        x = E, r = -Gamma0 C x, p = r
        repeat: q = A p, alpha = <r, r>_C0 / <p, q>_C0, x += alpha p, r' = r - alpha q,
                beta = <r', r'>_C0 / <r, r>_C0, p = r' + beta p, r = r'
    r = -Gamma0 : sigma(x) is Algorithm 1's increment at x, so the stopping test takes Algorithm 1's
    measure ||r|| / ||eps^(0)|| (l2 over the pattern of the Frobenius norm).  Every application of A
    (one forward and one inverse transform) counts as one iteration; history[k] is the measure of the
    k-th iterate, reached after k + 1 transforms.

    Rounding leaves every update a part outside the compatible fields of relative size ~u (the unit
    roundoff); A annihilates that part, so once the residual is at the rounding level of the first one
    the step lengths are undefined.  The iteration therefore also stops when ||r_k|| <= 1024 u ||r_0||
    (u = 2^-53), which includes r_0 = 0 (E is then the exact discrete solution).

    Gamma0 C0 must be a projector at every frequency: ``boundary='zero'``, or 'literal' on a lattice
    without boundary frequencies (every divisor odd).  A warm start is refused: the iterates stay in
    eps^(0) + the compatible fields, so an incompatible part of eps^(0) would never be removed.
    """
    lat = M if isinstance(M, Lattice) else Lattice(M)
    d, m = lat.d, lat.m
    phase = np.asarray(phase, dtype=np.int64)
    stiff = np.asarray(stiff, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    if eps0 is not None:
        raise ValueError("the conjugate-gradient scheme starts from eps = E")
    if C0_tensor is None:
        lam0, mu0 = C0
        C0t = el.iso_tensor(lam0, mu0, d)
    else:
        C0t = np.asarray(C0_tensor, dtype=np.float64)
    h = lat.h.astype(np.float64)
    if L is not None:
        h = h @ np.linalg.inv(np.asarray(L, dtype=np.float64))
    nz = np.any(lat.h != 0, axis=1)
    bmask = boundary_mask(lat)
    if boundary != 'zero' and bmask.any():
        raise ValueError("the conjugate-gradient scheme needs boundary='zero' on lattices with boundary frequencies")

    def apply_A(v):
        """Gamma0 : (C : v) with the mean and the boundary frequencies set to zero."""
        t_hat = _transform(lat, _phase_ddot(stiff, phase, v), False, transform)
        out = np.zeros_like(t_hat)
        if C0_tensor is None:
            out[nz] = el.gamma_iso_apply(h[nz], t_hat[nz], lam0, mu0)
        else:
            out[nz] = el.gamma_general_apply(C0t, h[nz], t_hat[nz])
        out[bmask] = 0.0
        return _transform(lat, out, True, transform).real

    def dot_c0(a, c):
        return float(np.einsum('yij,ijkl,ykl->', a, C0t, c))

    nE = np.sqrt(el.frob2(E))
    norm0 = np.sqrt(m) * nE if nE > 0 else 1.0
    x = np.broadcast_to(E, (m, d, d)).copy()
    history = []
    it = 0
    if maxit > 0:
        r = -apply_A(x)
        it = 1
        history.append(float(np.sqrt(el.frob2(r).sum()) / norm0))
        p = r.copy()
        gamma = dot_c0(r, r)
        floor = 1024 * 2.0 ** -53 * history[0]
        while not history[-1] < tol and it < maxit and not history[-1] <= floor:
            q = apply_A(p)
            it += 1
            delta = dot_c0(p, q)
            alpha = gamma / delta if delta != 0 else 0.0
            x = x + alpha * p
            r = r - alpha * q
            history.append(float(np.sqrt(el.frob2(r).sum()) / norm0))
            gamma_new = dot_c0(r, r)
            beta = gamma_new / gamma if gamma != 0 else 0.0
            p = r + beta * p
            gamma = gamma_new
    sigma = _phase_ddot(stiff, phase, x)
    return dict(eps=x, sigma=sigma, sigma_bar=sigma.mean(axis=0), iters=it, history=history)


def _inverse_on_sym(C):
    """Inverse of the linear map eps -> C : eps on symmetric d x d tensors, as a (d, d, d, d) tensor
    with the minor symmetries (via the orthonormal Mandel basis)."""
    d = C.shape[0]
    pairs = [(i, i) for i in range(d)] + [(i, j) for i in range(d) for j in range(i + 1, d)]
    B = []
    for (i, j) in pairs:
        e = np.zeros((d, d))
        if i == j:
            e[i, i] = 1.0
        else:
            e[i, j] = e[j, i] = np.sqrt(0.5)
        B.append(e)
    A = np.array([[np.einsum('ij,ijkl,kl', a, C, b) for b in B] for a in B])
    Ai = np.linalg.inv(A)
    return np.einsum('pq,pij,qkl->ijkl', Ai, np.array(B), np.array(B))


def filtered_start(M, phase, stiff, C0, E, eps0, rho, **kw):
    """(G^2(eps0) - rho^2 eps0) / (1 - rho^2), G one step of Algorithm 1 (not in the paper).

    G is affine with fixed point eps*, so the error of the result is p(T)(eps0 - eps*) with T the
    linear part of G and p(t) = (t^2 - rho^2) / (1 - rho^2): p(1) = 1 keeps eps*, p(+-rho) = 0
    removes the error components of eigenvalue +-rho.
    """
    g2 = basic_scheme(M, phase, stiff, C0, E, tol=0.0, maxit=2, eps0=eps0, **kw)['eps']
    return (g2 - rho * rho * np.asarray(eps0, dtype=np.float64)) / (1.0 - rho * rho)


def unit_load(d, a):
    """Unit load case a in Voigt order: eps_11 = 1, ..., or eps_ij = eps_ji = 1/2 for shear."""
    (i, j) = el.voigt_pairs(d)[a]
    E = np.zeros((d, d))
    if i == j:
        E[i, i] = 1.0
    else:
        E[i, j] = E[j, i] = 0.5
    return E


def effective_voigt(M, phase, stiff, C0, tol=1e-8, maxit=1000, **kw):
    """C^eff in Voigt form (engineering shear): column a = sigma_bar of unit load case a."""
    lat = M if isinstance(M, Lattice) else Lattice(M)
    d = lat.d
    n_c = len(el.voigt_pairs(d))
    Ceff = np.zeros((n_c, n_c))
    for a in range(n_c):
        res = basic_scheme(lat, phase, stiff, C0, unit_load(d, a), tol, maxit, **kw)
        Ceff[:, a] = el.sym_to_comps(res['sigma_bar'])
    return Ceff
