"""Classic Moulinec-Suquet Basic Scheme on a tensor-product grid, for the oracle's pins.

Test infrastructure only (see ``oracle/__init__``).

An independent implementation for M = diag(N_1, ..., N_d): no Smith normal
form, no pattern machinery.  Grid points x = j / N_i reduced into [-1/2, 1/2),
integer frequencies from numpy.fft.fftfreq (the symmetric cell), the
d-dimensional FFT of numpy, the closed-form isotropic Green operator at the
integer frequency, and the real part of the inverse transform.  Sec. 3.2
states that for a diagonal M the pattern scheme is this scheme; the pin test
compares the two.
"""
from __future__ import annotations

import numpy as np

from . import elasticity as el


def grid_points(N):
    """(m, d) numerators p = m y of the grid points in C order, y_i = j_i / N_i in [-1/2, 1/2)."""
    d = len(N)
    m = int(np.prod(N))
    idx = np.indices(N).reshape(d, -1).T
    y_num = np.empty_like(idx)
    for i in range(d):
        j = idx[:, i].copy()
        j[2 * j >= N[i]] -= N[i]
        y_num[:, i] = j * (m // N[i])
    return y_num


def classic_scheme(N, phase_grid, stiff, C0, E, tol=1e-8, maxit=1000):
    """MS98 basic scheme on the grid N (phase_grid has shape N); returns dict like scheme.basic_scheme."""
    N = tuple(int(n) for n in N)
    d = len(N)
    m = int(np.prod(N))
    lam0, mu0 = C0
    C0t = el.iso_tensor(lam0, mu0, d)
    dC = np.asarray(stiff) - C0t
    ph = np.asarray(phase_grid).reshape(-1)
    freqs = np.meshgrid(*[np.fft.fftfreq(n) * n for n in N], indexing='ij')
    k = np.stack([f.reshape(-1) for f in freqs], axis=-1)
    nz = np.any(k != 0, axis=1)
    eps = np.broadcast_to(E, (m, d, d)).copy()
    nE = np.sqrt(el.frob2(np.asarray(E)))
    norm0 = np.sqrt(m) * nE if nE > 0 else 1.0
    hist = []
    it = 0
    while it < maxit:
        tau = el.ddot(dC[ph], eps)
        th = np.fft.fftn(tau.reshape(N + (d, d)), axes=tuple(range(d))).reshape(m, d, d) / m
        eh = np.zeros_like(th)
        eh[nz] = -el.gamma_iso_apply(k[nz], th[nz], lam0, mu0)
        eh[~nz] = E
        new = (np.fft.ifftn(eh.reshape(N + (d, d)), axes=tuple(range(d))).reshape(m, d, d) * m).real
        r = np.sqrt(el.frob2(new - eps).sum()) / norm0
        eps = new
        it += 1
        hist.append(float(r))
        if r < tol:
            break
    sigma = el.ddot(np.asarray(stiff)[ph], eps)
    return dict(eps=eps, sigma=sigma, sigma_bar=sigma.mean(axis=0), iters=it, history=hist)
