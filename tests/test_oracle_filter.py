"""Pins of the start filter's premise on the oracle (tiny odd grid, so no frequency lies on the
boundary of the symmetric cell and Gamma0 is an exact projector).

With two phases whose stiffness is c_p C0 (lam = mu in each phase and in C0 = mean of the extremes),
the linear part T of one step of Algorithm 1 has the eigenvalues +-rho, rho = (k - 1) / (k + 1), on the
compatible strains confined to one phase; the exact solution is C0-orthogonal to them (equilibrium in
each phase, i.e. Gamma0 sigma* = 0), so the cold start's error has no such component.  The filter
(G^2(s) - rho^2 s) / (1 - rho^2) keeps eps* and removes those components from any start s.
"""
import numpy as np
import pytest

from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme, filtered_start

N = 7
K = 9.0


def _setup():
    lat = Lattice([[N, 0], [0, N]])
    pts = (lat.p // (lat.m // N)) % N            # integer grid coordinates in lattice order
    r2 = (pts[:, 0] - 3) ** 2 + (pts[:, 1] - 3) ** 2
    phase = (r2 <= 5).astype(np.int64)           # 21-point inclusion (phase 1), matrix phase 0
    stiff = np.array([el.iso_tensor(1.0, 1.0, 2), el.iso_tensor(K, K, 2)])
    C0 = (0.5 * (1 + K), 0.5 * (1 + K))
    E = np.array([[1.0, 0.3], [0.3, -0.5]])
    return lat, phase, stiff, C0, E


def _sym_basis(m):
    """Orthonormal basis of symmetric 2x2 fields on m points (3 m vectors, shape (m, 2, 2))."""
    B = []
    for y in range(m):
        for (i, j) in ((0, 0), (1, 1), (0, 1)):
            e = np.zeros((m, 2, 2))
            if i == j:
                e[y, i, i] = 1.0
            else:
                e[y, 0, 1] = e[y, 1, 0] = np.sqrt(0.5)
            B.append(e)
    return B


def _coords(f, B):
    return np.array([np.sum(f * b) for b in B])


@pytest.fixture(scope="module")
def system():
    lat, phase, stiff, C0, E = _setup()
    m = lat.m
    G = lambda eps: basic_scheme(lat, phase, stiff, C0, E, tol=0.0, maxit=1, eps0=eps)['eps']
    b = G(np.zeros((m, 2, 2)))
    B = _sym_basis(m)
    T = np.array([_coords(G(e) - b, B) for e in B]).T       # T[:, j] = coords of T e_j
    sol = basic_scheme(lat, phase, stiff, C0, E, tol=1e-15, maxit=3000)
    return dict(lat=lat, phase=phase, stiff=stiff, C0=C0, E=E, T=T, B=B, sol=sol)


def _eigspace(T, lam, tol=1e-9):
    u, s, vt = np.linalg.svd(T - lam * np.eye(len(T)))
    return vt[s < tol].T                                       # columns span ker(T - lam I)


def test_slow_eigenvalues_are_the_confined_compatible_fields(system):
    T, phase = system["T"], system["phase"]
    rho = (K - 1) / (K + 1)
    assert np.abs(np.linalg.eigvals(T)).max() <= rho + 1e-9   # spectrum within [-rho, rho]
    minus, plus = _eigspace(T, -rho), _eigspace(T, rho)
    # dimension count: confined fields (3 |S_p|) meet the compatible zero-mean ones (2 (m - 1))
    m = len(phase)
    n_incl = int(phase.sum())
    assert minus.shape[1] >= 3 * n_incl + 2 * (m - 1) - 3 * m
    assert plus.shape[1] >= 3 * (m - n_incl) + 2 * (m - 1) - 3 * m
    # -rho (stiff phase) fields vanish in the matrix, +rho (soft matrix) fields in the inclusion
    on_point = np.repeat(phase, 3)
    assert np.abs(minus[on_point == 0]).max() < 1e-8
    assert np.abs(plus[on_point == 1]).max() < 1e-8


def test_exact_solution_is_c0_orthogonal_to_the_slow_fields(system):
    T, B, sol = system["T"], system["B"], system["sol"]
    rho = (K - 1) / (K + 1)
    # with C0 = c0 iso(1, 1) the C0 inner product of two strain fields is c0 <e : iso(1,1) : f>
    iso = el.iso_tensor(1.0, 1.0, 2)
    for V in (_eigspace(T, -rho), _eigspace(T, rho)):
        for v in V.T:
            field = sum(c * b for c, b in zip(v, B))
            inner = np.sum(el.ddot(iso, field) * sol["eps"])
            assert abs(inner) < 1e-9 * np.linalg.norm(sol["eps"]) * np.linalg.norm(field)


def test_filter_keeps_the_solution_and_removes_slow_components(system):
    lat, phase, stiff, C0, E, T, B, sol = (system[k] for k in ("lat", "phase", "stiff", "C0", "E", "T", "B", "sol"))
    rho = (K - 1) / (K + 1)
    f = filtered_start(lat, phase, stiff, C0, E, sol["eps"], rho)
    assert np.abs(f - sol["eps"]).max() < 1e-12
    rng = np.random.default_rng(3)
    start = sol["eps"] + 0.1 * rng.standard_normal(sol["eps"].shape)
    start = 0.5 * (start + start.transpose(0, 2, 1))
    err = _coords(filtered_start(lat, phase, stiff, C0, E, start, rho) - sol["eps"], B)
    err0 = _coords(start - sol["eps"], B)
    for V in (_eigspace(T, -rho), _eigspace(T, rho)):
        Q, _ = np.linalg.qr(V)
        assert np.linalg.norm(Q.T @ err0) > 1e-3                 # the start had slow components
        # T is not symmetric in these coordinates: test with the eigen-decomposition instead of projections
    w, X = np.linalg.eig(T)
    c = np.linalg.solve(X, err)
    c0 = np.linalg.solve(X, err0)
    slow = np.abs(np.abs(w) - rho) < 1e-9
    assert np.abs(c[slow]).max() < 1e-10 * np.abs(c0[slow]).max()
    # every other component is multiplied by p(t) = (t^2 - rho^2) / (1 - rho^2)
    fast = ~slow & (np.abs(c0) > 1e-6 * np.abs(c0).max())
    p = (w ** 2 - rho ** 2) / (1 - rho ** 2)
    assert np.abs(c[fast] - p[fast] * c0[fast]).max() < 1e-8 * np.abs(c0).max()


def test_filter_rho_host_logic():
    # the package's rate for the filter: lam = mu phases against C0 = mean of extremes give (k - 1) / (k + 1);
    # a general phase gives the extreme generalized eigenvalue of (C_p - C0, C0) in Mandel form
    from scipy.linalg import eigh
    from paper_1605_05712_gb300 import synth
    from paper_1605_05712_gb300.warmstart import filter_rho
    for k in (0.1, 3.0, 100.0):
        C0 = (0.5 * (1 + k), 0.5 * (1 + k))
        assert abs(filter_rho([synth.iso_voigt(1, 1), synth.iso_voigt(k, k)], C0) - abs(k - 1) / (k + 1)) < 1e-12
    w = synth.hashin_workload()
    W = np.diag([1, 1, 1, np.sqrt(2), np.sqrt(2), np.sqrt(2)])
    M0 = W @ synth.iso_voigt(*w["C0"]) @ W
    ref = max(np.abs(eigh(W @ V @ W - M0, M0, eigvals_only=True)).max() for V in w["stiffness"])
    assert abs(filter_rho(w["stiffness"], w["C0"]) - ref) < 1e-12
