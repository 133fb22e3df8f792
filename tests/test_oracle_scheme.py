"""Pins of oracle.scheme (Algorithm 1, Sec. 3.2) against closed forms, invariants and the classic scheme."""
import json
import os

import numpy as np
import pytest

from oracle import analytic as an
from oracle import elasticity as el
from oracle.classic import classic_scheme, grid_points
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme, boundary_mask
from oracle.transform import dft_fast
from paper_1605_05712_gb300 import synth

RNG = np.random.default_rng(5)


def two_phase(d, l1=1.0, m1=1.0, l2=10.0, m2=10.0):
    return np.array([el.iso_tensor(l1, m1, d), el.iso_tensor(l2, m2, d)])


def sym(d):
    a = RNG.standard_normal((d, d))
    return a + a.T


@pytest.mark.parametrize("M", [[[8, -4], [2, 7]], [[4, 1, 0], [0, 4, 2], [2, 0, 4]]])
def test_homogeneous_reference_one_iteration(M):
    L = Lattice(M)
    d = L.d
    E = sym(d)
    C0 = (1.5, 0.9)
    stiff = np.array([el.iso_tensor(*C0, d)])
    r = basic_scheme(L, np.zeros(L.m, int), stiff, C0, E, tol=1e-14, maxit=10)
    assert r["iters"] == 1 and r["history"][0] == 0.0
    assert np.abs(r["eps"] - E).max() < 1e-14


@pytest.mark.parametrize("M", [[[8, -4], [2, 7]], [[4, 1, 0], [0, 4, 2], [2, 0, 4]]])
def test_homogeneous_other_medium(M):
    L = Lattice(M)
    d = L.d
    E = sym(d)
    C = el.iso_tensor(3.0, 2.0, d)
    r = basic_scheme(L, np.zeros(L.m, int), np.array([C]), (1.0, 0.5), E, tol=1e-14, maxit=5)
    assert np.abs(r["eps"] - E).max() < 1e-13
    assert np.abs(r["sigma_bar"] - el.ddot(C, E)).max() < 1e-12 * max(1.0, np.abs(el.ddot(C, E)).max())


def test_mean_strain_is_E_every_iteration():
    L = Lattice([[16, 4], [0, 8]])
    ph = synth.laminate_phase(L.p, L.m, [1, 2])
    E = sym(2)
    for k in (1, 2, 5):
        r = basic_scheme(L, ph, two_phase(2), (5.5, 5.5), E, tol=0.0, maxit=k)
        assert np.abs(r["eps"].mean(axis=0) - E).max() < 1e-13


@pytest.mark.parametrize("M,n_int", [([[64, 192], [0, 1]], [1, 3]), ([[4096, 12288], [0, 1]], [1, 3]),
                                     ([[32, 0], [0, 8]], [1, 0]), ([[8, 0, 0], [0, 4, 0], [0, 0, 16]], [0, 0, 1])])
def test_aligned_laminate_is_exact(M, n_int):
    # every frequency the laminate excites is parallel to n: the discrete fixed point is the analytic laminate
    L = Lattice(M)
    d = L.d
    ph = synth.laminate_phase(L.p, L.m, n_int)
    f1 = float(np.mean(ph == 0))
    assert f1 == 0.5
    E = sym(d)
    S = two_phase(d)
    r = basic_scheme(L, ph, S, (5.5, 5.5), E, tol=1e-15, maxit=200)
    e1, e2, sb = an.laminate_fields(S[0], S[1], f1, np.array(n_int, float), E)
    ex = np.where(ph[:, None, None] == 0, e1, e2)
    assert np.abs(r["eps"] - ex).max() < 1e-12 * max(1.0, np.abs(ex).max())
    assert np.abs(r["sigma_bar"] - sb).max() < 1e-12 * max(1.0, np.abs(sb).max())


def test_laminate_closed_forms_agree_with_milton():
    for d in (2, 3):
        S = two_phase(d, 1.0, 1.0, 7.0, 3.0)
        n = RNG.standard_normal(d)
        E = sym(d)
        for f1 in (0.25, 0.5, 0.8):
            e1, e2, sb = an.laminate_fields(S[0], S[1], f1, n, E)
            assert np.abs(f1 * e1 + (1 - f1) * e2 - E).max() < 1e-13
            nn = n / np.linalg.norm(n)
            t1, t2 = el.ddot(S[0], e1) @ nn, el.ddot(S[1], e2) @ nn
            assert np.abs(t1 - t2).max() < 1e-12                       # traction continuity
            D = e2 - e1                                                  # compatibility: sym(a (x) n)
            P = np.eye(d) - np.outer(nn, nn)
            assert np.abs(P @ D @ P).max() < 1e-12
            Ce = an.laminate_ceff_milton(S[0], S[1], f1, n)
            assert np.abs(el.ddot(Ce, E) - sb).max() < 1e-11


@pytest.mark.parametrize("N", [(8, 8), (6, 10), (3, 4), (5, 7), (4, 4, 4), (2, 6, 4), (3, 5, 9)])
def test_diagonal_lattice_equals_classic_grid_scheme(N):
    d = len(N)
    M = np.diag(N).tolist()
    L = Lattice(M)
    incl = synth.random_inclusions(17, d, 2, 0.3)
    ph_lat = synth.inclusions_phase(L.p, L.m, incl)
    gp = grid_points(N)
    ph_grid = synth.inclusions_phase(gp, L.m, incl)
    E = sym(d)
    S = two_phase(d)
    a = basic_scheme(L, ph_lat, S, (5.5, 5.5), E, tol=0.0, maxit=12)
    b = classic_scheme(N, ph_grid.reshape(N), S, (5.5, 5.5), E, tol=0.0, maxit=12)
    idx = {tuple(p): i for i, p in enumerate(gp.tolist())}
    perm = np.array([idx[tuple(p)] for p in L.p.tolist()])
    assert np.abs(a["eps"] - b["eps"][perm]).max() < 1e-13 * max(1, np.abs(b["eps"]).max())
    assert np.allclose(a["history"], b["history"], rtol=1e-11, atol=1e-15)


def test_real_part_reading_equals_averaged_green_operator():
    # boundary frequencies (even divisors): Re F^{-1}(-Gamma0(h(k)) tau_hat) equals F^{-1} of
    # -1/2 (Gamma0(h(k)) + Gamma0(h(-k))) tau_hat, which is what the CUDA path evaluates
    L = Lattice([[8, 2], [0, 4]])
    assert boundary_mask(L).any()
    d, m = L.d, L.m
    tau = np.stack([sym(d) for _ in range(m)])
    th = dft_fast(L, tau)
    h = L.h.astype(float)
    nz = np.any(L.h != 0, axis=1)
    e = np.array(L.e)
    neg = (-L.lam) % e
    flat = np.zeros(m, dtype=int)
    for j in range(d):
        flat = flat * e[j] + neg[:, j]
    lit = np.zeros_like(th)
    lit[nz] = -el.gamma_iso_apply(h[nz], th[nz], 2.0, 1.0)
    avg = np.zeros_like(th)
    avg[nz] = -0.5 * (el.gamma_iso_apply(h[nz], th[nz], 2.0, 1.0) + el.gamma_iso_apply(h[flat][nz], th[nz], 2.0, 1.0))
    a = dft_fast(L, lit, inverse=True)
    b = dft_fast(L, avg, inverse=True)
    assert np.abs(a.real - b.real).max() < 1e-13 and np.abs(b.imag).max() < 1e-13


def test_general_laminate_converges_under_refinement():
    E = np.array([[1.0, 0.0], [0.0, 0.0]])
    S = two_phase(2)
    errs = []
    for N in (8, 16, 32):
        L = Lattice([[N, 0], [0, N]])
        ph = synth.laminate_phase(L.p, L.m, [1, 2])
        r = basic_scheme(L, ph, S, (5.5, 5.5), E, tol=1e-10, maxit=2000)
        e1, e2, sb = an.laminate_fields(S[0], S[1], 0.5, np.array([1.0, 2.0]), E)
        errs.append(np.linalg.norm(r["sigma_bar"] - sb) / np.linalg.norm(sb))
    assert errs[2] < errs[1] < errs[0]


def test_paper_subsampling_trend():
    # Sec. 5.2 / Fig. 7: the rank-1 sub lattice M_b needs far fewer iterations and gives a smaller
    # strain error than the 8x8 pixel grid M_c of equal size; the full grid M_a sits in between
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_subsampling_fig7.json")))
    E = np.array([[1.0, 0.0], [0.0, 0.0]])
    S = two_phase(2)
    out = {}
    for name, M in (("M_a", [[64, 0], [0, 64]]), ("M_b", [[64, 32], [0, 1]]), ("M_c", [[8, 0], [0, 8]])):
        L = Lattice(M)
        ph = synth.laminate_phase(L.p, L.m, [2, 1])
        r = basic_scheme(L, ph, S, (5.5, 5.5), E, tol=g["threshold"], maxit=2000)
        e1, e2, sb = an.laminate_fields(S[0], S[1], 0.5, np.array([2.0, 1.0]), E)
        ex = np.where(ph[:, None, None] == 0, e1, e2)
        el2 = np.sqrt(el.frob2(r["eps"] - ex).sum() / el.frob2(ex).sum())
        out[name] = (r["iters"], el2)
    it, e = g["iterations"], g["e_l2"]
    assert (out["M_b"][0] < out["M_a"][0] / 3) == (it["M_b"] < it["M_a"] / 3)
    assert (out["M_b"][0] < out["M_c"][0] / 3) == (it["M_b"] < it["M_c"] / 3)
    assert (out["M_b"][1] < out["M_a"][1] < out["M_c"][1]) == (e["M_b"] < e["M_a"] < e["M_c"])
