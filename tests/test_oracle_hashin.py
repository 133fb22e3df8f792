"""Pins of the generalized Hashin structure (Sec. 4.2) in oracle.analytic and of the scheme on it.

The analytic field carries three readings of garbled formulas (depolarization factors, grad rho,
rotation); these tests check the field against what mechanics fixes: the interface conditions
(traction continuity, rank-one strain jumps), equilibrium inside the coating, neutrality of the
matrix, Sum d_i = 1 with the paper's closed forms as special cases, and convergence of the oracle's
Algorithm 1 towards the analytic effective stress under refinement.
"""
import numpy as np
import pytest

from oracle import elasticity as el
from oracle.analytic import Hashin, depolarization, ellipsoidal_radius, rotation_to
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme
from paper_1605_05712_gb300 import synth


def test_depolarization_factors():
    assert np.allclose(depolarization([0.2, 0.2, 0.2], 0.0), 1.0 / 3.0, atol=1e-13)
    for c in ([0.1, 0.15, 0.2], [0.05, 0.3, 0.31], [0.1, 0.1, 0.4]):
        for rho in (0.0, 0.05):
            d = depolarization(c, rho)
            assert abs(d.sum() - 1.0) < 1e-12
            assert np.allclose(d, synth._depol_carlson(c, rho), atol=1e-12, rtol=0)   # Carlson R_D agrees
    # prolate spheroid c1 = c2 < c3 (Sec. 4.2 with the garble fixed: d3 carries "- 1", d1 = d2 = (1 - d3)/2)
    d = depolarization([0.1, 0.1, 0.3], 0.0)
    dl = np.sqrt(1 - (0.1 / 0.3) ** 2)
    d3 = (1 - dl ** 2) / dl ** 2 * (np.log((1 + dl) / (1 - dl)) / (2 * dl) - 1)
    assert abs(d[2] - d3) < 1e-12 and abs(d[0] - (1 - d3) / 2) < 1e-12
    # oblate c1 < c2 = c3: d1 as printed, d2 = d3 = (1 - d1)/2
    d = depolarization([0.1, 0.3, 0.3], 0.0)
    dl = np.sqrt(1 - (0.1 / 0.3) ** 2)
    d1 = (1 - np.sqrt(1 - dl ** 2) / dl * np.arcsin(dl)) / dl ** 2
    assert abs(d[0] - d1) < 1e-12 and abs(d[1] - (1 - d1) / 2) < 1e-12
    # elliptic cylinder as printed
    d = depolarization([0.05, 0.35, np.inf], 0.09)
    l1, l2 = np.sqrt(0.05 ** 2 + 0.09), np.sqrt(0.35 ** 2 + 0.09)
    assert np.allclose(d, [l2 / (l1 + l2), l1 / (l1 + l2), 0.0])


def test_ellipsoidal_radius_and_rotation():
    c = np.array([0.1, 0.15, 0.2])
    rng = np.random.default_rng(0)
    x = rng.uniform(-0.4, 0.4, (50, 3))
    r = ellipsoidal_radius(c, x)
    assert np.abs(np.sum(x ** 2 / (c ** 2 + r[:, None]), axis=1) - 1).max() < 1e-12
    n = rng.standard_normal(3)
    R = rotation_to(n)
    assert np.allclose(R @ [1, 0, 0], n / np.linalg.norm(n)) and np.allclose(R @ R.T, np.eye(3))


@pytest.mark.parametrize("case", ["triaxial", "cylinder"])
def test_analytic_field_satisfies_mechanics(case):
    rng = np.random.default_rng(1)
    if case == "triaxial":
        w = synth.hashin_workload()
        H = Hashin(w["c"], w["rho_c"], w["rho_e"], 10, 10, 1, 1, R=w["R"])
        Cm = el.voigt6_to_tensor(w["stiffness"][2], 3)
        assert np.abs(H.eps0 - w["eps0"]).max() < 1e-13
    else:   # Example 4.1: c = (0.05, 0.35, inf), rho_c = 0, rho_e = 0.09, 60 degree rotation
        R = rotation_to([0.5, np.sqrt(3) / 2, 0.0])
        H = Hashin([0.05, 0.35, np.inf], 0.0, 0.09, 10, 10, 1, 1, R=R)
        C1 = el.iso_tensor(1, 1, 3)
        u = H.ceff_eps0 - el.ddot(C1, H.eps0)
        Cm = C1 + np.einsum('ij,kl->ijkl', u, u) / np.einsum('ij,ij', u, H.eps0)
    # neutrality of the matrix: C_m : eps0 = C^eff eps0, and C_m positive definite
    assert np.abs(el.ddot(Cm, H.eps0) - H.ceff_eps0).max() < 1e-13
    from oracle.analytic import to_mandel
    assert np.linalg.eigvalsh(to_mandel(Cm)).min() > 0
    fin = np.isfinite(H.c)
    for rho0, C_in, C_out in ((H.rho_e, H.Ce, Cm), (H.rho_c, H.Cc, H.Ce)):
        for _ in range(8):
            s = rng.standard_normal(3)
            if not fin[2]:
                s[2] = 0.0
            s /= np.linalg.norm(s)
            l = np.where(fin, np.sqrt(np.where(fin, H.c, 0) ** 2 + rho0), 0.0)
            xt = l * s
            x = H.R @ xt
            nt = np.where(fin, xt / np.where(fin, l, 1) ** 2, 0.0)
            nrm = H.R @ nt
            nrm /= np.linalg.norm(nrm)
            h = 1e-8
            e_in = H.strain((x - h * nrm)[None])[0]
            e_out = H.strain((x + h * nrm)[None])[0]
            t_in, t_out = el.ddot(C_in, e_in) @ nrm, el.ddot(C_out, e_out) @ nrm
            assert np.abs(t_in - t_out).max() < 1e-5 * np.abs(t_in).max()       # traction continuity
            P = np.eye(3) - np.outer(nrm, nrm)
            assert np.abs(P @ (e_out - e_in) @ P).max() < 1e-5                    # rank-one (compatible) jump
    # equilibrium inside the coating: div (C_e : eps) = 0
    for _ in range(4):
        while True:
            x = rng.uniform(-0.45, 0.45, 3)
            if not fin[2]:
                x[2] = 0.0
            if H.region(x[None])[0][0] == 1:
                break
        h = 2e-6
        div = np.zeros(3)
        for j in range(3 if fin[2] else 2):
            e = np.zeros(3)
            e[j] = h
            sp = el.ddot(H.Ce, H.strain((x + e)[None])[0])
            sm = el.ddot(H.Ce, H.strain((x - e)[None])[0])
            div += (sp[:, j] - sm[:, j]) / (2 * h)
        assert np.abs(div).max() < 1e-5 * np.abs(el.ddot(H.Ce, H.strain(x[None])[0])).max()


@pytest.mark.slow
def test_scheme_converges_to_hashin_effective_stress():
    # Algorithm 1 on the coated ellipsoid: the effective stress error shrinks under refinement
    w = synth.hashin_workload()
    S = np.array([el.voigt6_to_tensor(V, 3) for V in w["stiffness"]])
    errs = []
    for N in (16, 32):
        L = Lattice(np.diag([N, N, N]).tolist())
        ph = synth.coated_ellipsoid_phase(L.p, L.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
        r = basic_scheme(L, ph, S, w["C0"], w["eps0"], tol=1e-6, maxit=300)
        errs.append(np.linalg.norm(r["sigma_bar"] - w["ceff_eps0"]) / np.linalg.norm(w["ceff_eps0"]))
        assert np.abs(r["eps"].mean(axis=0) - w["eps0"]).max() < 1e-12
    assert errs[1] < errs[0] < 0.05
