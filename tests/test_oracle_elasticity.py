"""Pins of oracle.elasticity: stiffness, Voigt maps and the Green operator (Sec. 3.1)."""
import numpy as np
import pytest

from oracle import elasticity as el

RNG = np.random.default_rng(3)


def sym(d):
    a = RNG.standard_normal((d, d))
    return a + a.T


@pytest.mark.parametrize("d", [2, 3])
def test_iso_symmetries_and_voigt_roundtrip(d):
    C = el.iso_tensor(1.3, 0.7, d)
    assert np.allclose(C, C.transpose(1, 0, 2, 3)) and np.allclose(C, C.transpose(0, 1, 3, 2))
    assert np.allclose(C, C.transpose(2, 3, 0, 1))
    assert np.allclose(el.voigt6_to_tensor(el.iso_voigt6(1.3, 0.7), d), C)
    C3 = el.iso_tensor(1.3, 0.7, 3)
    assert np.allclose(el.tensor_to_voigt6(C3), el.iso_voigt6(1.3, 0.7))
    e = sym(d)
    # C : eps = lam tr(eps) I + 2 mu eps
    assert np.allclose(el.ddot(C, e), 1.3 * np.trace(e) * np.eye(d) + 1.4 * e)
    c = el.sym_to_comps(e)
    assert np.allclose(el.comps_to_sym(c, d), e)


@pytest.mark.parametrize("d", [2, 3])
def test_gamma_closed_form_equals_operator_definition(d):
    for _ in range(10):
        lam0, mu0 = RNG.uniform(0.1, 5), RNG.uniform(0.1, 5)
        C0 = el.iso_tensor(lam0, mu0, d)
        k = RNG.standard_normal(d)
        t = sym(d)
        G = el.gamma_tensor(C0, k)
        ref = np.einsum('ijkl,kl->ij', G, t)
        assert np.abs(el.gamma_iso_apply(k, t, lam0, mu0) - ref).max() < 1e-13
        assert np.abs(el.gamma_general_apply(C0, k, t) - ref).max() < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_gamma_projector_identities(d):
    lam0, mu0 = 2.0, 0.8
    C0 = el.iso_tensor(lam0, mu0, d)
    for _ in range(10):
        k = RNG.standard_normal(d)
        G = el.gamma_tensor(C0, k)
        # Gamma0 : C0 : Gamma0 = Gamma0
        assert np.abs(np.einsum('ijab,abcd,cdkl->ijkl', G, C0, G) - G).max() < 1e-12
        # compatible strains sym(a (x) k) are reproduced by Gamma0 : C0
        a = RNG.standard_normal(d)
        s = 0.5 * (np.outer(a, k) + np.outer(k, a))
        assert np.abs(el.gamma_iso_apply(k, el.ddot(C0, s), lam0, mu0) - s).max() < 1e-12
        # equilibrated stresses (sigma k = 0) are annihilated
        P = np.eye(d) - np.outer(k, k) / k.dot(k)
        sig = P @ sym(d) @ P
        assert np.abs(el.gamma_iso_apply(k, sig, lam0, mu0)).max() < 1e-12
        # symmetries and homogeneity of degree 0
        assert np.allclose(G, G.transpose(1, 0, 2, 3)) and np.allclose(G, G.transpose(2, 3, 0, 1))
        assert np.allclose(el.gamma_tensor(C0, 3.7 * k), G) and np.allclose(el.gamma_tensor(C0, -k), G)
