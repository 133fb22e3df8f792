"""Pins of the warm-start network reference (oracle/warmstart.py): the forward convolution against
scipy's periodic correlation, and every gradient against central finite differences."""
import numpy as np
import pytest

from oracle import warmstart as ws


def test_conv3_is_periodic_correlation():
    from scipy.ndimage import correlate
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 6, 4))
    W = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(2)
    y = ws.conv3(x, W, b)
    for co in range(2):
        ref = np.full(x.shape[1:], b[co])
        for ci in range(3):
            k = W[:, ci, co].reshape(3, 3, 3)          # taps lexicographic in (dz, dy, dx)
            ref += correlate(x[ci], k, mode='wrap')
        assert np.abs(y[co] - ref).max() < 1e-12


def _fd_check(f, x, grad, n=6, h=1e-6, seed=1):
    rng = np.random.default_rng(seed)
    flat = x.reshape(-1)
    g = grad.reshape(-1)
    for i in rng.choice(flat.size, size=n, replace=False):
        old = flat[i]
        flat[i] = old + h
        fp = f()
        flat[i] = old - h
        fm = f()
        flat[i] = old
        assert abs((fp - fm) / (2 * h) - g[i]) < 1e-6 * max(1.0, abs(g[i]))


def test_layer_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 4, 4, 4))
    W = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(2)
    R = rng.standard_normal((2, 4, 4, 4))
    loss = lambda: float(np.sum(ws.conv3(x, W, b) * R))
    dx, dW, db = ws.conv3_backward(x, W, R)
    _fd_check(loss, x, dx)
    _fd_check(loss, W, dW)
    _fd_check(loss, b, db, n=2)
    Rp = rng.standard_normal((3, 2, 2, 2))
    _fd_check(lambda: float(np.sum(ws.pool(x) * Rp)), x, ws.pool_backward(Rp))
    Ru = rng.standard_normal((3, 8, 8, 8))
    _fd_check(lambda: float(np.sum(ws.up(x) * Ru)), x, ws.up_backward(Ru))
    H = rng.standard_normal((3, 5))
    hb = rng.standard_normal(5)
    Rh = rng.standard_normal((5, 4, 4, 4))
    dxh, dH, dhb = ws.head_backward(x, H, Rh)
    _fd_check(lambda: float(np.sum(ws.head(x, H, hb) * Rh)), x, dxh)
    _fd_check(lambda: float(np.sum(ws.head(x, H, hb) * Rh)), H, dH)


def test_network_gradient_by_finite_differences():
    p = ws.init_params(3, C=4, cout=5)
    p["head.W"] = np.random.default_rng(9).standard_normal((4, 5))
    # small channel count for speed: convs 4 -> 4
    for k in list(p):
        if k.endswith(".W") and not k.startswith("head"):
            p[k] = p[k][:, :4, :4]
    rng = np.random.default_rng(4)
    x0 = rng.standard_normal((4, 8, 8, 8))
    T = rng.standard_normal((5, 8, 8, 8))

    def L():
        y, _ = ws.forward(p, x0)
        return ws.mse(y, T)[0]
    y, cache = ws.forward(p, x0)
    _, dy = ws.mse(y, T)
    g = ws.backward(p, cache, dy)
    for name in ("c0.W", "c3.W", "d1.W", "d0.b", "head.W"):
        _fd_check(L, p[name], g[name], n=4, h=1e-5)


def test_localization_preserves_mean_strain():
    rng = np.random.default_rng(5)
    y = rng.standard_normal((36, 4, 4, 4))
    E = rng.standard_normal(6)
    eps = ws.localization_to_strain(y, E)
    assert np.abs(eps.reshape(6, -1).mean(axis=1) - E).max() < 1e-13


def test_centered_loss_gradient_and_invariances():
    rng = np.random.default_rng(6)
    t = rng.standard_normal((5, 4, 4, 4))
    y = rng.standard_normal((5, 4, 4, 4))
    L, g = ws.centered_rel_loss(y, t)
    _fd_check(lambda: ws.centered_rel_loss(y, t)[0], y, g, n=8, h=1e-6)
    shift = rng.standard_normal((5, 1, 1, 1))
    assert abs(ws.centered_rel_loss(y + shift, t)[0] - L) < 1e-12            # channel means are not trained
    assert ws.centered_rel_loss(t + shift, t)[0] < 1e-14                       # perfect up to the mean
    tc = t - t.mean(axis=(1, 2, 3), keepdims=True)
    zero = ws.centered_rel_loss(np.zeros_like(t), t)[0]
    assert abs(zero - np.sum(tc ** 2) / (np.sum(tc ** 2) + t.size * 1e-6)) < 1e-15   # trivial predictor ~ 1
    assert np.abs(g.mean(axis=(1, 2, 3))).max() < 1e-15


def test_targets_and_strain_reconstruction_agree():
    # a prediction equal to the training targets reproduces every unit load case's strain field
    rng = np.random.default_rng(7)
    E_unit = np.diag([1.0, 1.0, 1.0, 0.5, 0.5, 0.5])
    fluct = rng.standard_normal((6, 6, 3, 4, 5))
    fluct -= fluct.mean(axis=(2, 3, 4), keepdims=True)
    eps_unit = fluct + E_unit[:, :, None, None, None]
    y = ws.localization_targets(eps_unit, E_unit)
    assert y.shape == (36, 3, 4, 5)
    for j in range(6):
        assert np.abs(ws.localization_to_strain(y, E_unit[j]) - eps_unit[j]).max() < 1e-13
    # superposition: a general E is the Voigt combination of the unit cases
    E = rng.standard_normal(6)
    Eu = E.copy()
    Eu[3:] *= 2.0
    ref = np.einsum('j,jixyz->ixyz', Eu, eps_unit)
    assert np.abs(ws.localization_to_strain(y, E) - ref).max() < 1e-12


def test_features_are_the_voigt_upper_triangle_over_mu0():
    # the 21 input channels are the upper triangle of the 6x6 Voigt stiffness (row by row) divided by
    # mu0, then 11 zero channels; written out for isotropic phases (lam, mu): diagonal lam + 2 mu on the
    # normal block, lam off the diagonal of the normal block, mu on the shear diagonal, zero elsewhere
    from oracle.elasticity import iso_voigt6
    mu0 = 2.5
    phases = [(1.0, 3.0), (7.0, 0.5)]
    phase = np.array([[[0, 1], [1, 0]], [[1, 1], [0, 0]]], dtype=np.int64)   # a 2x2x2 grid
    f = ws.features([iso_voigt6(*p) for p in phases], phase, mu0)
    assert f.shape == (32,) + phase.shape
    for q, (lam, mu) in enumerate(phases):
        a, b = (lam + 2 * mu) / mu0, lam / mu0
        s = mu / mu0
        expect = [a, b, b, 0, 0, 0,
                  a, b, 0, 0, 0,
                  a, 0, 0, 0,
                  s, 0, 0,
                  s, 0,
                  s] + [0] * 11
        sel = phase == q
        for c in range(32):
            assert np.all(f[c][sel] == expect[c]), c
