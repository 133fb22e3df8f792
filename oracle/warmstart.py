"""CPU reference of the learned warm-start network (test infrastructure, float64).

Test infrastructure only (see ``oracle/__init__``).  The warm start is not in the
paper: it predicts the strain-localization field A (eps = A : E) from the
stiffness field so that Algorithm 1 can start from eps^(0) = A : E instead of E;
the scheme then runs to the same tolerance and checks the result.

Network (a periodic 3-D U-Net with 4 levels and 32 channels):
    x0 = features (21 stiffness components, zero-padded to 32 channels); relu is leaky (slope 0.1)
    s0 = relu(conv3(x0))                      level 0
    s1 = relu(conv3(pool(s0)))                level 1 (half resolution)
    s2 = relu(conv3(pool(s1)))                level 2
    s3 = relu(conv3(pool(s2)))                level 3
    u2 = relu(conv3(up(s3) + s2))
    u1 = relu(conv3(up(u2) + s1))
    u0 = relu(conv3(up(u1) + s0))
    y  = head(u0)                             1x1x1 convolution to 36 channels
conv3 is a 3x3x3 cross-correlation with periodic wrap-around (the microstructure
is periodic), pool the 2x2x2 average, up the 2x2x2 nearest-neighbour copy.
Arrays are (channels, n0, n1, n2); conv weights W[t, ci, co] with the 27 taps t
in lexicographic order of (dz, dy, dx) in {-1, 0, 1}^3, so that
    conv3(x)[co, v] = b[co] + sum_t sum_ci W[t, ci, co] x[ci, v + offset(t)].
"""
from __future__ import annotations

import numpy as np

TAPS = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]


def shift(x, off):
    """x[:, v + off] with periodic wrap (np.roll moves the other way)."""
    return np.roll(x, shift=(-off[0], -off[1], -off[2]), axis=(1, 2, 3))


def conv3(x, W, b):
    Co = W.shape[2]
    out = np.zeros((Co,) + x.shape[1:])
    for t, off in enumerate(TAPS):
        out += np.einsum('co,cxyz->oxyz', W[t], shift(x, off))
    return out + b[:, None, None, None]


def conv3_backward(x, W, dout):
    """Gradients of conv3 with respect to x, W and b given dL/d(out)."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for t, off in enumerate(TAPS):
        xs = shift(x, off)
        dW[t] = np.einsum('cxyz,oxyz->co', xs, dout)
        # out[v] depends on x[v + off]: dx[u] += W^T dout[u - off]
        dx += shift(np.einsum('co,oxyz->cxyz', W[t], dout), (-off[0], -off[1], -off[2]))
    db = dout.sum(axis=(1, 2, 3))
    return dx, dW, db


LEAK = 0.1


def relu(x):
    """Leaky ReLU: x for x > 0, LEAK x otherwise."""
    return np.where(x > 0, x, LEAK * x)


def relu_grad(y):
    """Derivative of the leaky ReLU in terms of its output (same sign as its input)."""
    return np.where(y > 0, 1.0, LEAK)


def pool(x):
    C, a, b, c = x.shape
    return x.reshape(C, a // 2, 2, b // 2, 2, c // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(dout):
    return np.repeat(np.repeat(np.repeat(dout, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_backward(dout):
    C, a, b, c = dout.shape
    return dout.reshape(C, a // 2, 2, b // 2, 2, c // 2, 2).sum(axis=(2, 4, 6))


def head(x, H, hb):
    return np.einsum('cj,cxyz->jxyz', H, x) + hb[:, None, None, None]


def head_backward(x, H, dout):
    return np.einsum('cj,jxyz->cxyz', H, dout), np.einsum('cxyz,jxyz->cj', x, dout), dout.sum(axis=(1, 2, 3))


CONV_NAMES = ["c0", "c1", "c2", "c3", "d2", "d1", "d0"]


def init_params(seed, C=32, cin=32, cout=36):
    rng = np.random.default_rng(seed)
    p = {}
    for name in CONV_NAMES:
        fan = 27 * C
        p[name + ".W"] = rng.standard_normal((27, C, C)) * np.sqrt(2.0 / fan)
        p[name + ".b"] = np.zeros(C)
    p["head.W"] = np.zeros((C, cout))      # training starts from the trivial predictor A' = 0
    p["head.b"] = np.zeros(cout)
    return p


def forward(p, x0):
    """Network forward; returns (y, cache)."""
    cache = {"x0": x0}
    s0 = relu(conv3(x0, p["c0.W"], p["c0.b"]))
    p1 = pool(s0)
    s1 = relu(conv3(p1, p["c1.W"], p["c1.b"]))
    p2 = pool(s1)
    s2 = relu(conv3(p2, p["c2.W"], p["c2.b"]))
    p3 = pool(s2)
    s3 = relu(conv3(p3, p["c3.W"], p["c3.b"]))
    i2 = up(s3) + s2
    u2 = relu(conv3(i2, p["d2.W"], p["d2.b"]))
    i1 = up(u2) + s1
    u1 = relu(conv3(i1, p["d1.W"], p["d1.b"]))
    i0 = up(u1) + s0
    u0 = relu(conv3(i0, p["d0.W"], p["d0.b"]))
    y = head(u0, p["head.W"], p["head.b"])
    cache.update(s0=s0, p1=p1, s1=s1, p2=p2, s2=s2, p3=p3, s3=s3, i2=i2, u2=u2, i1=i1, u1=u1, i0=i0, u0=u0)
    return y, cache


def backward(p, cache, dy):
    """Gradients of all parameters given dL/dy (reverse of ``forward``)."""
    g = {}
    c = cache
    du0, g["head.W"], g["head.b"] = head_backward(c["u0"], p["head.W"], dy)
    di0, g["d0.W"], g["d0.b"] = conv3_backward(c["i0"], p["d0.W"], du0 * relu_grad(c["u0"]))
    ds0 = di0.copy()
    du1 = up_backward(di0)
    di1, g["d1.W"], g["d1.b"] = conv3_backward(c["i1"], p["d1.W"], du1 * relu_grad(c["u1"]))
    ds1 = di1.copy()
    du2 = up_backward(di1)
    di2, g["d2.W"], g["d2.b"] = conv3_backward(c["i2"], p["d2.W"], du2 * relu_grad(c["u2"]))
    ds2 = di2.copy()
    ds3 = up_backward(di2)
    dp3, g["c3.W"], g["c3.b"] = conv3_backward(c["p3"], p["c3.W"], ds3 * relu_grad(c["s3"]))
    ds2 = ds2 + pool_backward(dp3)
    dp2, g["c2.W"], g["c2.b"] = conv3_backward(c["p2"], p["c2.W"], ds2 * relu_grad(c["s2"]))
    ds1 = ds1 + pool_backward(dp2)
    dp1, g["c1.W"], g["c1.b"] = conv3_backward(c["p1"], p["c1.W"], ds1 * relu_grad(c["s1"]))
    ds0 = ds0 + pool_backward(dp1)
    _, g["c0.W"], g["c0.b"] = conv3_backward(c["x0"], p["c0.W"], ds0 * relu_grad(c["s0"]))
    return g


def mse(y, target):
    """Mean squared error over all entries and its gradient."""
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def localization_targets(eps_unit, E_unit):
    """Training targets (36, ...) from the strains of the six unit load cases.

    eps_unit[j, i] is component i (Voigt order, tensor components) of the strain field of unit load
    case j and E_unit[j, i] its mean; channel 6 i + j of the result is eps_unit[j, i] - E_unit[j, i].
    """
    eps_unit = np.asarray(eps_unit, dtype=np.float64)
    t = eps_unit - np.asarray(E_unit, dtype=np.float64).reshape(6, 6, *([1] * (eps_unit.ndim - 2)))
    return t.transpose(1, 0, *range(2, eps_unit.ndim)).reshape((36,) + eps_unit.shape[2:])


def centered_rel_loss(y, t, eps0=1e-6):
    """Training loss: relative squared error of the zero-mean parts of y and t, and dL/dy.

    L = sum (y~ - t~)^2 / (sum t~^2 + N eps0), with x~ = x minus its mean over space in each channel
    (axis 0 holds channels) and N the number of entries.  The mean of a prediction is discarded when
    it is used (<A'> = 0), so it is not trained.  Because y~ - t~ has zero mean in each channel, the
    gradient 2 (y~ - t~) / den is already the projection of dL/dy~ onto mean-free fields.
    """
    ax = tuple(range(1, y.ndim))
    yc = y - y.mean(axis=ax, keepdims=True)
    tc = t - t.mean(axis=ax, keepdims=True)
    den = float(np.sum(tc * tc)) + tc.size * eps0
    d = yc - tc
    return float(np.sum(d * d)) / den, 2.0 * d / den


def features(stiff_voigt, phase, mu0):
    """21 upper-triangle Voigt components of C(y) / mu0, zero-padded to 32 channels, shape (32, n0, n1, n2)."""
    iu = np.triu_indices(6)
    vals = np.array([np.asarray(V)[iu] for V in stiff_voigt]) / mu0     # (n_phases, 21)
    f = vals[phase.reshape(-1)].T                                         # (21, m)
    out = np.zeros((32,) + phase.shape)
    out[:21] = f.reshape((21,) + phase.shape)
    return out


def localization_to_strain(y, E):
    """eps = (I + A') : E with A' the network output after mean removal; y (36, ...) -> eps (6, ...).

    Channel 6 i + j holds A'_{ij}: the tensor component i of the strain of unit load case j
    (Voigt order, tensor components; unit shear load cases carry eps_ij = 1/2).
    """
    A = y.reshape(6, 6, -1)
    A = A - A.mean(axis=2, keepdims=True)          # <A'> = 0, hence <eps> = E exactly
    Eu = np.asarray(E, dtype=np.float64).copy()
    Eu[3:] *= 2.0                                    # E as combination of the unit load cases
    eps = np.einsum('ijm,j->im', A, Eu) + np.asarray(E)[:, None]
    return eps.reshape((6,) + y.shape[1:])
