"""Learned warm start for the lattice Basic Scheme: binding of the lat_wsnet_* entry points and the
training loop (argument marshalling and orchestration; every layer runs in liblatms).

The network predicts the strain-localization field A of a cubic tensor grid from its stiffness
field; eps^(0) = A : E starts basic_scheme_solve, which then runs to the same tolerance as a cold
start and so checks the prediction.  Training data are plain-scheme solutions of seeded random
ellipsoidal-inclusion microstructures.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from .api import _check, _stream, lib

N_PARAMS_CONV = 27 * 32 * 32 + 32


def _L():
    L = lib()
    vp, cvp = ctypes.c_void_p, ctypes.c_void_p
    L.lat_wsnet_param_bytes.restype = ctypes.c_size_t
    L.lat_wsnet_num_params.restype = ctypes.c_int64
    L.lat_wsnet_work_bytes.argtypes = [ctypes.c_int]
    L.lat_wsnet_work_bytes.restype = ctypes.c_size_t
    L.lat_wsnet_set_params.argtypes = [vp, ctypes.POINTER(ctypes.c_float), cvp]
    L.lat_wsnet_get_params.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), cvp]
    L.lat_wsnet_features.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_size_t, cvp]
    L.lat_wsnet_forward.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_size_t, cvp]
    L.lat_wsnet_backward.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_size_t, cvp]
    L.lat_wsnet_train_step.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), vp, ctypes.c_size_t, cvp]
    L.lat_wsnet_predict.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, vp, vp,
                                    ctypes.c_size_t, cvp]
    L.lattice_start_filter.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_size_t, cvp]
    L.lattice_start_filter.restype = ctypes.c_int
    L.lat_wsnet_get_activation.argtypes = [vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_float), cvp]
    for f in ("lat_wsnet_get_activation", "lat_wsnet_set_params", "lat_wsnet_get_params", "lat_wsnet_features", "lat_wsnet_forward",
              "lat_wsnet_backward", "lat_wsnet_train_step", "lat_wsnet_predict"):
        getattr(L, f).restype = ctypes.c_int
    return L


def feature_table(stiffness, mu0):
    """Per phase the 21 upper-triangle Voigt entries / mu0 (float32, flattened)."""
    iu = np.triu_indices(6)
    return np.ascontiguousarray(np.array([np.asarray(V)[iu] for V in stiffness], dtype=np.float32) / np.float32(mu0))


class WarmStartNet:
    """Parameters (device) of the warm-start U-Net plus a work buffer per grid size."""

    def __init__(self, device, seed=0, params=None):
        import torch
        self.L = _L()
        self.device = device
        self.n_params = int(self.L.lat_wsnet_num_params())
        self.pbuf = torch.zeros(int(self.L.lat_wsnet_param_bytes()), dtype=torch.uint8, device=device)
        self.works = {}
        self.step_count = 0
        self.set_params(self.init_params(seed) if params is None else params)

    def init_params(self, seed):
        rng = np.random.default_rng(seed)
        out = []
        for _ in range(7):
            out.append(rng.standard_normal(27 * 32 * 32) * np.sqrt(2.0 / (27 * 32)))
            out.append(np.zeros(32))
        out.append(np.zeros(32 * 36))      # zero head: training starts from the trivial predictor A' = 0
        out.append(np.zeros(36))
        return np.concatenate(out).astype(np.float32)

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(self.L.lat_wsnet_set_params(ctypes.c_void_p(self.pbuf.data_ptr()),
                                           p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream(None)))
        self.step_count = 0

    def get_params(self, grads=False):
        p = np.empty(self.n_params, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32) if grads else None
        _check(self.L.lat_wsnet_get_params(ctypes.c_void_p(self.pbuf.data_ptr()),
                                           p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if grads else None,
                                           _stream(None)))
        return (p, g) if grads else p

    def work(self, n):
        import torch
        if n not in self.works:
            nb = int(self.L.lat_wsnet_work_bytes(n))
            if nb == 0:
                raise ValueError("grid size %d not supported (16..256, divisible by 8)" % n)
            self.works[n] = torch.empty(nb, dtype=torch.uint8, device=self.device)
        return self.works[n]

    def _w(self, n):
        w = self.work(n)
        return ctypes.c_void_p(w.data_ptr()), w.numel()

    def _arg(self, t, name, dtype, numel=None, per=None):
        """A device argument of the network's kernels: contiguous, on the parameters' device, of the given
        type and number of entries (numel, or a positive multiple of per); the kernels get its raw pointer."""
        import torch
        ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.device == self.pbuf.device and t.is_contiguous()
              and t.dtype == dtype and (numel is None or t.numel() == numel)
              and (per is None or (t.numel() > 0 and t.numel() % per == 0)))
        if not ok:
            raise TypeError("%s must be a contiguous %s CUDA tensor on %s%s" % (
                name, dtype, self.pbuf.device, "" if numel is None else " with %d entries" % numel))
        return t

    def features(self, phase, table, n):
        import torch
        self._arg(phase, "phase", torch.uint8, n ** 3)
        tab = torch.from_numpy(np.ascontiguousarray(table, dtype=np.float32).reshape(-1)).to(self.device)
        w, nb = self._w(n)
        _check(self.L.lat_wsnet_features(ctypes.c_void_p(phase.data_ptr()), ctypes.c_void_p(tab.data_ptr()), n, w, nb,
                                         _stream(None)))

    def forward(self, n):
        import torch
        y = torch.empty((n ** 3, 36), dtype=torch.float32, device=self.device)
        w, nb = self._w(n)
        _check(self.L.lat_wsnet_forward(ctypes.c_void_p(self.pbuf.data_ptr()), n, ctypes.c_void_p(y.data_ptr()), w,
                                        nb, _stream(None)))
        return y

    def backward(self, n, dy):
        import torch
        w, nb = self._w(n)
        dy = self._arg(dy.contiguous(), "dy", torch.float32, 36 * n ** 3)
        _check(self.L.lat_wsnet_backward(ctypes.c_void_p(self.pbuf.data_ptr()), n, ctypes.c_void_p(dy.data_ptr()), w,
                                         nb, _stream(None)))

    def train_step(self, phase, table_dev, eps_unit, n, lr):
        import torch
        self._arg(phase, "phase", torch.uint8, n ** 3)
        self._arg(table_dev, "table_dev", torch.float32, per=21)
        self._arg(eps_unit, "eps_unit", torch.float64, 36 * n ** 3)
        self.step_count += 1
        loss = ctypes.c_double()
        w, nb = self._w(n)
        _check(self.L.lat_wsnet_train_step(ctypes.c_void_p(self.pbuf.data_ptr()), ctypes.c_void_p(phase.data_ptr()),
                                           ctypes.c_void_p(table_dev.data_ptr()), ctypes.c_void_p(eps_unit.data_ptr()),
                                           n, float(lr), self.step_count, ctypes.byref(loss), w, nb, _stream(None)))
        return loss.value

    ACT = {"x0": 0, "s0": 1, "s1": 2, "s2": 3, "s3": 4, "p1": 5, "p2": 6, "p3": 7, "i0": 8, "u0": 9, "i1": 10,
           "u1": 11, "i2": 12, "u2": 13}

    def activation(self, n, name):
        """A forward activation (host float32, shape (n_l^3, 32)) of the last forward pass at size n."""
        which = self.ACT[name]
        level = 0 if which in (0, 1, 8, 9) else {2: 1, 5: 1, 10: 1, 11: 1, 3: 2, 6: 2, 12: 2, 13: 2}.get(which, 3)
        out = np.empty(((n >> level) ** 3, 32), dtype=np.float32)
        w, nb = self._w(n)
        _check(self.L.lat_wsnet_get_activation(w, nb, n, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               _stream(None)))
        return out

    def predict(self, phase, table_dev, n, E):
        import torch
        self._arg(phase, "phase", torch.uint8, n ** 3)
        self._arg(table_dev, "table_dev", torch.float32, per=21)
        E = np.ascontiguousarray(np.asarray(E, dtype=np.float64).reshape(-1, 6))
        eps0 = torch.empty((E.shape[0], 6, n ** 3), dtype=torch.float64, device=self.device)
        w, nb = self._w(n)
        _check(self.L.lat_wsnet_predict(ctypes.c_void_p(self.pbuf.data_ptr()), ctypes.c_void_p(phase.data_ptr()),
                                        ctypes.c_void_p(table_dev.data_ptr()), n,
                                        E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), E.shape[0],
                                        ctypes.c_void_p(eps0.data_ptr()), w, nb, _stream(None)))
        return eps0


def random_microstructure(seed, n, device, contrast_log10=(-1.0, 2.0)):
    """Seeded two-phase ellipsoidal-inclusion microstructure on the n^3 grid (phase ids, materials, C0).

    Generated on the GPU with torch (input generation only): 1-8 periodic ellipsoids, volume
    fraction U(0.05, 0.4), inclusion Lame constants lam = mu = 10^U(contrast_log10), matrix (1, 1).
    """
    import torch
    from . import synth
    rng = np.random.default_rng(seed)
    n_incl = int(rng.integers(1, 9))
    incl = synth.random_inclusions(int(rng.integers(1 << 30)), 3, n_incl, float(rng.uniform(0.05, 0.4)))
    g = torch.arange(n, device=device, dtype=torch.float64) / n
    Z, Y, X = torch.meshgrid(g, g, g, indexing="ij")
    pts = torch.stack([Z.reshape(-1), Y.reshape(-1), X.reshape(-1)], dim=1)
    ph = torch.zeros(n ** 3, dtype=torch.uint8, device=device)
    for c, a, R in zip(incl["centers"], incl["axes"], incl["rots"]):
        z = pts - torch.as_tensor(c, device=device)
        z = z - torch.round(z)
        zt = z @ torch.as_tensor(R, device=device)
        inside = torch.sum((zt / torch.as_tensor(a, device=device)) ** 2, dim=1) <= 1.0
        ph[inside] = 1
    k = 10.0 ** rng.uniform(*contrast_log10)
    stiff = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(k, k)]
    C0 = synth.c0_mean_extremes([1.0, k], [1.0, k])
    return ph, stiff, C0


UNIT_E = np.diag([1.0, 1.0, 1.0, 0.5, 0.5, 0.5])


def train(net, n, n_samples, steps_per_sample=1, lr=1e-3, seed0=1000, tol=1e-4, log=None):
    """Generate n_samples microstructures, solve the six unit load cases (mixed precision, tol), and take
    Adam steps on each.  Returns the per-sample losses."""
    import torch
    from . import basic_scheme_solve, lattice_plan
    P = lattice_plan(np.diag([n, n, n]).tolist())
    eps = torch.empty((6, 6, n ** 3), dtype=torch.float64, device=net.device)
    ws = torch.empty(P.workspace_bytes(6, 1), dtype=torch.uint8, device=net.device)
    losses = []
    t0 = time.time()
    for s in range(n_samples):
        ph, stiff, C0 = random_microstructure(seed0 + s, n, net.device)
        basic_scheme_solve(P, ph, stiff, C0, UNIT_E, tol=tol, maxit=3000, precision="mixed", workspace=ws,
                           eps_out=eps)
        tab = torch.from_numpy(feature_table(stiff, C0[1]).reshape(-1)).to(net.device)
        for _ in range(steps_per_sample):
            losses.append(net.train_step(ph, tab, eps, n, lr))
        if log and (s % max(1, n_samples // 10) == 0):
            log("sample %d loss %.4e (%.1f s)" % (s, losses[-1], time.time() - t0))
    return losses


def filter_rho(stiffness, C0):
    """Largest |eigenvalue| of C0^-1 (C_p - C0) over the phases (Mandel form): the rate of the slowest error
    components of the iteration, the ones lattice_start_filter removes."""
    from . import synth
    W = np.diag([1.0, 1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0), np.sqrt(2.0)])
    M0 = W @ synth.iso_voigt(*C0) @ W
    L = np.linalg.cholesky(M0)
    Li = np.linalg.inv(L)
    rho = 0.0
    for V in stiffness:
        A = Li @ (W @ np.asarray(V, dtype=np.float64) @ W - M0) @ Li.T
        rho = max(rho, float(np.abs(np.linalg.eigvalsh(0.5 * (A + A.T))).max()))
    return rho


def start_filter(out, eps_g2, eps0, rho):
    """out = (G^2(eps0) - rho^2 eps0) / (1 - rho^2) on device binary64 tensors of equal size (C-ABI kernel)."""
    import torch
    for name, t in (("out", out), ("eps_g2", eps_g2), ("eps0", eps0)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == out.device and t.is_contiguous()
                and t.dtype == torch.float64 and t.numel() == out.numel()):
            raise TypeError("start_filter: %s must be a contiguous float64 CUDA tensor of %d entries on %s"
                            % (name, out.numel(), out.device))
    _check(_L().lattice_start_filter(ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(eps_g2.data_ptr()),
                                     ctypes.c_void_p(eps0.data_ptr()), float(rho), out.numel(), _stream(None)))
    return out


def solve_filtered(plan, phase, stiffness, C0, E, tol=1e-6, maxit=5000, precision="fp64", eps0=None, **kw):
    """basic_scheme_solve from the filtered start (G^2(s) - rho^2 s) / (1 - rho^2), s = eps0 (or E).

    Two plain iterations make the filter; 'iters' counts them too.  The filter keeps the fixed point and
    removes the error components of rate rho (see lattice_start_filter)."""
    import torch
    from . import basic_scheme_solve
    E = np.asarray(E, dtype=np.float64).reshape(-1, 6)
    rho = filter_rho(stiffness, C0)
    if eps0 is None:
        m = int(phase.numel())
        eps0 = torch.from_numpy(E).to(phase.device)[:, :, None].expand(E.shape[0], 6, m).contiguous()
    else:
        eps0 = eps0.to(device=phase.device, dtype=torch.float64).contiguous()
    g2 = basic_scheme_solve(plan, phase, stiffness, C0, E, tol=0.0, maxit=2, precision=precision, eps0=eps0)["eps"]
    start = start_filter(g2, g2, eps0, rho)
    out = basic_scheme_solve(plan, phase, stiffness, C0, E, tol=tol, maxit=maxit, precision=precision, eps0=start,
                             **kw)
    out["iters"] = out["iters"] + 2
    out["rho"] = rho
    return out


def solve_warm(plan, net, phase, stiffness, C0, E, n, tol=1e-6, maxit=5000, precision="fp64", filtered=True,
               fallback=True, **kw):
    """basic_scheme_solve started from the network's prediction eps^(0) = E + A' : E.

    filtered=True passes the prediction through the two-iteration start filter first (a prediction's
    error has components of the slowest rate rho that the exact solution, hence the cold start's error,
    lacks).  The plain scheme runs to the same tolerance; if it does not converge, the cold start is run
    instead (fallback).  'iters' counts every iteration taken, 'warm_used' whether the warm result stands.
    """
    import torch
    from . import basic_scheme_solve
    E = np.asarray(E, dtype=np.float64).reshape(-1, 6)
    tab = torch.from_numpy(feature_table(stiffness, C0[1]).reshape(-1)).to(phase.device)
    eps0 = net.predict(phase, tab, n, E)
    if filtered:
        out = solve_filtered(plan, phase, stiffness, C0, E, tol=tol, maxit=maxit, precision=precision, eps0=eps0,
                             **kw)
    else:
        out = basic_scheme_solve(plan, phase, stiffness, C0, E, tol=tol, maxit=maxit, precision=precision,
                                 eps0=eps0, **kw)
    out["warm_used"] = True
    if fallback and out["status"] != 0:
        spent = out["iters"]
        out = basic_scheme_solve(plan, phase, stiffness, C0, E, tol=tol, maxit=maxit, precision=precision, **kw)
        out["iters"] = out["iters"] + spent
        out["warm_used"] = False
    return out
