"""Python binding of liblatms (ctypes): argument marshalling only.

Every step of the lattice Basic Scheme runs in the CUDA library; this module
allocates device buffers with torch (plumbing), passes raw pointers and the
current CUDA stream through the C ABI of ``include/lattice_ms.h`` and turns
status codes into exceptions.  There is no CPU fallback: if the shared
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB

LAT_OK, LAT_NOT_CONVERGED, LAT_DIVERGED = 0, 1, 2
LAT_ERR_ARG = -1
LAT_SCHEME_BASIC, LAT_SCHEME_EYRE_MILTON, LAT_SCHEME_CG = 0, 1, 2
_SCHEMES = {"basic": LAT_SCHEME_BASIC, "eyre_milton": LAT_SCHEME_EYRE_MILTON, "cg": LAT_SCHEME_CG}
LAT_WS_CG = 256   # OR into the precision of a workspace query: room for the conjugate-gradient vectors
LAT_FP64, LAT_MIXED, LAT_DF64 = 0, 1, 2
LAT_BOUNDARY_AVERAGE, LAT_BOUNDARY_ZERO = 0, 1
HIST_CAP = 4096
BATCH_MAX_PHASES = 16

_lib = None


class LatticeError(RuntimeError):
    """A negative status returned by liblatms."""

    def __init__(self, code, msg):
        super().__init__("liblatms error %d: %s" % (code, msg))
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("boundary", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("resid_history", ctypes.POINTER(ctypes.c_double)),
                ("mixed_increment", ctypes.c_int), ("mixed_restart", ctypes.c_int),
                ("plain_launches", ctypes.c_int), ("scheme", ctypes.c_int)]


def lib():
    """Load liblatms.so (built in-tree by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError("liblatms.so is not built (%s); run __graft_entry__.build()" % LIB)
    L = ctypes.CDLL(LIB)
    vp, i64p, i32p, f64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int), \
        ctypes.POINTER(ctypes.c_double)
    L.lattice_plan.argtypes = [i64p, ctypes.c_int, ctypes.POINTER(vp)]
    L.lattice_plan.restype = ctypes.c_int
    L.lattice_plan_destroy.argtypes = [vp]
    L.lattice_plan_destroy.restype = None
    L.lattice_plan_info.argtypes = [vp, i64p, i32p, i64p]
    L.lattice_points.argtypes = [vp, i64p]
    L.lattice_freqs.argtypes = [vp, i64p]
    L.lattice_last_error.restype = ctypes.c_char_p
    L.lattice_fft_workspace_bytes.argtypes = [vp, ctypes.c_int]
    L.lattice_fft_workspace_bytes.restype = ctypes.c_size_t
    L.lattice_fft.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, vp]
    L.lattice_workspace_bytes.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.lattice_workspace_bytes.restype = ctypes.c_size_t
    L.basic_scheme_solve.argtypes = [vp, vp, ctypes.c_int, f64p, f64p, f64p, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.POINTER(_Opts), vp, vp, f64p, i32p, f64p, vp,
                                     ctypes.c_size_t, vp]
    for f in ("lattice_plan", "lattice_plan_info", "lattice_points", "lattice_freqs", "lattice_fft",
              "basic_scheme_solve"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc < 0:
        raise LatticeError(rc, lib().lattice_last_error().decode())
    return rc


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _on_device(t, device):
    """True for a contiguous tensor on the given CUDA device: the kernels receive its raw pointer, so a
    host tensor, a tensor of another device or a strided view must not reach them."""
    import torch
    return isinstance(t, torch.Tensor) and t.is_cuda and t.device == device and t.is_contiguous()


def _strain_buffer(t, name, numel, device):
    """A caller's strain (or stress) buffer: float64, numel entries, on the solve's device."""
    import torch
    if not (_on_device(t, device) and t.dtype == torch.float64 and t.numel() == numel):
        raise TypeError("%s must be a contiguous float64 CUDA tensor of %d entries on %s" % (name, numel, device))
    return t


def _fill_start(eps, eps0, numel):
    """Copy a warm start (any device, float64, numel entries) into the solve's strain buffer."""
    import torch
    if not (isinstance(eps0, torch.Tensor) and eps0.dtype == torch.float64 and eps0.numel() == numel):
        raise TypeError("eps0 must be a float64 tensor of %d entries (n_loads, n_c, m)" % numel)
    eps.view(-1).copy_(eps0.reshape(-1))


def _workspace(t, nbytes, device):
    """The caller's workspace (a contiguous CUDA tensor on the solve's device, any dtype) or a new uint8
    one of nbytes; returns the tensor and its size in bytes (the library checks that it suffices)."""
    import torch
    if t is None:
        t = torch.empty(nbytes, dtype=torch.uint8, device=device)
    elif not _on_device(t, device):
        raise TypeError("workspace must be a contiguous CUDA tensor on %s" % device)
    return t, t.numel() * t.element_size()


class LatticePlan:
    """Plan for the pattern P(M) of a regular integer matrix M (d = 2 or 3)."""

    def __init__(self, M):
        M = np.asarray(M, dtype=np.int64)
        if M.ndim != 2 or M.shape[0] != M.shape[1]:
            raise ValueError("M must be square")
        self.M = M.copy()
        self.d = M.shape[0]
        self._h = ctypes.c_void_p()
        Mc = np.ascontiguousarray(M)
        _check(lib().lattice_plan(Mc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), self.d,
                                  ctypes.byref(self._h)))
        m = ctypes.c_int64()
        dM = ctypes.c_int()
        div = (ctypes.c_int64 * 3)()
        _check(lib().lattice_plan_info(self._h, ctypes.byref(m), ctypes.byref(dM), div))
        self.m = m.value
        self.d_M = dM.value
        self.divisors = [div[i] for i in range(self.d)]
        self.n_c = self.d * (self.d + 1) // 2

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.lattice_plan_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def points(self):
        """(m, d) int64 numerators p of the pattern points y = p / m, in plan order."""
        p = np.empty((self.m, self.d), dtype=np.int64)
        _check(lib().lattice_points(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return p

    def freqs(self):
        """(m, d) int64 frequencies h in G(M^T), in the spectral order of lattice_fft."""
        h = np.empty((self.m, self.d), dtype=np.int64)
        _check(lib().lattice_freqs(self._h, h.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return h

    def set_cell(self, L=None):
        """Transformed pattern P_L(M) (Sec. 3.3): the cell is L [-1/2, 1/2)^d, the point y sits at
        x = L y and the Green operator is evaluated at L^{-T} h (lattice_plan_set_cell); None resets."""
        f = lib().lattice_plan_set_cell
        f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        f.restype = ctypes.c_int
        if L is None:
            _check(f(self._h, None))
            return
        a, ap = _f64(np.asarray(L, dtype=np.float64).reshape(self.d, self.d))
        _check(f(self._h, ap))

    def layout(self):
        """The FFT decomposition of the plan (lattice_plan_layout): dict(ax_len, groups, split); the last
        logical axis is the contiguous row, group g covers logical axes [a0, a1) and group 0 applies
        the Green operator."""
        f = lib().lattice_plan_layout
        f.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 5
        f.restype = ctypes.c_int
        nax, ng, split = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ax = (ctypes.c_int * 6)()
        grp = (ctypes.c_int * 6)()
        _check(f(self._h, ctypes.byref(nax), ax, ctypes.byref(ng), grp, ctypes.byref(split)))
        return dict(ax_len=[ax[i] for i in range(nax.value)],
                    groups=[(grp[2 * g], grp[2 * g + 1]) for g in range(ng.value)], split=split.value)

    def workspace_bytes(self, n_loads=1, precision=LAT_FP64):
        return int(lib().lattice_workspace_bytes(self._h, n_loads, precision))

    def autotune(self, n_items=1, precision="fp64", stream=None):
        """Time the launch shapes of a solve with n_items items and keep the fastest in the plan
        (lattice_autotune).  Returns tune_info(n_items, precision)."""
        import torch
        prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
        L = lib()
        L.lattice_autotune_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.lattice_autotune_workspace_bytes.restype = ctypes.c_size_t
        nb = int(L.lattice_autotune_workspace_bytes(self._h, n_items, prec))
        if nb == 0:
            raise LatticeError(LAT_ERR_ARG, "lattice_autotune_workspace_bytes: unsupported plan or arguments")
        ws = torch.empty(nb, dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
        L.lattice_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_void_p]
        L.lattice_autotune.restype = ctypes.c_int
        _check(L.lattice_autotune(self._h, n_items, prec, ctypes.c_void_p(ws.data_ptr()), nb, _stream(stream)))
        return self.tune_info(n_items, precision)

    def tune_info(self, n_items=1, precision="fp64"):
        """dict(rpc, w, ms) of the tuned bucket, or None if it is not tuned."""
        prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
        rpc = ctypes.c_int(0)
        ng = ctypes.c_int(0)
        w = (ctypes.c_int * 3)()
        ms = (ctypes.c_float * 4)()
        L = lib()
        L.lattice_tune_info.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_int)]
        L.lattice_tune_info.restype = ctypes.c_int
        r = _check(L.lattice_tune_info(self._h, n_items, prec, ctypes.byref(rpc), w, ms, ctypes.byref(ng)))
        if r == 0:
            return None
        return dict(rpc=rpc.value, w=[w[k] for k in range(ng.value)], ms=[ms[k] for k in range(1 + ng.value)])


def lattice_plan(M):
    return LatticePlan(M)


def lattice_fft(plan, x, inverse=False, stream=None):
    """Pattern DFT F(M) (forward, with 1/m) or its inverse of complex128 CUDA data (n_fields, m)."""
    import torch
    if x.dtype != torch.complex128 or not x.is_cuda or x.numel() == 0 or x.numel() % plan.m:
        raise TypeError("x must be a complex128 CUDA tensor of n_fields x m entries")
    x = x.contiguous()
    n_f = x.numel() // plan.m
    out = torch.empty_like(x)
    L = lib()
    L.lattice_fft_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.lattice_fft_workspace_bytes.restype = ctypes.c_size_t
    nb = int(L.lattice_fft_workspace_bytes(plan.handle, n_f))
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=x.device) if nb else None
    _check(L.lattice_fft(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n_f,
                         1 if inverse else 0, ctypes.c_void_p(ws.data_ptr()) if ws is not None else None, nb,
                         _stream(stream)))
    return out


def basic_scheme_solve(plan, phase, stiffness, C0, E, tol=1e-8, maxit=1000, precision="fp64",
                       boundary="average", eps0=None, want_sigma=False, history=False, workspace=None,
                       eps_out=None, stream=None, mixed_increment=True, plain_launches=False,
                       mixed_restart=True, scheme="basic"):
    """Algorithm 1 on the GPU.  Returns a dict of torch/numpy results.

    scheme     "basic" (Algorithm 1), "eyre_milton" (accelerated fixed point, same discrete solution at
               the same C0) or "cg" (conjugate gradients; fp64/df64, cold start, boundary "zero" on
               lattices with an even largest divisor)

    phase      uint8 CUDA tensor (m,), plan order
    stiffness  (n_phases, 6, 6) Voigt matrices (host)
    C0         (lam0, mu0)
    E          (n_loads, n_c) tensor components (host)
    eps0       optional float64 tensor of n_loads x n_c x m entries (n_loads, n_c, m): warm start, copied
               into the strain buffer (any device, any strides)
    eps_out    optional strain buffer: a contiguous float64 CUDA tensor of n_loads x n_c x m entries on
               the phase field's device (refused otherwise: the kernels get its raw pointer)
    workspace  optional contiguous CUDA tensor on the same device, any dtype (its size in bytes counts)
    """
    import torch
    stiff, stiff_p = _f64(np.asarray(stiffness, dtype=np.float64).reshape(-1, 36))
    n_ph = stiff.shape[0]
    C0a, C0p = _f64(np.asarray(C0, dtype=np.float64).reshape(2))
    E = np.asarray(E, dtype=np.float64).reshape(-1, plan.n_c)
    n_loads = E.shape[0]
    Ea, Ep = _f64(E)
    prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
    bnd = {"average": LAT_BOUNDARY_AVERAGE, "zero": LAT_BOUNDARY_ZERO}[boundary]
    if phase.dtype != torch.uint8 or not phase.is_cuda or not phase.is_contiguous() or phase.numel() != plan.m:
        raise TypeError("phase must be a uint8 CUDA tensor with m entries")
    dev = phase.device
    numel = n_loads * plan.n_c * plan.m
    if eps_out is not None:
        eps = _strain_buffer(eps_out, "eps_out", numel, dev)
    else:
        eps = torch.empty((n_loads, plan.n_c, plan.m), dtype=torch.float64, device=dev)
    if eps0 is not None:
        _fill_start(eps, eps0, numel)
    sigma = torch.empty_like(eps) if want_sigma else None
    wsb = plan.workspace_bytes(n_loads, prec | (LAT_WS_CG if scheme == "cg" else 0))
    ws, wsn = _workspace(workspace, wsb, dev)
    sbar = np.zeros((n_loads, plan.n_c))
    iters = np.zeros(n_loads, dtype=np.int32)
    resid = np.zeros(n_loads)
    hist = np.zeros((n_loads, max(maxit, 1))) if history else None
    opts = _Opts(prec, bnd, 1 if eps0 is not None else 0,
                 hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if history else None,
                 1 if mixed_increment else 0, 0 if mixed_restart else -1, 1 if plain_launches else 0,
                 _SCHEMES[scheme])
    rc = lib().basic_scheme_solve(
        plan.handle, ctypes.c_void_p(phase.data_ptr()), n_ph, stiff_p, C0p, Ep, n_loads, float(tol), int(maxit),
        ctypes.byref(opts), ctypes.c_void_p(eps.data_ptr()),
        ctypes.c_void_p(sigma.data_ptr()) if sigma is not None else None,
        sbar.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(ws.data_ptr()), wsn,
        _stream(stream))
    _check(rc)
    out = dict(status=rc, eps=eps, sigma=sigma, sigma_bar=sbar, iters=iters, resid=resid)
    if history:
        out["history"] = [hist[i, :min(int(iters[i]), maxit, HIST_CAP)] for i in range(n_loads)]
    return out


VOIGT_TRIU = [(i, j) for i in range(6) for j in range(i, 6)]   # plane order of a stiffness field


def voigt_field(voigts):
    """(m, 6, 6) per-point Voigt matrices -> the (21, m) plane layout of basic_scheme_solve_field."""
    v = np.asarray(voigts, dtype=np.float64)
    return np.ascontiguousarray(np.stack([v[:, i, j] for i, j in VOIGT_TRIU]))


def basic_scheme_solve_field(plan, field, C0, E, tol=1e-8, maxit=1000, precision="fp64", boundary="average",
                             eps0=None, want_sigma=False, history=False, workspace=None, eps_out=None, stream=None,
                             mixed_increment=True, mixed_restart=True, plain_launches=False):
    """Algorithm 1 with a per-point stiffness field (basic_scheme_solve_field).

    field  float64 CUDA tensor (21, m): plane p = upper-triangle entry p of each point's 6x6 Voigt matrix
           in plan order (voigt_field builds it from (m, 6, 6) matrices)
    Other arguments and the returned dict as for basic_scheme_solve.
    """
    import torch
    if field.dtype != torch.float64 or not field.is_cuda or tuple(field.shape) != (21, plan.m):
        raise TypeError("field must be a float64 CUDA tensor of shape (21, m)")
    field = field.contiguous()
    C0a, C0p = _f64(np.asarray(C0, dtype=np.float64).reshape(2))
    E = np.asarray(E, dtype=np.float64).reshape(-1, plan.n_c)
    n_loads = E.shape[0]
    Ea, Ep = _f64(E)
    prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
    bnd = {"average": LAT_BOUNDARY_AVERAGE, "zero": LAT_BOUNDARY_ZERO}[boundary]
    dev = field.device
    numel = n_loads * plan.n_c * plan.m
    if eps_out is not None:
        eps = _strain_buffer(eps_out, "eps_out", numel, dev)
    else:
        eps = torch.empty((n_loads, plan.n_c, plan.m), dtype=torch.float64, device=dev)
    if eps0 is not None:
        _fill_start(eps, eps0, numel)
    sigma = torch.empty_like(eps) if want_sigma else None
    L = lib()
    L.lattice_field_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    L.lattice_field_workspace_bytes.restype = ctypes.c_size_t
    wsb = int(L.lattice_field_workspace_bytes(plan.handle, n_loads, prec))
    ws, wsn = _workspace(workspace, wsb, dev)
    sbar = np.zeros((n_loads, plan.n_c))
    iters = np.zeros(n_loads, dtype=np.int32)
    resid = np.zeros(n_loads)
    hist = np.zeros((n_loads, max(maxit, 1))) if history else None
    opts = _Opts(prec, bnd, 1 if eps0 is not None else 0,
                 hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if history else None,
                 1 if mixed_increment else 0, 0 if mixed_restart else -1, 1 if plain_launches else 0,
                 LAT_SCHEME_BASIC)
    f = L.basic_scheme_solve_field
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp] + [ctypes.POINTER(ctypes.c_double)] * 2 + \
        [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Opts), vp, vp,
         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), vp,
         ctypes.c_size_t, vp]
    f.restype = ctypes.c_int
    rc = f(plan.handle, vp(field.data_ptr()), C0p, Ep, n_loads, float(tol), int(maxit), ctypes.byref(opts),
           vp(eps.data_ptr()), vp(sigma.data_ptr()) if sigma is not None else None,
           sbar.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
           resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), vp(ws.data_ptr()), wsn, _stream(stream))
    _check(rc)
    out = dict(status=rc, eps=eps, sigma=sigma, sigma_bar=sbar, iters=iters, resid=resid)
    if history:
        out["history"] = [hist[i, :min(int(iters[i]), maxit, HIST_CAP)] for i in range(n_loads)]
    return out


def basic_scheme_solve_async(plan, phase, stiffness, C0, E, tol=1e-8, maxit=1000, precision="fp64",
                             boundary="average", eps0=None, want_sigma=False, workspace=None, eps_out=None,
                             stream=None, mixed_increment=True, mixed_restart=True, scheme="basic"):
    """Algorithm 1 enqueued on the stream without a host synchronization (basic_scheme_solve_async): returns
    at once with device tensors sigma_bar (n_loads, n_c), iters, resid and status (n_loads) that are valid
    once the stream has passed the solve (e.g. after torch.cuda.synchronize())."""
    import torch
    stiff, stiff_p = _f64(np.asarray(stiffness, dtype=np.float64).reshape(-1, 36))
    n_ph = stiff.shape[0]
    C0a, C0p = _f64(np.asarray(C0, dtype=np.float64).reshape(2))
    E = np.asarray(E, dtype=np.float64).reshape(-1, plan.n_c)
    n_loads = E.shape[0]
    Ea, Ep = _f64(E)
    prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
    bnd = {"average": LAT_BOUNDARY_AVERAGE, "zero": LAT_BOUNDARY_ZERO}[boundary]
    if phase.dtype != torch.uint8 or not phase.is_cuda or not phase.is_contiguous() or phase.numel() != plan.m:
        raise TypeError("phase must be a uint8 CUDA tensor with m entries")
    dev = phase.device
    numel = n_loads * plan.n_c * plan.m
    if eps_out is not None:
        eps = _strain_buffer(eps_out, "eps_out", numel, dev)
    else:
        eps = torch.empty((n_loads, plan.n_c, plan.m), dtype=torch.float64, device=dev)
    if eps0 is not None:
        _fill_start(eps, eps0, numel)
    sigma = torch.empty_like(eps) if want_sigma else None
    wsb = plan.workspace_bytes(n_loads, prec | (LAT_WS_CG if scheme == "cg" else 0))
    ws, wsn = _workspace(workspace, wsb, dev)
    sbar = torch.empty((n_loads, plan.n_c), dtype=torch.float64, device=dev)
    iters = torch.empty(n_loads, dtype=torch.int32, device=dev)
    resid = torch.empty(n_loads, dtype=torch.float64, device=dev)
    status = torch.empty(n_loads, dtype=torch.int32, device=dev)
    opts = _Opts(prec, bnd, 1 if eps0 is not None else 0, None, 1 if mixed_increment else 0,
                 0 if mixed_restart else -1, 0, _SCHEMES[scheme])
    f = lib().basic_scheme_solve_async
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_double)] * 3 + \
        [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Opts), vp, vp, vp, vp, vp, vp, vp,
         ctypes.c_size_t, vp]
    f.restype = ctypes.c_int
    rc = f(plan.handle, vp(phase.data_ptr()), n_ph, stiff_p, C0p, Ep, n_loads, float(tol), int(maxit),
           ctypes.byref(opts), vp(eps.data_ptr()), vp(sigma.data_ptr()) if sigma is not None else None,
           vp(sbar.data_ptr()), vp(iters.data_ptr()), vp(resid.data_ptr()), vp(status.data_ptr()),
           vp(ws.data_ptr()), wsn, _stream(stream))
    _check(rc)
    # the tensors the enqueued work reads or writes are returned so that they outlive it
    return dict(eps=eps, sigma=sigma, sigma_bar=sbar, iters=iters, resid=resid, status=status, workspace=ws)


def lattice_pass_times(plan, phase, stiffness, C0, E, precision="fp64", n_reps=20, stream=None):
    """Average device milliseconds per launch of each kernel of one iteration (profiling helper); E is
    (n_c,) or (n_loads, n_c): the load cases run as one batch, as in basic_scheme_solve."""
    import torch
    stiff, stiff_p = _f64(np.asarray(stiffness, dtype=np.float64).reshape(-1, 36))
    C0a, C0p = _f64(np.asarray(C0, dtype=np.float64).reshape(2))
    Ea, Ep = _f64(np.asarray(E, dtype=np.float64).reshape(-1, plan.n_c))
    n_loads = Ea.shape[0]
    prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
    if phase.dtype != torch.uint8 or not phase.is_cuda or not phase.is_contiguous() or phase.numel() != plan.m:
        raise TypeError("phase must be a contiguous uint8 CUDA tensor with m entries")
    eps = torch.empty((n_loads, plan.n_c, plan.m), dtype=torch.float64, device=phase.device)
    ws = torch.empty(plan.workspace_bytes(n_loads, prec), dtype=torch.uint8, device=phase.device)
    ms = (ctypes.c_float * 8)()
    n = ctypes.c_int()
    L = lib()
    L.lattice_pass_times.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + \
        [ctypes.POINTER(ctypes.c_double)] * 3 + [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]
    L.lattice_pass_times.restype = ctypes.c_int
    _check(L.lattice_pass_times(plan.handle, ctypes.c_void_p(phase.data_ptr()), stiff.shape[0], stiff_p, C0p, Ep,
                                n_loads, prec, int(n_reps), ctypes.c_void_p(eps.data_ptr()),
                                ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream), ms, ctypes.byref(n)))
    return [ms[i] for i in range(n.value)]


def basic_scheme_solve_noalloc(plan, phase, stiffness, C0, E, tol=1e-8, maxit=1000, precision="fp64",
                               boundary="average", eps_out=None, want_sigma=False, stream=None, scheme="basic"):
    """basic_scheme_solve through the no-allocation entry point of the C ABI.

    For callers that cannot allocate device memory inside the call: the library uses its own
    static 16 MiB device scratch array instead of a workspace.  The outputs (eps, sigma) are
    still the caller's: pass ``eps_out`` (float64 CUDA, (n_loads, n_c, m)) to avoid any
    allocation here as well.
    """
    import torch
    stiff, stiff_p = _f64(np.asarray(stiffness, dtype=np.float64).reshape(-1, 36))
    C0a, C0p = _f64(np.asarray(C0, dtype=np.float64).reshape(2))
    E = np.asarray(E, dtype=np.float64).reshape(-1, plan.n_c)
    n_loads = E.shape[0]
    Ea, Ep = _f64(E)
    prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
    bnd = {"average": LAT_BOUNDARY_AVERAGE, "zero": LAT_BOUNDARY_ZERO}[boundary]
    if phase.dtype != torch.uint8 or not phase.is_cuda or not phase.is_contiguous() or phase.numel() != plan.m:
        raise TypeError("phase must be a uint8 CUDA tensor with m entries")
    if eps_out is not None:
        eps = _strain_buffer(eps_out, "eps_out", n_loads * plan.n_c * plan.m, phase.device)
    else:
        eps = torch.empty((n_loads, plan.n_c, plan.m), dtype=torch.float64, device=phase.device)
    sigma = torch.empty_like(eps) if want_sigma else None
    sbar = np.zeros((n_loads, plan.n_c))
    iters = np.zeros(n_loads, dtype=np.int32)
    resid = np.zeros(n_loads)
    opts = _Opts(prec, bnd, 0, None, 1, 0, 1, _SCHEMES[scheme])
    L = lib()
    f = L.basic_scheme_solve_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.POINTER(ctypes.c_double)] * 3 + \
        [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Opts), ctypes.c_void_p, ctypes.c_void_p,
         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
         ctypes.c_void_p]
    f.restype = ctypes.c_int
    rc = f(plan.handle, ctypes.c_void_p(phase.data_ptr()), stiff.shape[0], stiff_p, C0p, Ep, n_loads, float(tol),
           int(maxit), ctypes.byref(opts), ctypes.c_void_p(eps.data_ptr()),
           ctypes.c_void_p(sigma.data_ptr()) if sigma is not None else None,
           sbar.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
           resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream))
    _check(rc)
    return dict(status=rc, eps=eps, sigma=sigma, sigma_bar=sbar, iters=iters, resid=resid)


class _BatchItem(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_void_p), ("n_phases", ctypes.c_int), ("stiffness", ctypes.POINTER(ctypes.c_double)),
                ("C0", ctypes.c_double * 2), ("E", ctypes.POINTER(ctypes.c_double)), ("eps", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p)]


def basic_scheme_solve_batch(plan, phases, stiffnesses, C0s, Es, tol=1e-8, maxit=1000, precision="fp64",
                             boundary="average", want_sigma=False, history=False, workspace=None, eps_out=None,
                             stream=None, mixed_increment=True, plain_launches=False, mixed_restart=True,
                             scheme="basic"):
    """Algorithm 1 for a batch of independent microstructures on one lattice, in one set of launches.

    phases       list of uint8 CUDA tensors (m,)
    stiffnesses  list of (n_phases_i, 6, 6) Voigt matrices (n_phases_i <= 16)
    C0s          list of (lam0, mu0)
    Es           (n_items, n_c) macroscopic strains
    Returns dict(eps (n_items, n_c, m) torch, sigma, sigma_bar, iters, resid, status[, history]).
    """
    import torch
    n = len(phases)
    Es = np.asarray(Es, dtype=np.float64).reshape(n, plan.n_c)
    dev = phases[0].device
    if eps_out is not None:
        eps = _strain_buffer(eps_out, "eps_out", n * plan.n_c * plan.m, dev)
    else:
        eps = torch.empty((n, plan.n_c, plan.m), dtype=torch.float64, device=dev)
    sigma = torch.empty_like(eps) if want_sigma else None
    eps_i = eps.view(n, plan.n_c, plan.m)
    sigma_i = sigma.view(n, plan.n_c, plan.m) if sigma is not None else None
    prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
    bnd = {"average": LAT_BOUNDARY_AVERAGE, "zero": LAT_BOUNDARY_ZERO}[boundary]
    keep = []
    items = (_BatchItem * n)()
    for i in range(n):
        if phases[i].dtype != torch.uint8 or not phases[i].is_cuda or not phases[i].is_contiguous() or \
                phases[i].numel() != plan.m or phases[i].device != dev:
            raise TypeError("phase %d must be a uint8 CUDA tensor with m entries on %s" % (i, dev))
        st_i, st_p = _f64(np.asarray(stiffnesses[i], dtype=np.float64).reshape(-1, 36))
        e_i, e_p = _f64(Es[i])
        keep += [st_i, e_i]
        it = items[i]
        it.phase = phases[i].data_ptr()
        it.n_phases = st_i.shape[0]
        it.stiffness = st_p
        it.C0[0], it.C0[1] = float(C0s[i][0]), float(C0s[i][1])
        it.E = e_p
        it.eps = eps_i[i].data_ptr()
        it.sigma = sigma_i[i].data_ptr() if sigma is not None else None
    L = lib()
    L.lattice_batch_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    L.lattice_batch_workspace_bytes.restype = ctypes.c_size_t
    wsb = int(L.lattice_batch_workspace_bytes(plan.handle, n, prec | (LAT_WS_CG if scheme == "cg" else 0)))
    ws, wsn = _workspace(workspace, wsb, dev)
    sbar = np.zeros((n, plan.n_c))
    iters = np.zeros(n, dtype=np.int32)
    resid = np.zeros(n)
    hist = np.zeros((n, max(maxit, 1))) if history else None
    opts = _Opts(prec, bnd, 0, hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if history else None,
                 1 if mixed_increment else 0, 0 if mixed_restart else -1, 1 if plain_launches else 0,
                 _SCHEMES[scheme])
    f = L.basic_scheme_solve_batch
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(_BatchItem), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                  ctypes.POINTER(_Opts), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                  ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    f.restype = ctypes.c_int
    rc = f(plan.handle, items, n, float(tol), int(maxit), ctypes.byref(opts),
           sbar.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
           resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(ws.data_ptr()), wsn,
           _stream(stream))
    _check(rc)
    out = dict(status=rc, eps=eps, sigma=sigma, sigma_bar=sbar, iters=iters, resid=resid)
    if history:
        out["history"] = [hist[i, :min(int(iters[i]), maxit, HIST_CAP)] for i in range(n)]
    return out


class _MultiItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("phase", ctypes.c_void_p), ("n_phases", ctypes.c_int),
                ("stiffness", ctypes.POINTER(ctypes.c_double)), ("C0", ctypes.c_double * 2),
                ("E", ctypes.POINTER(ctypes.c_double)), ("n_loads", ctypes.c_int), ("eps", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("sigma_bar", ctypes.POINTER(ctypes.c_double)),
                ("iters", ctypes.POINTER(ctypes.c_int)), ("resid", ctypes.POINTER(ctypes.c_double))]


def basic_scheme_solve_multi(problems, tol=1e-8, maxit=1000, precision="fp64", boundary="average",
                             want_sigma=False, workspace=None, stream=None, mixed_increment=True,
                             plain_launches=False, warm_start=False, mixed_restart=True, scheme="basic"):
    """Algorithm 1 for independent problems on different lattices in one call (one CUDA graph).

    problems  list of dicts: plan (LatticePlan), phase (uint8 CUDA tensor (m,)), stiffness
              ((n_phases <= 16, 6, 6) Voigt), C0 (lam0, mu0), E ((n_loads, n_c) tensor components), and
              optionally eps (CUDA float64 (n_loads, n_c, m): output buffer; with warm_start=True it holds
              eps^(0) on entry)
    Returns (status, list of dicts eps, sigma, sigma_bar, iters, resid per problem).
    """
    import torch
    n = len(problems)
    prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
    bnd = {"average": LAT_BOUNDARY_AVERAGE, "zero": LAT_BOUNDARY_ZERO}[boundary]
    items = (_MultiItem * n)()
    keep, outs = [], []
    for i, pb in enumerate(problems):
        plan, phase = pb["plan"], pb["phase"]
        if phase.dtype != torch.uint8 or not phase.is_cuda or not phase.is_contiguous() or \
                phase.numel() != plan.m or phase.device != problems[0]["phase"].device:
            raise TypeError("problem %d: phase must be a uint8 CUDA tensor with m entries on the device of "
                            "problem 0" % i)
        E = np.asarray(pb["E"], dtype=np.float64).reshape(-1, plan.n_c)
        nl = E.shape[0]
        eps = pb.get("eps")
        if eps is not None:
            _strain_buffer(eps, "problem %d: eps" % i, nl * plan.n_c * plan.m, phase.device)
        else:
            if warm_start:
                raise ValueError("problem %d: warm_start needs eps" % i)
            eps = torch.empty((nl, plan.n_c, plan.m), dtype=torch.float64, device=phase.device)
        sigma = torch.empty_like(eps) if want_sigma else None
        st_i, st_p = _f64(np.asarray(pb["stiffness"], dtype=np.float64).reshape(-1, 36))
        e_i, e_p = _f64(E)
        o = dict(eps=eps, sigma=sigma, sigma_bar=np.zeros((nl, plan.n_c)), iters=np.zeros(nl, dtype=np.int32),
                 resid=np.zeros(nl))
        keep += [st_i, e_i]
        outs.append(o)
        it = items[i]
        it.plan = plan.handle
        it.phase = phase.data_ptr()
        it.n_phases = st_i.shape[0]
        it.stiffness = st_p
        it.C0[0], it.C0[1] = float(pb["C0"][0]), float(pb["C0"][1])
        it.E = e_p
        it.n_loads = nl
        it.eps = eps.data_ptr()
        it.sigma = sigma.data_ptr() if sigma is not None else None
        it.sigma_bar = o["sigma_bar"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        it.iters = o["iters"].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        it.resid = o["resid"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    L = lib()
    L.lattice_multi_workspace_bytes.argtypes = [ctypes.POINTER(_MultiItem), ctypes.c_int, ctypes.c_int]
    L.lattice_multi_workspace_bytes.restype = ctypes.c_size_t
    wsb = int(L.lattice_multi_workspace_bytes(items, n, prec | (LAT_WS_CG if scheme == "cg" else 0)))
    if wsb == 0:
        raise LatticeError(LAT_ERR_ARG, "lattice_multi_workspace_bytes: invalid items")
    dev = problems[0]["phase"].device
    ws, wsn = _workspace(workspace, wsb, dev)
    opts = _Opts(prec, bnd, 1 if warm_start else 0, None, 1 if mixed_increment else 0, 0 if mixed_restart else -1,
                 1 if plain_launches else 0, _SCHEMES[scheme])
    f = L.basic_scheme_solve_multi
    f.argtypes = [ctypes.POINTER(_MultiItem), ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Opts),
                  ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    f.restype = ctypes.c_int
    rc = f(items, n, float(tol), int(maxit), ctypes.byref(opts), ctypes.c_void_p(ws.data_ptr()), wsn,
           _stream(stream))
    _check(rc)
    return rc, outs


def multi_workspace_bytes(problems, precision="fp64", scheme="basic"):
    """Workspace bytes basic_scheme_solve_multi needs for these problems."""
    n = len(problems)
    items = (_MultiItem * n)()
    for i, pb in enumerate(problems):
        items[i].plan = pb["plan"].handle
        items[i].phase = 1                     # only checked for NULL
        items[i].n_phases = len(pb["stiffness"])
        items[i].stiffness = ctypes.cast(1, ctypes.POINTER(ctypes.c_double))
        items[i].E = ctypes.cast(1, ctypes.POINTER(ctypes.c_double))
        items[i].eps = 16
        items[i].n_loads = int(np.asarray(pb["E"]).reshape(-1, pb["plan"].n_c).shape[0])
    L = lib()
    L.lattice_multi_workspace_bytes.argtypes = [ctypes.POINTER(_MultiItem), ctypes.c_int, ctypes.c_int]
    L.lattice_multi_workspace_bytes.restype = ctypes.c_size_t
    prec = {"fp64": LAT_FP64, "mixed": LAT_MIXED, "df64": LAT_DF64}[precision]
    return int(L.lattice_multi_workspace_bytes(items, n, prec | (LAT_WS_CG if scheme == "cg" else 0)))


def gather_map(src_plan, dst_plan):
    """For every point of P(dst) in its plan order, the plan-order slot of the same point in P(src)
    (lattice_gather_map): dst a subpattern of src (M_src = J M_dst, Sec. 2.1) or pattern-congruent
    to it (Sec. 2.2).  Host numpy int32 array of dst.m entries; raises if P(dst) is not in P(src)."""
    out = np.empty(dst_plan.m, dtype=np.int32)
    f = lib().lattice_gather_map
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    f.restype = ctypes.c_int
    _check(f(src_plan.handle, dst_plan.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return out


def gather(x, index_map, stream=None):
    """out[..., s] = x[..., index_map[s]] on the GPU (lattice_gather): fields (..., m_src) on P(src)
    sampled onto P(dst).  x a contiguous CUDA tensor, index_map a CUDA int32 tensor from gather_map."""
    import torch
    if not (x.is_cuda and index_map.is_cuda and index_map.dtype == torch.int32 and x.is_contiguous()
            and index_map.is_contiguous() and index_map.device == x.device):
        raise TypeError("gather: x must be a contiguous CUDA tensor and index_map a contiguous CUDA int32 tensor "
                        "on the same device")
    lead = tuple(x.shape[:-1])
    n_f = int(np.prod(lead)) if lead else 1
    n = index_map.numel()
    out = torch.empty(lead + (n,), dtype=x.dtype, device=x.device)
    f = lib().lattice_gather
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(index_map.data_ptr()),
             n, x.element_size(), n_f, x.shape[-1], n, _stream(stream)))
    return out
