"""Host-side checks of the conjugate-gradient option of the C ABI (no GPU): the workspace queries with
LAT_WS_CG make room for the four vectors, and the solve refuses the cases the method does not cover
before it touches the device (mixed precision, warm start, boundary frequencies kept)."""
import ctypes

import numpy as np
import pytest

from paper_1605_05712_gb300 import api, lattice_plan, multi_workspace_bytes


def test_workspace_has_room_for_the_vectors():
    for M in ([[512, 16], [0, 512]], [[16, 4, 0], [0, 16, 4], [0, 0, 16]], [[4096, 12288], [0, 1]]):
        P = lattice_plan(M)
        for prec in (api.LAT_FP64, api.LAT_DF64):
            for n in (1, 3):
                base = P.workspace_bytes(n, prec)
                cg = P.workspace_bytes(n, prec | api.LAT_WS_CG)
                assert base > 0 and cg >= base + 4 * n * P.n_c * P.m * 8
        probs = [dict(plan=P, stiffness=[np.eye(6)], E=np.zeros((2, P.n_c)))]
        assert multi_workspace_bytes(probs, "fp64", scheme="cg") >= multi_workspace_bytes(probs) + 4 * 2 * P.n_c * P.m * 8


def _solve_rc(M, precision, boundary, warm, scheme=api.LAT_SCHEME_CG):
    """basic_scheme_solve through the ABI with placeholder device pointers: the argument checks run
    first and return before any device access."""
    L = api.lib()
    P = lattice_plan(M)
    stiff = np.eye(6).reshape(1, 36).copy()
    C0 = np.array([1.0, 1.0])
    E = np.zeros(P.n_c)
    E[0] = 1.0
    opts = api._Opts(precision, boundary, warm, None, 1, 0, 0, scheme)
    dp = ctypes.POINTER(ctypes.c_double)
    fake = ctypes.c_void_p(256)
    rc = L.basic_scheme_solve(P.handle, fake, 1, stiff.ctypes.data_as(dp), C0.ctypes.data_as(dp),
                              E.ctypes.data_as(dp), 1, 1e-6, 10, ctypes.byref(opts), fake, None, None, None, None,
                              fake, 0, None)
    return rc, L.lattice_last_error().decode()


@pytest.mark.parametrize("case", [
    dict(precision=api.LAT_MIXED, boundary=api.LAT_BOUNDARY_ZERO, warm=0, msg="LAT_FP64 or LAT_DF64"),
    dict(precision=api.LAT_FP64, boundary=api.LAT_BOUNDARY_ZERO, warm=1, msg="starts from eps = E"),
    dict(precision=api.LAT_FP64, boundary=api.LAT_BOUNDARY_AVERAGE, warm=0, msg="LAT_BOUNDARY_ZERO"),
])
def test_refusals(case):
    rc, msg = _solve_rc([[16, 4], [0, 8]], case["precision"], case["boundary"], case["warm"])
    assert rc == api.LAT_ERR_ARG and case["msg"] in msg


def test_boundary_zero_passes_the_checks():
    # the argument checks pass; the call then stops at the workspace size (0 bytes given), still before
    # any device access
    rc, msg = _solve_rc([[16, 4], [0, 8]], api.LAT_DF64, api.LAT_BOUNDARY_ZERO, 0)
    assert rc == -4 and "workspace" in msg


def test_chirp_z_plans_take_conjugate_gradients_in_binary64():
    # a largest divisor with no split into two passes (chirp-z rows): binary64 CG passes the argument
    # checks (odd largest divisor: either boundary option; even: boundary frequencies zeroed), pairs are
    # refused as for every scheme on these plans; the workspace holds the four vectors and two partial sums
    # for each of up to 1024 point blocks
    for M, bnd in (([[2053, 7], [0, 1]], api.LAT_BOUNDARY_AVERAGE), ([[2, 0], [0, 4106]], api.LAT_BOUNDARY_ZERO),
                   ([[3, 0, 0], [0, 1, 0], [0, 0, 3093]], api.LAT_BOUNDARY_ZERO)):
        P = lattice_plan(M)
        assert P.layout()["split"] == 2
        rc, msg = _solve_rc(M, api.LAT_FP64, bnd, 0)
        assert rc == -4 and "workspace" in msg, msg
        rc, msg = _solve_rc(M, api.LAT_DF64, bnd, 0)
        assert rc == -5 and "LAT_FP64" in msg, msg
        for n in (1, 2):
            base = P.workspace_bytes(n, api.LAT_FP64)
            assert P.workspace_bytes(n, api.LAT_FP64 | api.LAT_WS_CG) >= base + 4 * n * P.n_c * P.m * 8
            assert base >= n * 2 * 1024 * 8
    rc, msg = _solve_rc([[2, 0], [0, 4106]], api.LAT_FP64, api.LAT_BOUNDARY_AVERAGE, 0)
    assert rc == api.LAT_ERR_ARG and "LAT_BOUNDARY_ZERO" in msg


def test_multi_workspace_with_chirp_z_problems():
    # a multi call mixing a chirp-z lattice with power-of-two and general ones: the conjugate-gradient
    # query makes room for every problem's four vectors and is at least each problem's own workspace
    plans = [lattice_plan(M) for M in ([[2053, 7], [0, 1]], [[64, 1], [0, 64]], [[3, 0], [0, 5]])]
    probs = [dict(plan=P, stiffness=[np.eye(6)], E=np.zeros((2, P.n_c))) for P in plans]
    base = multi_workspace_bytes(probs, "fp64")
    cg = multi_workspace_bytes(probs, "fp64", scheme="cg")
    assert base > 0 and cg >= base + sum(4 * 2 * P.n_c * P.m * 8 for P in plans)
    for P in plans:
        assert cg >= P.workspace_bytes(2, api.LAT_FP64 | api.LAT_WS_CG)
