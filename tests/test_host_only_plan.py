"""A plan made without a CUDA device is host-only (CPU test).

lattice_plan uploads the plan's twiddle tables to the device current at the call, so that no solve
allocates.  Where no device exists the plan still serves the host queries (points, frequencies, gather
maps) and every solve returns LAT_ERR_CUDA before touching device memory.
"""
import ctypes

import numpy as np
import pytest

from paper_1605_05712_gb300 import lattice_plan
from paper_1605_05712_gb300.api import lib


def test_host_only_plan_refuses_solves():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: the plan is not host-only")
    P = lattice_plan([[64, 8], [0, 32]])
    assert P.points().shape == (P.m, 2) and P.freqs().shape == (P.m, 2)
    L = lib()
    f = L.basic_scheme_solve
    stiff = np.ascontiguousarray(np.eye(6).reshape(-1))
    C0 = np.array([5.5, 5.5])
    E = np.array([1.0, 0.0, 0.0])
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    fake = ctypes.c_void_p(256)          # never dereferenced: the call stops at the device check
    rc = f(P.handle, fake, 1, dp(stiff), dp(C0), dp(E), 1, 1e-8, 10, None, fake, None, None, None, None, fake,
           ctypes.c_size_t(1 << 40), None)
    assert rc == -6
    assert b"without a CUDA device" in L.lattice_last_error()
