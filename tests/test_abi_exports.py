"""liblatms.so builds, loads without a GPU and exports every function include/*.h declares."""
import pytest
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            if m.group(1) not in ("defined",):
                names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1605_05712_gb300._build import build
    lib_path = build()
    L = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert {"lattice_plan", "basic_scheme_solve", "lattice_fft", "basic_scheme_solve_noalloc"} <= names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def _fft_ws(P, n_fields):
    from paper_1605_05712_gb300.api import lib
    f = lib().lattice_fft_workspace_bytes
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_size_t
    return int(f(P.handle, n_fields))


def test_host_side_plan_without_gpu():
    # plan construction, points and frequencies are host code; they work with no GPU present
    import numpy as np
    from oracle.lattice import Lattice
    from paper_1605_05712_gb300 import LatticeError, lattice_plan
    for M in ([[8, -4], [2, 7]], [[512, 16], [0, 512]], [[16, 4, 0], [0, 16, 4], [0, 0, 16]],
              [[3, 0], [0, 5]], [[6, 2], [0, 10]], [[3072, 0], [0, 1]], [[1, 0, 0], [0, 3, 0], [0, 0, 45]]):
        P = lattice_plan(M)
        L = Lattice(M)
        assert P.m == L.m and P.divisors == L.e
        assert set(map(tuple, P.points().tolist())) == set(map(tuple, L.p.tolist()))
        assert set(map(tuple, P.freqs().tolist())) == set(map(tuple, L.h.tolist()))
        assert _fft_ws(P, 2) == 0   # in-place passes: no scratch
    # a largest divisor with no split into two passes (a prime beyond the pass length, or such a prime
    # times a small factor) keeps its rows whole for the chirp-z transform: layout split = 2
    for M in ([[4099, 0], [0, 1]], [[2053, 7], [0, 1]], [[2, 0], [0, 4106]], [[1031, 0, 0], [5, 1, 0], [7, 0, 1]],
              [[3, 0, 0], [0, 1, 0], [0, 0, 3093]]):
        P = lattice_plan(M)
        L = Lattice(M)
        lay = P.layout()
        assert lay["split"] == 2 and lay["ax_len"][-1] == L.e[-1]
        # the convolution lines: n_c planes x m / p rows x L >= 2p - 1 (power of two) complex binary64 per
        # load case, in the solve workspace and in lattice_fft's
        p = L.e[-1]
        Lc = 1 << (2 * p - 2).bit_length()
        lines = P.n_c * (P.m // p)
        assert P.workspace_bytes(1) >= lines * Lc * 16
        assert P.workspace_bytes(2) - P.workspace_bytes(1) >= lines * Lc * 16
        assert _fft_ws(P, 3) == 3 * (P.m // p) * Lc * 16
        assert P.m == L.m and P.divisors == L.e
        assert set(map(tuple, P.points().tolist())) == set(map(tuple, L.p.tolist()))
        assert set(map(tuple, P.freqs().tolist())) == set(map(tuple, L.h.tolist()))
    # singular; a divisor longer than one mixed-radix pass that is not the largest; a prime largest divisor
    # beyond the longest chirp-z row (2^22 points)
    for bad, code in (([[2, 4], [1, 2]], -2), ([[3000, 0], [0, 3000]], -5), ([[4194319, 0], [0, 1]], -5)):
        try:
            lattice_plan(bad)
            raise AssertionError("expected an error")
        except LatticeError as e:
            assert e.code == code


def test_set_cell_validates_on_the_host():
    from paper_1605_05712_gb300 import LatticeError, lattice_plan
    P = lattice_plan([[16, 4], [0, 8]])
    P.set_cell([[1.3, 0.4], [-0.2, 0.9]])
    P.set_cell(None)
    with pytest.raises(LatticeError):
        P.set_cell([[1.0, 2.0], [0.5, 1.0]])            # singular
    with pytest.raises(LatticeError):
        P.set_cell([[float("nan"), 0.0], [0.0, 1.0]])


def test_binding_constants_equal_the_header():
    # every LAT_* constant the Python binding defines has the value the C header defines
    from paper_1605_05712_gb300 import api
    header = open(os.path.join(ROOT, "include", "lattice_ms.h")).read()
    defs = {}
    for name, val in re.findall(r"^#define (LAT_\w+)\s+(-?\d+)", header, flags=re.M):
        defs[name] = int(val)
    names = [n for n in dir(api) if n.startswith("LAT_") and isinstance(getattr(api, n), int)]
    assert {"LAT_OK", "LAT_FP64", "LAT_SCHEME_CG", "LAT_WS_CG", "LAT_BOUNDARY_ZERO"} <= set(names)
    for n in names:
        assert n in defs, n
        assert getattr(api, n) == defs[n], n
