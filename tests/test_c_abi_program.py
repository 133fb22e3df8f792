"""The boundary is a plain C ABI: a C99 program (tests/c_abi/host_queries.c) compiled with gcc against
include/lattice_ms.h alone (no CUDA or torch headers, -pedantic -Werror) and linked to liblatms.so makes
the host-side calls -- plan, info, layout, workspace queries, points, frequencies, destroy, the error
path -- and reports the same values as the Python binding, in the same order.  No GPU is used."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MATS = [[[3, 0], [0, 5]], [[8, -4], [2, 7]], [[512, 16], [0, 512]], [[2053, 7], [0, 1]],
        [[2, 1, 0], [0, 3, 1], [1, 0, 4]], [[16, 4, 0], [0, 16, 4], [0, 0, 16]], [[1, 0], [0, 1]]]


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1605_05712_gb300 import api
    api.lib()                                     # the library is built and loads
    native = os.path.join(ROOT, "paper_1605_05712_gb300", "_native")
    exe = str(tmp_path_factory.mktemp("cabi") / "host_queries")
    cmd = [gcc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi", "host_queries.c"), "-L", native, "-llatms",
           "-Wl,-rpath," + native, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _run(exe, M):
    d = len(M)
    r = subprocess.run([exe, str(d)] + [str(x) for row in M for x in row], capture_output=True, text=True,
                       timeout=60)
    assert r.returncode == 0, r.stderr
    out = {"point": [], "freq": []}
    for line in r.stdout.splitlines():
        key, *vals = line.split(" ", 1)
        vals = vals[0] if vals else ""
        if key in ("point", "freq"):
            out[key].append([int(v) for v in vals.split()])
        elif key == "err":
            out[key] = vals
        else:
            out[key] = [int(v) for v in vals.split()]
    return out


@pytest.mark.parametrize("M", MATS)
def test_c_program_reports_what_the_binding_reports(program, M):
    from paper_1605_05712_gb300 import api, lattice_plan
    c = _run(program, M)
    P = lattice_plan(M)
    d = len(M)
    assert c["rc"] == [0]
    assert c["info"] == [P.m, P.d_M] + P.divisors
    lay = P.layout()
    assert c["layout"] == [len(lay["ax_len"]), lay["split"]] + lay["ax_len"]
    assert c["ws"] == [P.workspace_bytes(2, api.LAT_FP64), P.workspace_bytes(2, api.LAT_FP64 | api.LAT_WS_CG)]
    assert np.array_equal(np.array(c["point"], dtype=np.int64).reshape(P.m, d), P.points())
    assert np.array_equal(np.array(c["freq"], dtype=np.int64).reshape(P.m, d), P.freqs())


def test_c_program_error_path(program):
    c = _run(program, [[2, 4], [1, 2]])               # singular
    assert c["rc"] == [-2] and "det" in c["err"]
