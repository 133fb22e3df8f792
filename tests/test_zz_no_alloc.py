"""The no-allocation entry point against the workspace entry point (GPU).

basic_scheme_solve_noalloc serves callers that cannot allocate device memory
(a fixed memory budget, a foreign allocator that owns the device memory): it
runs the same kernels on a static device scratch array.  This file is
collected last so that a run stopping at the first failure has run every other
test before it; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1605_05712_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-10    # the tolerance of the binary64 parity tests


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_noalloc_matches_workspace_entry_point_twice(cuda):
    import torch
    from paper_1605_05712_gb300 import LatticeError, basic_scheme_solve, lattice_plan
    from paper_1605_05712_gb300.api import basic_scheme_solve_noalloc
    P = lattice_plan([[512, 16], [0, 512]])          # m = 262144, rank-2, four-step split
    ph = torch.from_numpy(synth.laminate_phase(P.points(), P.m, [1, 3])).to(cuda)
    stiff = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(10.0, 10.0)]
    E = np.array([[1.0, 0.0, 0.0], [0.2, -0.4, 0.3]])
    ref = basic_scheme_solve(P, ph, stiff, (5.5, 5.5), E, tol=1e-8, maxit=300, want_sigma=True)
    out_eps = torch.empty_like(ref["eps"])
    for call in range(2):                              # second call reuses the scratch left by the first
        out_eps.fill_(float("nan"))
        g = basic_scheme_solve_noalloc(P, ph, stiff, (5.5, 5.5), E, tol=1e-8, maxit=300, eps_out=out_eps,
                                       want_sigma=True)
        assert g["status"] == ref["status"] == 0
        assert np.array_equal(g["iters"], ref["iters"])
        assert _rel(g["eps"].cpu().numpy(), ref["eps"].cpu().numpy()) < RTOL
        assert _rel(g["sigma"].cpu().numpy(), ref["sigma"].cpu().numpy()) < RTOL
        assert _rel(g["sigma_bar"], ref["sigma_bar"]) < RTOL
        assert _rel(g["resid"], ref["resid"]) < 1e-9
    # a solve larger than the static scratch is refused with a size error, not run
    Pb = lattice_plan([[128, 0, 0], [0, 128, 0], [0, 0, 128]])
    phb = torch.zeros(Pb.m, dtype=torch.uint8, device=cuda)
    with pytest.raises(LatticeError) as ei:
        basic_scheme_solve_noalloc(Pb, phb, stiff[:1], (5.5, 5.5), np.eye(6)[:1], tol=1e-8, maxit=2)
    assert ei.value.code == -4


@pytest.mark.parametrize("scheme,C0,boundary", [("eyre_milton", (np.sqrt(10.0), np.sqrt(10.0)), "average"),
                                                ("cg", (5.5, 5.5), "zero")])
def test_noalloc_accelerated_schemes(cuda, scheme, C0, boundary):
    # the accelerated schemes through the no-allocation entry point (plain launches on the static scratch;
    # conjugate gradients need four more strain-sized vectors there) equal the workspace entry point
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    from paper_1605_05712_gb300.api import basic_scheme_solve_noalloc
    P = lattice_plan([[128, 16], [0, 256]])   # m = 32768: the vectors fit the 16 MiB scratch
    ph = torch.from_numpy(synth.laminate_phase(P.points(), P.m, [1, 3])).to(cuda)
    stiff = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(10.0, 10.0)]
    E = np.array([[1.0, 0.0, 0.0], [0.2, -0.4, 0.3]])
    ref = basic_scheme_solve(P, ph, stiff, C0, E, tol=1e-9, maxit=500, boundary=boundary, scheme=scheme)
    g = basic_scheme_solve_noalloc(P, ph, stiff, C0, E, tol=1e-9, maxit=500, boundary=boundary, scheme=scheme)
    assert g["status"] == ref["status"] == 0
    assert np.array_equal(g["iters"], ref["iters"])
    assert _rel(g["eps"].cpu().numpy(), ref["eps"].cpu().numpy()) < RTOL
    assert _rel(g["sigma_bar"], ref["sigma_bar"]) < RTOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_first_on_a_fresh_plan(cuda, precision):
    # the no-allocation entry point as the first solve on newly made plans (the plan's own tables, made by
    # lattice_plan, serve it; the mixed path's binary64-accurate restart uses the pair tables), then the
    # workspace entry point on other fresh plans of the same lattices: equal results
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    from paper_1605_05712_gb300.api import basic_scheme_solve_noalloc
    stiff = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(10.0, 10.0)]
    # the mixed solve also holds a binary64 spectrum for its restart: a smaller 2-D lattice fits the scratch
    M2 = [[512, 16], [0, 512]] if precision == "fp64" else [[256, 16], [0, 256]]
    for M in (M2, [[32, 4, 0], [0, 32, 4], [0, 0, 32]]):
        P = lattice_plan(M)
        d = len(M)
        incl = synth.random_inclusions(3, d, 4, 0.3)
        ph = torch.from_numpy(synth.inclusions_phase(P.points(), P.m, incl)).to(cuda)
        E = np.eye(P.n_c)[:2]
        tol = 1e-6 if precision == "mixed" else 1e-8
        g = basic_scheme_solve_noalloc(P, ph, stiff, (5.5, 5.5), E, tol=tol, maxit=500, precision=precision)
        P2 = lattice_plan(M)
        ref = basic_scheme_solve(P2, ph, stiff, (5.5, 5.5), E, tol=tol, maxit=500, precision=precision)
        assert g["status"] == ref["status"] == 0
        assert np.array_equal(g["iters"], ref["iters"])
        assert _rel(g["eps"].cpu().numpy(), ref["eps"].cpu().numpy()) < RTOL
        assert _rel(g["sigma_bar"], ref["sigma_bar"]) < RTOL


def test_noalloc_refuses_a_capturing_stream(cuda):
    # the call synchronizes its stream every iteration, so on a stream under capture it returns LAT_ERR_ARG
    # before enqueuing anything (the capture itself stays valid and ends normally)
    import torch
    from paper_1605_05712_gb300 import LatticeError, lattice_plan
    from paper_1605_05712_gb300.api import basic_scheme_solve_noalloc
    P = lattice_plan([[64, 8], [0, 32]])
    ph = torch.zeros(P.m, dtype=torch.uint8, device=cuda)
    eps = torch.empty((1, 3, P.m), dtype=torch.float64, device=cuda)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.graph(graph):
        try:
            basic_scheme_solve_noalloc(P, ph, [synth.iso_voigt(1.0, 1.0)], (5.5, 5.5), np.eye(3)[:1], tol=1e-8,
                                       maxit=5, eps_out=eps)
        except LatticeError as e:
            code = e.code
    assert code == -1
