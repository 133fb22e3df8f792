"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances: the binary64 path must agree with the oracle to 1e-10 relative
(max |difference| / max |value| per field and per component group: normal and shear entries of a tensor
field each against their own maximum); residual histories likewise; the mixed path within its stated
bounds (max relative strain error 1e-5, mean stress 1e-6, over the whole field); the
iteration count of a converged solve must match exactly unless the oracle's
residual at the stopping iteration lies within 1e-6 relative of tol.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme
from oracle.transform import dft_fast, dft_naive
from paper_1605_05712_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _index(rows):
    return {tuple(r): i for i, r in enumerate(rows.tolist())}


def to_oracle_order(plan_pts, lat):
    """perm[i] = oracle index of plan slot i (matching exact point numerators)."""
    idx = _index(lat.p)
    return np.array([idx[tuple(p)] for p in plan_pts.tolist()])


def stiff_tensors(voigts, d):
    return np.array([el.voigt6_to_tensor(v, d) for v in voigts])


def comps_to_tensor(comps, d):
    # (n_c, m) -> (m, d, d)
    return el.comps_to_sym(np.asarray(comps).T, d)


GROUP_FLOOR = 1e-3   # a component group whose values are all below 1e-3 of the field's maximum is measured
                     # against that floor (an identically zero group would otherwise divide rounding by zero)


def relerr(a, b):
    """Max |a - b| / max |b|, per component group for real tensor fields (..., d, d): the normal (diagonal)
    and the shear (off-diagonal) entries are measured against their own maxima, so small shear components
    are held to the same relative bound as the normal ones; other arrays against their overall maximum."""
    a, b = np.asarray(a), np.asarray(b)
    if b.ndim >= 2 and b.shape[-1] == b.shape[-2] and b.shape[-1] in (2, 3) and not np.iscomplexobj(b):
        d = b.shape[-1]
        scale = np.abs(b).max()
        worst = 0.0
        for mask in (np.eye(d, dtype=bool), ~np.eye(d, dtype=bool)):
            den = max(np.abs(b[..., mask]).max(), GROUP_FLOOR * scale, 1e-300)
            worst = max(worst, np.abs(a[..., mask] - b[..., mask]).max() / den)
        return worst
    return relerr_global(a, b)


def relerr_global(a, b):
    """Max |a - b| / max |b| over the whole array (the measure of the stated mixed-precision bounds)."""
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


FFT_MATS = [[[1, 0], [0, 1]], [[2, 0], [0, 1]], [[8, -4], [2, 7]], [[4, 4], [-4, 4]], [[16, 0], [4, 8]],
            [[64, 1], [0, 64]], [[512, 16], [0, 512]], [[512, 1], [0, 512]], [[64, 0], [0, 64]],
            [[8, 0, 0], [0, 8, 0], [0, 0, 8]], [[8, 1, 0], [0, 8, 1], [0, 0, 8]], [[4, 0, 0], [0, 8, 0], [0, 0, 1]],
            [[16, 4, 0], [0, 16, 4], [0, 0, 16]], [[64, 0, 0], [0, 64, 0], [0, 0, 64]],
            [[128, 1, 0], [0, 128, 1], [0, 0, 64]]]
# elementary divisors that are not powers of two (mixed-radix kernels): (1,15), (1,60) rank-1, rank-1
# m = 3 * 2^10 (four-step 48 x 64), (5,5), (6,12), (2,30), rank-1 m = 9216 (96 x 96), 3-D (1,3,45), (3,3,15),
# (1,1,25), (45,45,45) and a rank-1 lattice of prime length 1009
GEN_MATS = [[[3, 0], [0, 5]], [[6, 1], [0, 10]], [[3072, 0], [0, 1]], [[5, 0], [0, 5]], [[12, 0], [0, 6]],
            [[6, 2], [0, 10]], [[96, 1], [0, 96]], [[1009, 0], [0, 1]], [[1, 0, 0], [0, 3, 0], [0, 0, 45]],
            [[3, 0, 0], [0, 3, 0], [0, 0, 15]], [[2, 1, 0], [0, 3, 1], [1, 0, 4]],
            [[45, 0, 0], [0, 45, 0], [0, 0, 45]]]
# largest divisors with no split into two passes (chirp-z rows): rank-1 primes 2053 (2-D) and 1031 (3-D),
# (2, 2 x 2053), rank-1 2 x 4099, and 3-D (1, 3, 3 x 1031) whose chirp-z row meets a column pass
BLUE_MATS = [[[2053, 7], [0, 1]], [[1031, 0, 0], [5, 1, 0], [7, 0, 1]], [[2, 0], [0, 4106]], [[8198, 3], [0, 1]],
             [[3, 0, 0], [0, 1, 0], [0, 0, 3093]]]
FFT_MATS = FFT_MATS + GEN_MATS + BLUE_MATS


@pytest.mark.parametrize("M", FFT_MATS)
def test_lattice_fft_matches_oracle(cuda, M):
    import torch
    from paper_1605_05712_gb300 import lattice_fft, lattice_plan
    P = lattice_plan(M)
    L = Lattice(M)
    perm = to_oracle_order(P.points(), L)
    hidx = _index(L.h)
    hperm = np.array([hidx[tuple(h)] for h in P.freqs().tolist()])
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, P.m)) + 1j * rng.standard_normal((2, P.m))
    X = lattice_fft(P, torch.from_numpy(x).to(cuda)).cpu().numpy()
    a = np.empty((P.m, 2), dtype=complex)
    a[perm] = x.T
    ref = (dft_naive(L, a) if L.m <= 512 else dft_fast(L, a))[hperm].T
    assert relerr(X, ref) < 1e-12
    back = lattice_fft(P, torch.from_numpy(X).to(cuda), inverse=True).cpu().numpy()
    assert relerr(back, x) < 1e-12


def run_pair(M, phase_fn, voigts, C0, E, tol, maxit, boundary="average", warm=None, cuda=None, precision="fp64",
             cell=None, scheme="basic"):
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    P = lattice_plan(M)
    if cell is not None:
        P.set_cell(cell)
    L = Lattice(M)
    d = L.d
    ph_plan = phase_fn(P.points(), P.m)
    ph_or = phase_fn(L.p, L.m)
    perm = to_oracle_order(P.points(), L)
    assert np.array_equal(ph_plan, ph_or[perm])
    E = np.atleast_2d(E)
    eps0 = None
    if warm is not None:
        eps0 = torch.from_numpy(np.ascontiguousarray(warm)).to(cuda)
    g = basic_scheme_solve(P, torch.from_numpy(ph_plan).to(cuda), voigts, C0, E, tol=tol, maxit=maxit,
                           boundary=boundary, history=True, want_sigma=True, eps0=eps0, precision=precision,
                           scheme=scheme)
    g["precision"] = precision
    S = stiff_tensors(voigts, d)
    outs = []
    for lc in range(E.shape[0]):
        Et = el.comps_to_sym(E[lc], d)
        w0 = None
        if warm is not None:
            w0 = np.empty((L.m, d, d))
            w0[perm] = comps_to_tensor(warm[lc], d)
        o = basic_scheme(L, ph_or, S, C0, Et, tol=tol, maxit=maxit, eps0=w0,
                         boundary=("zero" if boundary == "zero" else "literal"), L=cell,
                         scheme=scheme)
        outs.append(o)
    return P, L, perm, g, outs


def check_pair(P, L, perm, g, outs, d, rtol=RTOL, check_iters=True, tol=0.0, hist_atol=None):
    for lc, o in enumerate(outs):
        eg = comps_to_tensor(g["eps"][lc].cpu().numpy(), d)
        assert relerr(eg, o["eps"][perm]) < rtol, "strain field"
        sg = comps_to_tensor(g["sigma"][lc].cpu().numpy(), d)
        assert relerr(sg, o["sigma"][perm]) < rtol, "stress field"
        sb = el.comps_to_sym(g["sigma_bar"][lc], d)
        assert relerr(sb, o["sigma_bar"]) < rtol, "mean stress"
        if check_iters:
            if int(g["iters"][lc]) != o["iters"]:
                h = o["history"]
                assert tol > 0 and abs(h[min(len(h), int(g["iters"][lc])) - 1] - tol) < 1e-6 * tol
        n = min(len(g["history"][lc]), len(o["history"]))
        hg, ho = np.array(g["history"][lc][:n]), np.array(o["history"][:n])
        # absolute floor: the strain's rounding, relative to the normalisation sqrt(m) |E| of r -- 2^-53 in
        # binary64, 2^-48 for double-float pairs (seen once the increments are ~1e-8 of the strain)
        atol = 1e-13 if g.get("precision") == "df64" else 1e-15
        if hist_atol is not None:
            atol = hist_atol
        assert np.all(np.abs(hg - ho) <= 1e-9 * np.maximum(ho, 1e-14) + atol), "residual history"


LAM2 = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(10.0, 10.0)]


def laminate(n_int):
    return lambda p, m: synth.laminate_phase(p, m, n_int)


def inclusions(seed, d, n, vf):
    incl = synth.random_inclusions(seed, d, n, vf)
    return lambda p, m: synth.inclusions_phase(p, m, incl)


SOLVE_2D = [[[1, 0], [0, 1]], [[2, 0], [0, 1]], [[2, 1], [0, 2]], [[8, -4], [2, 7]], [[4, 4], [-4, 4]],
            [[16, 0], [4, 8]], [[64, 1], [0, 64]], [[64, 32], [0, 1]], [[32, 0], [0, 64]], [[256, 16], [0, 256]],
            [[128, 1], [0, 128]], [[4096, 12288], [0, 1]], [[2048, 0], [0, 4]],
            # general plans (mixed-radix kernels)
            [[3, 0], [0, 5]], [[6, 1], [0, 10]], [[3072, 0], [0, 1]], [[12, 0], [0, 6]], [[96, 1], [0, 96]],
            [[45, 9], [0, 45]]]


# "df64": the binary64-accurate path on double-float pairs, held to the same 1e-10 as binary64
@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", SOLVE_2D)
def test_solve_fp64_fixed_iterations_2d(cuda, M, prec):
    E = np.array([[1.0, 0.0, 0.0], [0.3, -0.2, 0.4]])
    out = run_pair(M, inclusions(3, 2, 3, 0.3), LAM2, (5.5, 5.5), E, tol=0.0, maxit=7, cuda=cuda, precision=prec)
    check_pair(*out, d=2)


SOLVE_3D = [[[2, 0, 0], [0, 2, 0], [0, 0, 2]], [[8, 0, 0], [0, 8, 0], [0, 0, 8]], [[8, 1, 0], [0, 8, 1], [0, 0, 8]],
            [[4, 0, 0], [0, 8, 0], [0, 0, 1]], [[16, 4, 0], [0, 16, 4], [0, 0, 16]],
            [[64, 0, 0], [0, 64, 0], [0, 0, 32]], [[32, 1, 0], [0, 32, 1], [0, 0, 64]],
            # general plans (mixed-radix kernels)
            [[1, 0, 0], [0, 3, 0], [0, 0, 45]], [[3, 0, 0], [0, 3, 0], [0, 0, 15]], [[24, 0, 0], [0, 24, 0], [0, 0, 24]],
            [[12, 1, 0], [0, 12, 1], [0, 0, 12]], [[2, 1, 0], [0, 3, 1], [1, 0, 4]]]


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", SOLVE_3D)
def test_solve_fp64_fixed_iterations_3d(cuda, M, prec):
    E = np.array([[1.0, 0.0, 0.0, 0.0, 0.0, 0.0], [0.1, -0.3, 0.2, 0.25, -0.15, 0.4]])
    voigts = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(10.0, 10.0), synth.iso_voigt(3.0, 0.5)]

    def ph(p, m):
        a = inclusions(5, 3, 2, 0.2)(p, m)
        b = inclusions(9, 3, 1, 0.1)(p, m)
        return np.where(b == 1, 2, a).astype(np.uint8)
    out = run_pair(M, ph, voigts, (5.5, 5.5), E, tol=0.0, maxit=5, cuda=cuda, precision=prec)
    check_pair(*out, d=3)


def _orthotropic_voigts(rng, n):
    """n seeded axis-aligned orthotropic stiffness matrices (Voigt form): a random positive definite normal
    block and a positive shear diagonal, no normal-shear coupling."""
    out = np.zeros((n, 6, 6))
    for i in range(n):
        A = rng.standard_normal((3, 3))
        out[i, :3, :3] = 2.0 * np.eye(3) + A @ A.T
        out[i, 3:, 3:] = np.diag(10 ** rng.uniform(-0.3, 0.8, 3))
    return out


# phase tables beyond the isotropic ones: axis-aligned orthotropic and fully anisotropic stiffness (every
# entry of the tensor-component matrix in play)
@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("kind", ["orthotropic", "anisotropic"])
@pytest.mark.parametrize("M", [[[16, 4], [0, 8]], [[64, 32], [0, 1]], [[8, 1, 0], [0, 8, 1], [0, 0, 8]],
                               [[4096, 0, 0], [0, 1, 0], [0, 0, 1]], [[6, 1], [0, 10]]])
def test_solve_fixed_iterations_anisotropic_tables(cuda, M, kind, prec):
    d = len(M)
    n_c = d * (d + 1) // 2
    rng = np.random.default_rng(31)
    voigts = list(_orthotropic_voigts(rng, 3) if kind == "orthotropic" else _random_spd_voigts(rng, 3))
    E = np.ones((2, n_c)) * 0.2
    E[0, 0] = 1.0

    def ph(p, m):
        a = inclusions(5, d, 2, 0.2)(p, m)
        b = inclusions(9, d, 1, 0.1)(p, m)
        return np.where(b == 1, 2, a).astype(np.uint8)
    out = run_pair(M, ph, voigts, (5.0, 4.0), E, tol=0.0, maxit=5, cuda=cuda, precision=prec)
    check_pair(*out, d=d)


@pytest.mark.parametrize("kind", ["orthotropic", "anisotropic"])
@pytest.mark.parametrize("M", [[[256, 16], [0, 256]], [[32, 1, 0], [0, 32, 1], [0, 0, 32]]])
def test_mixed_anisotropic_tables_against_fp64(cuda, M, kind):
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    d = len(M)
    n_c = d * (d + 1) // 2
    rng = np.random.default_rng(32)
    voigts = list(_orthotropic_voigts(rng, 2) if kind == "orthotropic" else _random_spd_voigts(rng, 2))
    # reference medium 2 mu0 = the mean of the extreme Mandel eigenvalues, lam0 = 0 (a contraction)
    w = np.sqrt(2.0)
    scale = np.outer([1, 1, 1, w, w, w], [1, 1, 1, w, w, w])
    ev = np.concatenate([np.linalg.eigvalsh(v * scale) for v in voigts])
    C0 = (0.0, 0.25 * (ev.min() + ev.max()))
    P = lattice_plan(M)
    phd = torch.from_numpy(inclusions(3, d, 4, 0.3)(P.points(), P.m)).to(cuda)
    E = np.eye(n_c)[:2]
    ref = basic_scheme_solve(P, phd, voigts, C0, E, tol=1e-6, maxit=3000)
    mx = basic_scheme_solve(P, phd, voigts, C0, E, tol=1e-6, maxit=3000, precision="mixed")
    assert ref["status"] == 0 and mx["status"] == 0
    assert float((mx["eps"] - ref["eps"]).abs().max() / ref["eps"].abs().max()) <= MIXED_STRAIN_RTOL
    assert np.abs(mx["sigma_bar"] - ref["sigma_bar"]).max() <= MIXED_CEFF_RTOL * np.abs(ref["sigma_bar"]).max()


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", [[[64, 0], [0, 64]], [[512, 16], [0, 512]], [[8, 1, 0], [0, 8, 1], [0, 0, 8]],
                               [[60, 0], [0, 60]], [[45, 1], [0, 45]], [[12, 1, 0], [0, 12, 1], [0, 0, 12]]])
def test_solve_fp64_converged(cuda, M, prec):
    d = len(M)
    n_c = d * (d + 1) // 2
    E = np.zeros((1, n_c))
    E[0, 0] = 1.0
    ph = laminate([1, 3]) if d == 2 else inclusions(2, 3, 3, 0.25)
    out = run_pair(M, ph, LAM2, (5.5, 5.5), E, tol=1e-8, maxit=500, cuda=cuda, precision=prec)
    check_pair(*out, d=d, tol=1e-8)
    assert out[3]["status"] == 0


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_boundary_zero_option(cuda, prec):
    out = run_pair([[16, 2], [0, 8]], inclusions(4, 2, 2, 0.3), LAM2, (5.5, 5.5), np.array([[0.2, 1.0, 0.3]]),
                   tol=0.0, maxit=6, boundary="zero", cuda=cuda, precision=prec)
    check_pair(*out, d=2)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_warm_start_continues_the_iteration(cuda, prec):
    M = [[32, 4], [0, 16]]
    P_L = Lattice(M)
    from paper_1605_05712_gb300 import lattice_plan
    P = lattice_plan(M)
    perm = to_oracle_order(P.points(), P_L)
    ph = inclusions(8, 2, 2, 0.3)
    E = np.array([[1.0, 0.5, -0.25]])
    S = stiff_tensors(LAM2, 2)
    o3 = basic_scheme(P_L, ph(P_L.p, P_L.m), S, (5.5, 5.5), el.comps_to_sym(E[0], 2), tol=0.0, maxit=3)
    warm = el.sym_to_comps(o3["eps"][perm]).T[None]
    out = run_pair(M, ph, LAM2, (5.5, 5.5), E, tol=0.0, maxit=4, warm=warm, cuda=cuda, precision=prec)
    o7 = basic_scheme(P_L, ph(P_L.p, P_L.m), S, (5.5, 5.5), el.comps_to_sym(E[0], 2), tol=0.0, maxit=7)
    g = out[3]
    eg = comps_to_tensor(g["eps"][0].cpu().numpy(), 2)
    assert relerr(eg, o7["eps"][perm]) < RTOL


def test_edge_cases(cuda):
    import torch
    from paper_1605_05712_gb300 import LatticeError, basic_scheme_solve, lattice_plan
    P = lattice_plan([[16, 0], [4, 8]])
    ph = torch.from_numpy(synth.laminate_phase(P.points(), P.m, [1, 1])).to(cuda)
    # maxit = 0: eps = E, no iteration
    g = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), np.array([[1.0, 2.0, 3.0]]), tol=1e-8, maxit=0)
    assert int(g["iters"][0]) == 0 and g["status"] == 1
    e = g["eps"][0].cpu().numpy()
    assert np.all(e[0] == 1.0) and np.all(e[1] == 2.0) and np.all(e[2] == 3.0)
    # E = 0: the solution is zero
    g = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), np.zeros((1, 3)), tol=1e-8, maxit=10)
    assert np.abs(g["eps"].cpu().numpy()).max() == 0.0 and g["status"] == 0
    # invalid inputs are reported, not run
    with pytest.raises(LatticeError):
        lattice_plan([[2, 4], [1, 2]])          # singular
    # odd and non-power-of-two divisors are planned (mixed-radix kernels); a divisor too long for one pass
    # that is not the largest is refused
    assert lattice_plan([[3, 0], [0, 5]]).divisors == [1, 15]
    with pytest.raises(LatticeError):
        lattice_plan([[3000, 0], [0, 3000]])
    with pytest.raises(LatticeError):
        basic_scheme_solve(P, ph, LAM2, (1.0, -1.0), np.ones((1, 3)), tol=1e-8, maxit=3)   # mu0 <= 0


def test_aligned_laminate_m4096_matches_analytic(cuda):
    # 2-D rank-1 lattice M = [[4096, 12288], [0, 1]]: all frequencies parallel to (1,3); exact laminate
    import torch
    from oracle import analytic as an
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    P = lattice_plan(synth.LATTICES["laminate4096_aligned"])
    ph = synth.laminate_phase(P.points(), P.m, [1, 3])
    E = np.array([[1.0, 0.0, 0.0]])
    g = basic_scheme_solve(P, torch.from_numpy(ph).to(cuda), LAM2, synth.c0_mean_extremes([1, 10], [1, 10]), E,
                           tol=1e-14, maxit=100)
    S = stiff_tensors(LAM2, 2)
    e1, e2, sb = an.laminate_fields(S[0], S[1], 0.5, np.array([1.0, 3.0]), el.comps_to_sym(E[0], 2))
    ex = np.where(ph[:, None, None] == 0, e1, e2)
    assert relerr(comps_to_tensor(g["eps"][0].cpu().numpy(), 2), ex) < 1e-12
    assert relerr(el.comps_to_sym(g["sigma_bar"][0], 2), sb) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_aligned_laminate_262144_matches_analytic(cuda, prec):
    # the aligned rank-1 lattice of the m = 262144 laminate, M = [[262144, 786432], [0, 1]]: every frequency
    # is parallel to (1,3), so the converged discrete solution is the analytic laminate point by point -- a
    # full-size check without an oracle run; three unit load cases in one solve
    import torch
    from oracle import analytic as an
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    P = lattice_plan([[262144, 786432], [0, 1]])
    ph = synth.laminate_phase(P.points(), P.m, [1, 3])
    E = np.eye(3)
    E[2, 2] = 0.5
    g = basic_scheme_solve(P, torch.from_numpy(ph).to(cuda), LAM2, (5.5, 5.5), E, tol=1e-14, maxit=300,
                           precision=prec)
    S = stiff_tensors(LAM2, 2)
    for lc in range(3):
        e1, e2, sb = an.laminate_fields(S[0], S[1], 0.5, np.array([1.0, 3.0]), el.comps_to_sym(E[lc], 2))
        ex = np.where(ph[:, None, None] == 0, e1, e2)
        assert relerr(comps_to_tensor(g["eps"][lc].cpu().numpy(), 2), ex) < (1e-12 if prec == "fp64" else 1e-11)
        assert relerr(el.comps_to_sym(g["sigma_bar"][lc], 2), sb) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("name", ["grid512", "rank1_262144", "rank2_262144"])
def test_full_size_262144_fixed_iterations(cuda, name, prec):
    # the benchmark workload: laminate n = (1,3), m = 262144, three unit load cases, compared field-wise
    E = np.eye(3)
    E[2, 2] = 0.5
    out = run_pair(synth.LATTICES[name], laminate([1, 3]), LAM2, (5.5, 5.5), E, tol=0.0, maxit=4, cuda=cuda,
                   precision=prec)
    check_pair(*out, d=2)


# ---------------------------------------------------------------- mixed precision (binary32 bulk)
MIXED_STRAIN_RTOL = 1e-5     # max relative strain-field error against the binary64 oracle at tol 1e-6
MIXED_CEFF_RTOL = 1e-6       # relative error of the mean stress (a column of C^eff)


# the last five are general plans (mixed-radix binary32 kernels and their pair restart): (45, 45) sheared,
# rank-1 m = 9216 (four-step 96 x 96), (1, 3, 45), 24^3, and 3-D rank-1 m = 1728
@pytest.mark.parametrize("M", [[[256, 0], [0, 256]], [[512, 16], [0, 512]], [[64, 1], [0, 64]],
                               [[32, 0, 0], [0, 32, 0], [0, 0, 32]], [[64, 1, 0], [0, 64, 1], [0, 0, 64]],
                               [[45, 9], [0, 45]], [[96, 1], [0, 96]], [[1, 0, 0], [0, 3, 0], [0, 0, 45]],
                               [[24, 0, 0], [0, 24, 0], [0, 0, 24]], [[12, 1, 0], [0, 12, 1], [0, 0, 12]]])
def test_mixed_precision_within_stated_tolerance(cuda, M):
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    d = len(M)
    P = lattice_plan(M)
    L = Lattice(M)
    incl = synth.random_inclusions(3, d, 4, 0.3)
    ph_p = synth.inclusions_phase(P.points(), P.m, incl)
    ph_o = synth.inclusions_phase(L.p, L.m, incl)
    perm = to_oracle_order(P.points(), L)
    C0 = synth.c0_mean_extremes([1, 10], [1, 10])
    E = np.zeros((2, P.n_c))
    E[0, 0] = 1.0
    E[1, -1] = 0.5
    g = basic_scheme_solve(P, torch.from_numpy(ph_p).to(cuda), LAM2, C0, E, tol=1e-6, maxit=2000, precision="mixed")
    assert g["status"] == 0
    S = stiff_tensors(LAM2, d)
    for lc in range(2):
        o = basic_scheme(L, ph_o, S, C0, el.comps_to_sym(E[lc], d), tol=1e-6, maxit=2000)
        # the increment form reports the same residual sequence up to rounding: same stopping iteration
        assert abs(int(g["iters"][lc]) - o["iters"]) <= 1
        eg = comps_to_tensor(g["eps"][lc].cpu().numpy(), d)
        assert relerr_global(eg, o["eps"][perm]) < MIXED_STRAIN_RTOL
        assert relerr_global(el.comps_to_sym(g["sigma_bar"][lc], d), o["sigma_bar"]) < MIXED_CEFF_RTOL


# ---------------------------------------------------------------- batches of microstructures
@pytest.mark.parametrize("M,prec", [([[128, 8], [0, 64]], "fp64"), ([[16, 4, 0], [0, 16, 4], [0, 0, 16]], "fp64"),
                                    ([[256, 16], [0, 256]], "mixed")])
def test_batch_of_microstructures_matches_oracle(cuda, M, prec):
    # items with different phase fields, phase counts, stiffness, reference media and strains, one launch set
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve_batch, lattice_plan
    d = len(M)
    P = lattice_plan(M)
    L = Lattice(M)
    perm = to_oracle_order(P.points(), L)
    rng = np.random.default_rng(11)
    phases, stiffs, C0s, Es, ph_or = [], [], [], [], []
    for i in range(5):
        incl = synth.random_inclusions(100 + i, d, 1 + i, 0.1 + 0.05 * i)
        ph_p = synth.inclusions_phase(P.points(), P.m, incl)
        ph_o = synth.inclusions_phase(L.p, L.m, incl)
        if i % 2:                                    # a third phase in some items
            ph_p = np.where(P.points()[:, 0] > P.m // 4, 2, ph_p).astype(np.uint8)
            ph_o = np.where(L.p[:, 0] > L.m // 4, 2, ph_o).astype(np.uint8)
        contrast = 10.0 ** rng.uniform(-1, 1)
        st = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(contrast, contrast), synth.iso_voigt(2.0, 0.7)][:2 + i % 2]
        lams = [1.0, contrast, 2.0][:2 + i % 2]
        mus = [1.0, contrast, 0.7][:2 + i % 2]
        phases.append(torch.from_numpy(ph_p).to(cuda))
        ph_or.append(ph_o)
        stiffs.append(st)
        C0s.append(synth.c0_mean_extremes(lams, mus))
        Es.append(rng.standard_normal(P.n_c))
    tol = 1e-6 if prec == "mixed" else 1e-9
    g = basic_scheme_solve_batch(P, phases, stiffs, C0s, np.array(Es), tol=tol, maxit=3000, precision=prec)
    for i in range(5):
        S = stiff_tensors(stiffs[i], d)
        o = basic_scheme(L, ph_or[i], S, C0s[i], el.comps_to_sym(Es[i], d), tol=tol, maxit=3000)
        eg = comps_to_tensor(g["eps"][i].cpu().numpy(), d)
        sb = el.comps_to_sym(g["sigma_bar"][i], d)
        if prec == "fp64":
            assert int(g["iters"][i]) == o["iters"]
            assert relerr(eg, o["eps"][perm]) < RTOL and relerr(sb, o["sigma_bar"]) < RTOL
        else:
            assert abs(int(g["iters"][i]) - o["iters"]) <= 1
            assert relerr_global(eg, o["eps"][perm]) < MIXED_STRAIN_RTOL
            assert relerr_global(sb, o["sigma_bar"]) < MIXED_CEFF_RTOL


# ---------------------------------------------------------------- generalized Hashin structure (3-D)
def _hashin_case(M, cuda, precision, tol, maxit):
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    w = synth.hashin_workload()
    P = lattice_plan(M)
    ph = synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
    E = np.eye(6)
    E[3:, 3:] *= 0.5                                   # unit load cases in tensor components
    g = basic_scheme_solve(P, torch.from_numpy(ph).to(cuda), w["stiffness"], w["C0"], E, tol=tol, maxit=maxit,
                           precision=precision)
    return w, P, ph, E, g


@pytest.mark.parametrize("M", [[[32, 0, 0], [0, 32, 0], [0, 0, 32]], [[32, 1, 0], [0, 32, 1], [0, 0, 32]],
                               [[32, 4, 0], [0, 32, 4], [0, 0, 32]]])
def test_hashin_mixed_six_load_cases_against_oracle(cuda, M):
    # the coated-ellipsoid shape at m = 32768: mixed precision, the six unit load cases in one batch, tol 1e-6
    w, P, ph, E, g = _hashin_case(M, cuda, "mixed", 1e-6, 2000)
    assert g["status"] == 0
    L = Lattice(M)
    perm = to_oracle_order(P.points(), L)
    ph_o = synth.coated_ellipsoid_phase(L.p, L.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
    S = np.array([el.voigt6_to_tensor(V, 3) for V in w["stiffness"]])
    Ceff = np.zeros((6, 6))
    for lc in range(6):
        o = basic_scheme(L, ph_o, S, w["C0"], el.comps_to_sym(E[lc], 3), tol=1e-6, maxit=2000)
        assert abs(int(g["iters"][lc]) - o["iters"]) <= 1
        eg = comps_to_tensor(g["eps"][lc].cpu().numpy(), 3)
        assert relerr_global(eg, o["eps"][perm]) < MIXED_STRAIN_RTOL
        assert relerr_global(el.comps_to_sym(g["sigma_bar"][lc], 3), o["sigma_bar"]) < MIXED_CEFF_RTOL
        Ceff[:, lc] = g["sigma_bar"][lc]
    # C^eff eps0 from the six columns against the analytic value (discretisation error at 32^3)
    e0 = el.sym_to_comps(w["eps0"])
    e0_eng = e0 * np.array([1, 1, 1, 2, 2, 2])
    ce = el.comps_to_sym(Ceff @ e0_eng, 3)
    assert np.linalg.norm(ce - w["ceff_eps0"]) / np.linalg.norm(w["ceff_eps0"]) < 0.05


@pytest.mark.parametrize("name", ["grid128", "rank1_2097152", "sheared128"])
def test_hashin_full_size_fp64_fixed_iterations(cuda, name):
    # the full coated-ellipsoid size (m = 2^21), the eps0 load case, binary64, two iterations compared field-wise
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    w = synth.hashin_workload()
    M = synth.LATTICES[name]
    P = lattice_plan(M)
    L = Lattice(M)
    perm = to_oracle_order(P.points(), L)
    ph = synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
    ph_o = synth.coated_ellipsoid_phase(L.p, L.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
    E = el.sym_to_comps(w["eps0"])[None]
    g = basic_scheme_solve(P, torch.from_numpy(ph).to(cuda), w["stiffness"], w["C0"], E, tol=0.0, maxit=2)
    S = np.array([el.voigt6_to_tensor(V, 3) for V in w["stiffness"]])
    o = basic_scheme(L, ph_o, S, w["C0"], w["eps0"], tol=0.0, maxit=2)
    assert relerr(comps_to_tensor(g["eps"][0].cpu().numpy(), 3), o["eps"][perm]) < RTOL
    assert relerr(el.comps_to_sym(g["sigma_bar"][0], 3), o["sigma_bar"]) < RTOL


@pytest.mark.parametrize("name", ["grid128", "rank1_2097152"])
def test_hashin_full_size_mixed_against_oracle(cuda, name):
    # the mixed path at the full coated-ellipsoid size (m = 2^21): the 128^3 grid takes the four-pass column path, the rank-1
    # lattice the two-pass four-step split of its 2^21-point axis.  Six unit load cases batched as in the
    # workload; the eps0 load case and one shear unit load case against the oracle (separable FFTs),
    # four fixed iterations, at the stated bounds
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    w = synth.hashin_workload()
    M = synth.LATTICES[name]
    P = lattice_plan(M)
    L = Lattice(M)
    perm = to_oracle_order(P.points(), L)
    ph = synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
    ph_o = synth.coated_ellipsoid_phase(L.p, L.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
    E = np.eye(6)
    E[3:, 3:] *= 0.5
    E[0] = el.sym_to_comps(w["eps0"])
    g = basic_scheme_solve(P, torch.from_numpy(ph).to(cuda), w["stiffness"], w["C0"], E, tol=1e-6, maxit=4,
                           precision="mixed")
    S = np.array([el.voigt6_to_tensor(V, 3) for V in w["stiffness"]])
    for lc in (0, 4):
        o = basic_scheme(L, ph_o, S, w["C0"], el.comps_to_sym(E[lc], 3), tol=1e-6, maxit=4)
        assert int(g["iters"][lc]) == o["iters"] == 4
        eg = comps_to_tensor(g["eps"][lc].cpu().numpy(), 3)
        e_strain = relerr_global(eg, o["eps"][perm])
        e_sb = relerr_global(el.comps_to_sym(g["sigma_bar"][lc], 3), o["sigma_bar"])
        print("%s lc %d: strain %.2e (per group %.2e), sigma_bar %.2e, residual history %s vs %s"
              % (name, lc, e_strain, relerr(eg, o["eps"][perm]), e_sb, g["resid"][lc], o["history"][-1]))
        assert e_strain < MIXED_STRAIN_RTOL
        assert e_sb < MIXED_CEFF_RTOL
        assert abs(g["resid"][lc] - o["history"][-1]) < 1e-5 * o["history"][-1]


@pytest.mark.parametrize("name", ["grid128", "rank1_2097152", "sheared128"])
def test_hashin_full_size_mixed_converged_against_fp64(cuda, name):
    # converged to r < 1e-6 at the full coated-ellipsoid size (m = 2^21): the mixed path's strain and C^eff against the binary64
    # path (itself held to the oracle at this size above) on the six unit load cases
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    w = synth.hashin_workload()
    P = lattice_plan(synth.LATTICES[name])
    ph = torch.from_numpy(synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"],
                                                       R=w["R"])).to(cuda)
    E = np.eye(6)
    E[3:, 3:] *= 0.5
    a = basic_scheme_solve(P, ph, w["stiffness"], w["C0"], E, tol=1e-6, maxit=2000, precision="mixed")
    b = basic_scheme_solve(P, ph, w["stiffness"], w["C0"], E, tol=1e-6, maxit=2000)
    assert a["status"] == b["status"] == 0
    assert np.all(np.abs(a["iters"] - b["iters"]) <= 1)
    for lc in range(6):
        es = float((a["eps"][lc] - b["eps"][lc]).abs().max() / b["eps"][lc].abs().max())
        ec = np.abs(a["sigma_bar"][lc] - b["sigma_bar"][lc]).max() / np.abs(b["sigma_bar"][lc]).max()
        assert es <= MIXED_STRAIN_RTOL and ec <= MIXED_CEFF_RTOL, (lc, es, ec)


def test_plain_launches_equal_graph_loop(cuda):
    # the plain-launch iteration (host convergence check) runs the same kernels in the same order
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    for M, prec in (([[512, 16], [0, 512]], "fp64"), ([[32, 4, 0], [0, 32, 4], [0, 0, 32]], "mixed")):
        P = lattice_plan(M)
        d = len(M)
        ph = torch.from_numpy(inclusions(3, d, 4, 0.3)(P.points(), P.m)).to(cuda)
        E = np.eye(3 if d == 2 else 6)[:2]
        a = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=1e-7, maxit=500, precision=prec)
        b = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=1e-7, maxit=500, precision=prec, plain_launches=True)
        assert a["status"] == b["status"] == 0
        assert np.array_equal(a["iters"], b["iters"])
        assert torch.equal(a["eps"], b["eps"])
        assert np.array_equal(a["sigma_bar"], b["sigma_bar"])


@pytest.mark.parametrize("M,prec", [([[512, 16], [0, 512]], "fp64"), ([[512, 16], [0, 512]], "df64"),
                                    ([[64, 0, 0], [0, 64, 0], [0, 0, 64]], "mixed"),
                                    ([[128, 1, 0], [0, 128, 1], [0, 0, 64]], "mixed")])
def test_autotuned_shapes_give_the_same_fields(cuda, M, prec):
    # the tuner regroups lines into blocks; every line's arithmetic is unchanged, so the fields are equal
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    P = lattice_plan(M)
    d = len(M)
    ph = torch.from_numpy(inclusions(3, d, 4, 0.3)(P.points(), P.m)).to(cuda)
    E = np.eye(P.n_c)[:2]
    a = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=0.0, maxit=6, precision=prec)
    assert P.tune_info(2, prec) is None
    info = P.autotune(2, prec)
    assert info is not None and info["rpc"] >= 1 and len(info["w"]) == len(info["ms"]) - 1
    b = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=0.0, maxit=6, precision=prec)
    assert torch.equal(a["eps"], b["eps"])
    c = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=1e-7, maxit=500, precision=prec)
    assert c["status"] == 0


# ---------------------------------------------------------------- transformed pattern P_L(M) (Sec. 3.3)
CELL2 = [[1.3, 0.4], [-0.2, 0.9]]
CELL3 = [[1.1, 0.3, -0.2], [0.0, 0.8, 0.25], [0.15, -0.1, 1.2]]


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", [[[16, 4], [0, 8]], [[512, 16], [0, 512]], [[64, 1], [0, 64]],
                               [[8, 1, 0], [0, 8, 1], [0, 0, 8]], [[16, 4, 0], [0, 16, 4], [0, 0, 16]]])
def test_transformed_cell_fixed_iterations(cuda, M, prec):
    d = len(M)
    E = np.eye(d * (d + 1) // 2)[:2] + 0.1
    out = run_pair(M, inclusions(6, d, 3, 0.3), LAM2, (5.5, 5.5), E, tol=0.0, maxit=5, cuda=cuda, precision=prec,
                   cell=CELL2 if d == 2 else CELL3)
    check_pair(*out, d=d)


@pytest.mark.parametrize("M", [[[256, 0], [0, 256]], [[32, 1, 0], [0, 32, 1], [0, 0, 32]]])
def test_transformed_cell_mixed_within_stated_tolerance(cuda, M):
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    d = len(M)
    P = lattice_plan(M)
    P.set_cell(CELL2 if d == 2 else CELL3)
    ph = torch.from_numpy(inclusions(7, d, 4, 0.3)(P.points(), P.m)).to(cuda)
    E = np.eye(P.n_c)[:2]
    a = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=1e-6, maxit=2000, precision="mixed")
    b = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=1e-6, maxit=2000)
    assert a["status"] == b["status"] == 0
    assert float((a["eps"] - b["eps"]).abs().max() / b["eps"].abs().max()) <= MIXED_STRAIN_RTOL
    assert np.abs(a["sigma_bar"] - b["sigma_bar"]).max() <= MIXED_CEFF_RTOL * np.abs(b["sigma_bar"]).max()


def test_transformed_aligned_laminate_is_analytic(cuda):
    # all frequencies of M = [[4096, 12288], [0, 1]] are parallel to (1, 3); in the cell L the laminate
    # is the analytic one with the physical normal L^{-T} (1, 3)
    import torch
    from oracle import analytic as an
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    P = lattice_plan([[4096, 12288], [0, 1]])
    P.set_cell(CELL2)
    ph = synth.laminate_phase(P.points(), P.m, [1, 3])
    E = np.array([[0.6, 0.0, 0.25]])
    g = basic_scheme_solve(P, torch.from_numpy(ph).to(cuda), LAM2, (5.5, 5.5), E, tol=1e-14, maxit=500)
    S = stiff_tensors(LAM2, 2)
    n_phys = np.linalg.inv(np.array(CELL2)).T @ np.array([1.0, 3.0])
    e1, e2, sb = an.laminate_fields(S[0], S[1], 0.5, n_phys, el.comps_to_sym(E[0], 2))
    ex = np.where(ph[:, None, None] == 0, e1, e2)
    eg = comps_to_tensor(g["eps"][0].cpu().numpy(), 2)
    assert relerr(eg, ex) < 1e-10
    assert relerr(el.comps_to_sym(g["sigma_bar"][0], 2), sb) < 1e-10


# ---------------------------------------------------------------- Eyre-Milton iteration (scheme option)
@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", [[[16, 4], [0, 8]], [[512, 16], [0, 512]], [[64, 1], [0, 64]],
                               [[8, 1, 0], [0, 8, 1], [0, 0, 8]], [[16, 4, 0], [0, 16, 4], [0, 0, 16]]])
def test_eyre_milton_fixed_iterations(cuda, M, prec):
    d = len(M)
    E = np.eye(d * (d + 1) // 2)[:2] + 0.1
    g = np.sqrt(10.0)
    out = run_pair(M, inclusions(6, d, 3, 0.3), LAM2, (g, g), E, tol=0.0, maxit=5, cuda=cuda, precision=prec,
                   scheme="eyre_milton")
    check_pair(*out, d=d)


@pytest.mark.parametrize("M", [[[256, 16], [0, 256]], [[32, 1, 0], [0, 32, 1], [0, 0, 32]]])
def test_eyre_milton_solution_and_iterations(cuda, M):
    import torch
    from paper_1605_05712_gb300 import LatticeError, basic_scheme_solve, lattice_plan
    d = len(M)
    P = lattice_plan(M)
    ph = torch.from_numpy(inclusions(7, d, 4, 0.3)(P.points(), P.m)).to(cuda)
    k = 100.0
    S = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(k, k)]
    E = np.eye(P.n_c)[:2]
    # same reference medium: the same discrete solution as Algorithm 1
    b = basic_scheme_solve(P, ph, S, ((1 + k) / 2, (1 + k) / 2), E, tol=1e-11, maxit=20000)
    e = basic_scheme_solve(P, ph, S, ((1 + k) / 2, (1 + k) / 2), E, tol=1e-11, maxit=20000, scheme="eyre_milton")
    assert b["status"] == e["status"] == 0
    assert float((b["eps"] - e["eps"]).abs().max() / b["eps"].abs().max()) < 1e-7
    # at its own reference (geometric mean) it converges in a fraction of the iterations
    b6 = basic_scheme_solve(P, ph, S, ((1 + k) / 2, (1 + k) / 2), E, tol=1e-6, maxit=20000)
    e6 = basic_scheme_solve(P, ph, S, (np.sqrt(k), np.sqrt(k)), E, tol=1e-6, maxit=20000, scheme="eyre_milton")
    assert int(e6["iters"].max()) < int(b6["iters"].max()) / 3
    # mixed precision within the stated tolerances of its binary64 counterpart
    m6 = basic_scheme_solve(P, ph, S, (np.sqrt(k), np.sqrt(k)), E, tol=1e-6, maxit=20000, scheme="eyre_milton",
                            precision="mixed")
    assert m6["status"] == 0
    assert float((m6["eps"] - e6["eps"]).abs().max() / e6["eps"].abs().max()) <= MIXED_STRAIN_RTOL
    assert np.abs(m6["sigma_bar"] - e6["sigma_bar"]).max() <= MIXED_CEFF_RTOL * np.abs(e6["sigma_bar"]).max()
    with pytest.raises(LatticeError):
        basic_scheme_solve(P, ph, S, (np.sqrt(k), np.sqrt(k)), E, tol=1e-6, maxit=10, scheme="eyre_milton",
                           boundary="zero")


# ---------------------------------------------------------------- conjugate gradients (scheme option)
# the rank-1 lattices with one point along x2 sample a line that misses the inclusions: a laminate there,
# with f1 = 3/10 (at f1 = 1/2 the square wave excites only odd harmonics, the boundary frequencies of
# these lattices, which are zeroed)
# The last five are general plans (mixed-radix kernels): (3, 5), (1, 60), rank-1 m = 3072 (four-step),
# 3-D (1, 3, 45) and (3, 3, 15).
CG_MATS = [[[16, 4], [0, 8]], [[256, 16], [0, 256]], [[64, 32], [0, 1]], [[4096, 12288], [0, 1]],
           [[8, 1, 0], [0, 8, 1], [0, 0, 8]], [[16, 4, 0], [0, 16, 4], [0, 0, 16]], [[2, 0], [0, 1]],
           [[3, 0], [0, 5]], [[6, 1], [0, 10]], [[3072, 0], [0, 1]], [[1, 0, 0], [0, 3, 0], [0, 0, 45]],
           [[3, 0, 0], [0, 3, 0], [0, 0, 15]]]


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", CG_MATS)
def test_cg_fixed_iterations(cuda, M, prec):
    # the oracle runs Hestenes-Stiefel CG, the kernels the Chronopoulos-Gear recurrences: equal iterates
    # up to rounding; [[2,0],[0,1]] converges at once and stops at the rounding floor on both sides
    d = len(M)
    E = np.eye(d * (d + 1) // 2)[:2] + 0.1
    ph = ((lambda p, m: synth.laminate_phase(p, m, [1, 3], Fraction(3, 10))) if d == 2 and M[1][1] == 1
          else inclusions(6, d, 3, 0.3))
    out = run_pair(M, ph, LAM2, (5.5, 5.5), E, tol=0.0, maxit=6, cuda=cuda, precision=prec,
                   scheme="cg", boundary="zero")
    # a residual at the rounding floor (<= 1024 u r_0) is rounding noise on both sides
    check_pair(*out, d=d, hist_atol=1e-13)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", [[[16, 4], [0, 8]], [[8, 1, 0], [0, 8, 1], [0, 0, 8]]])
def test_cg_transformed_cell_fixed_iterations(cuda, M, prec):
    # conjugate gradients on P_L(M): the Green operator at L^{-T} h, as in Algorithm 1
    d = len(M)
    E = np.eye(d * (d + 1) // 2)[:2] + 0.1
    out = run_pair(M, inclusions(6, d, 3, 0.3), LAM2, (5.5, 5.5), E, tol=0.0, maxit=5, cuda=cuda, precision=prec,
                   cell=CELL2 if d == 2 else CELL3, scheme="cg", boundary="zero")
    check_pair(*out, d=d, hist_atol=1e-13)


@pytest.mark.parametrize("M", [[[256, 16], [0, 256]], [[32, 1, 0], [0, 32, 1], [0, 0, 32]], [[96, 1], [0, 96]]])
def test_cg_solution_and_iterations(cuda, M):
    import torch
    from paper_1605_05712_gb300 import LatticeError, basic_scheme_solve, lattice_plan
    d = len(M)
    P = lattice_plan(M)
    ph = torch.from_numpy(inclusions(7, d, 4, 0.3)(P.points(), P.m)).to(cuda)
    k = 100.0
    S = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(k, k)]
    E = np.eye(P.n_c)[:2]
    C0 = ((1 + k) / 2, (1 + k) / 2)
    # Algorithm 1's discrete solution (boundary frequencies zeroed, where it does not depend on C0)
    b = basic_scheme_solve(P, ph, S, C0, E, tol=1e-11, maxit=20000, boundary="zero")
    c = basic_scheme_solve(P, ph, S, C0, E, tol=1e-11, maxit=2000, boundary="zero", scheme="cg")
    c2 = basic_scheme_solve(P, ph, S, (1.0, 3.0), E, tol=1e-11, maxit=2000, boundary="zero", scheme="cg")
    cd = basic_scheme_solve(P, ph, S, C0, E, tol=1e-11, maxit=2000, boundary="zero", scheme="cg", precision="df64")
    assert b["status"] == c["status"] == c2["status"] == cd["status"] == 0
    scale = float(b["eps"].abs().max())
    assert float((b["eps"] - c["eps"]).abs().max()) / scale < 1e-7
    assert float((c2["eps"] - c["eps"]).abs().max()) / scale < 1e-7
    assert float((cd["eps"] - c["eps"]).abs().max()) / scale < 1e-9
    assert np.abs(c["sigma_bar"] - b["sigma_bar"]).max() < 1e-7 * np.abs(b["sigma_bar"]).max()
    # far fewer transforms to the same tolerance
    b6 = basic_scheme_solve(P, ph, S, C0, E, tol=1e-6, maxit=20000, boundary="zero")
    c6 = basic_scheme_solve(P, ph, S, C0, E, tol=1e-6, maxit=2000, boundary="zero", scheme="cg")
    assert int(c6["iters"].max()) < int(b6["iters"].max()) / 4
    for kw in (dict(precision="mixed", boundary="zero"), dict(boundary="average"),
               dict(boundary="zero", eps0=c6["eps"].clone())):
        with pytest.raises(LatticeError):
            basic_scheme_solve(P, ph, S, C0, E, tol=1e-6, maxit=10, scheme="cg", **kw)


@pytest.mark.parametrize("plain", [False, True])
def test_cg_stops_in_the_prologue(cuda, plain):
    # a homogeneous medium has r = 0 after the first transform: one iteration, eps = E, and the loop that
    # follows the prologue must not run (its condition starts from the active count)
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    P = lattice_plan([[64, 8], [0, 32]])
    E = np.array([[0.3, -0.2, 0.1], [1.0, 0.0, 0.0]])
    zero = torch.zeros(P.m, dtype=torch.uint8, device=cuda)
    g = basic_scheme_solve(P, zero, [synth.iso_voigt(3.0, 2.0)], (1.0, 0.5), E, tol=1e-12, maxit=50,
                           boundary="zero", scheme="cg", plain_launches=plain, history=True)
    assert g["status"] == 0 and np.all(g["iters"] == 1)
    for lc in range(2):
        assert float((g["eps"][lc] - torch.tensor(E[lc], device=cuda)[:, None]).abs().max()) < 1e-14
    # maxit = 1 stops after the prologue too
    ph = torch.from_numpy(inclusions(2, 2, 3, 0.3)(P.points(), P.m)).to(cuda)
    g1 = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=1e-12, maxit=1, boundary="zero", scheme="cg",
                            plain_launches=plain)
    assert g1["status"] == 1 and np.all(g1["iters"] == 1)


def test_cg_batch_and_multi(cuda):
    # a batch where one item stops in the prologue and the others iterate; a multi call over two plans
    # equals its single solves bitwise, with the graph loop and with plain launches
    import torch
    from paper_1605_05712_gb300 import (basic_scheme_solve, basic_scheme_solve_batch, basic_scheme_solve_multi,
                                        lattice_plan)
    P = lattice_plan([[128, 8], [0, 64]])
    phs = [torch.from_numpy(inclusions(s, 2, 3, 0.3)(P.points(), P.m)).to(cuda) for s in (1, 2)]
    phs.append(torch.zeros(P.m, dtype=torch.uint8, device=cuda))
    Es = np.array([[1.0, 0.0, 0.0], [0.2, 0.5, -0.3], [0.4, 0.1, 0.2]])
    bt = basic_scheme_solve_batch(P, phs, [LAM2] * 3, [(5.5, 5.5)] * 3, Es, tol=1e-9, maxit=500, boundary="zero",
                                  scheme="cg")
    assert bt["status"] == 0 and bt["iters"][2] == 1 and bt["iters"][0] > 5
    for i in range(3):
        s = basic_scheme_solve(P, phs[i], LAM2, (5.5, 5.5), Es[i:i + 1], tol=1e-9, maxit=500, boundary="zero",
                               scheme="cg")
        assert int(s["iters"][0]) == int(bt["iters"][i])
        assert float((s["eps"][0] - bt["eps"][i]).abs().max()) <= 1e-12 * float(s["eps"].abs().max())
    P2 = lattice_plan([[8, 1, 0], [0, 8, 1], [0, 0, 16]])
    ph2 = torch.from_numpy(inclusions(4, 3, 2, 0.25)(P2.points(), P2.m)).to(cuda)
    probs = [dict(plan=P, phase=phs[0], stiffness=LAM2, C0=(5.5, 5.5), E=Es[:2]),
             dict(plan=P2, phase=ph2, stiffness=LAM2, C0=(2.0, 3.0), E=np.eye(6)[:2])]
    rc, outs = basic_scheme_solve_multi(probs, tol=1e-9, maxit=500, boundary="zero", scheme="cg")
    rc_p, outs_p = basic_scheme_solve_multi(probs, tol=1e-9, maxit=500, boundary="zero", scheme="cg",
                                            plain_launches=True)
    assert rc == rc_p == 0
    for pb, o, op in zip(probs, outs, outs_p):
        single = basic_scheme_solve(pb["plan"], pb["phase"], pb["stiffness"], pb["C0"], pb["E"], tol=1e-9,
                                    maxit=500, boundary="zero", scheme="cg")
        assert np.array_equal(o["iters"], single["iters"]) and np.array_equal(o["iters"], op["iters"])
        assert torch.equal(o["eps"], single["eps"]) and torch.equal(o["eps"], op["eps"])


# ---------------------------------------------------------------- failure detection (host-injected)
@pytest.mark.parametrize("where", ["stiffness", "E"])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "df64"])
def test_nan_input_reports_diverged(cuda, where, prec):
    # a NaN written on the host into a stiffness entry or the macroscopic strain makes the residual
    # non-finite: the solve stops at once with LAT_DIVERGED (2) and still writes its outputs
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    P = lattice_plan([[128, 8], [0, 64]])
    ph = torch.from_numpy(inclusions(3, 2, 3, 0.3)(P.points(), P.m)).to(cuda)
    stiff = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(10.0, 10.0)]
    E = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    if where == "stiffness":
        stiff[1] = stiff[1].copy()
        stiff[1][0, 0] = np.nan
    else:
        E[1, 0] = np.nan
    tol = 1e-6 if prec == "mixed" else 1e-8
    g = basic_scheme_solve(P, ph, stiff, (5.5, 5.5), E, tol=tol, maxit=300, precision=prec)
    assert g["status"] == 2
    bad = [1] if where == "E" else [0, 1]
    for lc in bad:
        assert not np.isfinite(g["resid"][lc]) and int(g["iters"][lc]) <= 2
    if where == "E":   # the other load case is untouched by the injected value
        assert np.isfinite(g["resid"][0]) and g["resid"][0] < tol


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_soft_reference_medium_reports_diverged(cuda, prec):
    # C0 at the softer phase of a contrast-100 composite: the iteration does not contract (its rate is
    # |c - c0| / c0 = 99); the residual grows geometrically, and the divergence rule stops the solve after
    # LAT_DIVERGE_STEPS growing iterations with a finite residual above 1, long before maxit.  The
    # double-float pairs carry binary32 exponents, so there the growing strain overflows first (about
    # 99^10 > 2^64, squared in the residual): a non-finite residual, LAT_DIVERGED as well
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    P = lattice_plan([[256, 16], [0, 256]])
    ph = torch.from_numpy(inclusions(7, 2, 4, 0.3)(P.points(), P.m)).to(cuda)
    stiff = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(100.0, 100.0)]
    g = basic_scheme_solve(P, ph, stiff, (1.0, 1.0), np.eye(3)[:1], tol=1e-8, maxit=1000, precision=prec,
                           history=True)
    h = np.asarray(g["history"][0])
    assert g["status"] == 2 and int(g["iters"][0]) < 100
    if np.isfinite(g["resid"][0]):
        assert int(g["iters"][0]) >= 16 and g["resid"][0] > 1.0
        assert np.all(np.diff(h[-16:]) > 0)
    else:
        assert prec == "df64" and np.all(np.diff(h[np.isfinite(h)]) > 0)
    # the same composite with an admissible reference medium converges
    ok = basic_scheme_solve(P, ph, stiff, (50.5, 50.5), np.eye(3)[:1], tol=1e-6, maxit=5000, precision=prec)
    assert ok["status"] == 0


# ---------------------------------------------------------------- general plans (mixed-radix kernels)
@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", [[[6, 1], [0, 10]], [[96, 1], [0, 96]], [[3, 0, 0], [0, 3, 0], [0, 0, 15]]])
def test_general_plan_eyre_milton_and_options(cuda, M, prec):
    # the Eyre-Milton scheme, the boundary-zero option (even divisors), a warm start and a transformed cell on
    # lattices with odd divisors, against the oracle field by field
    d = len(M)
    E = np.eye(d * (d + 1) // 2)[:2] + 0.1
    out = run_pair(M, inclusions(6, d, 3, 0.3), LAM2, (np.sqrt(10.0),) * 2, E, tol=0.0, maxit=5, cuda=cuda,
                   precision=prec, scheme="eyre_milton")
    check_pair(*out, d=d)
    out = run_pair(M, inclusions(4, d, 2, 0.3), LAM2, (5.5, 5.5), E, tol=0.0, maxit=5, boundary="zero", cuda=cuda,
                   precision=prec)
    check_pair(*out, d=d)
    out = run_pair(M, inclusions(5, d, 3, 0.3), LAM2, (5.5, 5.5), E, tol=0.0, maxit=4, cuda=cuda, precision=prec,
                   cell=CELL2 if d == 2 else CELL3)
    check_pair(*out, d=d)


def test_general_plan_warm_start_batch_multi_and_refusals(cuda):
    import torch
    from paper_1605_05712_gb300 import (LatticeError, basic_scheme_solve, basic_scheme_solve_batch,
                                        basic_scheme_solve_multi, lattice_plan)
    M = [[45, 9], [0, 45]]
    P = lattice_plan(M)
    L = Lattice(M)
    perm = to_oracle_order(P.points(), L)
    ph = inclusions(8, 2, 2, 0.3)
    E = np.array([[1.0, 0.5, -0.25]])
    S = stiff_tensors(LAM2, 2)
    o3 = basic_scheme(L, ph(L.p, L.m), S, (5.5, 5.5), el.comps_to_sym(E[0], 2), tol=0.0, maxit=3)
    o7 = basic_scheme(L, ph(L.p, L.m), S, (5.5, 5.5), el.comps_to_sym(E[0], 2), tol=0.0, maxit=7)
    warm = torch.from_numpy(np.ascontiguousarray(el.sym_to_comps(o3["eps"][perm]).T[None])).to(cuda)
    php = torch.from_numpy(ph(P.points(), P.m)).to(cuda)
    g = basic_scheme_solve(P, php, LAM2, (5.5, 5.5), E, tol=0.0, maxit=4, eps0=warm)
    assert relerr(comps_to_tensor(g["eps"][0].cpu().numpy(), 2), o7["eps"][perm]) < RTOL
    # a batch and a multi call (a general and a power-of-two plan in one graph) equal single solves
    phs = [php, torch.from_numpy(inclusions(9, 2, 3, 0.2)(P.points(), P.m)).to(cuda)]
    Es = np.array([[1.0, 0.0, 0.0], [0.2, 0.5, -0.3]])
    bt = basic_scheme_solve_batch(P, phs, [LAM2] * 2, [(5.5, 5.5)] * 2, Es, tol=1e-9, maxit=500)
    P2 = lattice_plan([[64, 8], [0, 32]])
    ph2 = torch.from_numpy(inclusions(4, 2, 2, 0.25)(P2.points(), P2.m)).to(cuda)
    rc, outs = basic_scheme_solve_multi([dict(plan=P, phase=phs[1], stiffness=LAM2, C0=(5.5, 5.5), E=Es[1:]),
                                         dict(plan=P2, phase=ph2, stiffness=LAM2, C0=(5.5, 5.5), E=Es[:1])],
                                        tol=1e-9, maxit=500)
    assert bt["status"] == 0 and rc == 0
    for i in range(2):
        s1 = basic_scheme_solve(P, phs[i], LAM2, (5.5, 5.5), Es[i:i + 1], tol=1e-9, maxit=500)
        assert int(s1["iters"][0]) == int(bt["iters"][i])
        assert torch.equal(s1["eps"][0], bt["eps"][i])
    s1 = basic_scheme_solve(P, phs[1], LAM2, (5.5, 5.5), Es[1:], tol=1e-9, maxit=500)
    assert torch.equal(s1["eps"], outs[0]["eps"])
    s2 = basic_scheme_solve(P2, ph2, LAM2, (5.5, 5.5), Es[:1], tol=1e-9, maxit=500)
    assert torch.equal(s2["eps"], outs[1]["eps"])


@pytest.mark.parametrize("M", [[[6, 1], [0, 10]], [[3, 0, 0], [0, 3, 0], [0, 0, 15]]])
def test_general_plan_mixed_forms(cuda, M):
    # binary32 on general plans: the Eyre-Milton scheme (whose first step is taken in full), the plain
    # (non-increment) form and a contrast-100 composite (the pair restart removes the binary32 offset),
    # within the stated bounds
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, lattice_plan
    d = len(M)
    P = lattice_plan(M)
    L = Lattice(M)
    perm = to_oracle_order(P.points(), L)
    incl = synth.random_inclusions(12, d, 3, 0.3)
    ph_p = torch.from_numpy(synth.inclusions_phase(P.points(), P.m, incl)).to(cuda)
    ph_o = synth.inclusions_phase(L.p, L.m, incl)
    E = np.eye(P.n_c)[:2] + 0.1
    for lam, kw, okw in (((10.0, 10.0), dict(scheme="eyre_milton"), dict(scheme="eyre_milton")),
                         ((10.0, 10.0), dict(mixed_increment=False), {}),
                         ((100.0, 100.0), {}, {})):
        voigts = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(*lam)]
        C0 = (np.sqrt(lam[0]),) * 2 if "scheme" in kw else synth.c0_mean_extremes([1, lam[0]], [1, lam[1]])
        g = basic_scheme_solve(P, ph_p, voigts, C0, E, tol=1e-6, maxit=3000, precision="mixed", **kw)
        assert g["status"] == 0
        S = stiff_tensors(voigts, d)
        for lc in range(2):
            o = basic_scheme(L, ph_o, S, C0, el.comps_to_sym(E[lc], d), tol=1e-6, maxit=3000, **okw)
            assert abs(int(g["iters"][lc]) - o["iters"]) <= 1
            eg = comps_to_tensor(g["eps"][lc].cpu().numpy(), d)
            assert relerr_global(eg, o["eps"][perm]) < MIXED_STRAIN_RTOL
            assert relerr_global(el.comps_to_sym(g["sigma_bar"][lc], d), o["sigma_bar"]) < MIXED_CEFF_RTOL


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", [[[1009, 0], [0, 1]], [[2018, 1], [0, 1]], [[1, 0, 0], [0, 1, 0], [0, 0, 1021]]])
def test_prime_length_lattice(cuda, M, prec):
    # a rank-1 pattern of prime length (1009, 2 x 1009, 1021): the direct p-point DFT stage.  The pattern
    # lies on a line, so the laminate with normal (1, 3[, 2]) is heterogeneous along it
    d = len(M)
    E = np.eye(d * (d + 1) // 2)[:2] + 0.1
    ph = laminate([1, 3] if d == 2 else [1, 3, 2])
    out = run_pair(M, ph, LAM2, (5.5, 5.5), E, tol=0.0, maxit=6, cuda=cuda, precision=prec)
    assert 0 < np.count_nonzero(ph(out[1].p, out[1].m)) < out[1].m
    # the direct p-point DFT sums p terms: its rounding grows like sqrt(p) u instead of log2(m) u, which
    # sets the absolute floor of the residual history once the laminate has converged (~1e-13 by step 5)
    check_pair(*out, d=d, hist_atol=1e-14 if prec == "fp64" else None)


@pytest.mark.parametrize("M", BLUE_MATS)
def test_chirp_z_lattice(cuda, M):
    # the chirp-z rows (Bluestein) against the oracle: Algorithm 1 on a laminate (rank-1 patterns lie on a
    # line, along which the laminate with normal (1, 3[, 2]) is heterogeneous) or on inclusions, then the
    # Eyre-Milton scheme and conjugate gradients; binary64 only (the other precisions are refused)
    from paper_1605_05712_gb300 import LatticeError, basic_scheme_solve, lattice_plan
    import torch
    d = len(M)
    E = np.eye(d * (d + 1) // 2)[:2] + 0.1
    P = lattice_plan(M)
    assert P.layout()["split"] == 2
    rank1 = P.divisors[:-1] == [1] * (d - 1)
    ph = laminate([1, 3] if d == 2 else [1, 3, 2]) if rank1 else inclusions(7, d, 2, 0.3)
    out = run_pair(M, ph, LAM2, (5.5, 5.5), E, tol=0.0, maxit=5, cuda=cuda)
    assert 0 < np.count_nonzero(ph(out[1].p, out[1].m)) < out[1].m
    check_pair(*out, d=d, hist_atol=1e-14)
    out = run_pair(M, ph, LAM2, (np.sqrt(10.0),) * 2, E, tol=0.0, maxit=4, cuda=cuda, scheme="eyre_milton")
    check_pair(*out, d=d, hist_atol=1e-14)
    # conjugate gradients (the boundary frequencies of an even largest divisor zeroed); a laminate with
    # f1 = 3/10 on the rank-1 lines, so that the even lattices' load is not all boundary harmonics
    phc = ((lambda p, m: synth.laminate_phase(p, m, [1, 3] if d == 2 else [1, 3, 2], Fraction(3, 10))) if rank1
           else ph)
    out = run_pair(M, phc, LAM2, (5.5, 5.5), E, tol=0.0, maxit=5, cuda=cuda, scheme="cg", boundary="zero")
    assert 0 < np.count_nonzero(phc(out[1].p, out[1].m)) < out[1].m
    check_pair(*out, d=d, hist_atol=1e-13)
    php = torch.from_numpy(ph(P.points(), P.m)).to(cuda)
    for kw in (dict(precision="df64"), dict(precision="mixed"), dict(precision="df64", scheme="cg", boundary="zero")):
        with pytest.raises(LatticeError) as ei:
            basic_scheme_solve(P, php, LAM2, (5.5, 5.5), E, tol=1e-6, maxit=10, **kw)
        assert ei.value.code == -5


# ---------------------------------------------------------------- asynchronous entry point
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_async_solve_matches_synchronous(cuda, prec):
    # basic_scheme_solve_async returns before the solve ends; after a synchronization its device results
    # equal basic_scheme_solve's bitwise (same kernels, same graph); a non-converged and a diverged item
    # report their outcome in the status array
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, basic_scheme_solve_async, lattice_plan
    for M in ([[256, 16], [0, 256]], [[32, 4, 0], [0, 32, 4], [0, 0, 32]], [[45, 9], [0, 45]]):
        P = lattice_plan(M)
        d = len(M)
        ph = torch.from_numpy(inclusions(3, d, 4, 0.3)(P.points(), P.m)).to(cuda)
        E = np.eye(P.n_c)[:2]
        ref = basic_scheme_solve(P, ph, LAM2, (5.5, 5.5), E, tol=1e-7, maxit=500, precision=prec)
        a = basic_scheme_solve_async(P, ph, LAM2, (5.5, 5.5), E, tol=1e-7, maxit=500, precision=prec)
        torch.cuda.synchronize()
        assert torch.equal(a["eps"], ref["eps"])
        assert np.array_equal(a["iters"].cpu().numpy(), ref["iters"])
        assert np.array_equal(a["sigma_bar"].cpu().numpy(), ref["sigma_bar"])
        assert np.array_equal(a["resid"].cpu().numpy(), ref["resid"])
        assert np.all(a["status"].cpu().numpy() == 0)
    P = lattice_plan([[64, 8], [0, 32]])
    ph = torch.from_numpy(inclusions(3, 2, 3, 0.3)(P.points(), P.m)).to(cuda)
    a = basic_scheme_solve_async(P, ph, LAM2, (5.5, 5.5), np.eye(3)[:1], tol=1e-12, maxit=3, precision=prec)
    stiff = [LAM2[0], LAM2[1].copy()]
    stiff[1][0, 0] = np.nan
    b = basic_scheme_solve_async(P, ph, stiff, (5.5, 5.5), np.eye(3)[:1], tol=1e-8, maxit=50, precision=prec)
    torch.cuda.synchronize()
    assert int(a["status"][0]) == 1 and int(a["iters"][0]) == 3
    assert int(b["status"][0]) == 2


# ---------------------------------------------------------------- per-point stiffness field
def _random_spd_voigts(rng, m):
    """m seeded anisotropic stiffness matrices: isotropic (lam, mu) per point plus a random positive
    semidefinite perturbation (Voigt form, engineering shear)."""
    out = np.empty((m, 6, 6))
    for i in range(m):
        lam, mu = 10 ** rng.uniform(-0.5, 1.0), 10 ** rng.uniform(-0.5, 1.0)
        A = rng.standard_normal((6, 6))
        out[i] = synth.iso_voigt(lam, mu) + 0.05 * mu * (A @ A.T) / 6
    return out


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("M", [[[16, 4], [0, 8]], [[8, 1, 0], [0, 8, 1], [0, 0, 8]], [[6, 1], [0, 10]],
                               [[3, 0, 0], [0, 3, 0], [0, 0, 15]]])
def test_field_solve_matches_oracle(cuda, M, prec):
    # a genuinely per-point anisotropic field: the oracle gives every point its own phase
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve_field, lattice_plan, voigt_field
    P, L = lattice_plan(M), Lattice(M)
    d = L.d
    perm = to_oracle_order(P.points(), L)
    rng = np.random.default_rng(21)
    V_or = _random_spd_voigts(rng, L.m)                     # oracle order
    V_plan = V_or[perm]
    field = torch.from_numpy(voigt_field(V_plan)).to(cuda)
    E = np.eye(P.n_c)[:2] + 0.1
    C0 = (5.0, 4.0)
    g = basic_scheme_solve_field(P, field, C0, E, tol=0.0, maxit=5, precision=prec, want_sigma=True, history=True)
    S = np.array([el.voigt6_to_tensor(v, d) for v in V_or])
    for lc in range(2):
        o = basic_scheme(L, np.arange(L.m), S, C0, el.comps_to_sym(E[lc], d), tol=0.0, maxit=5)
        assert relerr(comps_to_tensor(g["eps"][lc].cpu().numpy(), d), o["eps"][perm]) < RTOL
        assert relerr(comps_to_tensor(g["sigma"][lc].cpu().numpy(), d), o["sigma"][perm]) < RTOL
        assert relerr(el.comps_to_sym(g["sigma_bar"][lc], d), o["sigma_bar"]) < RTOL
        ho = np.array(o["history"])
        atol = 1e-13 if prec == "df64" else 1e-15
        assert np.all(np.abs(np.array(g["history"][lc]) - ho) <= 1e-9 * ho + atol)


# the last two are general plans: rank-1 m = 9216 (four-step 96 x 96, mixed-radix) and the 24^3 grid
@pytest.mark.parametrize("M", [[[256, 16], [0, 256]], [[32, 1, 0], [0, 32, 1], [0, 0, 32]], [[96, 1], [0, 96]],
                               [[24, 0, 0], [0, 24, 0], [0, 0, 24]]])
def test_field_solve_equals_phase_solve(cuda, M):
    # the field built from a phase field and its table solves the same problem as the phase form: binary64
    # and df64 to rounding, mixed within its stated bounds against binary64
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, basic_scheme_solve_field, lattice_plan, voigt_field
    P = lattice_plan(M)
    d = len(M)
    ph = inclusions(3, d, 4, 0.3)(P.points(), P.m)
    V = np.array(LAM2)[ph]
    field = torch.from_numpy(voigt_field(V)).to(cuda)
    phd = torch.from_numpy(ph).to(cuda)
    E = np.eye(P.n_c)[:2]
    ref = basic_scheme_solve(P, phd, LAM2, (5.5, 5.5), E, tol=1e-8, maxit=2000)
    for prec in ("fp64", "df64"):
        f = basic_scheme_solve_field(P, field, (5.5, 5.5), E, tol=1e-8, maxit=2000, precision=prec)
        assert f["status"] == 0 and np.array_equal(f["iters"], ref["iters"])
        assert float((f["eps"] - ref["eps"]).abs().max() / ref["eps"].abs().max()) < 1e-11
        assert np.abs(f["sigma_bar"] - ref["sigma_bar"]).max() < 1e-11 * np.abs(ref["sigma_bar"]).max()
    r6 = basic_scheme_solve(P, phd, LAM2, (5.5, 5.5), E, tol=1e-6, maxit=2000)
    fm = basic_scheme_solve_field(P, field, (5.5, 5.5), E, tol=1e-6, maxit=2000, precision="mixed")
    assert fm["status"] == 0
    assert float((fm["eps"] - r6["eps"]).abs().max() / r6["eps"].abs().max()) <= MIXED_STRAIN_RTOL
    assert np.abs(fm["sigma_bar"] - r6["sigma_bar"]).max() <= MIXED_CEFF_RTOL * np.abs(r6["sigma_bar"]).max()


@pytest.mark.parametrize("M", [[[2053, 7], [0, 1]], [[3, 0, 0], [0, 1, 0], [0, 0, 3093]]])
def test_field_solve_on_chirp_z_lattice(cuda, M):
    # a largest divisor with no split into two passes (chirp-z rows, binary64): the field built from a
    # phase field and its table solves the phase problem to rounding
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, basic_scheme_solve_field, lattice_plan, voigt_field
    P = lattice_plan(M)
    assert P.layout()["split"] == 2
    d = len(M)
    ph = inclusions(5, d, 3, 0.3)(P.points(), P.m)
    V = np.array(LAM2)[ph]
    field = torch.from_numpy(voigt_field(V)).to(cuda)
    phd = torch.from_numpy(ph).to(cuda)
    E = np.eye(P.n_c)[:2]
    ref = basic_scheme_solve(P, phd, LAM2, (5.5, 5.5), E, tol=1e-8, maxit=2000)
    f = basic_scheme_solve_field(P, field, (5.5, 5.5), E, tol=1e-8, maxit=2000)
    assert ref["status"] == 0 and f["status"] == 0 and np.array_equal(f["iters"], ref["iters"])
    assert float((f["eps"] - ref["eps"]).abs().max() / ref["eps"].abs().max()) < 1e-11
    assert np.abs(f["sigma_bar"] - ref["sigma_bar"]).max() < 1e-11 * np.abs(ref["sigma_bar"]).max()
