"""GPU tests of subsampling (Sec. 2.1, Sec. 5.2) and rearrangement (Sec. 2.2) through lattice_gather:
bit-exact against direct sampling on the target pattern, and the paper's subsampling experiment
(full 64 x 64 grid M_a, rank-1 subpattern M_b = [[64,32],[0,1]], pixel subgrid M_c = diag(8,8)) solved
on the GPU from fields gathered off the full grid, with the oracle's iteration counts."""
import numpy as np
import pytest

from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme
from paper_1605_05712_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Mf,Mt", [([[64, 0], [0, 64]], [[64, 32], [0, 1]]), ([[8, 4], [0, 4]], [[8, 12], [0, 4]]),
                                   ([[32, 0, 0], [0, 32, 0], [0, 0, 32]], [[32, 16, 0], [0, 2, 0], [0, 0, 32]])])
def test_gather_equals_direct_sampling(cuda, Mf, Mt):
    import torch
    from paper_1605_05712_gb300 import gather, gather_map, lattice_plan
    src, dst = lattice_plan(Mf), lattice_plan(Mt)
    mp = torch.from_numpy(gather_map(src, dst)).to(cuda)
    d = src.d
    n_int = [2, 1] if d == 2 else [1, 2, 3]
    ph_src = torch.from_numpy(synth.laminate_phase(src.points(), src.m, n_int)).to(cuda)
    ph_dst = synth.laminate_phase(dst.points(), dst.m, n_int)
    assert np.array_equal(gather(ph_src, mp).cpu().numpy(), ph_dst)
    # binary64 planes: the coordinates y = p / m of each point (equal rationals round alike)
    y_src = torch.from_numpy((src.points().T / src.m).copy()).to(cuda)
    y_dst = dst.points().T / dst.m
    assert np.array_equal(gather(y_src, mp).cpu().numpy(), y_dst)


def test_paper_subsampling_experiment_on_gpu(cuda):
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, gather, gather_map, lattice_plan
    Pa = lattice_plan([[64, 0], [0, 64]])
    ph_a = torch.from_numpy(synth.laminate_phase(Pa.points(), Pa.m, [2, 1])).to(cuda)
    S = [synth.iso_voigt(1.0, 1.0), synth.iso_voigt(10.0, 10.0)]
    E = np.array([[1.0, 0.0, 0.0]])
    its = {}
    for name, M in (("M_a", None), ("M_b", [[64, 32], [0, 1]]), ("M_c", [[8, 0], [0, 8]])):
        P, ph = (Pa, ph_a) if M is None else (lattice_plan(M), None)
        if M is not None:
            ph = gather(ph_a, torch.from_numpy(gather_map(Pa, P)).to(cuda))
        g = basic_scheme_solve(P, ph, S, (5.5, 5.5), E, tol=1e-9, maxit=2000)
        L = Lattice(M if M is not None else [[64, 0], [0, 64]])
        o = basic_scheme(L, synth.laminate_phase(L.p, L.m, [2, 1]), np.array([el.voigt6_to_tensor(v, 2) for v in S]),
                         (5.5, 5.5), el.comps_to_sym(E[0], 2), tol=1e-9, maxit=2000)
        assert int(g["iters"][0]) == o["iters"]
        its[name] = o["iters"]
    # Sec. 5.2: the directional subpattern converges in a fraction of the iterations of either grid
    assert its["M_b"] < its["M_a"] / 3 and its["M_b"] < its["M_c"] / 3
