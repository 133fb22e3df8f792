"""The Sec. 5.1 shear sweep on the GPU: the coated ellipse of Example 4.1 (one point along x3) on the
393 pattern matrices M_{j,k,alpha} and M~_j, all in one basic_scheme_solve_multi call.  Checks: every
problem converges; three of them agree with the oracle field by field at fixed iterations; the
Table-1 errors against the analytic solution (e_eff of C^eff eps0, e_l2 of the strain field) are in
the range the paper reports for this geometry (its Lame constants are not printed, so the values
are trend checks)."""
import numpy as np
import pytest

from oracle import analytic as an
from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme
from paper_1605_05712_gb300 import synth

pytestmark = pytest.mark.gpu

TABLE1 = ["M_7,0,0", "M~_7", "M_8,-240,0", "M_8,16,0", "M_8,272,0", "M_9,-496,0", "M_9,16,0", "M_7,256,1",
          "M_7,272,1"]


def _eps0_comps(e):
    return np.array([e[0, 0], e[1, 1], e[2, 2], e[1, 2], e[0, 2], e[0, 1]])


def _problems(cuda, w, mats):
    import torch
    from paper_1605_05712_gb300 import lattice_plan
    out = []
    for name, M in mats:
        P = lattice_plan(M)
        ph = synth.coated_ellipsoid_phase(P.points(), P.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
        out.append(dict(name=name, M=M, plan=P, phase=torch.from_numpy(ph).to(cuda), stiffness=w["stiffness"],
                        C0=w["C0"], E=_eps0_comps(w["eps0"])[None]))
    return out


def test_shear_sweep_on_gpu(cuda):
    from paper_1605_05712_gb300 import basic_scheme_solve_multi
    w = synth.hashin2d_workload()
    H = an.Hashin(w["c"], w["rho_c"], w["rho_e"], 10.0, 10.0, 1.0, 1.0, R=w["R"])
    assert np.abs(H.eps0 - w["eps0"]).max() < 1e-10                  # oracle and generator agree
    mats = synth.shear_sweep_matrices()
    assert len(mats) == 393
    probs = _problems(cuda, w, mats)
    rc, outs = basic_scheme_solve_multi(probs, tol=1e-8, maxit=3000)
    assert rc == 0
    ce_ref = np.array([w["ceff_eps0"][i, j] for (i, j) in ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))])
    Sv = np.array([el.voigt6_to_tensor(v, 3) for v in w["stiffness"]])
    e_eff, e_l2 = {}, {}
    for pb, o in zip(probs, outs):
        sb = o["sigma_bar"][0]
        e_eff[pb["name"]] = np.linalg.norm(el.comps_to_sym(sb, 3) - w["ceff_eps0"]) / np.linalg.norm(w["ceff_eps0"])
        if pb["name"] in TABLE1:
            x = pb["plan"].points() / pb["plan"].m
            ex = H.strain(x)
            eg = el.comps_to_sym(o["eps"][0].cpu().numpy().T, 3)
            e_l2[pb["name"]] = np.sqrt(el.frob2(eg - ex).sum() / el.frob2(ex).sum())
    for name in TABLE1:
        print("%-12s e_eff %.4f  e_l2 %.3f" % (name, e_eff[name], e_l2[name]))
    assert max(e_eff.values()) < 0.02 and max(e_l2.values()) < 0.2
    # direction matters: the best pattern of the sweep beats the axis-aligned grid M_7,0,0
    assert min(e_eff.values()) < e_eff["M_7,0,0"]
    assert np.abs(ce_ref).max() > 0


def test_shear_sweep_matches_oracle_fixed_iterations(cuda):
    from paper_1605_05712_gb300 import basic_scheme_solve_multi
    w = synth.hashin2d_workload()
    mats = [m for m in synth.shear_sweep_matrices() if m[0] in ("M_9,16,0", "M_7,272,1", "M~_8")]
    probs = _problems(cuda, w, mats)
    rc, outs = basic_scheme_solve_multi(probs, tol=0.0, maxit=4)
    Sv = np.array([el.voigt6_to_tensor(v, 3) for v in w["stiffness"]])
    for pb, o in zip(probs, outs):
        L = Lattice(pb["M"])
        idx = {tuple(r): i for i, r in enumerate(L.p.tolist())}
        perm = np.array([idx[tuple(r)] for r in pb["plan"].points().tolist()])
        ph = synth.coated_ellipsoid_phase(L.p, L.m, w["c"], w["rho_c"], w["rho_e"], R=w["R"])
        ref = basic_scheme(L, ph, Sv, w["C0"], w["eps0"], tol=0.0, maxit=4)
        got = el.comps_to_sym(o["eps"][0].cpu().numpy().T, 3)
        assert np.abs(got - ref["eps"][perm]).max() < 1e-10 * np.abs(ref["eps"]).max()
