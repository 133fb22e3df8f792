"""GPU tests of basic_scheme_solve_multi: independent problems on different lattices in one call (one
CUDA graph, a WHILE loop per plan, problems sharing a plan batched).

- fixed iterations against the oracle, element by element (binary64, 1e-10 relative);
- bitwise equality with one basic_scheme_solve per problem and with the plain-launch loop;
- the uneven serving sweep (256 problems, m = 2^12 .. 2^21, 2-D and 3-D, rank-1 / rank-2 / diagonal
  lattices, contrast 1e-2 .. 1e2) in mixed precision to a 1e-6 residual: every problem converges,
  the mean strain is E to binary32 rounding, and sampled problems agree with their binary64 solution within the mixed
  tolerances (strain 1e-5, effective stress 1e-6).
"""
import numpy as np
import pytest

from oracle import elasticity as el
from oracle.lattice import Lattice
from oracle.scheme import basic_scheme
from paper_1605_05712_gb300 import synth

pytestmark = pytest.mark.gpu


def _problems(sweep, cuda, plans=None):
    import torch
    from paper_1605_05712_gb300 import lattice_plan
    out = []
    for i, s in enumerate(sweep):
        P = plans[i] if plans is not None else lattice_plan(s["M"])
        ph = torch.from_numpy(synth.inclusions_phase(P.points(), P.m, s["incl"])).to(cuda)
        out.append(dict(plan=P, phase=ph, stiffness=s["stiffness"], C0=s["C0"], E=s["E"]))
    return out


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_multi_matches_oracle_fixed_iterations(cuda):
    from paper_1605_05712_gb300 import basic_scheme_solve_multi, lattice_plan
    sweep = synth.serving_sweep(n=9, seed=synth.BASE_SEED + 5000, m_exp=(6, 12))
    # two more problems on the lattice of the first: they batch with it
    extra = synth.serving_sweep(n=2, seed=synth.BASE_SEED + 6000, m_exp=(6, 6))
    for e in extra:
        e.update(d=sweep[0]["d"], M=sweep[0]["M"], m=sweep[0]["m"], E=sweep[0]["E"])
        if sweep[0]["d"] != len(e["incl"]["centers"][0]):
            e["incl"] = synth.random_inclusions(7, sweep[0]["d"], 2, 0.2)
    sweep = sweep + extra
    plans = [lattice_plan(s["M"]) for s in sweep[:9]]
    plans += [plans[0], plans[0]]
    probs = _problems(sweep, cuda, plans)
    maxit = 6
    rc, outs = basic_scheme_solve_multi(probs, tol=0.0, maxit=maxit)
    assert rc == 1                                   # LAT_NOT_CONVERGED: tol 0 runs maxit iterations
    for s, pb, o in zip(sweep, probs, outs):
        d = s["d"]
        L = Lattice(s["M"])
        idx = {tuple(r): i for i, r in enumerate(L.p.tolist())}
        perm = np.array([idx[tuple(r)] for r in pb["plan"].points().tolist()])
        ph = synth.inclusions_phase(L.p, L.m, s["incl"])
        S = np.array([el.voigt6_to_tensor(v, d) for v in s["stiffness"]])
        assert np.all(o["iters"] == maxit)
        for lc in range(len(s["E"])):
            ref = basic_scheme(L, ph, S, s["C0"], el.comps_to_sym(s["E"][lc], d), tol=0.0, maxit=maxit)
            got = el.comps_to_sym(o["eps"][lc].cpu().numpy().T, d)
            assert _relerr(got, ref["eps"][perm]) < 1e-10
            assert _relerr(el.comps_to_sym(o["sigma_bar"][lc], d), ref["sigma_bar"]) < 1e-10


def test_multi_equals_single_solves_and_plain_launches(cuda):
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, basic_scheme_solve_multi
    sweep = synth.serving_sweep(n=12, seed=synth.BASE_SEED + 7000, m_exp=(10, 16))
    probs = _problems(sweep, cuda)
    for prec in ("mixed", "fp64"):
        rc, outs = basic_scheme_solve_multi(probs, tol=1e-6, maxit=4000, precision=prec)
        rc_p, outs_p = basic_scheme_solve_multi(probs, tol=1e-6, maxit=4000, precision=prec, plain_launches=True)
        assert rc == rc_p == 0
        for pb, o, op in zip(probs, outs, outs_p):
            single = basic_scheme_solve(pb["plan"], pb["phase"], pb["stiffness"], pb["C0"], pb["E"], tol=1e-6,
                                        maxit=4000, precision=prec)
            assert np.array_equal(o["iters"], single["iters"]) and np.array_equal(o["iters"], op["iters"])
            assert torch.equal(o["eps"], single["eps"]) and torch.equal(o["eps"], op["eps"])
            assert np.array_equal(o["sigma_bar"], single["sigma_bar"])


def test_serving_sweep_256_mixed(cuda):
    import torch
    from paper_1605_05712_gb300 import basic_scheme_solve, basic_scheme_solve_multi
    sweep = synth.serving_sweep()
    probs = _problems(sweep, cuda)
    rc, outs = basic_scheme_solve_multi(probs, tol=1e-6, maxit=5000, precision="mixed")
    assert rc == 0
    for s, o in zip(sweep, outs):
        assert np.all(o["resid"] < 1e-6)
        # <eps> = E: the binary32 increments have zero mean up to their rounding, accumulated over the
        # iterations (about 1e-8 here; binary64 keeps it to 1e-15)
        mean = o["eps"].mean(dim=2).cpu().numpy()
        assert np.abs(mean - s["E"]).max() < 1e-6
    # sampled problems against their binary64 solution: the extremes of contrast and size
    order = np.argsort([s["contrast"] for s in sweep])
    sizes = np.argsort([s["m"] for s in sweep])
    for i in sorted(set([order[0], order[1], order[-1], order[-2], sizes[-1], sizes[0]])):
        pb, o = probs[i], outs[i]
        ref = basic_scheme_solve(pb["plan"], pb["phase"], pb["stiffness"], pb["C0"], pb["E"], tol=1e-6, maxit=5000)
        e_ref = ref["eps"]
        strain_err = float((o["eps"] - e_ref).abs().max() / e_ref.abs().max())
        ceff_err = float(np.abs(o["sigma_bar"] - ref["sigma_bar"]).max() / np.abs(ref["sigma_bar"]).max())
        assert strain_err <= 1e-5, (i, sweep[i]["contrast"], strain_err)
        assert ceff_err <= 1e-6, (i, sweep[i]["contrast"], ceff_err)
