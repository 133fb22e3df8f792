"""Host-side checks of the uneven serving sweep (256 independent problems on different lattices): the
generator's matrices have the divisors their kind promises (checked with the oracle's Smith normal
form), the generator is deterministic, and every problem's launch geometry fits (the solver's workspace
queries return 0 for a shape it would refuse)."""
import numpy as np

from oracle.lattice import smith_normal_form
from paper_1605_05712_gb300 import lattice_plan, multi_workspace_bytes, synth


def test_sweep_divisors_match_kind():
    sw = synth.serving_sweep()
    assert len(sw) == 256
    kinds = {k: 0 for k in ("rank1", "rank2", "diag")}
    for s in sw:
        M = np.array(s["M"], dtype=np.int64)
        m = s["m"]
        assert abs(round(np.linalg.det(M))) == m and 2 ** 12 <= m <= 2 ** 21
        _, e, _ = smith_normal_form(M)
        e = [int(x) for x in e]
        kinds[s["kind"]] += 1
        if s["kind"] == "rank1":
            assert e[:-1] == [1] * (s["d"] - 1) and e[-1] == m
        elif s["kind"] == "rank2":
            nontriv = [x for x in e if x > 1]
            assert len(nontriv) == 2 and nontriv[1] % nontriv[0] == 0
        else:
            assert np.count_nonzero(M - np.diag(np.diag(M))) == 0
        assert len(s["E"]) == s["d"] * (s["d"] + 1) // 2
        assert 0.01 <= s["contrast"] <= 100.0
    assert min(kinds.values()) > 50
    again = synth.serving_sweep(n=4)
    assert all(a["M"] == b["M"] and a["contrast"] == b["contrast"] for a, b in zip(again, sw[:4]))


def test_sweep_geometry_fits():
    sw = synth.serving_sweep()
    probs = [dict(plan=lattice_plan(s["M"]), stiffness=s["stiffness"], E=s["E"]) for s in sw]
    for prec in ("fp64", "mixed"):
        assert all(multi_workspace_bytes([p], prec) > 0 for p in probs)
        assert multi_workspace_bytes(probs, prec) >= sum(multi_workspace_bytes([p], prec) for p in probs)


def test_shear_sweep_matrices_and_workload():
    from oracle.lattice import smith_normal_form
    mats = synth.shear_sweep_matrices()
    assert len(mats) == 393
    for name, M in mats:
        det = abs(round(np.linalg.det(np.array(M, float))))
        assert det == (2 ** 13 if name.startswith("M~") else 2 ** 14)
        _, e, _ = smith_normal_form(M)
        assert int(e[0]) == 1                                  # one point along x3
        assert multi_workspace_bytes([dict(plan=lattice_plan(M), stiffness=[np.eye(6)], E=np.zeros((1, 6)))]) > 0
    w = synth.hashin2d_workload()
    assert w["rho_e"] == 0.09 and np.isinf(w["c"][2])
    assert np.linalg.eigvalsh(w["stiffness"][2]).min() > 0      # the neutral matrix is positive definite
