"""Pins of oracle.lattice: Smith normal form, pattern and generating set (Sec. 2.1-2.2)."""
import json
import math
import os
from itertools import combinations

import numpy as np
import pytest

from oracle.lattice import Lattice, brute_force_genset, brute_force_pattern, det, smith_normal_form

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_lattice_facts.json")))


def _matmul(A, B):
    return (np.array(A, dtype=object) @ np.array(B, dtype=object)).tolist()


def minors_gcd(M, k):
    d = len(M)
    g = 0
    for rows in combinations(range(d), k):
        for cols in combinations(range(d), k):
            g = math.gcd(g, abs(det([[M[r][c] for c in cols] for r in rows])))
    return g


RNG = np.random.default_rng(7)
RANDOM_M = [RNG.integers(-9, 10, size=(d, d)).tolist() for d in (2, 3) for _ in range(25)]
RANDOM_M = [M for M in RANDOM_M if det(M) != 0]


@pytest.mark.parametrize("M", RANDOM_M + [GOLD["fig1_same_size"]["M2"], [[512, 0], [16, 32]], [[128, 16, 0], [0, 128, 16], [0, 0, 128]]])
def test_snf_factorization_and_divisors(M):
    Q, e, R = smith_normal_form(M)
    d = len(M)
    E = [[e[i] if i == j else 0 for j in range(d)] for i in range(d)]
    assert _matmul(_matmul(Q, E), R) == [list(r) for r in M]
    assert abs(det(Q)) == 1 and abs(det(R)) == 1
    assert all(x > 0 for x in e)
    assert all(e[i + 1] % e[i] == 0 for i in range(d - 1))
    # elementary divisors from gcds of k x k minors: e_1 ... e_k = gcd of k-minors
    prod = 1
    for k in range(1, d + 1):
        prod *= e[k - 1]
        assert prod == minors_gcd(M, k)


def test_paper_divisors():
    # Sec. 2.2 / Fig. 1: M2, M3 rank-1 with 64 points; Sec. 5.1 M_{9,16,0} is rank-2 (16, 1024); Sec. 5.2 M_b rank-1
    g = GOLD["fig1_same_size"]
    for M in (g["M2"], g["M3"]):
        L = Lattice(M)
        assert L.m == g["abs_det"] and L.e == [1, 64]
    assert Lattice(g["M3"]).d_M == g["M3_pattern_dimension"]
    assert Lattice([[512, 0], [16, 32]]).e == [16, 1024]
    assert Lattice(GOLD["subsampling"]["M_b"]).e == [1, 64]
    f = GOLD["fig1_factorization"]
    assert _matmul(f["J"], f["N"]) == f["M1"]
    assert Lattice(f["M1"]).e == [8, 8]


@pytest.mark.parametrize("M", [M for M in RANDOM_M if abs(det(M)) <= 64] + [[[8, -4], [2, 7]], [[8, -1], [0, 8]], [[6, 2], [0, 10]]])
def test_pattern_and_genset_brute_force(M):
    L = Lattice(M)
    P = set(map(tuple, L.p.tolist()))
    H = set(map(tuple, L.h.tolist()))
    assert len(P) == L.m and len(H) == L.m          # |P(M)| = |G(M^T)| = |det M|
    assert P == brute_force_pattern(M)
    assert H == brute_force_genset(M)
    # every point in the symmetric cube, every frequency in the symmetric cell of M^T
    assert all(-L.m <= 2 * x < L.m for x in L.p.reshape(-1))
    for h in L.h[:50]:
        assert all(-0.5 <= float(f) < 0.5 for f in L.frac_gen(list(map(int, h))))


def test_scalar_definitions_match_arrays():
    for M in ([[8, -4], [2, 7]], [[4, 1, 0], [0, 4, 2], [2, 0, 4]], [[16, 0], [4, 8]]):
        L = Lattice(M)
        for i in range(0, L.m, max(1, L.m // 40)):
            lam = list(map(int, L.lam[i]))
            assert L.point_numerator(lam) == L.p[i].tolist()
            assert L.frequency(lam) == L.h[i].tolist()


def test_transpose_same_divisors():
    # Sec. 2.2: d_M = d_{M^T} and the elementary divisors of M and M^T agree
    for M in RANDOM_M[:20]:
        assert Lattice(M).e == Lattice(np.array(M).T.tolist()).e


def test_example_2_2_same_points_different_genset():
    mats = GOLD["example_2_2"]["matrices"]
    Ls = [Lattice(M) for M in mats]
    pts = [set(map(tuple, L.p.tolist())) for L in Ls]
    gens = [set(map(tuple, L.h.tolist())) for L in Ls]
    assert pts[0] == pts[1] == pts[2]
    assert gens[0] != gens[1] and gens[1] != gens[2] and gens[0] != gens[2]
    c = GOLD["congruence_shear"]
    base = set(map(tuple, Lattice([[c["m1"], 0], [0, c["m2"]]]).p.tolist()))
    for n in c["n"]:
        assert set(map(tuple, Lattice([[c["m1"], c["m2"] * n], [0, c["m2"]]]).p.tolist())) == base


def _scaled(L, M_big):
    # points of L expressed as numerators over the other lattice's m
    mb = abs(det(M_big))
    assert mb % L.m == 0
    return set(map(tuple, (L.p * (mb // L.m)).tolist()))


def test_subpattern_inclusion():
    # Sec. 2.1: M = J N  =>  P(N) subset P(M) and G(N^T) subset G(M^T)
    f = GOLD["fig1_factorization"]
    LM, LN = Lattice(f["M1"]), Lattice(f["N"])
    assert _scaled(LN, f["M1"]) <= set(map(tuple, LM.p.tolist()))
    assert set(map(tuple, LN.h.tolist())) <= set(map(tuple, LM.h.tolist()))
    s = GOLD["subsampling"]
    a = s["a"]
    J, N = [[1, -a // 2], [0, a]], [[a, a // 2], [0, 1]]
    assert _matmul(J, N) == s["M_a"]
    La, Lb, Lc = Lattice(s["M_a"]), Lattice(s["M_b"]), Lattice(s["M_c"])
    assert Lb.m == s["m_b"]
    Pa = set(map(tuple, La.p.tolist()))
    assert _scaled(Lb, s["M_a"]) <= Pa and _scaled(Lc, s["M_a"]) <= Pa


def test_shear_family_facts():
    g = GOLD["shear_family"]
    from paper_1605_05712_gb300.synth import shear_matrix
    for j in (7, 8, 9):
        for alpha in (0, 1):
            for k in (-512, -16, 0, 16, 272):
                assert abs(det(shear_matrix(j, k, alpha))) == g["abs_det_shear"]
        Mt = [[2 ** j // 2, 2 ** (14 - j) // 2], [-(2 ** j) // 2, 2 ** (14 - j) // 2]]
        assert abs(det(Mt)) == g["abs_det_quincunx"]
    cap = g["caption"]
    assert shear_matrix(7, 0, 0) == cap["M_7_0_0"]
    assert shear_matrix(8, 16, 0) == cap["M_8_16_0"]
    assert shear_matrix(9, 16, 0) == cap["M_9_16_0"]
    assert [[64, 64], [-64, 64]] == cap["Mtilde_7"]


def test_shear_congruent_same_pattern():
    from paper_1605_05712_gb300.synth import shear_matrix
    for grp in GOLD["shear_congruent"]["groups"]:
        pts = [set(map(tuple, Lattice(shear_matrix(*t)).p.tolist())) for t in grp]
        assert all(p == pts[0] for p in pts)
