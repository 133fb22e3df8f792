"""The C++ plan against the definitions of Sec. 2.1-2.2 on seeded random matrices (CPU, host-only plans).

For several hundred regular integer matrices M (2-D and 3-D, m = |det M| up to 4096, every kind of
divisor: powers of two, odd, mixed, primes beyond one pass) the plan's outputs are checked against the
definitions, with no Smith form and no oracle arithmetic:
  * points: every p satisfies M (p / m) in Z^d and p / m in [-1/2, 1/2)^d; m distinct points, so the
    set is the whole pattern P(M) = Lambda(M) cap [-1/2, 1/2)^d (|P(M)| = m);
  * frequencies: every h has M^{-T} h in [-1/2, 1/2)^d, m distinct ones, so the set is the whole
    generating set G(M^T) (one representative per class of Z^d / M^T Z^d);
  * divisors: e_1 ... e_k = gcd of the k x k minors (the Smith invariants), e_j | e_{j+1};
  * layout: the logical axes multiply to m.
Small patterns are also compared with a brute-force scan of Lambda(M).
"""
from itertools import combinations
from math import gcd

import numpy as np
import pytest

from oracle.lattice import brute_force_pattern


def _minor_gcds(M):
    """g_k = gcd of all k x k minors (k = 1..d), exact integers."""
    d = len(M)
    out = []
    for k in range(1, d + 1):
        g = 0
        for rows in combinations(range(d), k):
            for cols in combinations(range(d), k):
                sub = [[M[i][j] for j in cols] for i in rows]
                g = gcd(g, abs(_exact_det(sub)))
        out.append(g)
    return out


def _exact_det(A):
    n = len(A)
    if n == 1:
        return A[0][0]
    if n == 2:
        return A[0][0] * A[1][1] - A[0][1] * A[1][0]
    return sum((-1) ** j * A[0][j] * _exact_det([r[:j] + r[j + 1:] for r in A[1:]]) for j in range(n))


def _adjugate(M):
    d = len(M)
    return [[(-1) ** (i + j) * _exact_det([r[:i] + r[i + 1:] for k, r in enumerate(M) if k != j])
             for j in range(d)] for i in range(d)]


def _random_matrices(seed=20240611):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < 160:                        # dense 2-D
        M = rng.integers(-40, 41, size=(2, 2)).tolist()
        if 1 <= abs(_exact_det(M)) <= 4096:
            out.append(M)
    while len(out) < 320:                        # dense 3-D
        M = rng.integers(-9, 10, size=(3, 3)).tolist()
        if 1 <= abs(_exact_det(M)) <= 4096:
            out.append(M)
    primes = [q for q in range(2049, 4097) if all(q % k for k in range(2, 65))]
    for q in rng.choice(primes, size=8, replace=False).tolist():   # chirp-z rows: a prime beyond one pass
        out.append([[q, int(rng.integers(0, q))], [0, 1]])
        out.append([[1, 0, 0], [int(rng.integers(0, 5)), 1, 0], [int(rng.integers(0, 5)), 0, q]])
    for _ in range(60):                          # upper-triangular 2-D / 3-D with chosen diagonals
        a, c = (int(x) for x in rng.integers(1, 65, size=2))
        out.append([[a, int(rng.integers(-a, a + 1))], [0, c]])
        a, b, c = (int(x) for x in rng.integers(1, 17, size=3))
        out.append([[a, int(rng.integers(-a, a + 1)), 0], [0, b, int(rng.integers(-b, b + 1))], [0, 0, c]])
    return out


MATS = _random_matrices()


def test_random_plans_match_the_definitions():
    from paper_1605_05712_gb300 import lattice_plan
    kinds = set()
    for M in MATS:
        d = len(M)
        D = _exact_det(M)
        m = abs(D)
        P = lattice_plan(M)
        assert P.m == m, M
        # divisors: Smith invariants from the gcds of minors
        g = _minor_gcds(M)
        e = [g[0]] + [g[k] // g[k - 1] for k in range(1, d)]
        assert P.divisors == e, (M, P.divisors, e)
        assert all(e[k + 1] % e[k] == 0 for k in range(d - 1))
        kinds.add("pow2" if all(x & (x - 1) == 0 for x in e) else "general")
        if P.layout()["split"] == 2:
            kinds.add("chirp-z")
        # points: M p / m integral, p / m in [-1/2, 1/2)^d, m distinct
        p = P.points()
        assert p.shape == (m, d)
        Mi = np.asarray(M, dtype=np.int64)
        assert np.all((p @ Mi.T) % m == 0), M
        assert np.all(2 * p >= -m) and np.all(2 * p < m), M
        assert len(set(map(tuple, p.tolist()))) == m, M
        # frequencies: M^{-T} h = adj(M^T) h / det in [-1/2, 1/2)^d, m distinct
        h = P.freqs()
        assert h.shape == (m, d)
        A = np.asarray(_adjugate([list(r) for r in np.asarray(M).T.tolist()]), dtype=np.int64)
        u = (h @ A.T) * (1 if D > 0 else -1)        # |det| M^{-T} h
        assert np.all(2 * u >= -m) and np.all(2 * u < m), M
        assert len(set(map(tuple, h.tolist()))) == m, M
        # the FFT decomposition covers the pattern
        if m > 1:
            assert int(np.prod(P.layout()["ax_len"])) == m, M
        # brute force on small patterns
        if m ** d <= 40000:
            assert set(map(tuple, p.tolist())) == brute_force_pattern(M), M
    assert kinds == {"pow2", "general", "chirp-z"}


def test_plan_size_limits():
    # a divisor other than the largest takes one pass (2048 points in 2-D, 1024 in 3-D); the largest takes
    # at most two (one four-step split) or chirp-z rows of at most 2^22 points
    from paper_1605_05712_gb300 import LatticeError, lattice_plan
    planned = {((1, 0), (0, 1 << 23)): 1, ((1, 0, 0), (0, 1, 0), (0, 0, 1 << 21)): 1,
               ((1, 0), (0, 3 << 20)): 1, ((1, 0), (0, 5 ** 9)): 2, ((2048, 0), (0, 2048)): 0,
               ((1, 0, 0), (0, 1024, 0), (0, 0, 1024)): 0, ((1536, 0), (0, 1536)): 0}
    for M, split in planned.items():
        assert lattice_plan([list(r) for r in M]).layout()["split"] == split, M
    for M in ([[4096, 0], [0, 4096]], [[3072, 0], [0, 3072]], [[1, 0, 0], [0, 1155, 0], [0, 0, 1155]],
              [[1, 0], [0, 1 << 24]], [[1, 0, 0], [0, 1, 0], [0, 0, 1 << 22]], [[1, 0], [0, 9 << 20]]):
        with pytest.raises(LatticeError) as ei:
            lattice_plan(M)
        assert ei.value.code == -5, M
