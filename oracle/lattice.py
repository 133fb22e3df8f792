"""Lattice algebra of the oracle: Smith normal form, pattern and generating set.

Test infrastructure only (see ``oracle/__init__``).  Exact integer arithmetic:
the scalar methods use Python ints and are the definitions; the (m, d) arrays
are the same formulas evaluated with numpy int64 under an overflow guard.

Paper references (arXiv 1605.05712):
  * Sec. 2.1, "The pattern and the generating set": congruence mod M, the
    lattice Lambda(M) = M^{-1} Z^d, the pattern P(M) taken in the symmetric
    cube [-1/2, 1/2)^d, and G(M) = M P(M); |P(M)| = |G(M^T)| = |det M| = m.
  * Sec. 2.2: Smith normal form M = Q E R with unimodular Q, R and
    E = diag(e_1..e_d), e_j | e_{j+1}; pattern dimension d_M = #{e_j > 1};
    pattern basis (Eq. patternBasisV) and generating-set basis
    h_j = R^T e_j (Eq. genSetBasisV); lexicographic addressing by lambda.

Reading of the garbled pattern-basis index in Eq. patternBasisV: the basis
vector attached to divisor e_j is y_j = R^{-1} e_j / e_j (mod 1), which is
what M^{-1} = R^{-1} E^{-1} Q^{-1} gives; then h(k)^T y(lambda) =
sum_j k_j lambda_j / e_j (mod 1).  Lexicographic order has the LAST index
fastest.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product


def _ident(d):
    return [[int(i == j) for j in range(d)] for i in range(d)]


def _matmul(A, B):
    n, k, p = len(A), len(B), len(B[0])
    return [[sum(A[i][t] * B[t][j] for t in range(k)) for j in range(p)] for i in range(n)]


def _transpose(A):
    return [list(r) for r in zip(*A)]


def det(M):
    """Exact integer determinant by cofactor expansion (d <= 4)."""
    M = [list(map(int, r)) for r in M]
    d = len(M)
    if d == 1:
        return M[0][0]
    if d == 2:
        return M[0][0] * M[1][1] - M[0][1] * M[1][0]
    s = 0
    for j in range(d):
        minor = [r[:j] + r[j + 1:] for r in M[1:]]
        s += (-1) ** j * M[0][j] * det(minor)
    return s


def adjugate(M):
    """Exact adjugate: adj(M) M = M adj(M) = det(M) I."""
    d = len(M)
    if d == 1:
        return [[1]]
    A = [[0] * d for _ in range(d)]
    for i in range(d):
        for j in range(d):
            minor = [r[:j] + r[j + 1:] for k, r in enumerate(M) if k != i]
            A[j][i] = (-1) ** (i + j) * det(minor)
    return A


def inverse_unimodular(U):
    """Inverse of an integer matrix with det +-1 (integral)."""
    D = det(U)
    assert abs(D) == 1, "not unimodular"
    A = adjugate(U)
    return [[a * D for a in r] for r in A]


def smith_normal_form(M):
    """Return (Q, e, R) with M = Q diag(e) R, Q and R unimodular (Sec. 2.2).

    Textbook elimination: row operations accumulate into U and column
    operations into V so that U M V = diag(e); then Q = U^{-1}, R = V^{-1}.
    Divisors are positive and e_j divides e_{j+1}.
    """
    d = len(M)
    A = [list(map(int, r)) for r in M]
    if det(A) == 0:
        raise ValueError("M is singular")
    U = _ident(d)
    V = _ident(d)

    def swap_rows(i, j):
        A[i], A[j] = A[j], A[i]
        U[i], U[j] = U[j], U[i]

    def swap_cols(i, j):
        for X in (A, V):
            for r in X:
                r[i], r[j] = r[j], r[i]

    def add_row(dst, src, q):  # row_dst += q * row_src
        A[dst] = [a + q * b for a, b in zip(A[dst], A[src])]
        U[dst] = [a + q * b for a, b in zip(U[dst], U[src])]

    def add_col(dst, src, q):  # col_dst += q * col_src
        for X in (A, V):
            for r in X:
                r[dst] += q * r[src]

    for t in range(d):
        while True:
            # smallest nonzero |entry| of the trailing block becomes the pivot
            best = None
            for i in range(t, d):
                for j in range(t, d):
                    if A[i][j] != 0 and (best is None or abs(A[i][j]) < abs(A[best[0]][best[1]])):
                        best = (i, j)
            i, j = best
            if i != t:
                swap_rows(i, t)
            if j != t:
                swap_cols(j, t)
            p = A[t][t]
            clean = True
            for i in range(t + 1, d):
                q = A[i][t] // p
                if q:
                    add_row(i, t, -q)
                if A[i][t] != 0:
                    clean = False
            for j in range(t + 1, d):
                q = A[t][j] // p
                if q:
                    add_col(j, t, -q)
                if A[t][j] != 0:
                    clean = False
            if not clean:
                continue
            # divisibility of the trailing block by the pivot
            bad = None
            for i in range(t + 1, d):
                for j in range(t + 1, d):
                    if A[i][j] % p != 0:
                        bad = i
                        break
                if bad is not None:
                    break
            if bad is not None:
                add_row(t, bad, 1)
                continue
            break
        if A[t][t] < 0:
            A[t] = [-a for a in A[t]]
            U[t] = [-a for a in U[t]]
    e = [A[i][i] for i in range(d)]
    Q = inverse_unimodular(U)
    R = inverse_unimodular(V)
    return Q, e, R


class Lattice:
    """Pattern P(M) and generating set G(M^T) with the SNF orderings.

    Attributes
    ----------
    M, d, m     the integer matrix, dimension and m = |det M|
    Q, e, R     Smith normal form M = Q diag(e) R
    axes        indices j with e_j > 1 (the d_M pattern axes), in order
    shape       tuple(e_j for j in axes): array shape of spatial/spectral data
    lam         (m, d) list of lambda multi-indices in lexicographic order
                (last index fastest); entries for e_j = 1 axes are 0
    p           (m, d) integer numerators of the pattern points, y = p / m,
                every y in [-1/2, 1/2)^d, same order as lam
    h           (m, d) generating-set frequencies h(k) in G(M^T), k in the
                same lexicographic order (M^{-T} h in [-1/2, 1/2)^d)
    """

    def __init__(self, M):
        self.M = [list(map(int, r)) for r in M]
        self.d = d = len(self.M)
        self.det = det(self.M)
        if self.det == 0:
            raise ValueError("M is singular")
        self.m = m = abs(self.det)
        self.Q, self.e, self.R = smith_normal_form(self.M)
        self.axes = [j for j in range(d) if self.e[j] > 1]
        self.d_M = len(self.axes)
        self.shape = tuple(self.e[j] for j in self.axes)
        self.Rinv = inverse_unimodular(self.R)
        self.adjMT = adjugate(_transpose(self.M))
        self._build_arrays()

    def _build_arrays(self):
        """Vectorised (numpy int64) lam, p and h; the scalar methods below are the definitions."""
        import numpy as np
        d, m, e = self.d, self.m, self.e
        # guard: every intermediate below stays far inside int64
        amax = lambda X: max(abs(x) for r in X for x in r)
        b_p = d * m * amax(self.Rinv)
        b_g = d * max(e) * amax(self.R)
        b_u = 2 * d * b_g * amax(self.adjMT) + m
        b_h = b_g + d * (b_u // m + 2) * amax(self.M)
        if max(b_p, b_u, b_h) >= 2 ** 62:
            raise OverflowError("lattice entries too large for the int64 oracle arrays")
        grids = np.indices(tuple(e), dtype=np.int64).reshape(d, -1).T  # lexicographic, last fastest
        self.lam = grids
        scale = np.array([m // ej for ej in e], dtype=np.int64)
        Rinv = np.array(self.Rinv, dtype=np.int64)
        p = (grids * scale) @ Rinv.T
        p %= m
        p[2 * p >= m] -= m
        self.p = p
        R = np.array(self.R, dtype=np.int64)
        g = grids @ R                      # rows: (R^T k)^T
        A = np.array(self.adjMT, dtype=np.int64)
        D = self.det
        u = g @ A.T
        z = np.floor_divide(2 * u + D, 2 * D)
        MT = np.array(self.M, dtype=np.int64).T
        self.h = g - z @ MT.T

    # -- pattern (Sec. 2.1, Eq. patternBasisV) --------------------------
    def point_numerator(self, lam):
        """m * y(lambda), y = R^{-1} E^{-1} lambda reduced mod 1 into [-1/2, 1/2)."""
        m = self.m
        v = [lam[j] * (m // self.e[j]) for j in range(self.d)]
        p = [sum(self.Rinv[i][j] * v[j] for j in range(self.d)) for i in range(self.d)]
        out = []
        for x in p:
            x %= m
            if 2 * x >= m:
                x -= m
            out.append(x)
        return out

    # -- generating set (Sec. 2.1, Eq. genSetBasisV) ---------------------
    def frequency(self, k):
        """h(k): the representative of R^T k mod M^T Z^d with M^{-T} h in [-1/2,1/2)^d."""
        d = self.d
        g = [sum(self.R[j][i] * k[j] for j in range(d)) for i in range(d)]  # R^T k
        D = self.det
        # M^{-T} g = adj(M^T) g / det(M^T); det(M^T) = det(M) = D
        u = [sum(self.adjMT[i][j] * g[j] for j in range(d)) for i in range(d)]
        # z_i = floor(u_i / D + 1/2) exactly
        z = [Fraction(2 * ui + D, 2 * D).__floor__() for ui in u]
        MT = _transpose(self.M)
        return [g[i] - sum(MT[i][j] * z[j] for j in range(d)) for i in range(d)]

    def frac_gen(self, h):
        """M^{-T} h as exact fractions (checks the symmetric-cell condition)."""
        d = self.d
        u = [sum(self.adjMT[i][j] * h[j] for j in range(d)) for i in range(d)]
        return [Fraction(x, self.det) for x in u]

    def neg_index(self, k):
        """Lexicographic multi-index of -k (mod e)."""
        return [(-k[j]) % self.e[j] for j in range(self.d)]

    def flat(self, lam):
        idx = 0
        for j in range(self.d):
            idx = idx * self.e[j] + lam[j]
        return idx


def brute_force_pattern(M):
    """All y in Lambda(M) cap [-1/2,1/2)^d by scanning integer vectors, as numerators m*y.

    Independent of the SNF: y = M^{-1} z for z in Z^d; m*y = +-adj(M) z is an
    integer vector, and scanning z over the box [0, m)^d reaches every class
    mod 1 (adj(M) z mod m runs through all lattice points).  Only for tiny m.
    """
    d = len(M)
    D = det(M)
    m = abs(D)
    A = adjugate([list(r) for r in M])
    pts = set()
    assert m ** d <= 2 ** 22, "brute force is for tiny patterns only"
    for z in product(range(m), repeat=d):
        v = [sum(A[i][j] * z[j] for j in range(d)) * (1 if D > 0 else -1) for i in range(d)]
        q = []
        for x in v:
            x %= m
            if 2 * x >= m:
                x -= m
            q.append(x)
        pts.add(tuple(q))
    return pts


def brute_force_genset(M):
    """All h in Z^d with M^{-T} h in [-1/2,1/2)^d, by scanning a bounding box."""
    d = len(M)
    MT = _transpose([list(r) for r in M])
    D = det(MT)
    A = adjugate(MT)
    # |h_i| <= sum_j |MT_ij| / 2
    bound = [sum(abs(x) for x in MT[i]) // 2 + 1 for i in range(d)]
    out = set()
    for h in product(*[range(-b, b + 1) for b in bound]):
        ok = True
        for i in range(d):
            f = Fraction(sum(A[i][j] * h[j] for j in range(d)), D)
            if not (Fraction(-1, 2) <= f < Fraction(1, 2)):
                ok = False
                break
        if ok:
            out.add(tuple(h))
    return out
