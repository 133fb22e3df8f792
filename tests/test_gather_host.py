"""Host checks of lattice_gather_map (subsampling, Sec. 2.1; rearrangement between pattern-congruent
matrices, Sec. 2.2) against the oracle's own point sets."""
import numpy as np
import pytest

from oracle.lattice import Lattice
from paper_1605_05712_gb300 import LatticeError, gather_map, lattice_plan


def _check_map(Mf, Mt):
    src, dst = lattice_plan(Mf), lattice_plan(Mt)
    mp = gather_map(src, dst)
    pf, pt = src.points(), dst.points()
    assert np.array_equal(pf[mp], pt * (src.m // dst.m))         # the same points, exactly
    # the oracle's pattern of the target (independent enumeration) is the same point set
    Lt = Lattice(Mt)
    assert sorted(map(tuple, Lt.p.tolist())) == sorted(map(tuple, pt.tolist()))
    return mp


@pytest.mark.parametrize("Mf,Mt", [([[64, 0], [0, 64]], [[64, 32], [0, 1]]),      # Sec. 5.2: M_a -> M_b
                                   ([[64, 0], [0, 64]], [[8, 0], [0, 8]]),        # M_a -> M_c
                                   ([[8, 0, 0], [0, 8, 0], [0, 0, 8]], [[8, 4, 0], [0, 1, 0], [0, 0, 8]]),
                                   # divisors that are not powers of two: odd, mixed, a chirp-z prime
                                   ([[45, 0], [0, 45]], [[15, 0], [0, 9]]),
                                   ([[24, 0, 0], [0, 24, 0], [0, 0, 24]], [[8, 0, 0], [0, 12, 0], [0, 0, 6]]),
                                   ([[2053, 0], [0, 2]], [[2053, 0], [0, 1]])])
def test_subpattern_map(Mf, Mt):
    mp = _check_map(Mf, Mt)
    assert len(np.unique(mp)) == len(mp)


def test_congruent_patterns_permute():
    # M2 = Q M1 with Q unimodular has the same pattern (Example 2.2): the map is a permutation
    mp = _check_map([[8, 4], [0, 4]], [[8, 12], [0, 4]])
    assert sorted(mp.tolist()) == list(range(32))
    mp = _check_map([[6, 3], [0, 5]], [[6, 8], [0, 5]])            # odd and even divisors, (1, 30)
    assert sorted(mp.tolist()) == list(range(30))


def test_not_a_subpattern_is_refused():
    with pytest.raises(LatticeError):
        gather_map(lattice_plan([[64, 0], [0, 64]]), lattice_plan([[3, 0], [0, 1]]))
    with pytest.raises(LatticeError):
        gather_map(lattice_plan([[8, 0], [0, 8]]), lattice_plan([[16, 1], [0, 4]]))
