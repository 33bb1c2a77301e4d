"""The size-independent certificate (tests/certify.py) and the oracle's exact
checker reject wrong results.

Correct oracle results pass; each test then plants one plausible mistake in a
copy of the result, on the CPU, and checks that both the exact mode and the
Freivalds mode used at full size refuse it.
"""
import numpy as np
import pytest

import oracle
from paper_1301_4438_gb300 import workloads as W
from tests.certify import certify

CASES = [(40, 30, 17, 65521), (33, 50, 33, 8388593), (45, 45, 45, 2147483647), (24, 36, 11, 251)]


def _result(m, n, r, p):
    A, pl = W.planted(m, n, r, p, seed=m * n + r)
    LU, pp, pq, rr = oracle.pluq(A, p)
    assert rr == r
    return A, LU, pp, pq, rr


def _bump(x, p):
    return np.uint32((int(x) + 1) % p)


def _mutations(LU, pp, pq, r, p, g):
    m, n = LU.shape
    out = []
    i, j = int(g.integers(1, r)), 0
    j = int(g.integers(0, i))
    X = LU.copy(); X[i, j] = _bump(X[i, j], p)                    # an L entry
    out.append(("L entry", X, pp, pq, r))
    k = int(g.integers(0, r))
    X = LU.copy(); X[k, k] = _bump(X[k, k], p) or np.uint32(1)    # a U diagonal entry
    if X[k, k] != LU[k, k]:
        out.append(("U diagonal", X, pp, pq, r))
    if n > r:
        c = int(g.integers(r, n))
        X = LU.copy(); X[0, c] = _bump(X[0, c], p)               # a V entry
        out.append(("V entry", X, pp, pq, r))
    if m > r:
        i2 = int(g.integers(r, m))
        X = LU.copy(); X[i2, 0] = _bump(X[i2, 0], p)             # an M entry
        out.append(("M entry", X, pp, pq, r))
    if m > r and n > r:
        X = LU.copy(); X[m - 1, n - 1] = 1                       # trailing block not zero
        out.append(("trailing block", X, pp, pq, r))
    q = pp.copy(); q[[0, 1]] = q[[1, 0]]                          # two pivot rows swapped
    out.append(("pivot rows swapped", LU, q, pq, r))
    q = pq.copy(); q[[0, r - 1]] = q[[r - 1, 0]]                  # two pivot columns swapped
    out.append(("pivot columns swapped", LU, pp, q, r))
    q = pq.copy(); q[-1] = q[0]                                   # not a permutation
    out.append(("duplicate column", LU, pp, q, r))
    out.append(("rank too small", LU, pp, pq, r - 1))
    return out


@pytest.mark.parametrize("m,n,r,p", CASES)
def test_correct_results_pass(m, n, r, p):
    A, LU, pp, pq, r = _result(m, n, r, p)
    assert certify(A, p, LU, pp, pq, r, exact=True) == ""
    assert certify(A, p, LU, pp, pq, r, exact=False, trials=2) == ""
    assert oracle.check_pluq(A, p, LU, pp, pq, r) == 0


@pytest.mark.parametrize("m,n,r,p", CASES)
def test_planted_mistakes_are_rejected(m, n, r, p):
    A, LU, pp, pq, r = _result(m, n, r, p)
    g = np.random.Generator(np.random.PCG64(r + p))
    muts = _mutations(LU, pp, pq, r, p, g)
    assert len(muts) >= 6          # full rank leaves no V, M or trailing block
    for name, X, q1, q2, rr in muts:
        assert certify(A, p, X, q1, q2, rr, exact=True) != "", name
        assert certify(A, p, X, q1, q2, rr, exact=False, trials=3) != "", name
        if name not in ("pivot rows swapped", "pivot columns swapped"):
            # the exact checker tests the contract A = P [L;M][U V] Q, not the order
            assert oracle.check_pluq(A, p, X, q1.astype(np.int32), q2.astype(np.int32), rr) != 0, name
