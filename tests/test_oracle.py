"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: brute-force
ranks of every leading submatrix, a second literal reading of Algorithm 1,
textbook LU, planted rank profiles (Lemma 1), the LEU theorem (Theorem 1),
hand-derived fixtures, closed-form special cases.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1301_4438_gb300 import workloads as W
from tests import brute
from tests.certify import certify

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PRIMES = [2, 3, 5, 7, 251, 65521, 8388593, 2147483647]


def R_from_col(col_of_row, m, n):
    R = np.zeros((m, n), dtype=np.int64)
    for i, c in enumerate(col_of_row):
        if c >= 0:
            R[i, c] = 1
    return R


def R_from_pq(perm_p, perm_q, r, m, n):
    R = np.zeros((m, n), dtype=np.int64)
    R[np.asarray(perm_p[:r]), np.asarray(perm_q[:r])] = 1
    return R


# ---------------------------------------------------------------- field --

def test_is_prime_matches_sieve():
    N = 5000
    sieve = np.ones(N, dtype=bool)
    sieve[:2] = False
    for i in range(2, int(N ** 0.5) + 1):
        if sieve[i]:
            sieve[i * i::i] = False
    for x in range(N):
        assert oracle.is_prime(x) == bool(sieve[x]), x
    for p in PRIMES:
        assert oracle.is_prime(p)
    assert not oracle.is_prime(2147483647 * 1 - 2)      # 2^31 - 3 = 5 * 429496729 ... composite
    assert not oracle.is_prime(65535)


def test_rejects_bad_input():
    A = np.array([[1, 2], [3, 4]], dtype=np.uint32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.pluq(A, 4)
    assert e.value.code == -2                       # not prime
    with pytest.raises(oracle.OracleError) as e:
        oracle.pluq(A, 3)
    assert e.value.code == -3                       # entry >= p


# ------------------------------------------------- exhaustive tiny cases --

@pytest.mark.parametrize("m,n,p", [(4, 4, 2), (3, 3, 3), (2, 5, 2), (5, 2, 2), (3, 4, 2), (2, 3, 3)])
def test_rank_profile_exhaustive(m, n, p):
    """R from incremental row echelon == R from the ranks of all leading submatrices."""
    As = brute.all_matrices(m, n, p)
    Rb = brute.rank_profile_matrix(As, p)
    for b in range(As.shape[0]):
        col = oracle.rank_profile(As[b].astype(np.uint32), p)
        assert np.array_equal(R_from_col(col, m, n), Rb[b]), As[b]


@pytest.mark.parametrize("m,n,p", [(4, 4, 2), (3, 3, 3), (2, 5, 2), (5, 3, 2), (1, 6, 3), (6, 1, 3)])
def test_pluq_equals_literal_alg1_exhaustive(m, n, p):
    """Two independent readings of Algorithm 1 agree bit for bit, and both reveal R."""
    As = brute.all_matrices(m, n, p)
    Rb = brute.rank_profile_matrix(As, p)
    for b in range(As.shape[0]):
        A = As[b].astype(np.uint32)
        LU, pp, pq, r = oracle.pluq(A, p)
        LU1, pp1, pq1, r1 = oracle.pluq_alg1(A, p)
        assert r == r1
        assert np.array_equal(pp, pp1) and np.array_equal(pq, pq1), A
        assert np.array_equal(LU, LU1), A
        assert np.array_equal(R_from_pq(pp, pq, r, m, n), Rb[b])
        assert oracle.check_pluq(A, p, LU, pp, pq, r) == 0


def test_all_shapes_up_to_4_including_empty():
    for m in range(0, 5):
        for n in range(0, 5):
            if m * n > 12:
                As = brute.all_matrices(m, n, 2)[::7]
            elif m * n == 0:
                As = np.zeros((1, m, n), dtype=np.int64)
            else:
                As = brute.all_matrices(m, n, 2)
            for A in As:
                A = A.astype(np.uint32)
                LU, pp, pq, r = oracle.pluq(A, 2)
                LU1, pp1, pq1, r1 = oracle.pluq_alg1(A, 2)
                assert (r, pp.tolist(), pq.tolist()) == (r1, pp1.tolist(), pq1.tolist())
                assert np.array_equal(LU, LU1)
                assert certify(A, 2, LU, pp, pq, r, exact=True) == ""


# --------------------------------------------------------- random small --

def _structured(g, m, n, p):
    kind = g.integers(0, 5)
    if kind == 0:                                    # dense uniform
        return g.integers(0, p, (m, n)).astype(np.uint32)
    if kind == 1:                                    # sparse
        A = g.integers(0, p, (m, n)) * (g.random((m, n)) < 0.15)
        return A.astype(np.uint32)
    if kind == 2:                                    # low rank planted
        r = int(g.integers(0, min(m, n) + 1))
        A, _ = W.planted(m, n, r, p, int(g.integers(1 << 30)))
        return A
    if kind == 3:                                    # zero rows / cols, duplicated rows
        A = g.integers(0, p, (m, n))
        A[g.random(m) < 0.3, :] = 0
        A[:, g.random(n) < 0.3] = 0
        if m > 2:
            A[m - 1] = A[0]
        return A.astype(np.uint32)
    r = int(g.integers(0, min(m, n) + 1))            # rank r product of random factors
    X = g.integers(0, p, (m, r))
    Y = g.integers(0, p, (r, n))
    return brute.matmul_mod(X, Y, p).astype(np.uint32)


@pytest.mark.parametrize("p", PRIMES)
def test_pluq_equals_literal_alg1_random(p):
    g = np.random.Generator(np.random.PCG64(p))
    for _ in range(40):
        m, n = int(g.integers(1, 41)), int(g.integers(1, 41))
        A = _structured(g, m, n, p)
        LU, pp, pq, r = oracle.pluq(A, p)
        LU1, pp1, pq1, r1 = oracle.pluq_alg1(A, p)
        assert r == r1
        assert np.array_equal(pp, pp1) and np.array_equal(pq, pq1)
        assert np.array_equal(LU, LU1)
        assert certify(A, p, LU, pp, pq, r, exact=True) == ""


@pytest.mark.parametrize("p", [3, 65521, 8388593, 2147483647])
def test_pluq_equals_literal_alg1_at_leaf_size(p):
    """The order function against the literal Algorithm 1 at the sizes the GPU
    base case handles (64 x 64 to 128 x 128): planted profiles whose rows and
    columns are paired at random (many descents), the anti-diagonal profile
    (every pair of pivots a descent), dense, sparse and low-rank products."""
    g = np.random.Generator(np.random.PCG64(4242 + p))
    shapes = [(64, 64), (128, 128), (96, 128), (128, 100), (127, 65), (80, 113)]
    for k, (m, n) in enumerate(shapes):
        r = min(m, n) // 2 + k
        cases = [W.planted(m, n, r, p, 900 + k)[0], _structured(g, m, n, p)]
        # anti-diagonal rank profile matrix: L0 R U0 with R[i, q - 1 - i] = 1
        q = min(m, n)
        L0 = np.tril(g.integers(0, p, (m, m)), -1) + np.eye(m, dtype=np.int64)
        U0 = np.triu(g.integers(0, p, (n, n)), 1) + np.eye(n, dtype=np.int64)
        R = np.zeros((m, n), dtype=np.int64)
        R[np.arange(q), q - 1 - np.arange(q)] = 1
        cases.append(brute.matmul_mod(brute.matmul_mod(L0, R, p), U0, p).astype(np.uint32))
        for A in cases:
            LU, pp, pq, rk = oracle.pluq(A, p)
            LU1, pp1, pq1, rk1 = oracle.pluq_alg1(A, p)
            assert rk == rk1, (m, n)
            assert np.array_equal(pp, pp1) and np.array_equal(pq, pq1), (m, n)
            assert np.array_equal(LU, LU1), (m, n)
        # the anti-diagonal case does exercise descents at every level
        _, pp, pq, rk = oracle.pluq(cases[-1], p)
        assert rk == q and not np.array_equal(pq[:rk], np.sort(pq[:rk]))


@pytest.mark.parametrize("p", [2, 5, 65521])
def test_leading_submatrix_rank_profiles(p):
    """Corollary of Lemma 2: rank profiles of every leading (k,t) submatrix are read off R."""
    g = np.random.Generator(np.random.PCG64(1000 + p))
    for _ in range(6):
        m, n = int(g.integers(2, 9)), int(g.integers(2, 9))
        A = _structured(g, m, n, p)
        LU, pp, pq, r = oracle.pluq(A, p)
        R = R_from_pq(pp, pq, r, m, n)
        for k in range(1, m + 1):
            for t in range(1, n + 1):
                sub = A[:k, :t].astype(np.int64)
                # row rank profile of the leading block, greedily by rank tests
                rows, cols = [], []
                for i in range(k):
                    if brute.batch_rank(sub[rows + [i]][None], p)[0] > len(rows):
                        rows.append(i)
                for j in range(t):
                    if brute.batch_rank(sub[:, cols + [j]][None], p)[0] > len(cols):
                        cols.append(j)
                Rk = R[:k, :t]
                assert rows == sorted(np.nonzero(Rk.any(axis=1))[0].tolist())
                assert cols == sorted(np.nonzero(Rk.any(axis=0))[0].tolist())


def test_leu_theorem_random():
    """Theorem 1: P [L 0; M Y] P^T unit lower and Q^T [U V; 0 Z] Q upper."""
    g = np.random.Generator(np.random.PCG64(77))
    for _ in range(60):
        p = int(g.choice(PRIMES))
        m, n = int(g.integers(1, 30)), int(g.integers(1, 30))
        A = _structured(g, m, n, p)
        LU, pp, pq, r = oracle.pluq(A, p)
        Lfull = np.zeros((m, m), dtype=np.int64)
        Lfull[:, :r] = np.tril(LU[:, :r].astype(np.int64), -1)
        Y = np.tril(g.integers(0, p, (m - r, m - r)), -1)
        Lfull[r:, r:] = Y
        np.fill_diagonal(Lfull, 1)
        Pm = np.zeros((m, m), dtype=np.int64)
        Pm[pp, np.arange(m)] = 1
        Lbar = Pm @ Lfull @ Pm.T
        assert np.array_equal(Lbar, np.tril(Lbar)) and np.all(np.diagonal(Lbar) == 1)
        for Zkind in ("I", "upper", "zero"):
            Ufull = np.zeros((n, n), dtype=np.int64)
            Ufull[:r, :] = np.triu(LU[:r, :].astype(np.int64))
            if Zkind == "I":
                Ufull[r:, r:] = np.eye(n - r, dtype=np.int64)
            elif Zkind == "upper":
                Ufull[r:, r:] = np.triu(g.integers(0, p, (n - r, n - r)))
            Qm = np.zeros((n, n), dtype=np.int64)
            Qm[np.arange(n), pq] = 1
            Ubar = Qm.T @ Ufull @ Qm
            assert np.array_equal(Ubar, np.triu(Ubar))


def test_oracle_leu_pinned():
    """oracle.leu against the Corollary's properties, not against itself:
    Lbar unit lower, Ubar upper, Lbar E Ubar = A with E the rank profile matrix
    from the independent row-echelon routine, and for a generic matrix (all
    leading minors nonzero, so P = Q = I) the plain [L 0; M I] and [U V; 0 0]."""
    g = np.random.Generator(np.random.PCG64(78))
    for it in range(40):
        p = int(g.choice(PRIMES))
        m, n = int(g.integers(1, 25)), int(g.integers(1, 25))
        A = _structured(g, m, n, p)
        LU, pp, pq, r = oracle.pluq(A, p)
        Lb, Ub = oracle.leu(LU, pp, pq, r)
        Lb = Lb.astype(np.int64)
        Ub = Ub.astype(np.int64)
        assert np.array_equal(Lb, np.tril(Lb)) and np.all(np.diagonal(Lb) == 1)
        assert np.array_equal(Ub, np.triu(Ub))
        col = oracle.rank_profile(A, p)
        E = np.zeros((m, n), dtype=object)
        for i, c in enumerate(col):
            if c >= 0:
                E[i, c] = 1
        rec = (Lb.astype(object).dot(E).dot(Ub.astype(object))) % p
        assert np.array_equal(rec, A.astype(object) % p), (m, n, p)
    # generic: leading minors nonzero -> P = Q = I
    p = 65521
    n = 12
    L0 = np.tril(g.integers(0, p, (n, n)), -1) + np.eye(n, dtype=np.int64)
    U0 = np.triu(g.integers(1, p, (n, n)))
    A = (L0.astype(object).dot(U0.astype(object)) % p).astype(np.uint32)
    LU, pp, pq, r = oracle.pluq(A, p)
    Lb, Ub = oracle.leu(LU, pp, pq, r)
    assert np.array_equal(pp, np.arange(n)) and np.array_equal(pq, np.arange(n))
    assert np.array_equal(Lb.astype(np.int64), L0) and np.array_equal(Ub.astype(np.int64), U0)


# ------------------------------------------------------- planted / sizes --

@pytest.mark.parametrize("m,n,r,p", [(50, 60, 20, 65521), (64, 64, 64, 8388593),
                                      (100, 37, 30, 2147483647), (200, 200, 100, 251),
                                      (40, 90, 0, 7), (33, 17, 17, 2)])
def test_planted_rank_profile_recovered(m, n, r, p):
    A, pl = W.planted(m, n, r, p, seed=m * 1000 + n + r)
    col = oracle.rank_profile(A, p)
    assert np.array_equal(col, pl.rank_profile())
    LU, pp, pq, rr = oracle.pluq(A, p)
    assert rr == r
    assert certify(A, p, LU, pp, pq, rr, exact=True, expected_col_of_row=pl.rank_profile()) == ""


def test_planted_config_256():
    cfg = W.CONFIGS["planted_256"]
    A, pl = W.make(cfg)
    LU, pp, pq, r = oracle.pluq(A, cfg.p)
    assert r == 200
    assert certify(A, cfg.p, LU, pp, pq, r, exact=True, expected_col_of_row=pl.rank_profile()) == ""


def test_generator_entries_exact():
    """Sampled entries of A = L0[:,rows] U0[cols,:] recomputed with Python integers."""
    for (m, n, r, p) in [(60, 70, 25, 2147483647), (40, 40, 40, 8388593)]:
        A, pl = W.planted(m, n, r, p, seed=5)
        g = np.random.Generator(np.random.PCG64(9))
        for _ in range(50):
            i, j = int(g.integers(m)), int(g.integers(n))
            v = sum(int(pl.Lc[i, t]) * int(pl.Ur[t, j]) for t in range(r)) % p
            assert int(A[i, j]) == v


# ------------------------------------------------- special closed forms --

@pytest.mark.parametrize("n,p", [(8, 65521), (17, 2147483647), (24, 251)])
def test_generic_rank_profile_is_plain_lu(n, p):
    """All leading principal minors nonzero => P = Q = I and L, U = LU without pivoting."""
    g = np.random.Generator(np.random.PCG64(n))
    while True:
        A = g.integers(0, p, (n, n)).astype(np.uint32)
        lu = brute.doolittle(A, p)
        if lu is not None:
            break
    L, U = lu
    LU, pp, pq, r = oracle.pluq(A, p)
    assert r == n
    assert np.array_equal(pp, np.arange(n)) and np.array_equal(pq, np.arange(n))
    assert np.array_equal(np.tril(LU.astype(np.int64), -1), np.tril(L, -1))
    assert np.array_equal(np.triu(LU.astype(np.int64)), U)


@pytest.mark.parametrize("m,n", [(0, 0), (0, 5), (5, 0), (7, 9), (1, 1)])
def test_zero_matrix(m, n):
    A = np.zeros((m, n), dtype=np.uint32)
    LU, pp, pq, r = oracle.pluq(A, 65521)
    assert r == 0
    assert np.array_equal(pp, np.arange(m)) and np.array_equal(pq, np.arange(n))
    assert not LU.any()


def test_scaled_partial_permutation():
    """R of a scaled partial permutation matrix is its support; L = I and U = diag."""
    g = np.random.Generator(np.random.PCG64(3))
    p = 65521
    for _ in range(20):
        m, n = int(g.integers(1, 40)), int(g.integers(1, 40))
        r = int(g.integers(0, min(m, n) + 1))
        rows = g.choice(m, r, replace=False)
        cols = g.choice(n, r, replace=False)
        vals = g.integers(1, p, r)
        A = np.zeros((m, n), dtype=np.uint32)
        A[rows, cols] = vals
        LU, pp, pq, rr = oracle.pluq(A, p)
        assert rr == r
        assert np.array_equal(R_from_pq(pp, pq, r, m, n), (A != 0).astype(np.int64))
        expect = np.zeros((m, n), dtype=np.uint32)
        expect[np.arange(r), np.arange(r)] = A[pp[:r], pq[:r]]
        assert np.array_equal(LU, expect)


# ------------------------------------------------------ golden fixtures --

def _load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_golden_rotation_base_case():
    """A 2 x 6 case where a transposition in the m = 1 base case would report the
    column rank profile {1, 2}; the rank definition gives {0, 2}."""
    gd = _load_golden("rotation_2x6.json")
    A = np.array(gd["A"], dtype=np.uint32)
    p = gd["p"]
    for f in (oracle.pluq, oracle.pluq_alg1):
        LU, pp, pq, r = f(A, p)
        assert r == gd["rank"]
        assert sorted(pq[:r].tolist()) == gd["col_rank_profile"]
        assert sorted(pp[:r].tolist()) == gd["row_rank_profile"]
        assert [[int(a), int(b)] for a, b in zip(pp[:r], pq[:r])] == gd["pivots_in_order"]


def test_golden_alg1_order_8x8():
    """A case where Algorithm 2's growing leading submatrix would meet pivot (3,4)
    before (2,6); Algorithm 1 (and the canonical order) put (2,6) first."""
    gd = _load_golden("alg1_order_8x8.json")
    A = np.array(gd["A"], dtype=np.uint32)
    p = gd["p"]
    for f in (oracle.pluq, oracle.pluq_alg1):
        LU, pp, pq, r = f(A, p)
        assert [[int(a), int(b)] for a, b in zip(pp[:r], pq[:r])] == gd["pivots_in_order"]


# ------------------------------------------------ BLAS-like subroutines --

def test_matmul_sub_against_python_integers():
    g = np.random.Generator(np.random.PCG64(11))
    for p in (2, 65521, 2147483647):
        for (M, N, K) in [(5, 7, 3), (16, 9, 33), (1, 1, 1), (4, 6, 0)]:
            A = g.integers(0, p, (M, K)).astype(np.uint32)
            B = g.integers(0, p, (K, N)).astype(np.uint32)
            C = g.integers(0, p, (M, N)).astype(np.uint32)
            got = oracle.matmul_sub(C, A, B, p)
            want = (C.astype(object) - brute.matmul_mod(A, B, p).astype(object)) % p
            assert np.array_equal(got.astype(np.int64), want.astype(np.int64))


def test_trsm_solves():
    g = np.random.Generator(np.random.PCG64(12))
    for p in (3, 65521, 2147483647):
        for (r, N) in [(1, 5), (7, 3), (20, 20)]:
            L = np.tril(g.integers(0, p, (r, r)), -1)
            Lu = L + np.eye(r, dtype=np.int64)
            B = g.integers(0, p, (r, N)).astype(np.uint32)
            X = oracle.trsm_left_lower_unit((L + 5 * np.eye(r, dtype=np.int64)) % p, B, p)
            assert np.array_equal(brute.matmul_mod(Lu, X, p), B.astype(np.int64))
            U = np.triu(g.integers(1, p, (r, r)))
            B2 = g.integers(0, p, (N, r)).astype(np.uint32)
            X2 = oracle.trsm_right_upper(U, B2, p)
            assert np.array_equal(brute.matmul_mod(X2, U, p), B2.astype(np.int64))


def test_descent_free_profiles_are_met_in_row_order():
    """When the ones of R have increasing columns in row order, Algorithm 1's
    recursion meets them in row order (checked against the literal reading)."""
    g = np.random.Generator(np.random.PCG64(21))
    for _ in range(40):
        m, n = int(g.integers(2, 40)), int(g.integers(2, 40))
        r = int(g.integers(0, min(m, n) + 1))
        rows = np.sort(g.choice(m, r, replace=False))
        cols = np.sort(g.choice(n, r, replace=False))        # increasing with the rows
        col = np.full(m, -1, dtype=np.int32)
        col[rows] = cols
        pr, pc = oracle.canonical_order(m, n, col)
        assert np.array_equal(pr, rows) and np.array_equal(pc, cols)
        # and the literal Algorithm 1 agrees on a matrix with that profile
        Lc = np.tril(g.integers(0, 7, (m, m)), -1) + np.eye(m, dtype=np.int64)
        Uc = np.triu(g.integers(0, 7, (n, n)), 1) + np.eye(n, dtype=np.int64)
        Rm = np.zeros((m, n), dtype=np.int64)
        Rm[rows, cols] = 1
        A = brute.matmul_mod(brute.matmul_mod(Lc, Rm, 7), Uc, 7).astype(np.uint32)
        _, pp, pq, rr = oracle.pluq_alg1(A, 7)
        assert rr == r and np.array_equal(pp[:r], rows) and np.array_equal(pq[:r], cols)


# ------------------------------------------- uses of the decomposition --
# Sec. 1: linear systems, the determinant and the nullspace.  The oracle
# computes them from the RREF and from elimination with row exchanges; these
# pins check them against enumeration, the Leibniz formula and Cramer's rule.

def _profiles_brute(A, p):
    """(row rank profile, column rank profile) from the brute-force R."""
    m, n = A.shape
    if m == 0 or n == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    R = brute.rank_profile_matrix(A, p)[0]
    rows, cols = np.nonzero(R)
    return np.sort(rows), np.sort(cols)


def _tiny_cases(g, p, shapes, per_shape=6):
    for m, n in shapes:
        for t in range(per_shape):
            r = int(g.integers(0, min(m, n) + 1))
            if t % 3 == 2:
                A = g.integers(0, p, (m, n)).astype(np.uint32)
            else:
                A, _ = W.planted(m, n, r, p, seed=int(g.integers(1 << 30)))
            yield A


@pytest.mark.parametrize("p", [2, 3, 5, 7, 65521, 2147483647])
def test_determinant_matches_leibniz(p):
    g = np.random.Generator(np.random.PCG64(p + 11))
    for n in range(0, 7):
        for t in range(8):
            if t % 2:
                A = g.integers(0, p, (n, n)).astype(np.uint32)
            else:
                A, _ = W.planted(n, n, int(g.integers(0, n + 1)), p, seed=int(g.integers(1 << 30)))
            assert oracle.determinant(A, p) == brute.leibniz_det(A, p), (n, t)


@pytest.mark.parametrize("n,p", [(40, 65521), (33, 2147483647), (50, 3)])
def test_determinant_planted_closed_form(n, p):
    """A = L0 Pi U0 with unit triangular L0, U0: det A = sgn of the planted
    pairing (rows are 0..n-1, row j has its one in column cols[j])."""
    A, pl = W.planted(n, n, n, p, seed=n)
    sgn = brute.permutation_sign(pl.cols)
    assert oracle.determinant(A, p) == sgn % p
    B, _ = W.planted(n, n, n - 1, p, seed=n + 1)
    assert oracle.determinant(B, p) == 0


def test_determinant_multiplicative():
    p = 65521
    g = np.random.Generator(np.random.PCG64(5))
    for n in (1, 5, 12):
        A = g.integers(0, p, (n, n)).astype(np.uint32)
        B = g.integers(0, p, (n, n)).astype(np.uint32)
        AB = brute.matmul_mod(A, B, p).astype(np.uint32)
        assert oracle.determinant(AB, p) == oracle.determinant(A, p) * oracle.determinant(B, p) % p


@pytest.mark.parametrize("p", [2, 3, 5])
def test_right_nullspace_brute_force(p):
    """ker A by enumeration equals the span of N's columns, and N is the
    identity on the coordinates outside the column rank profile."""
    g = np.random.Generator(np.random.PCG64(100 + p))
    shapes = [(3, 4), (4, 3), (2, 5), (5, 2), (4, 4), (1, 3)] if p < 5 else [(3, 4), (2, 4), (4, 3)]
    for A in _tiny_cases(g, p, shapes):
        m, n = A.shape
        N = oracle.right_nullspace(A, p).astype(np.int64)
        _, cols = _profiles_brute(A, p)
        r = cols.size
        assert N.shape == (n, n - r)
        free = np.setdiff1d(np.arange(n), cols)
        assert np.array_equal(N[free, :], np.eye(n - r, dtype=np.int64))
        X = brute.all_vectors(n, p)
        ker = {tuple(x) for x in X if not np.any(brute.matmul_mod(A, x[:, None], p))}
        Y = brute.all_vectors(n - r, p) if n > r else np.zeros((1, 0), dtype=np.int64)
        span = {tuple(v) for v in (brute.matmul_mod(N, Y.T, p).T if n > r else
                                   np.zeros((1, n), dtype=np.int64))}
        assert ker == span


@pytest.mark.parametrize("p", [2, 3])
def test_left_nullspace_brute_force(p):
    """{y : y A = 0} by enumeration equals the row span of the left basis,
    which is the identity on the rows outside the row rank profile."""
    g = np.random.Generator(np.random.PCG64(200 + p))
    for A in _tiny_cases(g, p, [(4, 3), (3, 4), (5, 2), (2, 2)]):
        m, n = A.shape
        N = oracle.left_nullspace(A, p).astype(np.int64)
        rows, _ = _profiles_brute(A, p)
        r = rows.size
        assert N.shape == (m - r, m)
        free = np.setdiff1d(np.arange(m), rows)
        assert np.array_equal(N[:, free], np.eye(m - r, dtype=np.int64))
        Y = brute.all_vectors(m, p)
        ker = {tuple(y) for y in Y if not np.any(brute.matmul_mod(y[None, :], A, p))}
        Z = brute.all_vectors(m - r, p) if m > r else np.zeros((1, 0), dtype=np.int64)
        span = {tuple(v) for v in (brute.matmul_mod(Z, N, p) if m > r else
                                   np.zeros((1, m), dtype=np.int64))}
        assert ker == span


@pytest.mark.parametrize("p", [2, 3, 5])
def test_solve_brute_force(p):
    """Per right-hand side: consistent iff enumeration finds a solution, and
    the returned one is the only solution that vanishes outside the column
    rank profile."""
    g = np.random.Generator(np.random.PCG64(300 + p))
    for A in _tiny_cases(g, p, [(3, 4), (4, 3), (4, 4), (2, 5)] if p < 5 else [(3, 4), (4, 3)]):
        m, n = A.shape
        k = 4
        B = g.integers(0, p, (m, k)).astype(np.uint32)
        B[:, 0] = brute.matmul_mod(A, g.integers(0, p, (n, 1)), p)[:, 0]   # one consistent column
        X, ok = oracle.solve(A, B, p)
        _, cols = _profiles_brute(A, p)
        free = np.setdiff1d(np.arange(n), cols)
        V = brute.all_vectors(n, p)
        AV = brute.matmul_mod(A, V.T, p).T                                 # (p^n, m)
        for c in range(k):
            sols = V[np.all(AV == B[:, c].astype(np.int64)[None, :], axis=1)]
            assert bool(ok[c]) == (len(sols) > 0)
            if len(sols):
                canon = sols[np.all(sols[:, free] == 0, axis=1)]
                assert len(canon) == 1
                assert np.array_equal(X[:, c].astype(np.int64), canon[0])
        assert ok[0]


def test_solve_cramer():
    """Nonsingular A: x_i = det(A with column i replaced by b) / det(A)."""
    p = 65521
    g = np.random.Generator(np.random.PCG64(9))
    for n in (1, 3, 5):
        A, _ = W.planted(n, n, n, p, seed=n + 50)
        b = g.integers(0, p, (n, 1)).astype(np.uint32)
        X, ok = oracle.solve(A, b, p)
        assert ok.all()
        d = brute.leibniz_det(A, p)
        dinv = pow(d, p - 2, p)
        for i in range(n):
            Ai = A.copy()
            Ai[:, i] = b[:, 0]
            assert int(X[i, 0]) == brute.leibniz_det(Ai, p) * dinv % p


def test_nullspace_and_solve_medium():
    """At 60 x 80: A N = 0, N A' = 0, A X = B on the consistent columns, with
    exact Python-integer products."""
    p = 8388593
    A, pl = W.planted(60, 80, 37, p, seed=3)
    N = oracle.right_nullspace(A, p)
    assert N.shape == (80, 43)
    assert not np.any(brute.matmul_mod(A, N, p))
    Nl = oracle.left_nullspace(A, p)
    assert Nl.shape == (23, 60)
    assert not np.any(brute.matmul_mod(Nl, A, p))
    g = np.random.Generator(np.random.PCG64(4))
    B = brute.matmul_mod(A, g.integers(0, p, (80, 3)), p).astype(np.uint32)
    X, ok = oracle.solve(A, B, p)
    assert ok.all()
    assert np.array_equal(brute.matmul_mod(A, X, p), B.astype(np.int64))
    B2 = g.integers(0, p, (60, 2)).astype(np.uint32)
    _, ok2 = oracle.solve(A, B2, p)
    assert not ok2.any()                 # random right-hand sides miss a rank-37 image


def test_use_pins_reject_plausible_mistakes():
    """The checks above would catch the usual slips: a determinant without the
    permutation signs, a kernel basis without the minus sign, a particular
    solution with nonzero free coordinates."""
    p = 5
    g = np.random.Generator(np.random.PCG64(77))
    # determinant: product of U's diagonal without sgn(P) sgn(Q)
    caught = False
    for _ in range(40):
        A = g.integers(0, p, (4, 4)).astype(np.uint32)
        LU, pp, pq, r = oracle.pluq(A, p)
        if r < 4:
            continue
        unsigned = int(np.prod([int(LU[i, i]) for i in range(4)], dtype=object) % p)
        assert oracle.determinant(A, p) == brute.leibniz_det(A, p)
        if unsigned != brute.leibniz_det(A, p):
            caught = True
    assert caught
    # nullspace: the pivot coordinates without the minus sign
    A = np.array([[1, 2, 3, 1], [0, 1, 4, 2]], dtype=np.uint32)
    N = oracle.right_nullspace(A, p).astype(np.int64)
    assert not np.any(brute.matmul_mod(A, N, p))
    _, pc = oracle.rref(A, p)
    wrong = N.copy()
    wrong[pc, :] = (p - wrong[pc, :]) % p
    assert np.any(brute.matmul_mod(A, wrong, p))
    # solve: a solution with a nonzero free coordinate is valid but not the one
    # the definition picks
    b = brute.matmul_mod(A, np.array([[1], [1], [1], [1]]), p).astype(np.uint32)
    X, ok = oracle.solve(A, b, p)
    free = np.setdiff1d(np.arange(4), pc)
    assert ok.all() and not np.any(X[free, 0])
    other = (X[:, 0].astype(np.int64) + N[:, 0]) % p
    assert not np.any(brute.matmul_mod(A, other[:, None], p) - b.astype(np.int64))
    assert np.any(other[free])


# ------------------------------------------------------------ PLE / CUP --
# Sec. 1 relates the PLUQ to the PLE (E in row echelon form, pivots on the
# column rank profile) and CUP (C in column echelon form, pivots on the row
# rank profile) decompositions.  The oracle writes them out from their
# definitions; these pins check every defining property against brute force.

def _greedy_profiles(A, p):
    """Row and column rank profiles by greedy rank tests (brute force)."""
    A = A.astype(np.int64)
    m, n = A.shape
    rows, cols = [], []
    for i in range(m):
        if brute.batch_rank(A[rows + [i]][None], p)[0] > len(rows):
            rows.append(i)
    for j in range(n):
        if brute.batch_rank(A[:, cols + [j]][None], p)[0] > len(cols):
            cols.append(j)
    return rows, cols


def _leading(v):
    nz = np.nonzero(v)[0]
    return int(nz[0]) if nz.size else -1


@pytest.mark.parametrize("p", [2, 3, 7, 65521, 2147483647])
def test_ple_cup_defining_properties(p):
    g = np.random.Generator(np.random.PCG64(777 + p))
    shapes = [(1, 1), (2, 5), (5, 2), (6, 6), (9, 7), (7, 12), (16, 16), (0, 4), (4, 0)]
    for (m, n) in shapes:
        for _ in range(3):
            A = _structured(g, m, n, p) if m and n else np.zeros((m, n), np.uint32)
            rows, cols = _greedy_profiles(A, p) if m and n else ([], [])
            r = len(rows)
            # PLE: A[P] = L E
            pp, L, E, rk = oracle.ple(A, p)
            assert rk == r
            assert sorted(pp.tolist()) == list(range(m))
            prod = brute.matmul_mod(L, E, p) if r else np.zeros((m, n), np.int64)
            assert np.array_equal(prod, A[pp].astype(np.int64))
            assert np.array_equal(np.triu(L, 1), np.zeros_like(L)) and all(L[t, t] == 1 for t in range(r))
            lead = [_leading(E[t]) for t in range(r)]
            assert lead == cols                      # row echelon on the column rank profile
            # CUP: A[:, Q] = C U
            pq, C, U, rk2 = oracle.cup(A, p)
            assert rk2 == r
            assert sorted(pq.tolist()) == list(range(n))
            prod = brute.matmul_mod(C, U, p) if r else np.zeros((m, n), np.int64)
            assert np.array_equal(prod, A[:, pq].astype(np.int64))
            assert np.array_equal(np.tril(U, -1), np.zeros_like(U)) and all(U[t, t] == 1 for t in range(r))
            lead_c = [_leading(C[:, t]) for t in range(r)]
            assert lead_c == rows                    # column echelon on the row rank profile
            # the pivot rows / columns come first, the others after in increasing order
            assert pp[r:].tolist() == sorted(set(range(m)) - set(pp[:r].tolist()))
            assert pq[r:].tolist() == sorted(set(range(n)) - set(pq[:r].tolist()))


def test_ple_cup_closed_form_2x2():
    """A = [[0, a], [b, c]] (a, b nonzero): the pivots (0, 1) and (1, 0) form a
    descent.  PLE: P swaps the rows, L = I, E = [[b, c], [0, a]].  CUP: Q swaps
    the columns, C = [[a, 0], [c, b]], U = I."""
    p = 65521
    g = np.random.Generator(np.random.PCG64(5))
    for _ in range(20):
        a, b = (int(x) for x in g.integers(1, p, 2))
        c = int(g.integers(0, p))
        A = np.array([[0, a], [b, c]], dtype=np.uint32)
        pp, L, E, r = oracle.ple(A, p)
        assert r == 2 and pp.tolist() == [1, 0]
        assert L.tolist() == [[1, 0], [0, 1]] and E.tolist() == [[b, c], [0, a]]
        pq, C, U, r = oracle.cup(A, p)
        assert r == 2 and pq.tolist() == [1, 0]
        assert C.tolist() == [[a, 0], [c, b]] and U.tolist() == [[1, 0], [0, 1]]


def test_ple_needs_more_than_permuting_the_pluq_factors():
    """The reading behind the GPU construction: Sec. 1 says a PLE follows from
    the PLUQ by permutations only.  On the 2x2 example with a descent, the
    rank-one terms of A = P [L; M] [U V] Q sorted by pivot column give a left
    factor that no row permutation bringing the pivot rows to the diagonal
    makes lower triangular, so the L of the PLE is not a permutation of the
    PLUQ's L (an r x r elimination without pivoting is needed)."""
    p = 65521
    A = np.array([[0, 3], [5, 2]], dtype=np.uint32)
    LU, pp, pq, r = oracle.pluq(A, p)
    assert r == 2 and pp.tolist() == [0, 1] and pq.tolist() == [1, 0]   # pivots (0,1), (1,0)
    Lp = np.tril(LU.astype(np.int64), -1) + np.eye(2, dtype=np.int64)    # [L; M] in packed order
    Lbar = np.zeros((2, 2), dtype=np.int64)
    Lbar[np.ix_(pp, pp)] = Lp                                             # P [L 0; M I] P^T
    order = np.argsort(pq[:r])                                            # pivots by column
    Lc = Lbar[:, pp[:r][order]]
    assert Lc[0, 1] != 0                          # (0,1) lies above the diagonal in any row order
    Pt = Lc[pp[:r][order]]                        # the row order that puts pivot rows on the diagonal
    assert not np.array_equal(np.triu(Pt, 1), np.zeros_like(Pt))
    _, L, _, _ = oracle.ple(A, p)
    assert L.tolist() == [[1, 0], [0, 1]]
