"""Per-kernel parity of the CUDA path against the CPU oracle (bit-exact).

Every case calls the C-ABI library through its binding and compares element
by element with the oracle on the same seeded inputs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1301_4438_gb300 import pluq, workloads as W
from tests import brute

pytestmark = pytest.mark.gpu
PRIMES = [2, 3, 251, 65521, 8388593, 2147483647]
KINDS = ["simt", "tensor"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.uint32)


def _structured(g, m, n, p):
    kind = int(g.integers(0, 4))
    if kind == 0:
        return g.integers(0, p, (m, n)).astype(np.uint32)
    if kind == 1:
        return (g.integers(0, p, (m, n)) * (g.random((m, n)) < 0.1)).astype(np.uint32)
    if kind == 2:
        r = int(g.integers(0, min(m, n) + 1))
        return W.planted(m, n, r, p, int(g.integers(1 << 30)))[0]
    A = g.integers(0, p, (m, n))
    A[g.random(m) < 0.3] = 0
    A[:, g.random(n) < 0.3] = 0
    return A.astype(np.uint32)


# ------------------------------------------------------------------ leaf --

@pytest.mark.parametrize("p", PRIMES)
def test_leaf_matches_oracle(p):
    g = np.random.Generator(np.random.PCG64(p + 1))
    lm, ln = pluq.leaf_max()
    shapes = [(1, 1), (1, 128), (128, 1), (128, 128), (127, 65), (3, 100), (64, 64), (2, 2)]
    shapes += [(int(g.integers(1, lm + 1)), int(g.integers(1, ln + 1))) for _ in range(12)]
    for (m, n) in shapes:
        A = _structured(g, m, n, p)
        LU0, pp0, pq0, r0 = oracle.pluq(A, p)
        d = dev(A)
        pp, pq, r = pluq.pluq_leaf(d, p)
        assert r == r0, (m, n)
        assert np.array_equal(pp.cpu().numpy(), pp0), (m, n)
        assert np.array_equal(pq.cpu().numpy(), pq0), (m, n)
        assert np.array_equal(host(d), LU0), (m, n)


@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
def test_leaf_left_looking_variant_matches_oracle(p):
    """The left-looking form of the base case's blocked elimination (the
    variant the base-case section mentions) gives the same result: generic
    blocks (all leading minors nonzero), blocks whose generic attempt fails
    late, rank-deficient blocks (elimination in Algorithm 1's order), wide and
    tall ones; then a whole decomposition with it."""
    g = np.random.Generator(np.random.PCG64(p + 31))
    old = pluq.pluq_get_leaf_variant()
    pluq.pluq_set_leaf_variant(True)
    try:
        cases = [g.integers(0, p, (128, 128)).astype(np.uint32),
                 g.integers(0, p, (100, 128)).astype(np.uint32),
                 g.integers(0, p, (128, 37)).astype(np.uint32),
                 _lu_product(g, 120, 128, p, 70),
                 W.planted(128, 128, 50, p, 5)[0],
                 W.planted(97, 120, 97, p, 6)[0],
                 _structured(g, 77, 66, p)]
        for A in cases:
            LU0, pp0, pq0, r0 = oracle.pluq(A, p)
            d = dev(A)
            pp, pq, r = pluq.pluq_leaf(d, p)
            assert r == r0, A.shape
            assert np.array_equal(pp.cpu().numpy(), pp0), A.shape
            assert np.array_equal(pq.cpu().numpy(), pq0), A.shape
            assert np.array_equal(host(d), LU0), A.shape
        A = W.planted(700, 500, 300, p, 7)[0]
        LU0, pp0, pq0, r0 = oracle.pluq(A, p)
        d = dev(A)
        pp, pq, r = pluq.pluq_mod_p(d, p)
        assert r == r0 and np.array_equal(host(d), LU0)
        assert np.array_equal(pp.cpu().numpy(), pp0) and np.array_equal(pq.cpu().numpy(), pq0)
    finally:
        pluq.pluq_set_leaf_variant(old)


def _lu_product(g, m, n, p, zero_at):
    """L0 U0 mod p with L0 unit lower (m x m) and U0 upper (m x n) whose
    diagonal is nonzero except at `zero_at`: the leading minors are nonzero
    exactly up to order zero_at."""
    L0 = np.tril(g.integers(0, p, (m, m)), -1) + np.eye(m, dtype=np.int64)
    U0 = np.triu(g.integers(0, p, (m, n)), 1)
    for k in range(min(m, n)):
        U0[k, k] = 0 if k == zero_at else int(g.integers(1, p))
    return (L0.astype(object).dot(U0.astype(object)) % p).astype(np.uint32)


@pytest.mark.parametrize("p", PRIMES)
def test_leaf_generic_rank_profile_and_late_fallback(p):
    """Blocks with all leading minors nonzero (the blocked path without
    pivoting) and blocks whose first zero minor comes only after one or more
    panels (the hand-over to the general path after work was done)."""
    g = np.random.Generator(np.random.PCG64(p + 77))
    cases = []
    for (m, n) in [(64, 64), (128, 128), (100, 37), (37, 100), (17, 1), (1, 17), (128, 50),
                   (33, 33)]:
        k = min(m, n)
        cases += [(m, n, None), (m, n, k - 1), (m, n, k // 2), (m, n, 0)]
    for (m, n, z) in cases:
        A = _lu_product(g, m, n, p, -1 if z is None else z)
        LU0, pp0, pq0, r0 = oracle.pluq(A, p)
        d = dev(A)
        pp, pq, r = pluq.pluq_leaf(d, p)
        assert r == r0, (m, n, z)
        assert np.array_equal(pp.cpu().numpy(), pp0), (m, n, z)
        assert np.array_equal(pq.cpu().numpy(), pq0), (m, n, z)
        assert np.array_equal(host(d), LU0), (m, n, z)


def test_leaf_exhaustive_gf2_4x4():
    As = brute.all_matrices(4, 4, 2)[::5]
    for A in As:
        A = A.astype(np.uint32)
        LU0, pp0, pq0, r0 = oracle.pluq(A, 2)
        d = dev(A)
        pp, pq, r = pluq.pluq_leaf(d, 2)
        assert r == r0 and np.array_equal(pp.cpu().numpy(), pp0)
        assert np.array_equal(pq.cpu().numpy(), pq0) and np.array_equal(host(d), LU0)


def test_leaf_in_place_inside_larger_matrix():
    p = 65521
    g = np.random.Generator(np.random.PCG64(5))
    big = g.integers(0, p, (200, 300)).astype(np.uint32)
    sub = W.planted(100, 90, 40, p, 3)[0]
    big[50:150, 70:160] = sub
    d = dev(big)
    pp, pq, r = pluq.pluq_leaf(d[50:150, 70:160], p)
    LU0, pp0, pq0, r0 = oracle.pluq(sub, p)
    out = host(d)
    assert r == r0 and np.array_equal(out[50:150, 70:160], LU0)
    mask = np.ones_like(big, dtype=bool)
    mask[50:150, 70:160] = False
    assert np.array_equal(out[mask], big[mask])      # nothing outside the block touched


# ---------------------------------------------------------------- modmm --

@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("p", PRIMES)
def test_modmm_matches_oracle(kind, p):
    g = np.random.Generator(np.random.PCG64(1000 + p))
    shapes = [(1, 1, 1), (64, 64, 64), (130, 257, 129), (7, 300, 1000), (300, 5, 77),
              (256, 256, 1500), (1, 513, 64), (200, 200, 0)]
    for (M, N, K) in shapes:
        A = g.integers(0, p, (M, K)).astype(np.uint32)
        B = g.integers(0, p, (K, N)).astype(np.uint32)
        C = g.integers(0, p, (M, N)).astype(np.uint32)
        want = oracle.matmul_sub(C, A, B, p)
        dC = dev(C)
        pluq.pluq_modmm(dC, dev(A), dev(B), p, mm=kind)
        assert np.array_equal(host(dC), want), (M, N, K)
        # assign form: C <- A B
        want2 = oracle.matmul_sub(np.zeros((M, N), np.uint32), A, B, p)
        want2 = ((p - want2.astype(np.int64)) % p).astype(np.uint32)
        dC2 = dev(C)
        pluq.pluq_modmm(dC2, dev(A), dev(B), p, assign=True, mm=kind)
        assert np.array_equal(host(dC2), want2), (M, N, K)


@pytest.mark.parametrize("kind", KINDS)
def test_modmm_strided_blocks(kind):
    p = 8388593
    g = np.random.Generator(np.random.PCG64(8))
    big = g.integers(0, p, (700, 900)).astype(np.uint32)
    d = dev(big)
    # C = rows 400..650 x cols 500..880, A = rows 400..650 x cols 0..300, B = rows 0..300 x 500..880
    C, A, B = big[400:650, 500:880], big[400:650, 0:300], big[0:300, 500:880]
    want = oracle.matmul_sub(C, A, B, p)
    pluq.pluq_modmm(d[400:650, 500:880], d[400:650, 0:300], d[0:300, 500:880], p, mm=kind)
    out = host(d)
    assert np.array_equal(out[400:650, 500:880], want)
    mask = np.ones_like(big, dtype=bool)
    mask[400:650, 500:880] = False
    assert np.array_equal(out[mask], big[mask])


# ----------------------------------------------------------------- trsm --

@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("p", [3, 65521, 2147483647])
def test_trsm_matches_oracle(kind, p):
    g = np.random.Generator(np.random.PCG64(2000 + p))
    for (r, other) in [(1, 5), (2, 1), (3, 300), (8, 129), (15, 1000), (16, 257), (17, 40),
                       (31, 7), (32, 33), (63, 10), (64, 64), (65, 200), (96, 17),
                       (127, 9), (128, 128), (129, 20), (200, 130), (517, 300)]:
        L = g.integers(0, p, (r, r)).astype(np.uint32)
        B = g.integers(0, p, (r, other)).astype(np.uint32)
        want = oracle.trsm_left_lower_unit(L, B, p)
        dB = dev(B)
        pluq.pluq_trsm_left_lower_unit(dev(L), dB, p, mm=kind)
        assert np.array_equal(host(dB), want), ("left", r, other)
        U = np.triu(g.integers(1, p, (r, r))).astype(np.uint32)
        U = (U + np.tril(g.integers(0, p, (r, r)), -1)).astype(np.uint32)   # lower part ignored
        B2 = g.integers(0, p, (other, r)).astype(np.uint32)
        want2 = oracle.trsm_right_upper(np.triu(U), B2, p)
        dB2 = dev(B2)
        pluq.pluq_trsm_right_upper(dev(U), dB2, p, mm=kind)
        assert np.array_equal(host(dB2), want2), ("right", r, other)


# ---------------------------------------------------------- permutations --

def test_perm_rows_cols():
    g = np.random.Generator(np.random.PCG64(9))
    # staged in shared memory (column stripes of 16, 8 or 4 / whole rows), and
    # the shapes past the staging limits that go through the scratch instead
    for (h, w) in [(1, 1), (5, 1000), (1000, 3), (257, 513), (2000, 37), (5000, 21),
                   (13000, 9), (3, 60000), (4500, 1001)]:
        X = g.integers(0, 1 << 31, (h, w)).astype(np.uint32)
        pr = g.permutation(h).astype(np.int32)
        pc = g.permutation(w).astype(np.int32)
        d = dev(X)
        pluq.pluq_perm_rows(d, torch.from_numpy(pr).cuda())
        assert np.array_equal(host(d), X[pr]), (h, w)
        pluq.pluq_perm_cols(d, torch.from_numpy(pc).cuda())
        assert np.array_equal(host(d), X[pr][:, pc]), (h, w)


@pytest.mark.parametrize("c0", [0, 1, 2, 3])
@pytest.mark.parametrize("ld", [1024, 1027])
def test_perm_strided_blocks_in_place(c0, ld):
    """Blocks starting at every 16-byte phase, with a 16-byte row stride (whole
    chunks move as uint4, partial chunks element by element) and without one
    (every element on its own); nothing outside the block changes."""
    g = np.random.Generator(np.random.PCG64(100 * c0 + ld))
    big = g.integers(0, 1 << 31, (300, ld)).astype(np.uint32)
    for (r0, h, w) in [(5, 257, 130), (1, 40, 700), (0, 299, 5)]:
        pr = g.permutation(h).astype(np.int32)
        pc = g.permutation(w).astype(np.int32)
        d = dev(big)
        blk = d[r0:r0 + h, c0:c0 + w]
        pluq.pluq_perm_rows(blk, torch.from_numpy(pr).cuda())
        want = big.copy()
        want[r0:r0 + h, c0:c0 + w] = big[r0:r0 + h, c0:c0 + w][pr]
        assert np.array_equal(host(d), want), ("rows", r0, h, w)
        pluq.pluq_perm_cols(blk, torch.from_numpy(pc).cuda())
        want[r0:r0 + h, c0:c0 + w] = want[r0:r0 + h, c0:c0 + w][:, pc]
        assert np.array_equal(host(d), want), ("cols", r0, h, w)


# -------------------------------------------------------- rank profiles --

def test_rank_profile_readouts():
    p = 65521
    A, pl = W.planted(300, 200, 120, p, 11)
    d = dev(A)
    pp, pq, r = pluq.pluq_mod_p(d, p, mm="simt")
    assert r == 120
    rows = pluq.row_rank_profile(pp, r).cpu().numpy()
    cols = pluq.col_rank_profile(pq, r).cpu().numpy()
    assert np.array_equal(rows, np.sort(pl.rows))
    assert np.array_equal(cols, np.sort(pl.cols))
    rr, cc = pluq.rank_profile_matrix(pp, pq, r)
    order = np.argsort(pl.rows)
    assert np.array_equal(rr.cpu().numpy(), pl.rows[order])
    assert np.array_equal(cc.cpu().numpy(), pl.cols[order])


@pytest.mark.parametrize("m,n,r,p", [(300, 200, 120, 65521), (150, 260, 150, 65521),
                                     (90, 70, 3, 2147483647), (40, 30, 0, 7)])
def test_extract_factors(m, n, r, p):
    """[L; M] and [U V] read out of the packed result: equal to the oracle's
    packed factors sliced by definition, and P [L; M] [U V] Q == A."""
    A, _ = W.planted(m, n, r, p, seed=m + n + r)
    LU0, pp0, pq0, r0 = oracle.pluq(A, p)
    d = dev(A)
    pp, pq, rk = pluq.pluq_mod_p(d, p, mm="tensor")
    assert rk == r0 == r
    L = pluq.pluq_extract_L(d, rk).cpu().numpy().astype(np.uint32)
    U = pluq.pluq_extract_U(d, rk).cpu().numpy().astype(np.uint32)
    L0 = np.tril(LU0[:, :r0].astype(np.int64), -1) + np.eye(m, r0, dtype=np.int64)
    U0 = np.triu(LU0[:r0, :].astype(np.int64))
    assert np.array_equal(L.astype(np.int64), L0)
    assert np.array_equal(U.astype(np.int64), U0)
    # reconstruction, exact in Python integers
    prod = np.array(L, dtype=object).dot(np.array(U, dtype=object)) % p if r0 else \
        np.zeros((m, n), dtype=object)
    Ap = A[pp0][:, pq0].astype(object)
    assert np.array_equal(prod, Ap)


@pytest.mark.parametrize("m,n,r,p", [(120, 90, 50, 65521), (64, 64, 64, 2147483647),
                                     (33, 70, 0, 7), (200, 150, 150, 8388593)])
def test_leu_and_leading_profiles(m, n, r, p):
    """LEU read-out bit-exact with the oracle's (its definition), and the rank
    profiles of leading k x t blocks, read from P and Q, equal the oracle's
    row-echelon rank profile of A[:k, :t]."""
    A, _ = W.planted(m, n, r, p, seed=3 * m + n + r)
    LU0, pp0, pq0, r0 = oracle.pluq(A, p)
    d = dev(A)
    pp, pq, rk = pluq.pluq_mod_p(d, p)
    assert rk == r0
    Lb, Ub = pluq.pluq_leu(d, pp, pq, rk)
    Lb0, Ub0 = oracle.leu(LU0, pp0, pq0, r0)
    assert np.array_equal(host(Lb), Lb0)
    assert np.array_equal(host(Ub), Ub0)
    g = np.random.Generator(np.random.PCG64(m * n + 1))
    blocks = [(m, n), (0, n), (m, 0), (1, 1)] + [(int(g.integers(0, m + 1)), int(g.integers(0, n + 1)))
                                                 for _ in range(8)]
    for (k, t) in blocks:
        rows, cols = pluq.pluq_leading_rank_profiles(pp, pq, rk, k, t)
        col = oracle.rank_profile(A[:k, :t], p) if k and t else np.zeros(0, np.int32)
        want_rows = np.nonzero(col >= 0)[0]
        want_cols = np.sort(col[col >= 0])
        assert np.array_equal(rows.cpu().numpy(), want_rows), (k, t)
        assert np.array_equal(cols.cpu().numpy(), want_cols), (k, t)


def test_extract_errors():
    d = torch.zeros((4, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(pluq.PluqError):
        pluq.pluq_extract_L(d, 5)          # r > min(m, n)
    with pytest.raises(pluq.PluqError):
        pluq.pluq_extract_U(d, -1)


# -------------------------------------------------------------- errors --

def test_error_statuses_leave_input_untouched():
    p = 65521
    A = np.full((10, 10), 5, dtype=np.uint32)
    A[3, 4] = p                      # not reduced
    d = dev(A)
    with pytest.raises(pluq.PluqError) as e:
        pluq.pluq_mod_p(d, p)
    assert e.value.status == -3
    assert np.array_equal(host(d), A)
    with pytest.raises(pluq.PluqError) as e:
        pluq.pluq_mod_p(dev(np.zeros((4, 4), np.uint32)), 65535)
    assert e.value.status == -2
    # a too-small workspace (the binding would replace it; call the library directly)
    lib = pluq.load()
    import ctypes
    r = ctypes.c_int64(0)
    z = dev(np.zeros((64, 64), np.uint32))
    pp = torch.empty(64, dtype=torch.int32, device="cuda")
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    st = lib.pluq_mod_p(ctypes.c_void_p(z.data_ptr()), 64, 64, 64, p, ctypes.c_void_p(pp.data_ptr()),
                        ctypes.c_void_p(pp.data_ptr()), ctypes.byref(r), ctypes.c_void_p(ws.data_ptr()),
                        16, 0, ctypes.c_void_p(0))
    assert st == -4


# ------------------------------------------- tensor-core exactness bound --

@pytest.mark.parametrize("p,x", [(65521, 32640), (8388593, 4161408), (2147483647, 1065320320),
                                 (251, 128)])
def test_tensor_exact_at_accumulation_bound(p, x):
    """Residues whose balanced digits have the largest magnitudes the split
    produces, so every partial sum of a K-chunk reaches the 2^24 bound; and the
    same with alternating signs (cancellation).  Must stay bit-exact."""
    assert pluq.tensor_limbs(p) in (1, 2, 3, 4)
    for K in (64, 256, 320, 512, 1024, 1600):
        for mixed in (False, True):
            A = np.full((130, K), x, np.uint32)
            B = np.full((K, 70), x, np.uint32)
            if mixed:
                A[:, 1::2] = p - x
                B[::3, :] = p - x
            C = np.zeros((130, 70), np.uint32)
            want = oracle.matmul_sub(C, A, B, p)
            dC = dev(C)
            pluq.pluq_modmm(dC, dev(A), dev(B), p, mm="tensor")
            assert np.array_equal(host(dC), want), (K, mixed)
