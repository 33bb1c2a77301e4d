"""Parity of the uses of the decomposition (Sec. 1: determinant, nullspaces,
linear systems) computed by the CUDA path through the C-ABI.

Small and medium sizes (several tiles, ragged tails, every limb count) are
compared element by element with the oracle, which computes them from the
textbook definitions (Gauss-Jordan RREF, elimination with row exchanges) and
never from a PLUQ.  At the 4096 x 4096 size of the dense workload the results
are checked by properties that hold at any size: the closed-form determinant
of a planted L0 Pi U0, A N = 0 by Freivalds' test with N the identity outside
the planted column profile, and exact recovery of a planted solution.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1301_4438_gb300 import pluq, workloads as W
from tests import brute
from tests.certify import _mulvec_mod

pytestmark = pytest.mark.gpu
KINDS = ["simt", "tensor"]

CASES = [
    (300, 257, 150, 65521), (257, 300, 257, 65521), (129, 400, 100, 8388593),
    (400, 129, 129, 2147483647), (512, 512, 300, 65521), (200, 150, 0, 251),
    (1, 300, 1, 7), (300, 1, 1, 65521), (384, 384, 384, 2147483647), (700, 650, 333, 3),
]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.uint32)


def factor(A, p, kind):
    d = dev(A)
    pp, pq, r = pluq.pluq_mod_p(d, p, mm=kind)
    return d, pp, pq, r


def u32(t):
    return int(t.item()) & 0xFFFFFFFF


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("m,n,r,p", CASES)
def test_right_nullspace_matches_oracle(kind, m, n, r, p):
    A, _ = W.planted(m, n, r, p, seed=m + 3 * n + r)
    d, pp, pq, rr = factor(A, p, kind)
    assert rr == r
    N = pluq.pluq_right_nullspace(d, pq, rr, p, mm=kind)
    torch.cuda.synchronize()
    assert np.array_equal(host(N), oracle.right_nullspace(A, p))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("m,n,r,p", CASES)
def test_left_nullspace_matches_oracle(kind, m, n, r, p):
    A, _ = W.planted(m, n, r, p, seed=2 * m + n + r)
    d, pp, pq, rr = factor(A, p, kind)
    K = pluq.pluq_left_nullspace(d, pp, rr, p, mm=kind)
    torch.cuda.synchronize()
    assert np.array_equal(host(K), oracle.left_nullspace(A, p))


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("m,n,r,p", CASES)
def test_solve_matches_oracle(kind, m, n, r, p):
    A, _ = W.planted(m, n, r, p, seed=m + n + 5 * r)
    g = np.random.Generator(np.random.PCG64(m * n + r))
    k = 7
    Xp = g.integers(0, p, (n, k)).astype(np.uint32)
    B = brute.matmul_mod(A, Xp, p).astype(np.uint32)
    B[:, 5:] = g.integers(0, p, (m, 2)).astype(np.uint32)   # solvable only if r = m
    X0, ok = oracle.solve(A, B, p)
    d, pp, pq, rr = factor(A, p, kind)
    X, flag = pluq.pluq_solve(d, pp, pq, rr, dev(B), p, mm=kind)
    torch.cuda.synchronize()
    assert u32(flag) == (0 if ok.all() else 1)
    X = host(X)
    assert np.array_equal(X[:, ok], X0[:, ok])
    # all right-hand sides solvable: the flag is clear and every column matches
    X, flag = pluq.pluq_solve(d, pp, pq, rr, dev(np.ascontiguousarray(B[:, :5])), p, mm=kind)
    torch.cuda.synchronize()
    assert u32(flag) == 0
    assert np.array_equal(host(X), X0[:, :5])


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,p", [(1, 65521), (2, 3), (37, 2147483647), (128, 65521),
                                 (129, 8388593), (300, 2), (513, 65521)])
def test_determinant_matches_oracle(kind, n, p):
    g = np.random.Generator(np.random.PCG64(n + p))
    mats = [g.integers(0, p, (n, n)).astype(np.uint32),
            W.planted(n, n, n, p, seed=n)[0],
            W.planted(n, n, max(n - 1, 0), p, seed=n + 1)[0]]
    for A in mats:
        d, pp, pq, r = factor(A, p, kind)
        det = pluq.pluq_determinant(d, pp, pq, r, p)
        torch.cuda.synchronize()
        assert u32(det) == oracle.determinant(A, p)


def test_degenerate_shapes():
    p = 65521
    for m, n in [(0, 0), (0, 5), (5, 0), (3, 3)]:
        A = np.zeros((m, n), dtype=np.uint32)
        d, pp, pq, r = factor(A, p, "tensor")
        assert r == 0
        N = pluq.pluq_right_nullspace(d, pq, r, p)
        K = pluq.pluq_left_nullspace(d, pp, r, p)
        X, flag = pluq.pluq_solve(d, pp, pq, r, dev(np.zeros((m, 2), dtype=np.uint32)), p)
        torch.cuda.synchronize()
        assert np.array_equal(host(N), np.eye(n, dtype=np.uint32))
        assert np.array_equal(host(K), np.eye(m, dtype=np.uint32))
        assert u32(flag) == 0 and not np.any(host(X))
        if m == n:
            det = pluq.pluq_determinant(d, pp, pq, r, p)
            torch.cuda.synchronize()
            assert u32(det) == (1 if n == 0 else 0)
    # no right-hand sides; full rank leaves empty nullspaces
    A, _ = W.planted(64, 64, 64, p, seed=1)
    d, pp, pq, r = factor(A, p, "tensor")
    X, flag = pluq.pluq_solve(d, pp, pq, r, dev(np.zeros((64, 0), dtype=np.uint32)), p)
    assert pluq.pluq_right_nullspace(d, pq, r, p).shape == (64, 0)
    assert pluq.pluq_left_nullspace(d, pp, r, p).shape == (0, 64)
    torch.cuda.synchronize()
    assert u32(flag) == 0 and X.shape == (64, 0)


def test_uses_argument_errors():
    p = 65521
    lib = pluq.load()
    d = dev(np.zeros((4, 4), dtype=np.uint32))
    pp = torch.arange(4, dtype=torch.int32, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    a, q, f, w = d.data_ptr(), pp.data_ptr(), flag.data_ptr(), ws.data_ptr()
    # r > n
    assert lib.pluq_right_nullspace(a, 4, 4, 4, 5, q, p, a, 4, 0, w, 1 << 20, None) == -1
    # modulus not prime
    assert lib.pluq_left_nullspace(a, 4, 4, 4, 0, q, 65535, a, 4, 0, w, 1 << 20, None) == -2
    # no workspace
    assert lib.pluq_solve(a, 4, 4, 4, 0, q, q, p, a, 4, 4, a, 4, f, 0, None, 0, None) == -4
    # lda < n
    assert lib.pluq_determinant(a, 4, 3, 4, q, q, p, f, w, 1 << 20, None) == -1
    # ldn < n - r
    assert lib.pluq_right_nullspace(a, 4, 4, 4, 0, q, p, a, 3, 0, w, 1 << 20, None) == -1
    torch.cuda.synchronize()


def _planted_device(m, n, r, p, seed):
    pl = W.planted_factors(m, n, r, p, seed)
    A = W.planted_matrix(pl, device="cuda").to(torch.int32).contiguous()
    return A, pl


@pytest.mark.parametrize("kind", KINDS)
def test_determinant_4096_closed_form(kind):
    """A = L0 Pi U0 with unit triangular L0, U0: det A = sgn(Pi)."""
    p = 65521
    A, pl = _planted_device(4096, 4096, 4096, p, seed=41)
    cols = [int(c) for c in pl.cols]
    seen, cycles = [False] * 4096, 0
    for i in range(4096):
        if not seen[i]:
            cycles += 1
            j = i
            while not seen[j]:
                seen[j] = True
                j = cols[j]
    sgn = 1 if (4096 - cycles) % 2 == 0 else p - 1
    pp, pq, r = pluq.pluq_mod_p(A, p, mm=kind)
    det = pluq.pluq_determinant(A, pp, pq, r, p)
    torch.cuda.synchronize()
    assert r == 4096 and u32(det) == sgn
    B, _ = _planted_device(4096, 4096, 4095, p, seed=42)
    pp, pq, r = pluq.pluq_mod_p(B, p, mm=kind)
    det = pluq.pluq_determinant(B, pp, pq, r, p)
    torch.cuda.synchronize()
    assert r == 4095 and u32(det) == 0


def test_nullspace_4096_planted():
    p = 65521
    A, pl = _planted_device(4096, 4096, 2048, p, seed=43)
    Ah = host(A)
    pp, pq, r = pluq.pluq_mod_p(A, p)          # A now holds the packed factors
    assert r == 2048
    N = host(pluq.pluq_right_nullspace(A, pq, r, p))
    K = host(pluq.pluq_left_nullspace(A, pp, r, p))
    free = np.setdiff1d(np.arange(4096), pl.cols)
    assert np.array_equal(N[free, :], np.eye(2048, dtype=np.uint32))
    free_rows = np.setdiff1d(np.arange(4096), pl.rows)
    assert np.array_equal(K[:, free_rows], np.eye(2048, dtype=np.uint32))
    g = np.random.Generator(np.random.PCG64(7))
    Kt = np.ascontiguousarray(K.T)
    At = np.ascontiguousarray(Ah.T)
    for _ in range(2):
        x = g.integers(0, p, 2048, dtype=np.int64)
        assert not np.any(_mulvec_mod(Ah, _mulvec_mod(N, x, p), p))     # A (N x) = 0
        assert not np.any(_mulvec_mod(At, _mulvec_mod(Kt, x, p), p))    # (x^T K A)^T = 0


def test_solve_4096_dense_recovers_planted_solution():
    p = 65521
    g = np.random.Generator(np.random.PCG64(4096))
    Ah = g.integers(0, p, (4096, 4096)).astype(np.uint32)
    X0 = g.integers(0, p, (4096, 8)).astype(np.int64)
    B = np.stack([_mulvec_mod(Ah, X0[:, c], p) for c in range(8)], axis=1).astype(np.uint32)
    LU = dev(Ah)
    pp, pq, r = pluq.pluq_mod_p(LU, p)
    if r < 4096:
        pytest.skip("the random matrix is singular")
    X, flag = pluq.pluq_solve(LU, pp, pq, r, dev(B), p)
    torch.cuda.synchronize()
    assert u32(flag) == 0
    assert np.array_equal(host(X).astype(np.int64), X0)
