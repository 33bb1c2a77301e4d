"""PLE and CUP decompositions (Sec. 1) built on the GPU from the packed PLUQ,
element by element against the oracle's definitions (elimination with the
pivots of the rank profile matrix taken in column / row order), on inputs
whose pivots form descents (so an elimination is needed besides
permutations), dense and rank-deficient, square and rectangular, every limb
count, both product forms, r = 0 and empty shapes; and at a size where the
triangle goes through the tensor-core products."""
import numpy as np
import pytest
import torch

import oracle
from paper_1301_4438_gb300 import pluq, workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.uint32)


def _cases(p):
    g = np.random.Generator(np.random.PCG64(p + 404))
    q = 9
    L0 = np.tril(g.integers(0, p, (q, q)), -1) + np.eye(q, dtype=np.int64)
    U0 = np.triu(g.integers(0, p, (q, q)), 1) + np.eye(q, dtype=np.int64)
    R = np.zeros((q, q), dtype=np.int64)
    R[np.arange(q), q - 1 - np.arange(q)] = 1                  # every pair a descent
    anti = (L0.astype(object).dot(R).dot(U0.astype(object)) % p).astype(np.uint32)
    return [
        np.array([[0, 3], [5, 2]], dtype=np.uint32) % p,
        anti,
        W.planted(60, 45, 30, p, 1)[0],
        W.planted(45, 70, 45, p, 2)[0],
        W.planted(300, 260, 200, p, 3)[0],
        g.integers(0, p, (130, 97)).astype(np.uint32),
        np.zeros((20, 30), dtype=np.uint32),
    ]


@pytest.mark.parametrize("mm", ["simt", "tensor"])
@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
def test_ple_cup_match_oracle(p, mm):
    for A in _cases(p):
        d = dev(A)
        pp, pq, r = pluq.pluq_mod_p(d, p, mm=mm)
        perm, L, E = pluq.pluq_ple(d, pp, pq, r, p, mm=mm)
        pp0, L0, E0, r0 = oracle.ple(A, p)
        assert r == r0, A.shape
        assert np.array_equal(perm.cpu().numpy(), pp0), A.shape
        assert np.array_equal(host(L), L0) and np.array_equal(host(E), E0), A.shape
        perm, C, U = pluq.pluq_cup(d, pp, pq, r, p, mm=mm)
        pq0, C0, U0, r0 = oracle.cup(A, p)
        assert np.array_equal(perm.cpu().numpy(), pq0), A.shape
        assert np.array_equal(host(C), C0) and np.array_equal(host(U), U0), A.shape


def test_ple_cup_empty_shapes():
    p = 65521
    for (m, n) in [(0, 5), (5, 0), (0, 0)]:
        A = np.zeros((m, n), dtype=np.uint32)
        d = torch.zeros((max(m, 1), max(n, 1)), dtype=torch.int32, device="cuda")[:m, :n]
        pp, pq, r = pluq.pluq_mod_p(d, p)
        perm, L, E = pluq.pluq_ple(d, pp, pq, r, p)
        assert r == 0 and perm.cpu().tolist() == list(range(m))
        perm, C, U = pluq.pluq_cup(d, pp, pq, r, p)
        assert perm.cpu().tolist() == list(range(n))


def test_ple_cup_large_planted_tensor():
    """1500 x 1200 of planted rank 900 mod 2^31 - 1: the 900 x 900 triangle's
    factorisation, solve and product run on the tensor-core path."""
    p = 2147483647
    A = W.planted(1500, 1200, 900, p, 8)[0]
    d = dev(A)
    pp, pq, r = pluq.pluq_mod_p(d, p, mm="tensor")
    perm, L, E = pluq.pluq_ple(d, pp, pq, r, p, mm="tensor")
    pp0, L0, E0, r0 = oracle.ple(A, p)
    assert r == r0 == 900
    assert np.array_equal(perm.cpu().numpy(), pp0)
    assert np.array_equal(host(L), L0) and np.array_equal(host(E), E0)
