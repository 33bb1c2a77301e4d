"""The allocation-free tensor-core product, for callers that cannot allocate.

Some users of this library cannot give it a device workspace: a plug-in living
in a process whose device memory belongs to another allocator (a framework's
caching allocator that has reserved the card), or a loop that must not risk an
allocation failing half way.  pluq_modmm_tensor_noalloc serves them from a
fixed device array built into the library.  This file checks, through the
C-ABI, that it returns exactly the CPU oracle's C - A B (or A B) mod p and what
the workspace-taking pluq_modmm returns, on two calls in a row with different
inputs (so leftovers of the first call cannot hide); that the largest square
product the header documents fits; and that one size past it is refused
without touching C.

The file is named so that pytest collects it after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1301_4438_gb300 import pluq

pytestmark = pytest.mark.gpu

ENOMEM = -4


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(C, A, B, p, assign):
    M, K = A.shape
    N = B.shape[1]
    return pluq.load().pluq_modmm_tensor_noalloc(_vp(C), C.stride(0), _vp(A), A.stride(0), _vp(B),
                                                 B.stride(0), M, N, K, p, int(assign),
                                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _expected(C0, A, B, p, assign):
    """Oracle product: C0 - A B mod p, or A B mod p (C - A B with C = 0, negated)."""
    if not assign:
        return oracle.matmul_sub(C0, A, B, p)
    neg = oracle.matmul_sub(np.zeros_like(C0), A, B, p).astype(np.int64)
    return ((p - neg) % p).astype(np.uint32)


@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
def test_noalloc_matches_oracle_and_workspace_entry_point_twice(p):
    g = np.random.Generator(np.random.PCG64(p))
    shapes = [(300, 257, 700), (129, 64, 1100)]          # ragged tiles, several K-chunks
    for call, (M, N, K) in enumerate(shapes):
        A_h = g.integers(0, p, (M, K)).astype(np.uint32)
        B_h = g.integers(0, p, (K, N)).astype(np.uint32)
        C0_h = g.integers(0, p, (M, N)).astype(np.uint32)
        A = torch.from_numpy(A_h.astype(np.int32)).cuda()
        B = torch.from_numpy(B_h.astype(np.int32)).cuda()
        C0 = torch.from_numpy(C0_h.astype(np.int32)).cuda()
        for assign in (False, True):
            want = _expected(C0_h, A_h, B_h, p, assign)
            ref = C0.clone()
            pluq.pluq_modmm(ref, A, B, p, assign=assign, mm="tensor")
            got = C0.clone()
            st = _noalloc(got, A, B, p, assign)
            assert st == 0, pluq.status_string(st)
            torch.cuda.synchronize()
            got_h = got.cpu().numpy().astype(np.uint32)
            assert np.array_equal(got_h, want), (call, assign)
            assert torch.equal(got, ref), (call, assign)


def test_noalloc_largest_documented_square_fits_and_next_is_refused():
    # the header documents M = N = K = 2000 as the largest square for p < 2^16
    p = 65521
    g = np.random.Generator(np.random.PCG64(2000))
    n = 2000
    A_h = g.integers(0, p, (n, n)).astype(np.uint32)
    B_h = g.integers(0, p, (n, n)).astype(np.uint32)
    C0_h = g.integers(0, p, (n, n)).astype(np.uint32)
    A = torch.from_numpy(A_h.astype(np.int32)).cuda()
    B = torch.from_numpy(B_h.astype(np.int32)).cuda()
    C = torch.from_numpy(C0_h.astype(np.int32)).cuda()
    assert _noalloc(C, A, B, p, False) == 0
    torch.cuda.synchronize()
    got = C.cpu().numpy().astype(np.uint32)
    rows = g.choice(n, 24, replace=False)           # sampled rows against the oracle
    want = oracle.matmul_sub(C0_h[rows], A_h[rows], B_h, p)
    assert np.array_equal(got[rows], want)
    n1 = n + 1
    A1 = torch.zeros((n1, n1), dtype=torch.int32, device="cuda")
    B1 = torch.zeros((n1, n1), dtype=torch.int32, device="cuda")
    C1 = torch.full((n1, n1), 7, dtype=torch.int32, device="cuda")
    assert _noalloc(C1, A1, B1, p, False) == ENOMEM
    torch.cuda.synchronize()
    assert bool((C1 == 7).all())


def test_noalloc_refuses_products_beyond_its_scratch():
    p = 65521
    M = N = K = 4096                       # limb planes need 128 MiB > the 32 MiB array
    A = torch.zeros((M, K), dtype=torch.int32, device="cuda")
    B = torch.zeros((K, N), dtype=torch.int32, device="cuda")
    C = torch.full((M, N), 7, dtype=torch.int32, device="cuda")
    assert _noalloc(C, A, B, p, False) == ENOMEM
    torch.cuda.synchronize()
    assert bool((C == 7).all())
