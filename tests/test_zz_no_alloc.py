"""The allocation-free tensor-core product, for callers that cannot allocate.

Some users of this library cannot give it a device workspace: they run inside
a CUDA graph capture (no cudaMalloc there), or live in a process whose device
memory belongs to another allocator, or sit in a loop that must not risk an
allocation failure.  pluq_modmm_tensor_noalloc serves them from a fixed device
array built into the library.  This file checks, through the C-ABI, that it
returns exactly what the workspace-taking pluq_modmm returns, on two calls in
a row with different inputs (so leftovers of the first call cannot hide), and
that a product too large for the array is refused without touching C.

The file is named so that pytest collects it after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
def test_noalloc_matches_workspace_entry_point_twice(p):
    g = np.random.Generator(np.random.PCG64(p))
    shapes = [(300, 257, 700), (129, 64, 1100)]          # ragged tiles, several K-chunks
    for call, (M, N, K) in enumerate(shapes):
        A = torch.from_numpy(g.integers(0, p, (M, K)).astype(np.int32)).cuda()
        B = torch.from_numpy(g.integers(0, p, (K, N)).astype(np.int32)).cuda()
        C0 = torch.from_numpy(g.integers(0, p, (M, N)).astype(np.int32)).cuda()
        for assign in (False, True):
            ref = C0.clone()
            pluq.pluq_modmm(ref, A, B, p, assign=assign, mm="tensor")
            got = C0.clone()
            st = _noalloc(got, A, B, p, assign)
            assert st == 0, pluq.status_string(st)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), (call, assign)


def test_noalloc_refuses_products_beyond_its_scratch():
    p = 65521
    M = N = K = 4096                       # limb planes need 128 MiB > the 32 MiB array
    A = torch.zeros((M, K), dtype=torch.int32, device="cuda")
    B = torch.zeros((K, N), dtype=torch.int32, device="cuda")
    C = torch.full((M, N), 7, dtype=torch.int32, device="cuda")
    assert _noalloc(C, A, B, p, False) == ENOMEM
    torch.cuda.synchronize()
    assert bool((C == 7).all())
