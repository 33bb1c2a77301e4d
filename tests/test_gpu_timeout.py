"""Failure detection on the GPU without a fault.

Every wait of a kernel on other warps is bounded (the tensor-core product's
pipeline barriers, the base case's step barrier).  pluq_set_wait_limit(0)
makes each such wait give up before its first try, so the give-up path runs
for real: the kernel records the error, winds down (its issued copies and MMAs
finish under their full bound, tensor memory is freed) and returns, and the
host reads PLUQ_ETIMEOUT.  Each test then restores the built-in bound and
checks that the next call is bit-exact against the oracle, i.e. that the
context is still usable.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1301_4438_gb300 import pluq, workloads as W

pytestmark = pytest.mark.gpu

ETIMEOUT = -6


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.uint32)


@pytest.fixture
def zero_wait_limit():
    pluq.pluq_device_status()              # no record left by earlier tests
    pluq.pluq_set_wait_limit(0)
    yield
    pluq.pluq_set_wait_limit(-1)
    pluq.pluq_device_status()


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_tensor_product_gives_up_then_recovers(zero_wait_limit, p):
    g = np.random.Generator(np.random.PCG64(p + 7))
    A = g.integers(0, p, (300, 400)).astype(np.uint32)
    B = g.integers(0, p, (400, 260)).astype(np.uint32)
    C0 = g.integers(0, p, (300, 260)).astype(np.uint32)
    C = dev(C0)
    pluq.pluq_modmm(C, dev(A), dev(B), p, mm="tensor")
    assert pluq.pluq_device_status() == ETIMEOUT
    assert pluq.pluq_device_status() == 0             # the record is cleared
    pluq.pluq_set_wait_limit(-1)
    C = dev(C0)
    pluq.pluq_modmm(C, dev(A), dev(B), p, mm="tensor")
    assert pluq.pluq_device_status() == 0
    assert np.array_equal(host(C), oracle.matmul_sub(C0, A, B, p))


def test_leaf_gives_up_then_recovers(zero_wait_limit):
    p = 8388593
    # a non-generic rank profile, so the base case reaches its step barrier
    A, _ = W.planted(120, 100, 40, p, seed=77)
    d = dev(A)
    _, _, r = pluq.pluq_leaf(d, p)
    assert r == -1
    assert pluq.pluq_device_status() == ETIMEOUT
    pluq.pluq_set_wait_limit(-1)
    d = dev(A)
    pp, pq, r = pluq.pluq_leaf(d, p)
    LU0, pp0, pq0, r0 = oracle.pluq(A, p)
    assert pluq.pluq_device_status() == 0
    assert r == r0 == 40
    assert np.array_equal(pp.cpu().numpy(), pp0) and np.array_equal(pq.cpu().numpy(), pq0)
    assert np.array_equal(host(d), LU0)


def test_decomposition_reports_timeout_then_recovers(zero_wait_limit):
    p = 65521
    A, _ = W.planted(300, 300, 100, p, seed=78)
    with pytest.raises(pluq.PluqError) as e:
        pluq.pluq_mod_p(dev(A), p)
    assert e.value.status == ETIMEOUT
    pluq.pluq_set_wait_limit(-1)
    d = dev(A)
    pp, pq, r = pluq.pluq_mod_p(d, p)
    LU0, pp0, pq0, r0 = oracle.pluq(A, p)
    assert r == r0 == 100
    assert np.array_equal(pp.cpu().numpy(), pp0) and np.array_equal(pq.cpu().numpy(), pq0)
    assert np.array_equal(host(d), LU0)
