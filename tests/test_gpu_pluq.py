"""End-to-end parity of pluq_mod_p (CUDA path through the C-ABI) with the oracle.

Small and medium sizes (several leaves and ragged tails) are compared element
by element with the oracle.  Full-size workloads are checked with the
size-independent certificate of tests/certify.py (reconstruction, LEU
triangularity => rank profile matrix, Algorithm 1's pivot order), plus the
planted rank profile where the input was built with one.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1301_4438_gb300 import pluq, workloads as W
from tests.certify import certify

pytestmark = pytest.mark.gpu
KINDS = ["simt", "tensor"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.uint32)


def run(A, p, kind):
    d = dev(A)
    pp, pq, r = pluq.pluq_mod_p(d, p, mm=kind)
    torch.cuda.synchronize()
    return host(d), pp.cpu().numpy(), pq.cpu().numpy(), r


def assert_same(A, p, kind):
    LU0, pp0, pq0, r0 = oracle.pluq(A, p)
    LU, pp, pq, r = run(A, p, kind)
    assert r == r0
    assert np.array_equal(pp, pp0)
    assert np.array_equal(pq, pq0)
    assert np.array_equal(LU, LU0)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("m,n,r,p", [
    (300, 257, 150, 65521), (257, 300, 257, 65521), (129, 1000, 100, 8388593),
    (1000, 129, 129, 2147483647), (512, 512, 300, 65521), (600, 450, 0, 251),
    (1, 700, 1, 7), (700, 1, 1, 65521), (2, 900, 2, 3), (384, 384, 384, 2147483647),
])
def test_pluq_planted_matches_oracle(kind, m, n, r, p):
    A, pl = W.planted(m, n, r, p, seed=m * 7 + n * 3 + r)
    assert_same(A, p, kind)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("m,n,p", [(520, 390, 65521), (260, 260, 2), (333, 777, 2147483647)])
def test_pluq_dense_and_structured(kind, m, n, p):
    g = np.random.Generator(np.random.PCG64(m + n + p))
    A = g.integers(0, p, (m, n)).astype(np.uint32)
    assert_same(A, p, kind)
    # zero rows / columns and duplicated rows
    B = A.copy()
    B[g.random(m) < 0.25] = 0
    B[:, g.random(n) < 0.25] = 0
    B[m // 2] = B[1]
    assert_same(B, p, kind)


@pytest.mark.parametrize("kind", KINDS)
def test_pluq_empty_and_zero(kind):
    for (m, n) in [(0, 0), (0, 10), (10, 0)]:
        d = torch.zeros((m, n), dtype=torch.int32, device="cuda")
        pp, pq, r = pluq.pluq_mod_p(d, 65521, mm=kind)
        assert r == 0 and pp.numel() == m and pq.numel() == n
    LU, pp, pq, r = run(np.zeros((300, 200), np.uint32), 65521, kind)
    assert r == 0 and not LU.any()
    assert np.array_equal(pp, np.arange(300)) and np.array_equal(pq, np.arange(200))


@pytest.mark.parametrize("kind", KINDS)
def test_config_planted_256(kind):
    cfg = W.CONFIGS["planted_256"]
    A, pl = W.make(cfg)
    assert_same(A, cfg.p, kind)


@pytest.mark.parametrize("kind", KINDS)
def test_config_dense_4096(kind):
    """4096 x 4096 uniform mod 65521 at full size: certificate."""
    cfg = W.CONFIGS["dense_4096"]
    A, _ = W.make(cfg)
    LU, pp, pq, r = run(A, cfg.p, kind)
    assert certify(A, cfg.p, LU, pp, pq, r, exact=False, trials=2) == ""


@pytest.mark.slow
@pytest.mark.parametrize("name", ["planted_16384", "rect_8192x32768"])
def test_config_large_planted(name):
    """Full-size planted workloads: certificate and the planted rank profile."""
    cfg = W.CONFIGS[name]
    At, pl = W.make(cfg, device="cuda")
    A32 = At.to(torch.int32)
    del At
    A = host(A32)
    pp, pq, r = pluq.pluq_mod_p(A32, cfg.p, mm="tensor")
    torch.cuda.synchronize()
    LU = host(A32)
    assert r == cfg.r
    assert certify(A, cfg.p, LU, pp.cpu().numpy(), pq.cpu().numpy(), r, exact=False, trials=1,
                   expected_col_of_row=pl.rank_profile()) == ""


def test_tuning_knobs_do_not_change_results():
    """Leaf size and product threshold change speed only."""
    p = 65521
    A, _ = W.planted(700, 650, 300, p, seed=12)
    old = pluq.pluq_get_tuning()
    outs = []
    try:
        for leaf, small in [(16, 0), (64, 1 << 25), (128, 1 << 40)]:
            pluq.pluq_set_tuning(leaf, small)
            outs.append(run(A, p, "tensor"))
    finally:
        pluq.pluq_set_tuning(*old)
    for o in outs[1:]:
        assert o[3] == outs[0][3]
        assert all(np.array_equal(x, y) for x, y in zip(o[:3], outs[0][:3]))
    LU0, pp0, pq0, r0 = oracle.pluq(A, p)
    assert np.array_equal(outs[0][0], LU0)


@pytest.mark.parametrize("node,ctas", [(2, 1), (1, 1), (0, 1), (1, 2), (2, 2), (1, 4), (2, 4), (1, 8), (2, 8)])
@pytest.mark.parametrize("p", [65521, 8388593, 2147483647])
def test_node_kernel_matches_oracle(p, node, ctas):
    """With the node kernel on, nodes of at most twice (levels 1) or four times
    (levels 2) the leaf size below rank-deficient nodes are computed in one
    thread block, or in a cluster of 2, 4 or 8 (F and G at once, the steps
    between them split); with it off they take the host-driven path.  Either way results stay element-wise equal to
    the oracle (planted profiles of several densities,
    a clustered profile, sparse and low-rank products, rectangular shapes)."""
    g = np.random.Generator(np.random.PCG64(p + 99))
    old, old_ctas = pluq.pluq_get_node_kernel(), pluq.pluq_get_node_cluster()
    pluq.pluq_set_node_kernel(node)
    pluq.pluq_set_node_cluster(ctas)
    try:
        cases = [W.planted(256, 256, 60, p, 1)[0], W.planted(300, 200, 150, p, 2)[0],
                 W.planted(700, 500, 120, p, 3)[0], W.planted(520, 900, 400, p, 4)[0],
                 W.planted(400, 400, 200, p, 5, pivot_rows=W.clustered_rows(400, 200, 100, 6))[0],
                 W.planted(1024, 1000, 990, p, 7)[0],       # nodes whose blocks are nearly full rank
                 (g.integers(0, p, (600, 450)) * (g.random((600, 450)) < 0.01)).astype(np.uint32)]
        X = g.integers(0, p, (640, 40)).astype(np.int64)
        Y = g.integers(0, p, (40, 610)).astype(np.int64)
        cases.append((X.astype(object).dot(Y.astype(object)) % p).astype(np.uint32))
        for A in cases:
            LU0, pp0, pq0, r0 = oracle.pluq(A, p)
            d = torch.from_numpy(A.astype(np.int32)).cuda()
            pp, pq, r = pluq.pluq_mod_p(d, p)
            assert r == r0, A.shape
            assert np.array_equal(pp.cpu().numpy(), pp0), A.shape
            assert np.array_equal(pq.cpu().numpy(), pq0), A.shape
            assert np.array_equal(d.cpu().numpy().astype(np.uint32), LU0), A.shape
    finally:
        pluq.pluq_set_node_kernel(old)
        pluq.pluq_set_node_cluster(old_ctas)
