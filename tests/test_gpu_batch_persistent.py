"""The uneven batch in one persistent launch (pluq_mod_p_batched_persistent)
against the oracle, element by element: every recursion depth the device runs
(a lone base case, then node steps of one to four levels), degenerate shapes,
three primes (both residue forms of the base case), per-matrix errors, and the
call captured in a CUDA graph and replayed on new inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_1301_4438_gb300 import pluq, workloads as W
from tests.certify import certify

pytestmark = pytest.mark.gpu

ERANGE = -3


def _matrix(m, n, kind, p, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    if m == 0 or n == 0 or kind == "zero":
        return np.zeros((m, n), dtype=np.uint32)
    if kind == "uniform":
        return g.integers(0, p, (m, n)).astype(np.uint32)
    if kind == "sparse":   # a few nonzero entries far from the origin
        A = np.zeros((m, n), dtype=np.uint32)
        for _ in range(3):
            A[g.integers(m // 2, m), g.integers(n // 2, n)] = g.integers(1, p)
        return A
    r = {"planted": min(m, n) // 2, "low": min(8, min(m, n))}[kind]
    A, _ = W.planted(m, n, r, p, seed=seed)
    return A


SHAPES = [  # (m, n, kind): sides up to 128 (base case), 256, 512, 1024, 2048 (four levels)
    (1, 1, "uniform"), (0, 7, "zero"), (7, 0, "zero"), (70, 130, "planted"),
    (200, 64, "uniform"), (129, 129, "planted"), (300, 257, "uniform"), (64, 700, "planted"),
    (33, 1, "uniform"), (1, 40, "sparse"), (257, 129, "planted"), (128, 128, "uniform"),
    (1, 1500, "sparse"), (1500, 1, "sparse"), (600, 900, "planted"), (1100, 600, "planted"),
    (520, 1030, "low"), (700, 700, "zero"), (2048, 40, "uniform"), (40, 2048, "planted"),
    (1030, 1030, "sparse"),
]
SHAPES_WIDE_P = [s for s in SHAPES if s[0] * s[1] <= 700 * 700]


def _check_batch(shapes, p, ctas, seed0):
    hosts = [_matrix(m, n, kind, p, seed0 + k) for k, (m, n, kind) in enumerate(shapes)]
    mats = [torch.from_numpy(A.astype(np.int32)).cuda() for A in hosts]
    pps, pqs, ranks = pluq.pluq_mod_p_batched_persistent(mats, p, ctas=ctas)
    torch.cuda.synchronize()
    for (m, n, kind), A, d, pp, pq, r in zip(shapes, hosts, mats, pps, pqs, ranks):
        LU0, pp0, pq0, r0 = oracle.pluq(A, p)
        assert r == r0, (m, n, kind, r, r0)
        assert np.array_equal(pp.cpu().numpy(), pp0), (m, n, kind)
        assert np.array_equal(pq.cpu().numpy(), pq0), (m, n, kind)
        assert np.array_equal(d.cpu().numpy().astype(np.uint32), LU0), (m, n, kind)


def test_persistent_batch_matches_oracle_p65521():
    # five thread blocks for 21 matrices: every block takes several
    _check_batch(SHAPES, 65521, ctas=5, seed0=500)


@pytest.mark.parametrize("p", [8388593, 2147483647])
def test_persistent_batch_matches_oracle_wide_primes(p):
    _check_batch(SHAPES_WIDE_P, p, ctas=0, seed0=700)


def test_persistent_batch_results_do_not_depend_on_ctas():
    p = 65521
    shapes = [(300, 400, "planted"), (129, 700, "planted"), (90, 90, "uniform"), (513, 257, "low")]
    hosts = [_matrix(m, n, kind, p, 900 + k) for k, (m, n, kind) in enumerate(shapes)]
    outs = []
    for ctas in (1, 3, 0):
        mats = [torch.from_numpy(A.astype(np.int32)).cuda() for A in hosts]
        pps, pqs, ranks = pluq.pluq_mod_p_batched_persistent(mats, p, ctas=ctas)
        torch.cuda.synchronize()
        outs.append(([d.cpu() for d in mats], [x.cpu() for x in pps], [x.cpu() for x in pqs], ranks))
    for o in outs[1:]:
        assert o[3] == outs[0][3]
        for a, b in zip(o[0] + o[1] + o[2], outs[0][0] + outs[0][1] + outs[0][2]):
            assert torch.equal(a, b)


def test_persistent_batch_reports_errors_per_matrix():
    p = 65521
    good = [_matrix(100, 100, "planted", p, 11), _matrix(50, 60, "uniform", p, 12)]
    bad = _matrix(300, 200, "uniform", p, 13)
    bad[123, 45] = p   # not reduced mod p
    hosts = [good[0], bad, good[1]]
    mats = [torch.from_numpy(A.astype(np.int32)).cuda() for A in hosts]
    pps, pqs, ranks = pluq.pluq_mod_p_batched_persistent(mats, p, ctas=2)
    torch.cuda.synchronize()
    assert ranks[1] == ERANGE
    assert np.array_equal(mats[1].cpu().numpy().astype(np.uint32), bad)   # untouched
    for i in (0, 2):
        LU0, pp0, pq0, r0 = oracle.pluq(hosts[i], p)
        assert ranks[i] == r0
        assert np.array_equal(mats[i].cpu().numpy().astype(np.uint32), LU0)
        assert np.array_equal(pps[i].cpu().numpy(), pp0) and np.array_equal(pqs[i].cpu().numpy(), pq0)
    # host-checked arguments
    with pytest.raises(pluq.PluqError):
        pluq.pluq_mod_p_batched_persistent([torch.zeros(2049, 3, dtype=torch.int32, device="cuda")], p)
    with pytest.raises(pluq.PluqError):
        pluq.pluq_mod_p_batched_persistent([torch.zeros(3, 3, dtype=torch.int32, device="cuda")], 65535)


def test_persistent_batch_graph_capture_and_replay():
    """Warm up once, capture the call (one memset, one launch) in a CUDA
    graph, then replay it twice on new contents of the same matrices."""
    p = 65521
    shapes = [(600, 500, "planted"), (257, 300, "uniform"), (64, 64, "planted"), (1, 90, "sparse"),
              (400, 130, "low"), (129, 1000, "planted")]
    mats = [torch.zeros(m, n, dtype=torch.int32, device="cuda") for m, n, _ in shapes]
    b = pluq.PersistentBatch(mats, p, ctas=torch.cuda.get_device_properties(0).multi_processor_count)

    def load_inputs(seed0):
        hosts = [_matrix(m, n, kind, p, seed0 + k) for k, (m, n, kind) in enumerate(shapes)]
        for d, A in zip(mats, hosts):
            d.copy_(torch.from_numpy(A.astype(np.int32)))
        return hosts

    def check(hosts):
        pps, pqs = b.perms()
        ranks = b.ranks()
        for A, d, pp, pq, r in zip(hosts, mats, pps, pqs, ranks):
            LU0, pp0, pq0, r0 = oracle.pluq(A, p)
            assert r == r0
            assert np.array_equal(pp.cpu().numpy(), pp0) and np.array_equal(pq.cpu().numpy(), pq0)
            assert np.array_equal(d.cpu().numpy().astype(np.uint32), LU0)

    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        hosts = load_inputs(1000)
        b.run()
    torch.cuda.synchronize()
    check(hosts)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()
    for seed0 in (2000, 3000):
        hosts = load_inputs(seed0)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        check(hosts)


@pytest.mark.slow
def test_persistent_batch_2000_planted():
    """The 2000-matrix uneven batch (m, n uniform in [64, 2048], rank
    floor(min/2), planted profiles, p = 65521) in one launch: every rank equals
    the planted one; a sample gets the full certificate with the planted rank
    profile matrix."""
    bt = W.batch_2000()
    mats, plants = [], []
    for m, n, r, s in zip(bt.ms, bt.ns, bt.rs, bt.seeds):
        A, rows, cols = W.planted_device(m, n, r, bt.p, s, "cuda")
        mats.append(A)
        plants.append((rows, cols))
    originals = {i: mats[i].cpu().numpy().astype(np.uint32) for i in range(0, 2000, 125)}
    pps, pqs, ranks = pluq.pluq_mod_p_batched_persistent(mats, bt.p)
    torch.cuda.synchronize()
    assert ranks == bt.rs
    for i, A in originals.items():
        col = np.full(bt.ms[i], -1, dtype=np.int32)
        col[plants[i][0]] = plants[i][1]
        assert certify(A, bt.p, mats[i].cpu().numpy().astype(np.uint32), pps[i].cpu().numpy(),
                       pqs[i].cpu().numpy(), ranks[i], exact=False, expected_col_of_row=col) == ""
