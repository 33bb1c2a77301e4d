"""Batched decompositions of uneven sizes (pluq_mod_p_batched) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1301_4438_gb300 import pluq, workloads as W
from tests.certify import certify

pytestmark = pytest.mark.gpu


def test_batch_small_uneven_matches_oracle():
    p = 65521
    g = np.random.Generator(np.random.PCG64(4))
    shapes = [(1, 1), (0, 7), (7, 0), (70, 130), (200, 64), (129, 129), (300, 257), (64, 700),
              (33, 1), (1, 40), (257, 129), (128, 128)]
    hosts, mats = [], []
    for k, (m, n) in enumerate(shapes):
        if m and n and k % 2:
            A, _ = W.planted(m, n, min(m, n) // 2, p, seed=100 + k)
        else:
            A = g.integers(0, p, (m, n)).astype(np.uint32)
        hosts.append(A)
        mats.append(torch.from_numpy(A.astype(np.int32)).cuda())
    pps, pqs, ranks = pluq.pluq_mod_p_batched(mats, p, workers=4)
    torch.cuda.synchronize()
    for A, d, pp, pq, r in zip(hosts, mats, pps, pqs, ranks):
        LU0, pp0, pq0, r0 = oracle.pluq(A, p)
        assert r == r0
        assert np.array_equal(pp.cpu().numpy(), pp0) and np.array_equal(pq.cpu().numpy(), pq0)
        assert np.array_equal(d.cpu().numpy().astype(np.uint32), LU0)


@pytest.mark.slow
def test_batch_2000_planted():
    """2000 matrices, m, n uniform in [64, 2048], rank floor(min/2), planted
    profiles, p = 65521: every rank equals the planted one; a sample gets the
    full certificate with the planted rank profile matrix."""
    bt = W.batch_2000()
    mats, plants = [], []
    for m, n, r, s in zip(bt.ms, bt.ns, bt.rs, bt.seeds):
        A, rows, cols = W.planted_device(m, n, r, bt.p, s, "cuda")
        mats.append(A)
        plants.append((rows, cols))
    originals = {i: mats[i].cpu().numpy().astype(np.uint32) for i in range(0, 2000, 125)}
    pps, pqs, ranks = pluq.pluq_mod_p_batched(mats, bt.p, workers=16)
    torch.cuda.synchronize()
    assert ranks == bt.rs
    for i, A in originals.items():
        col = np.full(bt.ms[i], -1, dtype=np.int32)
        col[plants[i][0]] = plants[i][1]
        assert certify(A, bt.p, mats[i].cpu().numpy().astype(np.uint32), pps[i].cpu().numpy(),
                       pqs[i].cpu().numpy(), ranks[i], exact=False, expected_col_of_row=col) == ""
