"""Size-independent certificate that a PLUQ result is the canonical one.

For a result (LU packed, perm_p, perm_q, r) of an m x n matrix A over Z/pZ:

1. perm_p, perm_q are permutations; U has a nonzero diagonal; the trailing
   (m-r) x (n-r) block is zero.
2. A = P [L;M] [U V] Q, checked exactly (small) or by Freivalds' test with
   random vectors (error probability <= p^-trials).
3. The LEU triangularity of Theorem 1 (Sec. 3) with Y = I and Z = I:
   P [L 0; M I] P^T is unit lower and Q^T [U V; 0 I] Q is upper triangular,
   and the non-pivot parts of perm_p / perm_q increase (so any unit lower Y and
   any upper Z keep the property).  Then A = Lbar . E . Ubar with
   E = P diag(I_r, 0) Q, and since multiplying by invertible lower (left) and
   upper (right) triangular matrices keeps the rank of every leading
   submatrix (Lemma 1, Sec. 4), E is the rank profile matrix of A.
4. The pivots appear in the order Algorithm 1 finds them (the oracle's
   canonical order of E's ones).

Given P and Q the packed factors are unique, so a result that passes all four
is, entry for entry, the oracle's.  This module is test infrastructure.
"""
from __future__ import annotations

import numpy as np

import oracle


def _mulvec_mod(M: np.ndarray, x: np.ndarray, p: int) -> np.ndarray:
    """(M @ x) mod p exactly for uint32 M (< 2^31) and x in [0, p)."""
    M64 = M.astype(np.int64, copy=False)
    lo = (x & 0xFFFF).astype(np.int64)
    hi = (x >> 16).astype(np.int64)
    out = np.zeros(M.shape[0], dtype=np.int64)
    step = 1 << 15
    for s in range(0, M.shape[1], step):
        e = min(M.shape[1], s + step)
        blk = M64[:, s:e]
        out = (out + (blk @ lo[s:e]) % p + ((blk @ hi[s:e]) % p) * (65536 % p)) % p
    return out


def reconstruct_freivalds(A, p, LU, perm_p, perm_q, r, trials=2, seed=0) -> bool:
    m, n = A.shape
    g = np.random.Generator(np.random.PCG64(seed))
    for _ in range(trials):
        x = g.integers(0, p, size=n, dtype=np.int64)
        # left: (P^T A Q^T) x = A z restricted to rows perm_p, z[perm_q[j]] = x[j]
        z = np.zeros(n, dtype=np.int64)
        z[perm_q] = x
        left = _mulvec_mod(A, z, p)[perm_p]
        # right: [L;M] ([U V] x)
        Uv = LU[:r, :].astype(np.int64)
        Uv = np.triu(Uv)                       # rows < r, upper part incl. V
        y = _mulvec_mod(Uv, x, p) if r else np.zeros(0, dtype=np.int64)
        Lm = np.tril(LU[:, :r].astype(np.int64), -1)
        right = _mulvec_mod(Lm, y, p) if r else np.zeros(m, dtype=np.int64)
        right[:r] = (right[:r] + y) % p         # unit diagonal of L
        if not np.array_equal(left % p, right % p):
            return False
    return True


def certify(A: np.ndarray, p: int, LU: np.ndarray, perm_p: np.ndarray,
            perm_q: np.ndarray, r: int, exact: bool = None, trials: int = 2,
            expected_col_of_row: np.ndarray = None) -> str:
    """'' if the result is the canonical PLUQ of A, else a reason."""
    A = np.asarray(A, dtype=np.uint32)
    LU = np.asarray(LU, dtype=np.uint32)
    perm_p = np.asarray(perm_p, dtype=np.int64)
    perm_q = np.asarray(perm_q, dtype=np.int64)
    m, n = A.shape
    if LU.shape != (m, n):
        return "shape"
    if not (0 <= r <= min(m, n)):
        return "rank out of range"
    if not np.array_equal(np.sort(perm_p), np.arange(m)):
        return "perm_p is not a permutation"
    if not np.array_equal(np.sort(perm_q), np.arange(n)):
        return "perm_q is not a permutation"
    if r and np.any(np.diagonal(LU)[:r] == 0):
        return "zero on U's diagonal"
    if np.any(LU[r:, r:] != 0):
        return "trailing block not zero"
    if np.any(LU >= p):
        return "entry >= p"
    # 3. LEU triangularity
    if r:
        Lpart = LU[:, :r]
        a, b = np.nonzero(np.tril(Lpart != 0, -1))
        if a.size and np.any(perm_p[a] <= perm_p[b]):
            return "P [L 0; M I] P^T not lower triangular"
        Upart = LU[:r, :]
        a, b = np.nonzero(np.triu(Upart != 0, 1))
        if a.size and np.any(perm_q[a] >= perm_q[b]):
            return "Q^T [U V; 0 I] Q not upper triangular"
    if np.any(np.diff(perm_p[r:]) <= 0) or np.any(np.diff(perm_q[r:]) <= 0):
        return "non-pivot rows/columns not increasing"
    # 4. canonical order of E's ones
    col_of_row = np.full(m, -1, dtype=np.int32)
    col_of_row[perm_p[:r]] = perm_q[:r]
    if expected_col_of_row is not None and not np.array_equal(col_of_row, expected_col_of_row):
        return "rank profile matrix differs from the expected one"
    pr, pc = oracle.canonical_order(m, n, col_of_row)
    if not (np.array_equal(pr, perm_p[:r]) and np.array_equal(pc, perm_q[:r])):
        return "pivot order differs from Algorithm 1's"
    # 2. reconstruction
    if exact is None:
        exact = m * n * max(r, 1) <= 1 << 24
    if exact:
        if oracle.check_pluq(A, p, LU, perm_p.astype(np.int32), perm_q.astype(np.int32), r) != 0:
            return "A != P [L;M][U V] Q"
    elif not reconstruct_freivalds(A, p, LU, perm_p, perm_q, r, trials=trials):
        return "Freivalds: A != P [L;M][U V] Q"
    return ""
