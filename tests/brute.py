"""Independent brute-force references for tiny inputs (test side only).

Nothing here shares code with the oracle or the CUDA library.  Ranks of every
leading submatrix are computed by a vectorised Gauss-Jordan elimination over a
batch of matrices, with Python's ``pow`` for inverses.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np


@functools.lru_cache(maxsize=None)
def _inverse_table(p: int) -> np.ndarray:
    return np.array([0] + [pow(x, p - 2, p) for x in range(1, p)], dtype=np.int64)


def batch_rank(M: np.ndarray, p: int) -> np.ndarray:
    """Rank over Z/pZ of each matrix of the batch M (B, k, t)."""
    M = (np.asarray(M, dtype=np.int64) % p).copy()
    B, k, t = M.shape
    rank = np.zeros(B, dtype=np.int64)
    if k == 0 or t == 0:
        return rank
    inv = _inverse_table(p) if p < 1 << 16 else None
    idx = np.arange(k)[None, :]
    for c in range(t):
        cand = (M[:, :, c] != 0) & (idx >= rank[:, None])
        has = cand.any(axis=1)
        b = np.nonzero(has)[0]
        if b.size == 0:
            continue
        piv = np.argmax(cand[b], axis=1)
        rb = rank[b]
        top = M[b, rb, :].copy()
        M[b, rb, :] = M[b, piv, :]
        M[b, piv, :] = top
        pv = M[b, rb, c]
        iv = inv[pv] if inv is not None else np.array([pow(int(x), p - 2, p) for x in pv])
        M[b, rb, :] = (M[b, rb, :] * iv[:, None]) % p
        f = M[b, :, c].copy()
        f[np.arange(b.size), rb] = 0
        M[b] = (M[b] - f[:, :, None] * M[b, rb, :][:, None, :]) % p
        rank[b] += 1
    return rank


def rho_table(A: np.ndarray, p: int) -> np.ndarray:
    """rho[b, k, t] = rank of the leading k x t submatrix of A[b]."""
    A = np.asarray(A, dtype=np.int64)
    if A.ndim == 2:
        A = A[None]
    B, m, n = A.shape
    rho = np.zeros((B, m + 1, n + 1), dtype=np.int64)
    for k in range(1, m + 1):
        for t in range(1, n + 1):
            rho[:, k, t] = batch_rank(A[:, :k, :t], p)
    return rho


def rank_profile_matrix(A: np.ndarray, p: int) -> np.ndarray:
    """R[b, k, t] = rho(k+1,t+1) - rho(k,t+1) - rho(k+1,t) + rho(k,t)."""
    rho = rho_table(A, p)
    return rho[:, 1:, 1:] - rho[:, :-1, 1:] - rho[:, 1:, :-1] + rho[:, :-1, :-1]


def all_matrices(m: int, n: int, p: int) -> np.ndarray:
    """Every m x n matrix over Z/pZ, as a (p^(mn), m, n) array."""
    vals = np.array(list(itertools.product(range(p), repeat=m * n)), dtype=np.int64)
    return vals.reshape(-1, m, n)


def matmul_mod(A, B, p: int) -> np.ndarray:
    """Exact product with Python integers (object arrays)."""
    A = np.asarray(A, dtype=object)
    B = np.asarray(B, dtype=object)
    if A.shape[1] == 0:
        return np.zeros((A.shape[0], B.shape[1]), dtype=np.int64)
    return (A.dot(B) % p).astype(np.int64)


def doolittle(A: np.ndarray, p: int):
    """Textbook LU without pivoting (Doolittle's formulas, entry by entry):
    U[i][j] = a_ij - sum_{l<i} L[i][l] U[l][j], L[j][i] = (a_ji - sum_{l<i} L[j][l] U[l][i]) / U[i][i].
    Returns (L, U) or None if a zero pivot appears."""
    A = [[int(x) % p for x in row] for row in np.asarray(A)]
    n = len(A)
    L = [[int(i == j) for j in range(n)] for i in range(n)]
    U = [[0] * n for _ in range(n)]
    for i in range(n):
        for j in range(i, n):
            U[i][j] = (A[i][j] - sum(L[i][l] * U[l][j] for l in range(i))) % p
        if U[i][i] == 0:
            return None
        inv = pow(U[i][i], p - 2, p)
        for j in range(i + 1, n):
            L[j][i] = ((A[j][i] - sum(L[j][l] * U[l][i] for l in range(i))) * inv) % p
    return np.array(L, dtype=np.int64), np.array(U, dtype=np.int64)


def leibniz_det(A, p: int) -> int:
    """Determinant by the Leibniz formula: the sum over all permutations s of
    sgn(s) prod_i A[i][s(i)], sgn(s) = (-1)^(number of inversions)."""
    A = [[int(x) for x in row] for row in np.asarray(A)]
    n = len(A)
    total = 0
    for s in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if s[i] > s[j])
        term = -1 if inv % 2 else 1
        for i in range(n):
            term *= A[i][s[i]]
        total += term
    return total % p


def permutation_sign(s) -> int:
    """+1 or -1: (-1)^(number of inversions of the sequence s)."""
    s = list(s)
    inv = sum(1 for i in range(len(s)) for j in range(i + 1, len(s)) if s[i] > s[j])
    return -1 if inv % 2 else 1


def all_vectors(n: int, p: int) -> np.ndarray:
    """Every vector of (Z/pZ)^n, as a (p^n, n) array."""
    return np.array(list(itertools.product(range(p), repeat=n)), dtype=np.int64).reshape(-1, n)
