"""CPU oracle for the rank-profile-revealing PLUQ decomposition over Z/pZ.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may load it.  It shares no code with the CUDA
library in ``paper_1301_4438_gb300`` and neither imports the other.

The arithmetic lives in ``pluq_oracle.c`` (plain C, exact, compiled with gcc);
this module only compiles it on demand and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pluq_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_is_prime.argtypes = [ctypes.c_uint32]
            lib.oracle_is_prime.restype = ctypes.c_int
            lib.oracle_rank_profile.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_uint32, _i32p]
            lib.oracle_rank_profile.restype = ctypes.c_int64
            lib.oracle_canonical_order.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p,
                                                   _i32p, _i32p, _i64p]
            lib.oracle_canonical_order.restype = ctypes.c_int
            lib.oracle_pluq.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_uint32, _u32p, ctypes.c_int64, _i32p, _i32p,
                                        _i64p]
            lib.oracle_pluq.restype = ctypes.c_int
            lib.oracle_pluq_alg1.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_uint32, _i32p, _i32p,
                                             _i64p]
            lib.oracle_pluq_alg1.restype = ctypes.c_int
            lib.oracle_matmul_sub.argtypes = [_u32p, ctypes.c_int64, _u32p, ctypes.c_int64,
                                              _u32p, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32]
            lib.oracle_matmul_sub.restype = None
            lib.oracle_trsm_left_lower_unit.argtypes = [_u32p, ctypes.c_int64, _u32p,
                                                        ctypes.c_int64, ctypes.c_int64,
                                                        ctypes.c_int64, ctypes.c_uint32]
            lib.oracle_trsm_left_lower_unit.restype = None
            lib.oracle_trsm_right_upper.argtypes = [_u32p, ctypes.c_int64, _u32p,
                                                    ctypes.c_int64, ctypes.c_int64,
                                                    ctypes.c_int64, ctypes.c_uint32]
            lib.oracle_trsm_right_upper.restype = None
            lib.oracle_check_pluq.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int64, ctypes.c_uint32, _u32p,
                                              ctypes.c_int64, _i32p, _i32p, ctypes.c_int64]
            lib.oracle_check_pluq.restype = ctypes.c_int
            lib.oracle_rref.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_uint32, _i32p]
            lib.oracle_rref.restype = ctypes.c_int64
            lib.oracle_determinant.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_uint32, _u32p]
            lib.oracle_determinant.restype = ctypes.c_int
            for nm in ("oracle_ple", "oracle_cup"):
                f = getattr(lib, nm)
                f.argtypes = [_u32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                              ctypes.c_uint32, _i32p, _u32p, _u32p, _i64p]
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def _u32(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def is_prime(p: int) -> bool:
    return bool(_load().oracle_is_prime(p))


def rank_profile(A: np.ndarray, p: int) -> np.ndarray:
    """col_of_row[i] = column of the one of R in row i, or -1 (R = rank profile matrix)."""
    A = _u32(A)
    m, n = A.shape
    col = np.full(max(m, 1), -1, dtype=np.int32)
    r = _load().oracle_rank_profile(_ptr(A, _u32p), m, n, max(n, 1), p, _ptr(col, _i32p))
    if r < 0:
        raise OracleError(int(r), "rank_profile")
    return col[:m]


def canonical_order(m: int, n: int, col_of_row: np.ndarray):
    """Pivots (rows, cols) of R in the order Algorithm 1 finds them."""
    col = np.ascontiguousarray(col_of_row, dtype=np.int32)
    if col.size == 0:
        col = np.full(1, -1, dtype=np.int32)
    cap = max(min(m, n), 1)
    pr = np.zeros(cap, dtype=np.int32)
    pc = np.zeros(cap, dtype=np.int32)
    r = ctypes.c_int64(0)
    st = _load().oracle_canonical_order(m, n, _ptr(col, _i32p), _ptr(pr, _i32p),
                                        _ptr(pc, _i32p), ctypes.byref(r))
    if st != 0:
        raise OracleError(st, "canonical_order")
    return pr[: r.value].copy(), pc[: r.value].copy()


def pluq(A: np.ndarray, p: int):
    """Returns (LU packed m x n, perm_p, perm_q, r)."""
    A = _u32(A)
    m, n = A.shape
    LU = np.zeros((max(m, 1), max(n, 1)), dtype=np.uint32)
    pp = np.zeros(max(m, 1), dtype=np.int32)
    pq = np.zeros(max(n, 1), dtype=np.int32)
    r = ctypes.c_int64(0)
    src = A if A.size else np.zeros((1, 1), dtype=np.uint32)
    st = _load().oracle_pluq(_ptr(src, _u32p), m, n, max(n, 1), p, _ptr(LU, _u32p),
                             max(n, 1), _ptr(pp, _i32p), _ptr(pq, _i32p), ctypes.byref(r))
    if st != 0:
        raise OracleError(st, "pluq")
    return LU[:m, :n].copy(), pp[:m].copy(), pq[:n].copy(), int(r.value)


def pluq_alg1(A: np.ndarray, p: int):
    """Literal recursive Algorithm 1 (rotation base cases). Returns (LU, perm_p, perm_q, r)."""
    A = _u32(A).copy()
    m, n = A.shape
    work = A if A.size else np.zeros((1, 1), dtype=np.uint32)
    pp = np.zeros(max(m, 1), dtype=np.int32)
    pq = np.zeros(max(n, 1), dtype=np.int32)
    r = ctypes.c_int64(0)
    st = _load().oracle_pluq_alg1(_ptr(work, _u32p), m, n, max(n, 1), p, _ptr(pp, _i32p),
                                  _ptr(pq, _i32p), ctypes.byref(r))
    if st != 0:
        raise OracleError(st, "pluq_alg1")
    return (work[:m, :n].copy() if A.size else np.zeros((m, n), dtype=np.uint32),
            pp[:m].copy(), pq[:n].copy(), int(r.value))


def matmul_sub(C: np.ndarray, A: np.ndarray, B: np.ndarray, p: int) -> np.ndarray:
    """MM(C, A, B): returns C - A B mod p."""
    C = _u32(C).copy()
    A = _u32(A)
    B = _u32(B)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2 and C.shape == (M, N)
    z = np.zeros((1, 1), dtype=np.uint32)
    _load().oracle_matmul_sub(_ptr(C if C.size else z, _u32p), max(N, 1),
                              _ptr(A if A.size else z, _u32p), max(K, 1),
                              _ptr(B if B.size else z, _u32p), max(N, 1), M, N, K, p)
    return C


def trsm_left_lower_unit(L: np.ndarray, B: np.ndarray, p: int) -> np.ndarray:
    """Returns L^{-1} B for L unit lower triangular (its diagonal is not read)."""
    L = _u32(L)
    B = _u32(B).copy()
    r, N = B.shape
    if r and N:
        _load().oracle_trsm_left_lower_unit(_ptr(L, _u32p), r, _ptr(B, _u32p), N, r, N, p)
    return B


def trsm_right_upper(U: np.ndarray, B: np.ndarray, p: int) -> np.ndarray:
    """Returns B U^{-1} for U upper triangular with nonzero diagonal."""
    U = _u32(U)
    B = _u32(B).copy()
    M, r = B.shape
    if M and r:
        _load().oracle_trsm_right_upper(_ptr(U, _u32p), r, _ptr(B, _u32p), r, M, r, p)
    return B


def check_pluq(A: np.ndarray, p: int, LU: np.ndarray, perm_p: np.ndarray,
               perm_q: np.ndarray, r: int) -> int:
    """0 iff (LU, perm_p, perm_q, r) satisfies Algorithm 1's output contract for A."""
    A = _u32(A)
    LU = _u32(LU)
    m, n = A.shape
    if m == 0 or n == 0:
        return 0 if r == 0 else 1
    pp = np.ascontiguousarray(perm_p, dtype=np.int32)
    pq = np.ascontiguousarray(perm_q, dtype=np.int32)
    return int(_load().oracle_check_pluq(_ptr(A, _u32p), m, n, n, p, _ptr(LU, _u32p), n,
                                         _ptr(pp, _i32p), _ptr(pq, _i32p), r))


def leu(LU: np.ndarray, perm_p: np.ndarray, perm_q: np.ndarray, r: int):
    """LEU decomposition read off a PLUQ (Corollary of the triangularity
    theorem, Sec. 3), written out as its definition:
        Lbar = P [L 0; M I_{m-r}] P^T,  Ubar = Q^T [U V; 0 0] Q,
    where P[perm_p[i], i] = 1 and Q[j, perm_q[j]] = 1.  Only entries move; no
    field arithmetic.  Returns (Lbar m x m, Ubar n x n) as uint32."""
    LU = np.asarray(LU, dtype=np.int64)
    m, n = LU.shape
    inner_l = np.eye(m, dtype=np.int64)                       # [L 0; M I]
    inner_l[:, :r] = np.tril(LU[:, :r], -1) + np.eye(m, r, dtype=np.int64)
    inner_u = np.zeros((n, n), dtype=np.int64)                # [U V; 0 0]
    inner_u[:r, :] = np.triu(LU[:r, :])
    P = np.zeros((m, m), dtype=np.int64)
    P[np.asarray(perm_p), np.arange(m)] = 1
    Q = np.zeros((n, n), dtype=np.int64)
    Q[np.arange(n), np.asarray(perm_q)] = 1
    Lbar = P @ inner_l @ P.T                                  # permutation products: entries move
    Ubar = Q.T @ inner_u @ Q
    return Lbar.astype(np.uint32), Ubar.astype(np.uint32)


# ------------------------------------------------ uses of the decomposition --
# Sec. 1 lists solving linear systems, the determinant and the nullspace among
# the uses of a triangular decomposition.  These are computed here from their
# textbook definitions (Gauss-Jordan RREF, elimination with row exchanges),
# independently of any PLUQ.


def rref(A: np.ndarray, p: int, npiv: int = None):
    """Reduced row echelon form of A (m x n); pivots only among the first
    npiv columns (default n).  Returns (E, pivot columns)."""
    E = _u32(A).copy()
    m, n = E.shape
    npiv = n if npiv is None else npiv
    pc = np.zeros(max(min(m, npiv), 1), dtype=np.int32)
    if m == 0 or n == 0:
        return E, pc[:0].copy()
    r = _load().oracle_rref(_ptr(E, _u32p), m, n, n, npiv, p, _ptr(pc, _i32p))
    if r < 0:
        raise OracleError(int(r), "rref")
    return E, pc[:r].copy()


def determinant(A: np.ndarray, p: int) -> int:
    """det A mod p for square A (1 for the 0 x 0 matrix)."""
    A = _u32(A)
    n, n2 = A.shape
    assert n == n2
    if n == 0:
        return 1
    d = np.zeros(1, dtype=np.uint32)
    st = _load().oracle_determinant(_ptr(A, _u32p), n, n, p, _ptr(d, _u32p))
    if st != 0:
        raise OracleError(st, "determinant")
    return int(d[0])


def right_nullspace(A: np.ndarray, p: int) -> np.ndarray:
    """Basis N (n x (n - r)) of {x : A x = 0}: column c is 1 at the c-th
    non-pivot column of the RREF (increasing), 0 at the other non-pivot
    columns, and minus the RREF's entries in that column at the pivot
    coordinates."""
    m, n = np.shape(A)
    E, pc = rref(A, p)
    r = pc.size
    free = np.setdiff1d(np.arange(n), pc)
    N = np.zeros((n, n - r), dtype=np.int64)
    N[free, np.arange(n - r)] = 1
    if r:
        N[pc, :] = (p - E[:r, free].astype(np.int64)) % p
    return N.astype(np.uint32)


def left_nullspace(A: np.ndarray, p: int) -> np.ndarray:
    """Basis ((m - r) x m) of {y : y A = 0}: the right nullspace of A^T,
    transposed (identity on the rows outside the row rank profile)."""
    return np.ascontiguousarray(right_nullspace(np.ascontiguousarray(np.asarray(A).T), p).T)


def solve(A: np.ndarray, B: np.ndarray, p: int):
    """A X = B (A m x n, B m x k).  Returns (X, consistent) where consistent[c]
    says whether column c has a solution, and X[:, c] is then the solution
    that is zero at every non-pivot coordinate (RREF of [A | B] with pivots
    taken in A's columns only)."""
    A = _u32(A)
    B = _u32(B)
    m, n = A.shape
    k = B.shape[1]
    E, pc = rref(np.concatenate([A, B], axis=1), p, npiv=n)
    r = pc.size
    Bt = E[:, n:]
    consistent = ~np.any(Bt[r:, :] != 0, axis=0)
    X = np.zeros((n, k), dtype=np.uint32)
    X[pc, :] = Bt[:r, :]
    return X, consistent


def ple(A: np.ndarray, p: int):
    """PLE decomposition (Sec. 1) from its definition: returns (perm_p, L, E, r)
    with A[perm_p] = L E, L (m x r) unit lower trapezoidal and E (r x n) in
    row echelon form whose leading entries sit on the column rank profile."""
    A = _u32(A)
    m, n = A.shape
    cap = max(min(m, n), 1)
    pp = np.zeros(max(m, 1), dtype=np.int32)
    L = np.zeros(max(m, 1) * cap, dtype=np.uint32)
    E = np.zeros(cap * max(n, 1), dtype=np.uint32)
    r = ctypes.c_int64(0)
    z = np.zeros(1, dtype=np.uint32)
    st = _load().oracle_ple(_ptr(A if A.size else z, _u32p), m, n, max(n, 1), p,
                            _ptr(pp, _i32p), _ptr(L, _u32p), _ptr(E, _u32p), ctypes.byref(r))
    if st != 0:
        raise OracleError(st, "ple")
    k = r.value
    return pp[:m].copy(), L[:m * k].reshape(m, k).copy(), E[:k * n].reshape(k, n).copy(), k


def cup(A: np.ndarray, p: int):
    """CUP decomposition (Sec. 1) from its definition: returns (perm_q, C, U, r)
    with A[:, perm_q] = C U, C (m x r) in column echelon form whose leading
    entries sit on the row rank profile and U (r x n) unit upper trapezoidal."""
    A = _u32(A)
    m, n = A.shape
    cap = max(min(m, n), 1)
    pq = np.zeros(max(n, 1), dtype=np.int32)
    C = np.zeros(max(m, 1) * cap, dtype=np.uint32)
    U = np.zeros(cap * max(n, 1), dtype=np.uint32)
    r = ctypes.c_int64(0)
    z = np.zeros(1, dtype=np.uint32)
    st = _load().oracle_cup(_ptr(A if A.size else z, _u32p), m, n, max(n, 1), p,
                            _ptr(pq, _i32p), _ptr(C, _u32p), _ptr(U, _u32p), ctypes.byref(r))
    if st != 0:
        raise OracleError(st, "cup")
    k = r.value
    return pq[:n].copy(), C[:m * k].reshape(m, k).copy(), U[:k * n].reshape(k, n).copy(), k
