"""Thin Python binding of libpluq (include/pluq.h).

Argument marshalling only: torch tensors are passed as raw device pointers and
the current CUDA stream; every step of the computation runs in the library's
CUDA kernels.  The library is loaded from this package directory on first use;
if it is missing or no CUDA device is present the calls raise.  There is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpluq.so")
_lock = threading.Lock()
_lib = None

MM_AUTO, MM_SIMT, MM_TENSOR = 0, 1, 2
_KIND = {"auto": MM_AUTO, "simt": MM_SIMT, "tensor": MM_TENSOR}

_c_i64 = ctypes.c_int64
_c_u32 = ctypes.c_uint32
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_szp = ctypes.POINTER(ctypes.c_size_t)

_SIGS = {
    "pluq_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pluq_tensor_limbs": (ctypes.c_int, [_c_u32]),
    "pluq_leaf_max_rows": (_c_i64, []),
    "pluq_leaf_max_cols": (_c_i64, []),
    "pluq_workspace_size": (ctypes.c_int, [_c_i64, _c_i64, _c_u32, _szp]),
    "pluq_mod_p": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_u32, _vp, _vp, _i64p, _vp,
                                  ctypes.c_size_t, ctypes.c_int, _vp]),
    "row_rank_profile": (ctypes.c_int, [_vp, _c_i64, _c_i64, _vp, _vp]),
    "col_rank_profile": (ctypes.c_int, [_vp, _c_i64, _c_i64, _vp, _vp]),
    "rank_profile_matrix": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, _c_i64, _vp, _vp, _vp]),
    "pluq_extract_L": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _c_i64, _vp]),
    "pluq_extract_U": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _c_i64, _vp]),
    "pluq_leu": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _vp, _vp, _c_i64, _vp,
                                _c_i64, _vp, ctypes.c_size_t, _vp]),
    "pluq_leading_rank_profiles": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, _c_i64, _c_i64, _c_i64,
                                                  _vp, _vp, _vp, _vp]),
    "pluq_uses_workspace_size": (ctypes.c_int, [_c_i64, _c_i64, _c_i64, _c_i64, _c_u32,
                                                ctypes.c_int, _szp]),
    "pluq_determinant": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _vp, _vp, _c_u32, _vp, _vp,
                                        ctypes.c_size_t, _vp]),
    "pluq_right_nullspace": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _c_u32, _vp,
                                            _c_i64, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "pluq_left_nullspace": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _c_u32, _vp,
                                           _c_i64, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "pluq_solve": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _vp, _c_u32, _vp,
                                  _c_i64, _c_i64, _vp, _c_i64, _vp, ctypes.c_int, _vp,
                                  ctypes.c_size_t, _vp]),
    "pluq_modmm_workspace_size": (ctypes.c_int, [_c_i64, _c_i64, _c_i64, _c_u32, ctypes.c_int,
                                                 _szp]),
    "pluq_modmm": (ctypes.c_int, [_vp, _c_i64, _vp, _c_i64, _vp, _c_i64, _c_i64, _c_i64, _c_i64,
                                  _c_u32, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "pluq_trsm_workspace_size": (ctypes.c_int, [_c_i64, _c_i64, _c_u32, ctypes.c_int, _szp]),
    "pluq_trsm_left_lower_unit": (ctypes.c_int, [_vp, _c_i64, _vp, _c_i64, _c_i64, _c_i64, _c_u32,
                                                 ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "pluq_trsm_right_upper": (ctypes.c_int, [_vp, _c_i64, _vp, _c_i64, _c_i64, _c_i64, _c_u32,
                                             ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "pluq_perm_rows": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _vp, _vp, ctypes.c_size_t,
                                      _vp]),
    "pluq_perm_cols": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _vp, _vp, ctypes.c_size_t,
                                      _vp]),
    "pluq_leaf": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_u32, _vp, _vp, _vp, _vp]),
    "pluq_modmm_tensor_noalloc": (ctypes.c_int, [_vp, _c_i64, _vp, _c_i64, _vp, _c_i64, _c_i64,
                                                 _c_i64, _c_i64, _c_u32, ctypes.c_int, _vp]),
    "pluq_batched_workspace_size": (ctypes.c_int, [_i64p, _i64p, _c_i64, _c_u32, ctypes.c_int, _szp]),
    "pluq_batched_persistent_workspace_size": (ctypes.c_int, [_c_i64, _c_i64, ctypes.c_int, _szp]),
    "pluq_mod_p_batched_persistent": (ctypes.c_int, [_vp, _vp, _vp, _vp, _c_i64, _c_i64, _c_i64,
                                                     _c_u32, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                                     ctypes.c_int, _vp]),
    "pluq_mod_p_batched": (ctypes.c_int, [ctypes.POINTER(_vp), _i64p, _i64p, _i64p, _c_i64, _c_u32,
                                          ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64p, _vp,
                                          ctypes.c_size_t, ctypes.c_int, ctypes.c_int, _vp]),
    "pluq_echelon_workspace_size": (ctypes.c_int, [_c_i64, _c_i64, _c_i64, _c_u32, ctypes.c_int,
                                                   _szp]),
    "pluq_ple": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _vp, _c_u32, _vp, _vp,
                                _c_i64, _vp, _c_i64, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "pluq_cup": (ctypes.c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _vp, _c_u32, _vp, _vp,
                                _c_i64, _vp, _c_i64, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    "pluq_set_tuning": (ctypes.c_int, [_c_i64, _c_i64]),
    "pluq_get_tuning": (ctypes.c_int, [_i64p, _i64p]),
    "pluq_set_branch_min": (ctypes.c_int, [_c_i64]),
    "pluq_get_branch_min": (ctypes.c_int64, []),
    "pluq_set_lazy_zero_test": (ctypes.c_int, [ctypes.c_int]),
    "pluq_set_wait_limit": (ctypes.c_int, [_c_i64]),
    "pluq_set_leaf_variant": (ctypes.c_int, [ctypes.c_int]),
    "pluq_get_leaf_variant": (ctypes.c_int, []),
    "pluq_set_node_kernel": (ctypes.c_int, [ctypes.c_int]),
    "pluq_get_node_kernel": (ctypes.c_int, []),
    "pluq_set_node_cluster": (ctypes.c_int, [ctypes.c_int]),
    "pluq_get_node_cluster": (ctypes.c_int, []),
    "pluq_device_status": (ctypes.c_int, [_vp]),
    "pluq_get_lazy_zero_test": (ctypes.c_int, []),
    "pluq_launch_count": (ctypes.c_longlong, []),
    "pluq_measure_mma_sync_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_double,
                                                  ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_double)]),
    "pluq_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "pluq_profile_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
}


class PluqError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


def load():
    """Load libpluq.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libpluq.so not built ({LIB_PATH}); run __graft_entry__.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def status_string(status: int) -> str:
    return load().pluq_status_string(status).decode()


def _check(status: int, what: str):
    if status != 0:
        raise PluqError(status, what)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else ctypes.c_void_p(0)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("libpluq works on CUDA tensors only")


def _u32_view(A: torch.Tensor) -> torch.Tensor:
    """uint32 data are carried in int32 tensors (same bits)."""
    if A.dtype not in (torch.int32,) and getattr(torch, "uint32", None) is not A.dtype:
        raise TypeError("matrix must be int32/uint32 holding residues in [0, p)")
    return A


def tensor_limbs(p: int) -> int:
    return int(load().pluq_tensor_limbs(p))


def leaf_max() -> tuple:
    lib = load()
    return int(lib.pluq_leaf_max_rows()), int(lib.pluq_leaf_max_cols())


def pluq_workspace_size(m: int, n: int, p: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().pluq_workspace_size(m, n, p, ctypes.byref(out)), "pluq_workspace_size")
    return int(out.value)


def pluq_mod_p(A: torch.Tensor, p: int, mm: str = "auto", workspace: torch.Tensor = None,
               stream=None):
    """In-place PLUQ of A (m x n int32 on the GPU, residues in [0, p)).
    Returns (perm_p, perm_q, r); A holds the packed [L\\U V; M 0]."""
    _need_cuda(A)
    _u32_view(A)
    m, n = A.shape
    lda = A.stride(0) if m > 0 else max(n, 1)
    if A.numel() and A.stride(1) != 1:
        raise ValueError("rows of A must be contiguous")
    dev = A.device
    pp = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    pq = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ws = pluq_workspace_size(m, n, p)
    if workspace is None or workspace.numel() < ws:
        workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
    r = ctypes.c_int64(0)
    st = load().pluq_mod_p(_ptr(A), m, n, lda, p, _ptr(pp), _ptr(pq), ctypes.byref(r),
                           _ptr(workspace), workspace.numel(), _KIND[mm], _stream(stream))
    _check(st, "pluq_mod_p")
    return pp[:m], pq[:n], int(r.value)


def row_rank_profile(perm_p: torch.Tensor, r: int, stream=None) -> torch.Tensor:
    _need_cuda(perm_p)
    out = torch.empty(max(r, 1), dtype=torch.int32, device=perm_p.device)
    _check(load().row_rank_profile(_ptr(perm_p), perm_p.numel(), r, _ptr(out), _stream(stream)),
           "row_rank_profile")
    return out[:r]


def col_rank_profile(perm_q: torch.Tensor, r: int, stream=None) -> torch.Tensor:
    _need_cuda(perm_q)
    out = torch.empty(max(r, 1), dtype=torch.int32, device=perm_q.device)
    _check(load().col_rank_profile(_ptr(perm_q), perm_q.numel(), r, _ptr(out), _stream(stream)),
           "col_rank_profile")
    return out[:r]


def rank_profile_matrix(perm_p: torch.Tensor, perm_q: torch.Tensor, r: int, stream=None):
    _need_cuda(perm_p, perm_q)
    rows = torch.empty(max(r, 1), dtype=torch.int32, device=perm_p.device)
    cols = torch.empty(max(r, 1), dtype=torch.int32, device=perm_p.device)
    _check(load().rank_profile_matrix(_ptr(perm_p), _ptr(perm_q), perm_p.numel(), perm_q.numel(),
                                      r, _ptr(rows), _ptr(cols), _stream(stream)),
           "rank_profile_matrix")
    return rows[:r], cols[:r]


def pluq_extract_L(LU: torch.Tensor, r: int, stream=None) -> torch.Tensor:
    """[L; M] (m x r, unit lower trapezoid) from the packed result of pluq_mod_p."""
    _need_cuda(LU)
    m, n = LU.shape
    L = torch.empty((m, max(r, 0)), dtype=LU.dtype, device=LU.device)
    _check(load().pluq_extract_L(_ptr(LU), m, n, LU.stride(0), r, _ptr(L), max(r, 1),
                                 _stream(stream)), "pluq_extract_L")
    return L


def pluq_extract_U(LU: torch.Tensor, r: int, stream=None) -> torch.Tensor:
    """[U V] (r x n, upper trapezoid) from the packed result of pluq_mod_p."""
    _need_cuda(LU)
    m, n = LU.shape
    U = torch.empty((max(r, 0), n), dtype=LU.dtype, device=LU.device)
    _check(load().pluq_extract_U(_ptr(LU), m, n, LU.stride(0), r, _ptr(U), max(n, 1),
                                 _stream(stream)), "pluq_extract_U")
    return U


def pluq_leu(LU: torch.Tensor, perm_p: torch.Tensor, perm_q: torch.Tensor, r: int, stream=None):
    """(Lbar, Ubar) of the LEU decomposition A = Lbar E Ubar; E is the rank
    profile matrix (rank_profile_matrix)."""
    _need_cuda(LU, perm_p, perm_q)
    m, n = LU.shape
    Lbar = torch.empty((m, m), dtype=LU.dtype, device=LU.device)
    Ubar = torch.empty((n, n), dtype=LU.dtype, device=LU.device)
    work = torch.empty(max(m + n, 1), dtype=torch.int32, device=LU.device)
    _check(load().pluq_leu(_ptr(LU), m, n, LU.stride(0) if m else max(n, 1), r, _ptr(perm_p),
                           _ptr(perm_q), _ptr(Lbar), max(m, 1), _ptr(Ubar), max(n, 1),
                           _ptr(work), work.numel() * 4, _stream(stream)), "pluq_leu")
    return Lbar, Ubar


def pluq_leading_rank_profiles(perm_p: torch.Tensor, perm_q: torch.Tensor, r: int, k: int, t: int,
                               stream=None):
    """(rows, cols): the row and column rank profiles of the leading k x t
    submatrix, read from P and Q without forming R; len(rows) is its rank."""
    _need_cuda(perm_p, perm_q)
    rows = torch.empty(max(r, 1), dtype=torch.int32, device=perm_p.device)
    cols = torch.empty(max(r, 1), dtype=torch.int32, device=perm_p.device)
    count = torch.zeros(1, dtype=torch.int32, device=perm_p.device)
    _check(load().pluq_leading_rank_profiles(_ptr(perm_p), _ptr(perm_q), perm_p.numel(),
                                             perm_q.numel(), r, k, t, _ptr(rows), _ptr(cols),
                                             _ptr(count), _stream(stream)),
           "pluq_leading_rank_profiles")
    c = int(count.item())
    return rows[:c], cols[:c]


def uses_workspace_size(m: int, n: int, r: int, k: int, p: int, mm: str = "auto") -> int:
    out = ctypes.c_size_t(0)
    _check(load().pluq_uses_workspace_size(m, n, r, k, p, _KIND[mm], ctypes.byref(out)),
           "pluq_uses_workspace_size")
    return int(out.value)


def _uses_ws(m, n, r, k, p, mm, workspace, dev):
    need = uses_workspace_size(m, n, r, k, p, mm)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    return workspace


def _ld(X: torch.Tensor, cols: int) -> int:
    return X.stride(0) if X.shape[0] > 0 else max(cols, 1)


def pluq_determinant(LU: torch.Tensor, perm_p: torch.Tensor, perm_q: torch.Tensor, r: int,
                     p: int, workspace=None, stream=None) -> torch.Tensor:
    """det A mod p (A square) from its PLUQ, as a one-element device tensor
    (int32 holding the uint32 value)."""
    _need_cuda(LU, perm_p, perm_q)
    n, n2 = LU.shape
    if n != n2:
        raise ValueError("the determinant needs a square matrix")
    det = torch.zeros(1, dtype=torch.int32, device=LU.device)
    ws = _uses_ws(n, n, r, 0, p, "auto", workspace, LU.device)
    _check(load().pluq_determinant(_ptr(LU), n, _ld(LU, n), r, _ptr(perm_p), _ptr(perm_q), p,
                                   _ptr(det), _ptr(ws), ws.numel(), _stream(stream)),
           "pluq_determinant")
    return det


def pluq_right_nullspace(LU: torch.Tensor, perm_q: torch.Tensor, r: int, p: int,
                         mm: str = "auto", workspace=None, stream=None) -> torch.Tensor:
    """N (n x (n - r)) with A N = 0: Q^T [-U^{-1} V; I]."""
    _need_cuda(LU, perm_q)
    m, n = LU.shape
    N = torch.empty((n, n - r), dtype=LU.dtype, device=LU.device)
    ws = _uses_ws(m, n, r, 0, p, mm, workspace, LU.device)
    _check(load().pluq_right_nullspace(_ptr(LU), m, n, _ld(LU, n), r, _ptr(perm_q), p, _ptr(N),
                                       max(n - r, 1), _KIND[mm], _ptr(ws), ws.numel(),
                                       _stream(stream)), "pluq_right_nullspace")
    return N


def pluq_left_nullspace(LU: torch.Tensor, perm_p: torch.Tensor, r: int, p: int,
                        mm: str = "auto", workspace=None, stream=None) -> torch.Tensor:
    """K ((m - r) x m) with K A = 0: [-M L^{-1}, I] P^T."""
    _need_cuda(LU, perm_p)
    m, n = LU.shape
    K = torch.empty((m - r, m), dtype=LU.dtype, device=LU.device)
    ws = _uses_ws(m, n, r, 0, p, mm, workspace, LU.device)
    _check(load().pluq_left_nullspace(_ptr(LU), m, n, _ld(LU, n), r, _ptr(perm_p), p, _ptr(K),
                                      max(m, 1), _KIND[mm], _ptr(ws), ws.numel(),
                                      _stream(stream)), "pluq_left_nullspace")
    return K


def pluq_solve(LU: torch.Tensor, perm_p: torch.Tensor, perm_q: torch.Tensor, r: int,
               B: torch.Tensor, p: int, mm: str = "auto", workspace=None, stream=None):
    """A X = B (B m x k, rows contiguous).  Returns (X n x k, inconsistent):
    inconsistent is a one-element device tensor, 1 if some column of B has no
    solution; X holds, per solvable column, the solution that is zero outside
    the column rank profile."""
    _need_cuda(LU, perm_p, perm_q, B)
    m, n = LU.shape
    if B.dim() != 2 or B.shape[0] != m:
        raise ValueError("B must be m x k")
    if B.numel() and B.stride(1) != 1:
        raise ValueError("rows of B must be contiguous")
    k = B.shape[1]
    X = torch.empty((n, k), dtype=LU.dtype, device=LU.device)
    flag = torch.empty(1, dtype=torch.int32, device=LU.device)
    ws = _uses_ws(m, n, r, k, p, mm, workspace, LU.device)
    _check(load().pluq_solve(_ptr(LU), m, n, _ld(LU, n), r, _ptr(perm_p), _ptr(perm_q), p,
                             _ptr(B), _ld(B, k), k, _ptr(X), max(k, 1), _ptr(flag), _KIND[mm],
                             _ptr(ws), ws.numel(), _stream(stream)), "pluq_solve")
    return X, flag


def modmm_workspace_size(M: int, N: int, K: int, p: int, mm: str = "auto") -> int:
    out = ctypes.c_size_t(0)
    _check(load().pluq_modmm_workspace_size(M, N, K, p, _KIND[mm], ctypes.byref(out)),
           "pluq_modmm_workspace_size")
    return int(out.value)


def pluq_modmm(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, p: int, assign: bool = False,
               mm: str = "auto", workspace: torch.Tensor = None, stream=None):
    """C <- C - A B (or A B) mod p, in place on C."""
    _need_cuda(C, A, B)
    M, K = A.shape
    K2, N = B.shape
    if K2 != K or tuple(C.shape) != (M, N):
        raise ValueError("shape mismatch")
    ws = modmm_workspace_size(M, N, K, p, mm)
    if ws and (workspace is None or workspace.numel() < ws):
        workspace = torch.empty(ws, dtype=torch.uint8, device=C.device)
    wsn = workspace.numel() if workspace is not None else 0
    _check(load().pluq_modmm(_ptr(C), C.stride(0) if M else max(N, 1), _ptr(A),
                             A.stride(0) if M else max(K, 1), _ptr(B),
                             B.stride(0) if K else max(N, 1), M, N, K, p, int(assign), _KIND[mm],
                             _ptr(workspace), wsn, _stream(stream)), "pluq_modmm")
    return C


def _trsm_ws(r, other, p, mm, workspace, dev):
    out = ctypes.c_size_t(0)
    _check(load().pluq_trsm_workspace_size(r, other, p, _KIND[mm], ctypes.byref(out)),
           "pluq_trsm_workspace_size")
    if workspace is None or workspace.numel() < out.value:
        workspace = torch.empty(max(out.value, 1), dtype=torch.uint8, device=dev)
    return workspace


def pluq_trsm_left_lower_unit(L: torch.Tensor, B: torch.Tensor, p: int, mm: str = "auto",
                              workspace=None, stream=None):
    """B <- L^{-1} B in place (L unit lower, diagonal not read)."""
    _need_cuda(L, B)
    r, N = B.shape
    ws = _trsm_ws(r, N, p, mm, workspace, B.device)
    _check(load().pluq_trsm_left_lower_unit(_ptr(L), L.stride(0) if r else 1, _ptr(B),
                                            B.stride(0) if r else max(N, 1), r, N, p, _KIND[mm],
                                            _ptr(ws), ws.numel(), _stream(stream)),
           "pluq_trsm_left_lower_unit")
    return B


def pluq_trsm_right_upper(U: torch.Tensor, B: torch.Tensor, p: int, mm: str = "auto",
                          workspace=None, stream=None):
    """B <- B U^{-1} in place (U upper, nonzero diagonal)."""
    _need_cuda(U, B)
    M, r = B.shape
    ws = _trsm_ws(r, M, p, mm, workspace, B.device)
    _check(load().pluq_trsm_right_upper(_ptr(U), U.stride(0) if r else 1, _ptr(B),
                                        B.stride(0) if M else max(r, 1), M, r, p, _KIND[mm],
                                        _ptr(ws), ws.numel(), _stream(stream)),
           "pluq_trsm_right_upper")
    return B


def pluq_perm_rows(X: torch.Tensor, perm: torch.Tensor, workspace=None, stream=None):
    _need_cuda(X, perm)
    count, width = X.shape
    if workspace is None:
        workspace = torch.empty(max(count * width * 4, 1), dtype=torch.uint8, device=X.device)
    _check(load().pluq_perm_rows(_ptr(X), X.stride(0) if count else max(width, 1), count, width,
                                 _ptr(perm), _ptr(workspace), workspace.numel(), _stream(stream)),
           "pluq_perm_rows")
    return X


def pluq_perm_cols(X: torch.Tensor, perm: torch.Tensor, workspace=None, stream=None):
    _need_cuda(X, perm)
    height, count = X.shape
    if workspace is None:
        workspace = torch.empty(max(count * height * 4, 1), dtype=torch.uint8, device=X.device)
    _check(load().pluq_perm_cols(_ptr(X), X.stride(0) if height else max(count, 1), height, count,
                                 _ptr(perm), _ptr(workspace), workspace.numel(), _stream(stream)),
           "pluq_perm_cols")
    return X


def pluq_leaf(A: torch.Tensor, p: int, stream=None):
    """Base case on a block of at most pluq_leaf_max_rows() x pluq_leaf_max_cols(), in place.
    Returns (perm_p, perm_q, r) with r read back after the stream synchronises."""
    _need_cuda(A)
    m, n = A.shape
    dev = A.device
    pp = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    pq = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    rk = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(load().pluq_leaf(_ptr(A), m, n, A.stride(0) if m else max(n, 1), p, _ptr(pp), _ptr(pq),
                            _ptr(rk), _stream(stream)), "pluq_leaf")
    return pp[:m], pq[:n], int(rk.item())


PROFILE_CLASSES = {"tensor_mm": 0, "simt_mm": 1, "leaf": 2, "move": 3, "split": 4, "tri_base": 5}


def pluq_launch_count() -> int:
    return int(load().pluq_launch_count())


def pluq_profile_enable(classes=True):
    """True: every class; False: stop; or an iterable of class names."""
    if classes is True:
        mask = (1 << len(PROFILE_CLASSES)) - 1
    elif not classes:
        mask = 0
    else:
        mask = 0
        for c in classes:
            mask |= 1 << PROFILE_CLASSES.get(c, c)
    _check(load().pluq_profile_enable(mask), "pluq_profile_enable")


def pluq_profile_read(kernel_class):
    """(launches, device ms, algorithmic work) of one kernel class since enable."""
    cls = PROFILE_CLASSES.get(kernel_class, kernel_class)
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0)
    w = ctypes.c_double(0)
    _check(load().pluq_profile_read(cls, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(w)),
           "pluq_profile_read")
    return int(n.value), float(ms.value), float(w.value)


def pluq_batched_workspace_size(shapes, p: int, workers: int = 8) -> int:
    cnt = len(shapes)
    ms = (ctypes.c_int64 * max(cnt, 1))(*[int(a) for a, _ in shapes])
    ns = (ctypes.c_int64 * max(cnt, 1))(*[int(b) for _, b in shapes])
    out = ctypes.c_size_t(0)
    _check(load().pluq_batched_workspace_size(ms, ns, cnt, p, workers, ctypes.byref(out)),
           "pluq_batched_workspace_size")
    return int(out.value)


def pluq_mod_p_batched(mats, p: int, mm: str = "auto", workers: int = 8, workspace=None,
                       stream=None):
    """In-place PLUQ of every matrix in `mats` (int32 CUDA tensors, rows
    contiguous).  Returns (list of perm_p, list of perm_q, list of ranks)."""
    _need_cuda(*mats)
    cnt = len(mats)
    if cnt == 0:
        return [], [], []
    dev = mats[0].device
    shapes = [tuple(A.shape) for A in mats]
    pps = [torch.empty(max(m, 1), dtype=torch.int32, device=dev) for m, _ in shapes]
    pqs = [torch.empty(max(n, 1), dtype=torch.int32, device=dev) for _, n in shapes]
    ws = pluq_batched_workspace_size(shapes, p, workers)
    if workspace is None or workspace.numel() < ws:
        workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
    VP = _vp * cnt
    I64 = ctypes.c_int64 * cnt
    a_ptrs = VP(*[A.data_ptr() if A.numel() else 0 for A in mats])
    p_ptrs = VP(*[t.data_ptr() for t in pps])
    q_ptrs = VP(*[t.data_ptr() for t in pqs])
    ms = I64(*[m for m, _ in shapes])
    ns = I64(*[n for _, n in shapes])
    lds = I64(*[(A.stride(0) if A.shape[0] else max(A.shape[1], 1)) for A in mats])
    ranks = I64()
    _check(load().pluq_mod_p_batched(a_ptrs, ms, ns, lds, cnt, p, p_ptrs, q_ptrs, ranks,
                                     _ptr(workspace), workspace.numel(), _KIND[mm], workers,
                                     _stream(stream)), "pluq_mod_p_batched")
    return ([pps[i][:shapes[i][0]] for i in range(cnt)], [pqs[i][:shapes[i][1]] for i in range(cnt)],
            [int(ranks[i]) for i in range(cnt)])


def pluq_batched_persistent_workspace_size(max_m: int, max_n: int, ctas: int = 0) -> int:
    out = ctypes.c_size_t(0)
    _check(load().pluq_batched_persistent_workspace_size(int(max_m), int(max_n), int(ctas),
                                                         ctypes.byref(out)),
           "pluq_batched_persistent_workspace_size")
    return int(out.value)


class PersistentBatch:
    """A batch for pluq_mod_p_batched_persistent: the device-side argument
    arrays (matrices largest first, by m n min(m, n)), the output vectors and
    the workspace, built once.  `run()` queues the call (one memset, one
    launch) on the current stream; after a first run it can be captured in a
    CUDA graph and replayed on new contents of the same matrices.  `ranks()`
    gives the ranks (or negative per-matrix statuses) in the order of `mats`."""

    def __init__(self, mats, p: int, ctas: int = 0, workspace=None):
        _need_cuda(*mats)
        for A in mats:
            if A.dim() != 2 or (A.shape[0] > 1 and A.shape[1] > 1 and A.stride(1) != 1):
                raise ValueError("matrices must be 2-D with contiguous rows")
        self.mats, self.p, self.ctas = list(mats), int(p), int(ctas)
        cnt = len(self.mats)
        dev = self.mats[0].device if cnt else torch.device("cuda")
        shapes = [tuple(A.shape) for A in self.mats]
        self.pps = [torch.empty(max(m, 1), dtype=torch.int32, device=dev) for m, _ in shapes]
        self.pqs = [torch.empty(max(n, 1), dtype=torch.int32, device=dev) for _, n in shapes]
        self.order = sorted(range(cnt), key=lambda i: -shapes[i][0] * shapes[i][1] *
                            min(shapes[i][0], shapes[i][1]))
        o = self.order

        def i64(vals):
            return torch.tensor(vals, dtype=torch.int64).to(dev)

        self.d_A = i64([self.mats[i].data_ptr() if self.mats[i].numel() else 0 for i in o])
        self.d_m = i64([shapes[i][0] for i in o])
        self.d_n = i64([shapes[i][1] for i in o])
        self.d_lda = i64([(self.mats[i].stride(0) if shapes[i][0] > 1 else max(shapes[i][1], 1))
                          for i in o])
        self.d_pp = i64([self.pps[i].data_ptr() for i in o])
        self.d_pq = i64([self.pqs[i].data_ptr() for i in o])
        self.d_rank = torch.zeros(max(cnt, 1), dtype=torch.int64, device=dev)
        self.max_m = max([m for m, _ in shapes], default=0)
        self.max_n = max([n for _, n in shapes], default=0)
        ws = pluq_batched_persistent_workspace_size(self.max_m, self.max_n, self.ctas)
        if workspace is None or workspace.numel() < ws:
            workspace = torch.empty(ws, dtype=torch.uint8, device=dev)
        self.workspace = workspace
        self._stream = None

    def run(self, stream=None):
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        _check(load().pluq_mod_p_batched_persistent(
            _ptr(self.d_A), _ptr(self.d_m), _ptr(self.d_n), _ptr(self.d_lda), len(self.mats),
            self.max_m, self.max_n, self.p, _ptr(self.d_pp), _ptr(self.d_pq), _ptr(self.d_rank),
            _ptr(self.workspace), self.workspace.numel(), self.ctas, _stream(self._stream)),
            "pluq_mod_p_batched_persistent")

    def ranks(self):
        """Waits for the stream of the last run(), then reads the ranks."""
        if self._stream is not None:
            self._stream.synchronize()
        got = self.d_rank.cpu().tolist()
        out = [0] * len(self.mats)
        for pos, i in enumerate(self.order):
            out[i] = int(got[pos])
        return out

    def perms(self):
        return ([self.pps[i][:A.shape[0]] for i, A in enumerate(self.mats)],
                [self.pqs[i][:A.shape[1]] for i, A in enumerate(self.mats)])


def pluq_mod_p_batched_persistent(mats, p: int, ctas: int = 0, workspace=None, stream=None):
    """In-place PLUQ of every matrix in `mats` (int32 CUDA tensors, rows
    contiguous, sides <= 2048) in one persistent launch.  Returns (list of
    perm_p, list of perm_q, list of ranks); a negative rank is that matrix's
    status (PLUQ_ERANGE, PLUQ_EINVAL, PLUQ_ETIMEOUT)."""
    if not mats:
        return [], [], []
    b = PersistentBatch(mats, p, ctas, workspace)
    b.run(stream)
    pps, pqs = b.perms()
    return pps, pqs, b.ranks()


def pluq_set_tuning(leaf: int, small_mm_macs: int):
    _check(load().pluq_set_tuning(int(leaf), int(small_mm_macs)), "pluq_set_tuning")


def pluq_get_tuning():
    a = ctypes.c_int64(0)
    b = ctypes.c_int64(0)
    _check(load().pluq_get_tuning(ctypes.byref(a), ctypes.byref(b)), "pluq_get_tuning")
    return int(a.value), int(b.value)


def pluq_set_branch_min(branch_min: int):
    _check(load().pluq_set_branch_min(int(branch_min)), "pluq_set_branch_min")


def pluq_get_branch_min() -> int:
    return int(load().pluq_get_branch_min())


def pluq_set_lazy_zero_test(lazy: bool):
    _check(load().pluq_set_lazy_zero_test(1 if lazy else 0), "pluq_set_lazy_zero_test")


def pluq_get_lazy_zero_test() -> bool:
    return bool(load().pluq_get_lazy_zero_test())


def pluq_set_wait_limit(tries: int):
    """Tries of every abortable device-side wait (negative: built-in bounds)."""
    _check(load().pluq_set_wait_limit(int(tries)), "pluq_set_wait_limit")


def pluq_device_status(stream=None) -> int:
    """Synchronise the stream; PLUQ_ETIMEOUT (-6) if a kernel gave up a wait."""
    return int(load().pluq_device_status(_stream(stream)))


def measure_mma_sync_peak(form: str = "s8", target_ms: float = 500.0):
    """(tera-ops/s, ms) of mma.sync s8 x s8 -> s32 (form 's8') or bf16 -> fp32
    ('bf16') with every SM busy for about target_ms."""
    tops = ctypes.c_double(0)
    ms = ctypes.c_double(0)
    _check(load().pluq_measure_mma_sync_peak({"s8": 0, "bf16": 1}[form], float(target_ms),
                                             ctypes.byref(tops), ctypes.byref(ms)),
           "pluq_measure_mma_sync_peak")
    return tops.value, ms.value


def pluq_set_leaf_variant(left_looking: bool):
    """Base case's blocked elimination: right-looking (False) or left-looking (True)."""
    _check(load().pluq_set_leaf_variant(1 if left_looking else 0), "pluq_set_leaf_variant")


def pluq_get_leaf_variant() -> bool:
    return bool(load().pluq_get_leaf_variant())


def _echelon(fn, LU, perm_p, perm_q, r, p, mm, stream, rows_out, left_shape, right_shape):
    _need_cuda(LU)
    m, n = LU.shape
    dev = LU.device
    size = ctypes.c_size_t(0)
    _check(load().pluq_echelon_workspace_size(m, n, r, p, _KIND[mm], ctypes.byref(size)),
           "pluq_echelon_workspace_size")
    ws = torch.empty(max(size.value, 1), dtype=torch.uint8, device=dev)
    perm = torch.empty(max(rows_out, 1), dtype=torch.int32, device=dev)
    X = torch.zeros((max(left_shape[0], 1), max(left_shape[1], 1)), dtype=torch.int32, device=dev)
    Y = torch.zeros((max(right_shape[0], 1), max(right_shape[1], 1)), dtype=torch.int32, device=dev)
    _check(fn(_ptr(LU), m, n, LU.stride(0) if m else max(n, 1), r, _ptr(perm_p), _ptr(perm_q), p,
              _ptr(perm), _ptr(X), X.stride(0), _ptr(Y), Y.stride(0), _KIND[mm], _ptr(ws),
              ws.numel(), _stream(stream)), fn.__name__)
    return perm[:rows_out], X[:left_shape[0], :left_shape[1]], Y[:right_shape[0], :right_shape[1]]


def pluq_ple(LU: torch.Tensor, perm_p: torch.Tensor, perm_q: torch.Tensor, r: int, p: int,
             mm: str = "auto", stream=None):
    """PLE decomposition from the packed PLUQ: returns (perm (m), L (m x r), E (r x n))
    with A[perm] = L E, L unit lower trapezoidal, E in row echelon form."""
    m, n = LU.shape
    return _echelon(load().pluq_ple, LU, perm_p, perm_q, r, p, mm, stream, m, (m, r), (r, n))


def pluq_cup(LU: torch.Tensor, perm_p: torch.Tensor, perm_q: torch.Tensor, r: int, p: int,
             mm: str = "auto", stream=None):
    """CUP decomposition from the packed PLUQ: returns (perm (n), C (m x r), U (r x n))
    with A[:, perm] = C U, C in column echelon form, U unit upper trapezoidal."""
    m, n = LU.shape
    return _echelon(load().pluq_cup, LU, perm_p, perm_q, r, p, mm, stream, n, (m, r), (r, n))


def pluq_set_node_kernel(levels: int):
    """Small nodes below rank-deficient ones in one thread block: 0 off, 1 up to
    2 x leaf, 2 up to 4 x leaf on a side (speed only)."""
    _check(load().pluq_set_node_kernel(int(levels)), "pluq_set_node_kernel")


def pluq_get_node_kernel() -> int:
    return int(load().pluq_get_node_kernel())


def pluq_set_node_cluster(ctas: int):
    """Thread blocks of a node kernel: 1, or a cluster of 2, 4 or 8 (speed only)."""
    _check(load().pluq_set_node_cluster(int(ctas)), "pluq_set_node_cluster")


def pluq_get_node_cluster() -> int:
    return int(load().pluq_get_node_cluster())
