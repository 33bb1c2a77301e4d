"""Seeded synthetic inputs for PLUQ over Z/pZ.

This module only draws random matrices; it holds none of the decomposition's
arithmetic and imports neither the CUDA binding nor the CPU oracle, so both can
be fed the same inputs.

Matrices of a prescribed rank profile follow the paper's experimental recipe
(Sec. 8): A = L0 . R . U0 with L0 unit lower triangular, U0 unit upper
triangular (entries uniform in [0, p)) and R a 0/1 matrix with r ones at
distinct rows and columns.  Left multiplication by an invertible lower
triangular matrix and right multiplication by an invertible upper triangular
matrix keep every leading submatrix's rank (Lemma 1 of Sec. 4, with its lower /
upper roles read as in its proof), so the rank profile matrix of A is exactly R.

Only the r columns of L0 and r rows of U0 that R selects matter:
A = L0[:, rows] . U0[cols, :].  The product is formed exactly: with numpy int64
and 16-bit limbs for small sizes, or on a CUDA device with float32 GEMMs on
8-bit unsigned limbs in K-slices of 256 (every partial sum stays below 2^24, so
it is exact in any summation order) for large ones.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

BASE_SEED = 13014438


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(m: int, n: int, p: int, seed: int) -> np.ndarray:
    """Dense m x n matrix with entries uniform in [0, p)."""
    return rng(seed).integers(0, p, size=(m, n), dtype=np.uint32)


@dataclass
class Planted:
    m: int
    n: int
    r: int
    p: int
    rows: np.ndarray          # pivot rows of R (R[rows[t], cols[t]] = 1), int64
    cols: np.ndarray
    Lc: np.ndarray            # m x r: column rows[t] of L0 in column t
    Ur: np.ndarray            # r x n: row cols[t] of U0 in row t

    def rank_profile(self) -> np.ndarray:
        """col_of_row: column of R's one in each row, -1 if none."""
        c = np.full(self.m, -1, dtype=np.int32)
        c[self.rows] = self.cols
        return c


def planted_factors(m: int, n: int, r: int, p: int, seed: int,
                    pivot_rows: Optional[np.ndarray] = None) -> Planted:
    """Random L0[:, rows], U0[cols, :] and the planted R (rows, cols)."""
    assert 0 <= r <= min(m, n)
    g = rng(seed)
    rows = np.sort(g.choice(m, size=r, replace=False)) if pivot_rows is None \
        else np.sort(np.asarray(pivot_rows, dtype=np.int64))
    assert rows.size == r
    cols = np.sort(g.choice(n, size=r, replace=False))
    cols = cols[g.permutation(r)]          # pair rows with columns at random
    rows = rows.astype(np.int64)
    cols = cols.astype(np.int64)
    Lc = g.integers(0, p, size=(m, r), dtype=np.uint32)
    Ur = g.integers(0, p, size=(r, n), dtype=np.uint32)
    ii = np.arange(m)[:, None]
    jj = np.arange(n)[None, :]
    # unit lower column: zeros above the diagonal entry, one on it
    Lc[ii < rows[None, :]] = 0
    Lc[rows, np.arange(r)] = 1
    # unit upper row: zeros left of the diagonal entry, one on it
    Ur[jj < cols[:, None]] = 0
    Ur[np.arange(r), cols] = 1
    return Planted(m, n, r, p, rows, cols, Lc, Ur)


def _product_numpy(Lc: np.ndarray, Ur: np.ndarray, p: int) -> np.ndarray:
    m, r = Lc.shape
    n = Ur.shape[1]
    out = np.zeros((m, n), dtype=np.int64)
    if r == 0:
        return out.astype(np.uint32)
    a = Lc.astype(np.int64)
    lo = (Ur & 0xFFFF).astype(np.int64)
    hi = (Ur >> 16).astype(np.int64)
    step = 1 << 15                      # products < 2^47, 2^15 of them < 2^62
    for s in range(0, r, step):
        e = min(r, s + step)
        out = (out + (a[:, s:e] @ lo[s:e]) % p + ((a[:, s:e] @ hi[s:e]) % p) * (65536 % p)) % p
    return out.astype(np.uint32)


def _product_torch(Lc: np.ndarray, Ur: np.ndarray, p: int, device: str):
    import torch
    m, r = Lc.shape
    n = Ur.shape[1]
    nl = max(1, (int(p - 1).bit_length() + 7) // 8)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        A = torch.from_numpy(Lc.astype(np.int64)).to(device)
        B = torch.from_numpy(Ur.astype(np.int64)).to(device)
        acc = [torch.zeros((m, n), dtype=torch.float64, device=device) for _ in range(2 * nl - 1)]
        KS = 256
        for s in range(0, r, KS):
            e = min(r, s + KS)
            al = [((A[:, s:e] >> (8 * i)) & 255).to(torch.float32) for i in range(nl)]
            bl = [((B[s:e] >> (8 * j)) & 255).to(torch.float32) for j in range(nl)]
            for i in range(nl):
                for j in range(nl):
                    acc[i + j] += (al[i] @ bl[j]).to(torch.float64)
        out = torch.zeros((m, n), dtype=torch.int64, device=device)
        for s_, a in enumerate(acc):
            w = pow(256, s_, p)
            out = (out + (a.to(torch.int64) % p) * w) % p
        return out
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def planted_matrix(pl: Planted, device: Optional[str] = None):
    """A = L0[:, rows] U0[cols, :] mod p.  numpy uint32 on the host, or (with
    device='cuda...') a torch int64 tensor on that device."""
    if device is None:
        return _product_numpy(pl.Lc, pl.Ur, pl.p)
    return _product_torch(pl.Lc, pl.Ur, pl.p, device)


def planted(m: int, n: int, r: int, p: int, seed: int,
            pivot_rows: Optional[np.ndarray] = None):
    """(A as numpy uint32, Planted)."""
    pl = planted_factors(m, n, r, p, seed, pivot_rows)
    return planted_matrix(pl), pl


def clustered_rows(m: int, r: int, top: int, seed: int) -> np.ndarray:
    """Pivot rows crowding the top `top` rows: all of them when r > top (the rest
    uniform below), else r of them drawn uniformly among the top rows."""
    g = rng(seed ^ 0x5A5A)
    if r <= top:
        return np.sort(g.choice(top, size=r, replace=False))
    rest = g.choice(np.arange(top, m), size=r - top, replace=False)
    return np.sort(np.concatenate([np.arange(top), rest]))


# ------------------------------------------------------------ named configs --

@dataclass
class Config:
    name: str
    m: int
    n: int
    p: int
    r: Optional[int]          # None: dense uniform (rank not planted)
    seed: int
    kind: str                 # "planted" | "uniform"
    cluster_top: Optional[int] = None
    note: str = ""


CONFIGS = {
    "planted_256": Config("planted_256", 256, 256, 65521, 200, BASE_SEED + 0, "planted",
                          note="256x256, p=65521, r=200, A = L0 R U0"),
    "dense_4096": Config("dense_4096", 4096, 4096, 65521, None, BASE_SEED + 1, "uniform",
                         note="4096x4096 uniform in [0,p), p=65521, full rank w.h.p."),
    "planted_16384": Config("planted_16384", 16384, 16384, 8388593, 8192, BASE_SEED + 2,
                            "planted", note="16384x16384, p=8388593, r=8192"),
    "rect_8192x32768": Config("rect_8192x32768", 8192, 32768, 2147483647, 6000,
                              BASE_SEED + 4, "planted", cluster_top=2048,
                              note="8192x32768, p=2^31-1, r=6000, pivot rows crowd the top 25%"),
}


def make(cfg: Config, device: Optional[str] = None):
    """(A, Planted-or-None).  A is numpy uint32 (device None) or a torch int64
    tensor on `device`."""
    if cfg.kind == "uniform":
        A = uniform(cfg.m, cfg.n, cfg.p, cfg.seed)
        if device is not None:
            import torch
            return torch.from_numpy(A.astype(np.int64)).to(device), None
        return A, None
    rows = None
    if cfg.cluster_top is not None:
        rows = clustered_rows(cfg.m, cfg.r, cfg.cluster_top, cfg.seed)
    pl = planted_factors(cfg.m, cfg.n, cfg.r, cfg.p, cfg.seed, rows)
    return planted_matrix(pl, device), pl


@dataclass
class Batch:
    p: int
    ms: List[int]
    ns: List[int]
    rs: List[int]
    seeds: List[int]


def batch_2000(count: int = 2000, lo: int = 64, hi: int = 2048, p: int = 65521,
               seed: int = BASE_SEED + 3) -> Batch:
    """Sizes of the uneven batch: m, n uniform in [lo, hi], r = floor(min(m, n)/2)."""
    g = rng(seed)
    ms = g.integers(lo, hi + 1, size=count).tolist()
    ns = g.integers(lo, hi + 1, size=count).tolist()
    rs = [min(a, b) // 2 for a, b in zip(ms, ns)]
    seeds = [seed * 7919 + i for i in range(count)]
    return Batch(p, ms, ns, rs, seeds)


def planted_device(m: int, n: int, r: int, p: int, seed: int, device: str):
    """Planted-profile matrix drawn with torch's generator on `device` (for
    batches too large to draw on the host).  Returns (A int32 tensor,
    rows, cols) with R[rows[t], cols[t]] = 1 as numpy int64 arrays."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rows = torch.sort(torch.randperm(m, generator=g, device=device)[:r]).values
    cols = torch.sort(torch.randperm(n, generator=g, device=device)[:r]).values
    cols = cols[torch.randperm(r, generator=g, device=device)]
    Lc = torch.randint(0, p, (m, r), generator=g, device=device, dtype=torch.int64)
    Ur = torch.randint(0, p, (r, n), generator=g, device=device, dtype=torch.int64)
    ii = torch.arange(m, device=device)[:, None]
    jj = torch.arange(n, device=device)[None, :]
    Lc = torch.where(ii < rows[None, :], torch.zeros_like(Lc), Lc)
    Lc[rows, torch.arange(r, device=device)] = 1
    Ur = torch.where(jj < cols[:, None], torch.zeros_like(Ur), Ur)
    Ur[torch.arange(r, device=device), cols] = 1
    if r == 0:
        A = torch.zeros((m, n), dtype=torch.int32, device=device)
    else:
        A = _product_torch_t(Lc, Ur, p).to(torch.int32)
    return A, rows.cpu().numpy().astype(np.int64), cols.cpu().numpy().astype(np.int64)


def _product_torch_t(A, B, p: int):
    """Exact (A B) mod p for int64 CUDA tensors with entries in [0, p)."""
    import torch
    m, r = A.shape
    n = B.shape[1]
    nl = max(1, (int(p - 1).bit_length() + 7) // 8)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        acc = [torch.zeros((m, n), dtype=torch.float64, device=A.device) for _ in range(2 * nl - 1)]
        for s in range(0, r, 256):
            e = min(r, s + 256)
            al = [((A[:, s:e] >> (8 * i)) & 255).to(torch.float32) for i in range(nl)]
            bl = [((B[s:e] >> (8 * j)) & 255).to(torch.float32) for j in range(nl)]
            for i in range(nl):
                for j in range(nl):
                    acc[i + j] += (al[i] @ bl[j]).to(torch.float64)
        out = torch.zeros((m, n), dtype=torch.int64, device=A.device)
        for s_, a in enumerate(acc):
            out = (out + (a.to(torch.int64) % p) * pow(256, s_, p)) % p
        return out
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
