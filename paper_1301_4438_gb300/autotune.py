"""Autotuner for the recursion cutoff and the product-kernel threshold.

The decomposition's result never depends on these knobs (the split points of
the recursion are fixed at floor(m/2), floor(n/2); the leaf and the products
are exact), only its speed does.  For a workload class (size rounded to a
power of two, number of limbs of p, dense or rank-deficient) the tuner times
`pluq_mod_p` on a seeded synthetic matrix of that class for each candidate
(leaf size, small-product threshold) and caches the fastest in a JSON file.
`apply()` looks the class up and sets the library's process-wide knobs.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import pluq, workloads

LEAVES = (32, 64, 128)
SMALL_MM = (1 << 24, 1 << 25, 1 << 27)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pluq_gb300", "tuning.json")


def _class_key(m: int, n: int, p: int, deficient: bool) -> str:
    def c(x):
        return 1 << max(0, int(np.ceil(np.log2(max(x, 1)))))
    return f"{c(m)}x{c(n)}:L{pluq.tensor_limbs(p)}:{'def' if deficient else 'full'}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _sample(m, n, p, deficient, seed=7):
    if deficient:
        A = workloads.planted_device(m, n, min(m, n) // 2, p, seed, "cuda")[0]
    else:
        A = torch.from_numpy(workloads.uniform(m, n, p, seed).astype(np.int32)).cuda()
    return A


def tune(m: int, n: int, p: int, deficient: bool = False, reps: int = 2,
         cache: str = DEFAULT_CACHE, budget_s: float = 60.0):
    """Time every candidate on one sample of the class and cache the best.
    Returns (leaf, small_mm_macs, ms)."""
    key = _class_key(m, n, p, deficient)
    A0 = _sample(m, n, p, deficient)
    ws = torch.empty(pluq.pluq_workspace_size(m, n, p), dtype=torch.uint8, device="cuda")
    old = pluq.pluq_get_tuning()
    best = None
    t_start = time.perf_counter()
    try:
        for leaf in LEAVES:
            for small in SMALL_MM:
                pluq.pluq_set_tuning(leaf, small)
                times = []
                for _ in range(reps + 1):
                    A = A0.clone()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    pluq.pluq_mod_p(A, p, workspace=ws)
                    torch.cuda.synchronize()
                    times.append(time.perf_counter() - t0)
                ms = 1e3 * min(times[1:])
                if best is None or ms < best[2]:
                    best = (leaf, small, ms)
                if time.perf_counter() - t_start > budget_s:
                    break
            if time.perf_counter() - t_start > budget_s:
                break
    finally:
        pluq.pluq_set_tuning(*old)
    data = _load(cache)
    data[key] = {"leaf": best[0], "small_mm_macs": best[1], "ms": best[2]}
    _store(cache, data)
    return best


def apply(m: int, n: int, p: int, deficient: bool = False, cache: str = DEFAULT_CACHE) -> bool:
    """Set the library's knobs from the cache; False if the class is unknown."""
    ent = _load(cache).get(_class_key(m, n, p, deficient))
    if not ent:
        return False
    pluq.pluq_set_tuning(int(ent["leaf"]), int(ent["small_mm_macs"]))
    return True
