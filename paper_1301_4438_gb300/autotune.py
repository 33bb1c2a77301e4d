"""Autotuner for the recursion cutoff, the product-kernel threshold and the
branch threshold.

The decomposition's result never depends on these knobs (the split points of
the recursion are fixed at floor(m/2), floor(n/2); the leaf and the products
are exact; PLUQ(F) and PLUQ(G) are independent), only its speed does.  For a
workload class (size rounded to a power of two, number of limbs of p, dense
or rank-deficient) the tuner times `pluq_mod_p` on a seeded synthetic matrix
of that class, one knob at a time from the defaults (leaf size, then
small-product threshold, the size above which PLUQ(G) runs on another host
thread, whether zero tests below rank-deficient nodes are awaited or read
lazily, the right- or left-looking base case, whether a node kernel (a small
node below a rank-deficient one in one launch) runs as one thread block or a
cluster of two, four or eight, then how many levels it covers), and caches
the fastest setting in a JSON file.  `apply()` looks
the class up and sets the library's process-wide knobs.
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
BRANCH = (32, 64, 128, 1 << 40)          # 2^40: never hand G to another thread
LAZY_ZERO = (0, 1)
LEAF_LEFT = (0, 1)                       # base case right- / left-looking
NODE = (1, 2, 0)                         # device-side levels of small deficient nodes
NODE_CTAS = (1, 2, 4, 8)                 # thread blocks of a node kernel
DEFAULT = (128, 1 << 25, 64, 0, 0, 1, 1)
KNOBS = (LEAVES, SMALL_MM, BRANCH, LAZY_ZERO, LEAF_LEFT, NODE, NODE_CTAS)
ORDER = (0, 1, 2, 3, 4, 6, 5)            # the cluster size before the node levels: a
                                         # larger cluster makes deeper node kernels pay
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
         cache: str = DEFAULT_CACHE, budget_s: float = 60.0, force: bool = False):
    """Time the candidates on one sample of the class, one knob at a time, and
    cache the best; a class already in the cache is returned as cached unless
    `force`.  Returns (leaf, small_mm_macs, branch_min, lazy_zero, leaf_left, node,
    node_ctas, ms)."""
    key = _class_key(m, n, p, deficient)
    if not force:
        ent = _load(cache).get(key)
        if ent and "node_ctas" in ent:
            return (int(ent["leaf"]), int(ent["small_mm_macs"]), int(ent["branch_min"]),
                    int(ent["lazy_zero"]), int(ent["leaf_left"]), int(ent["node"]),
                    int(ent["node_ctas"]), ent["ms"])
    A0 = _sample(m, n, p, deficient)
    ws = torch.empty(pluq.pluq_workspace_size(m, n, p), dtype=torch.uint8, device="cuda")
    old = pluq.pluq_get_tuning()
    old_branch = pluq.pluq_get_branch_min()
    old_lazy = pluq.pluq_get_lazy_zero_test()
    old_left = pluq.pluq_get_leaf_variant()
    old_node = pluq.pluq_get_node_kernel()
    old_ctas = pluq.pluq_get_node_cluster()
    t_start = time.perf_counter()

    def run(cand):
        pluq.pluq_set_tuning(cand[0], cand[1])
        pluq.pluq_set_branch_min(cand[2])
        pluq.pluq_set_lazy_zero_test(bool(cand[3]))
        pluq.pluq_set_leaf_variant(bool(cand[4]))
        pluq.pluq_set_node_kernel(int(cand[5]))
        pluq.pluq_set_node_cluster(int(cand[6]))
        times = []
        for _ in range(reps + 1):
            A = A0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pluq.pluq_mod_p(A, p, workspace=ws)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        return 1e3 * min(times[1:])

    try:
        best = DEFAULT
        best_ms = run(best)
        for knob in ORDER:
            for v in KNOBS[knob]:
                if time.perf_counter() - t_start > budget_s:
                    break
                cand = tuple(v if i == knob else best[i] for i in range(len(KNOBS)))
                if cand == best:
                    continue
                ms = run(cand)
                if ms < best_ms:
                    best, best_ms = cand, ms
    finally:
        pluq.pluq_set_tuning(*old)
        pluq.pluq_set_branch_min(old_branch)
        pluq.pluq_set_lazy_zero_test(old_lazy)
        pluq.pluq_set_leaf_variant(old_left)
        pluq.pluq_set_node_kernel(old_node)
        pluq.pluq_set_node_cluster(old_ctas)
    data = _load(cache)
    data[key] = {"leaf": best[0], "small_mm_macs": best[1], "branch_min": best[2],
                 "lazy_zero": best[3], "leaf_left": best[4], "node": best[5],
                 "node_ctas": best[6], "ms": best_ms}
    _store(cache, data)
    return best[0], best[1], best[2], best[3], best[4], best[5], best[6], best_ms


def apply(m: int, n: int, p: int, deficient: bool = False, cache: str = DEFAULT_CACHE) -> bool:
    """Set the library's knobs from the cache; False if the class is unknown."""
    ent = _load(cache).get(_class_key(m, n, p, deficient))
    if not ent:
        return False
    pluq.pluq_set_tuning(int(ent["leaf"]), int(ent["small_mm_macs"]))
    if "branch_min" in ent:
        pluq.pluq_set_branch_min(int(ent["branch_min"]))
    if "lazy_zero" in ent:
        pluq.pluq_set_lazy_zero_test(bool(ent["lazy_zero"]))
    if "leaf_left" in ent:
        pluq.pluq_set_leaf_variant(bool(ent["leaf_left"]))
    if "node" in ent:
        pluq.pluq_set_node_kernel(int(ent["node"]))
    if "node_ctas" in ent:
        pluq.pluq_set_node_cluster(int(ent["node_ctas"]))
    return True
