"""The C-ABI library builds, loads and exports every function include/pluq.h
declares (no GPU needed: no compute calls here)."""
import ctypes
import os
import re

from paper_1301_4438_gb300 import _build, pluq

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = []
    for fn in sorted(os.listdir(HEADER)):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(HEADER, fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "sizeof"):
                names.append(name)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("pluq_mod_p", "row_rank_profile", "col_rank_profile", "rank_profile_matrix",
                 "pluq_workspace_size", "pluq_status_string", "pluq_modmm",
                 "pluq_trsm_left_lower_unit", "pluq_trsm_right_upper", "pluq_perm_rows",
                 "pluq_perm_cols", "pluq_leaf"):
        assert must in names, must


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding covers every declared entry point with the same name
    assert set(declared_functions()) <= set(pluq.exported_symbols())


def test_host_only_queries():
    lib = pluq.load()
    assert lib.pluq_tensor_limbs(65521) == 2
    assert lib.pluq_tensor_limbs(8388593) == 3
    assert lib.pluq_tensor_limbs(2147483647) == 4
    assert lib.pluq_tensor_limbs(251) == 1
    assert pluq.status_string(-3) == "matrix entry not reduced modulo p"
    assert pluq.pluq_workspace_size(256, 256, 65521) > 256 * 256 * 4
    import pytest
    with pytest.raises(pluq.PluqError):
        pluq.pluq_workspace_size(10, 10, 65535)     # not prime


def test_modulus_validation_matches_trial_division():
    """The library's primality test (Miller-Rabin, bases 2, 7, 61) against
    trial division: small numbers, Carmichael numbers, strong pseudoprimes to
    small bases and the neighbourhood of 2^31."""
    import pytest

    def trial(n):
        if n < 2:
            return False
        d = 2
        while d * d <= n:
            if n % d == 0:
                return False
            d += 1
        return True

    cases = list(range(0, 2000)) + [561, 1105, 1729, 2465, 2821, 6601, 8911, 25326001,
                                     3215031751 % (1 << 31), 2047, 1373653, 9080191,
                                     4759123141 % (1 << 31), 65521, 65535, 65537, 8388593,
                                     8388607] + list(range((1 << 31) - 300, 1 << 31))
    for n in cases:
        if trial(n):
            assert pluq.pluq_workspace_size(4, 4, n) > 0, n
        else:
            with pytest.raises(pluq.PluqError):
                pluq.pluq_workspace_size(4, 4, n)


def test_uses_reject_bad_arguments_on_the_host():
    """The determinant / nullspace / solve entry points and their workspace
    query validate sizes, pointers and the modulus before any device work, so
    these calls need no GPU (the matrix pointer is never dereferenced)."""
    import ctypes
    lib = pluq.load()
    out = ctypes.c_size_t(0)
    ok, einval, enotprime = 0, -1, -2
    assert lib.pluq_uses_workspace_size(10, 8, 9, 0, 65521, 0, ctypes.byref(out)) == einval  # r > n
    assert lib.pluq_uses_workspace_size(10, 8, 4, -1, 65521, 0, ctypes.byref(out)) == einval  # k < 0
    assert lib.pluq_uses_workspace_size(10, 8, 4, 0, 65521, 7, ctypes.byref(out)) == einval   # kind
    assert lib.pluq_uses_workspace_size(10, 8, 4, 0, 65535, 0, ctypes.byref(out)) == enotprime
    assert lib.pluq_uses_workspace_size(10, 8, 4, 3, 65521, 0, ctypes.byref(out)) == ok
    small = out.value
    assert lib.pluq_uses_workspace_size(10, 8, 4, 300, 65521, 0, ctypes.byref(out)) == ok
    assert out.value >= small > 0
    fake = 4096                                   # never dereferenced: the calls stop first
    assert lib.pluq_determinant(fake, 4, 3, 4, fake, fake, 65521, fake, None, 0, None) == einval
    assert lib.pluq_determinant(fake, 4, 4, 4, fake, fake, 65521, None, None, 0, None) == einval
    assert lib.pluq_determinant(fake, 4, 4, 4, fake, fake, 65535, fake, None, 0, None) == enotprime
    assert lib.pluq_right_nullspace(fake, 4, 4, 4, 5, fake, 65521, fake, 1, 0, None, 0,
                                    None) == einval                                       # r > n
    assert lib.pluq_left_nullspace(fake, 4, 4, 4, 1, fake, 65535, fake, 4, 0, None, 0,
                                   None) == enotprime
    assert lib.pluq_left_nullspace(fake, 4, 4, 4, 1, fake, 65521, fake, 3, 0, None, 0,
                                   None) == einval                                        # ldk < m
    assert lib.pluq_solve(fake, 4, 4, 4, 2, fake, fake, 65521, fake, 4, -1, fake, 4, fake, 0,
                          None, 0, None) == einval                                        # k < 0
    assert lib.pluq_solve(fake, 4, 4, 4, 2, fake, fake, 65521, fake, 4, 2, fake, 4, None, 0,
                          None, 0, None) == einval                                        # no flag


def test_core_entry_points_reject_bad_arguments_on_the_host():
    """The decomposition, its batched form, the read-outs and the kernel-level
    calls check sizes, strides, pointers, the product form and the modulus
    before any device work (the device pointers below are never
    dereferenced), and report the statuses the header documents."""
    import ctypes
    lib = pluq.load()
    ok, einval, enotprime, enomem = 0, -1, -2, -4
    fake = 4096
    rank = ctypes.c_int64(-1)
    out = ctypes.c_size_t(0)
    # pluq_workspace_size / pluq_mod_p (Algorithm 1)
    assert lib.pluq_workspace_size(-1, 4, 65521, ctypes.byref(out)) == einval
    assert lib.pluq_workspace_size(4, 4, 65521, None) == einval
    assert lib.pluq_workspace_size(4, 4, 1, ctypes.byref(out)) == enotprime
    assert lib.pluq_workspace_size(4, 4, 2147483648 - 1, ctypes.byref(out)) == ok
    need = out.value
    mod_p = lib.pluq_mod_p
    assert mod_p(fake, 4, 4, 4, 65521, fake, fake, None, fake, need, 0, None) == einval   # no rank
    assert mod_p(fake, -1, 4, 4, 65521, fake, fake, ctypes.byref(rank), fake, need, 0, None) == einval
    assert mod_p(fake, 4, 4, 3, 65521, fake, fake, ctypes.byref(rank), fake, need, 0, None) == einval
    assert mod_p(None, 4, 4, 4, 65521, fake, fake, ctypes.byref(rank), fake, need, 0, None) == einval
    assert mod_p(fake, 4, 4, 4, 65521, None, fake, ctypes.byref(rank), fake, need, 0, None) == einval
    assert mod_p(fake, 4, 4, 4, 65521, fake, fake, ctypes.byref(rank), fake, need, 3, None) == einval
    assert mod_p(fake, 4, 4, 4, 65535, fake, fake, ctypes.byref(rank), fake, need, 0, None) == enotprime
    assert lib.pluq_workspace_size(4, 4, 65521, ctypes.byref(out)) == ok
    assert mod_p(fake, 4, 4, 4, 65521, fake, fake, ctypes.byref(rank), fake, out.value - 1, 0,
                 None) == enomem
    assert mod_p(fake, 4, 4, 4, 65521, fake, fake, ctypes.byref(rank), None, out.value, 0,
                 None) == enomem
    # pluq_batched_workspace_size / pluq_mod_p_batched
    I64 = ctypes.c_int64 * 2
    ms, ns = I64(3, 5), I64(4, 2)
    assert lib.pluq_batched_workspace_size(ms, ns, -1, 65521, 2, ctypes.byref(out)) == einval
    assert lib.pluq_batched_workspace_size(ms, ns, 2, 65521, 0, ctypes.byref(out)) == einval
    assert lib.pluq_batched_workspace_size(ms, ns, 2, 9, 2, ctypes.byref(out)) == enotprime
    assert lib.pluq_batched_workspace_size(I64(3, -5), ns, 2, 65521, 2, ctypes.byref(out)) == einval
    assert lib.pluq_batched_workspace_size(ms, ns, 2, 65521, 2, ctypes.byref(out)) == ok
    VP = ctypes.c_void_p * 2
    ptrs = VP(fake, fake)
    ranks = I64()
    batched = lib.pluq_mod_p_batched
    assert batched(ptrs, ms, ns, I64(4, 2), 2, 65521, ptrs, ptrs, ranks, fake, out.value, 0, 0,
                   None) == einval                                                # no workers
    assert batched(ptrs, ms, ns, I64(4, 1), 2, 65521, ptrs, ptrs, ranks, fake, out.value, 0, 2,
                   None) == einval                                                # lda < n
    assert batched(ptrs, ms, ns, I64(4, 2), 2, 65521, ptrs, ptrs, ranks, fake, out.value - 1, 0,
                   2, None) == enomem
    assert batched(ptrs, ms, ns, I64(4, 2), 0, 65521, ptrs, ptrs, ranks, None, 0, 0, 2,
                   None) == ok                                                    # empty batch
    # read-outs (Corollaries of Lemma 2, Sec. 4; Sec. 3)
    assert lib.row_rank_profile(fake, 3, 4, fake, None) == einval                 # r > m
    assert lib.col_rank_profile(fake, 3, -1, fake, None) == einval
    assert lib.rank_profile_matrix(fake, fake, 3, 5, 4, fake, fake, None) == einval
    assert lib.pluq_extract_L(fake, 4, 4, 4, 5, fake, 5, None) == einval         # r > n
    assert lib.pluq_extract_L(fake, 4, 4, 4, 2, fake, 1, None) == einval         # ldl < r
    assert lib.pluq_extract_U(fake, 4, 4, 4, 2, fake, 3, None) == einval         # ldu < n
    assert lib.pluq_leu(fake, 4, 4, 4, 2, fake, fake, None, 4, None, 4, fake, 64,
                        None) == einval                                           # no output
    assert lib.pluq_leu(fake, 4, 4, 4, 2, fake, fake, fake, 4, None, 4, fake, 31,
                        None) == enomem                                           # (m + n) ints
    assert lib.pluq_leading_rank_profiles(fake, fake, 4, 4, 2, 5, 1, fake, fake, fake,
                                          None) == einval                         # k > m
    # kernel-level calls
    assert lib.pluq_modmm(fake, 4, fake, 4, fake, 4, -1, 4, 4, 65521, 0, 0, fake, 0,
                          None) == einval
    assert lib.pluq_modmm(fake, 4, fake, 4, fake, 4, 4, 4, 4, 65521, 0, 5, fake, 0,
                          None) == einval                                         # form
    assert lib.pluq_modmm(fake, 4, fake, 4, fake, 4, 4, 4, 4, 15, 0, 0, fake, 0,
                          None) == enotprime
    assert lib.pluq_modmm(fake, 3, fake, 4, fake, 4, 4, 4, 4, 65521, 0, 0, fake, 0,
                          None) == einval                                         # ldc < N
    assert lib.pluq_trsm_left_lower_unit(fake, 4, fake, 4, 4, 4, 65521, 0, fake, 0,
                                         None) == enomem
    assert lib.pluq_trsm_left_lower_unit(fake, 3, fake, 4, 4, 4, 65521, 0, fake, 1 << 30,
                                         None) == einval                          # ldl < r
    assert lib.pluq_trsm_right_upper(fake, 4, fake, 4, 4, 4, 4, 0, fake, 1 << 30,
                                     None) == enotprime
    assert lib.pluq_perm_rows(fake, 4, -1, 4, fake, fake, 64, None) == einval
    assert lib.pluq_perm_rows(fake, 4, 0, 4, None, None, 0, None) == ok           # nothing moves
    assert lib.pluq_perm_rows(fake, 4, 4, 4, fake, fake, 63, None) == enomem
    assert lib.pluq_perm_cols(fake, 3, 4, 4, fake, fake, 1 << 20, None) == einval  # ldx < count
    assert lib.pluq_leaf(fake, 129, 4, 4, 65521, fake, fake, fake, None) == einval  # > base case
    assert lib.pluq_leaf(fake, 4, 4, 4, 65535, fake, fake, fake, None) == enotprime
    # process-wide knobs: accepted values round-trip, others are refused
    lf, sm = ctypes.c_int64(0), ctypes.c_int64(0)
    assert lib.pluq_get_tuning(ctypes.byref(lf), ctypes.byref(sm)) == ok
    assert lib.pluq_set_tuning(8, 0) == einval and lib.pluq_set_tuning(256, 0) == einval
    assert lib.pluq_set_tuning(64, 1 << 20) == ok
    l2, s2 = ctypes.c_int64(0), ctypes.c_int64(0)
    assert lib.pluq_get_tuning(ctypes.byref(l2), ctypes.byref(s2)) == ok and (l2.value, s2.value) == (64, 1 << 20)
    assert lib.pluq_set_tuning(lf.value, sm.value) == ok
    assert lib.pluq_set_node_cluster(3) == einval and lib.pluq_set_node_kernel(3) == einval
    assert lib.pluq_set_leaf_variant(2) == einval and lib.pluq_set_lazy_zero_test(-1) == einval
    assert lib.pluq_set_branch_min(0) == einval
    old = lib.pluq_get_node_cluster()
    assert lib.pluq_set_node_cluster(8) == ok and lib.pluq_get_node_cluster() == 8
    assert lib.pluq_set_node_cluster(old) == ok


def test_persistent_batch_rejects_bad_arguments_on_the_host():
    """The persistent batch entry point and its workspace query check sizes,
    the modulus, the argument arrays and the workspace before any device work
    (the device arrays are never dereferenced here)."""
    import ctypes
    lib = pluq.load()
    out = ctypes.c_size_t(0)
    ok, einval, enotprime, enomem = 0, -1, -2, -4
    f = lib.pluq_batched_persistent_workspace_size
    assert f(2049, 10, 4, ctypes.byref(out)) == einval     # beyond sixteen base-case blocks
    assert f(10, -1, 4, ctypes.byref(out)) == einval
    assert f(10, 10, -1, ctypes.byref(out)) == einval      # ctas < 0
    assert f(2048, 2048, 4, ctypes.byref(out)) == ok
    big = out.value
    assert big >= 4 * (2048 * 2048 + 1025 * 1025) * 4      # four blocks' stage and copy of I
    assert f(100, 30, 4, ctypes.byref(out)) == ok and 0 < out.value < big
    need = out.value
    fake = 4096
    run = lib.pluq_mod_p_batched_persistent
    assert run(fake, fake, fake, fake, -1, 100, 30, 65521, fake, fake, fake, fake, need, 4,
               None) == einval                                                 # count < 0
    assert run(fake, fake, fake, fake, 3, 2049, 30, 65521, fake, fake, fake, fake, need, 4,
               None) == einval                                                 # max_m
    assert run(fake, fake, fake, fake, 3, 100, 30, 65535, fake, fake, fake, fake, need, 4,
               None) == enotprime
    assert run(fake, None, fake, fake, 3, 100, 30, 65521, fake, fake, fake, fake, need, 4,
               None) == einval                                                 # no m array
    assert run(fake, fake, fake, fake, 3, 100, 30, 65521, fake, fake, fake, fake, need - 1, 4,
               None) == enomem
    assert run(fake, fake, fake, fake, 3, 100, 30, 65521, fake, fake, fake, fake + 4, need, 4,
               None) == einval                                                 # misaligned
    assert run(fake, fake, fake, fake, 0, 100, 30, 65521, fake, fake, fake, None, 0, 4,
               None) == ok                                                     # empty batch


def test_autotune_cache_lookup_on_the_host(tmp_path):
    """Workload classes round sizes up to powers of two and separate limb
    counts and dense / deficient inputs; apply() sets the library's knobs
    from the cache and leaves them alone for an unknown class."""
    import json
    from paper_1301_4438_gb300 import autotune
    assert autotune._class_key(4096, 4096, 65521, False) == "4096x4096:L2:full"
    assert autotune._class_key(3000, 5000, 2147483647, True) == "4096x8192:L4:def"
    assert autotune._class_key(1, 1, 251, False) == "1x1:L1:full"
    cache = tmp_path / "tuning.json"
    cache.write_text(json.dumps({"256x256:L2:def": {"leaf": 64, "small_mm_macs": 1 << 25,
                                                    "ms": 1.0}}))
    old = pluq.pluq_get_tuning()
    try:
        assert autotune.apply(200, 256, 65521, deficient=True, cache=str(cache))
        assert pluq.pluq_get_tuning() == (64, 1 << 25)
        assert not autotune.apply(200, 256, 65521, deficient=False, cache=str(cache))
        assert pluq.pluq_get_tuning() == (64, 1 << 25)
    finally:
        pluq.pluq_set_tuning(*old)
