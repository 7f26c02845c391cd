"""Parity at the two large workload sizes, checked on sampled outputs.

* 8e6 particles of a truncated Plummer sphere, Yukawa (kappa 0.5), theta 0.8, n 8, leaf and
  batch size autotuned over {500, 1000, 2000, 3000, 4000}: tree and lists bit-exact with the
  oracle at full size, the FP64 path against the oracle's Algorithm 1 on sampled batches,
  mixed against FP64 over all targets, and both against the direct sum on seeded targets
  (the error is sampled at a random subset of targets for large N, Sec. IV).
* 2.56e8 uniform particles, Coulomb, theta 0.8, n 10: the mixed treecode against the oracle's
  own direct sum on 64 seeded targets and against the GPU FP64 direct sum on 2048; tree and
  lists bit-exact with the oracle at full size; mixed against the FP64 treecode on six
  sampled batches; and determinism of a repeated solve.
"""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import (FP64_ELEM, FP64_REL2, MIXED_REL2, assert_close_abs, batch_targets, dev,
                         host, system)

pytestmark = pytest.mark.gpu


def _solve(gpu, X, p):
    import torch
    phi = torch.empty_like(X[0])
    b.bltc_solve(gpu.h, *X, p, phi)
    torch.cuda.synchronize()
    return host(phi)


def _direct_gpu(gpu, X, idx, p64):
    import torch
    T = [t.index_select(0, torch.from_numpy(idx).cuda()).contiguous() for t in X[:3]]
    ref = torch.empty_like(T[0])
    b.bltc_direct_sum(gpu.h, *T, *X[:3], X[3], p64, ref)
    torch.cuda.synchronize()
    return host(ref)


def test_plummer_8e6_yukawa_autotuned(gpu):
    n = 8_000_000
    x, y, z, q = system("plummer", n, 20031836 + 3)
    X = dev(x, y, z, q)
    p = b.params(8, 0.8, 2000, 2000, b.BLTC_KERNEL_YUKAWA, 0.5, b.BLTC_PRECISION_MIXED)
    best, ms = b.bltc_autotune(gpu.h, *X, p, leaf=(500, 1000, 2000, 3000, 4000), repeats=1)
    assert best.leaf_size in (500, 1000, 2000, 3000, 4000) and best.batch_size == best.leaf_size
    timed = {k: v for k, v in ms.items() if v == v}      # the screen's contenders
    if timed:
        assert ms[(best.leaf_size, best.batch_size)] == min(timed.values())
    again, _ = b.bltc_autotune(gpu.h, *X, p)          # cached: no timing
    assert again.leaf_size == best.leaf_size
    leaf = best.leaf_size

    # tree and lists, bit-exact at full size
    h = b.bltc_tree_build(gpu.h, *X, leaf)
    ot = oracle.Tree(x, y, z, leaf)
    try:
        gt = b.bltc_tree_export(gpu.h, h)
        for k in ("perm", "begin", "count", "parent", "n_children", "children"):
            assert np.array_equal(getattr(ot, k), gt[k].astype(getattr(ot, k).dtype)), k
        for k in ("lo", "hi", "center", "radius"):
            assert np.array_equal(getattr(ot, k).view(np.int64), gt[k].view(np.int64)), k
        L = b.bltc_lists_build(gpu.h, h, h, best)
        got = b.bltc_lists_export(gpu.h, L)
        b.bltc_lists_destroy(L)
        want = oracle.lists(ot, ot, 0.8, 8)
        for k in want:
            assert np.array_equal(want[k], got[k]), k
    finally:
        b.bltc_tree_destroy(h)

    p64 = b.params(8, 0.8, leaf, leaf, b.BLTC_KERNEL_YUKAWA, 0.5, b.BLTC_PRECISION_FP64)
    got64 = _solve(gpu, X, p64)
    gotmx = _solve(gpu, X, best)
    assert oracle.rel_err(got64, gotmx) <= MIXED_REL2

    nl = len(ot.leaves)
    pick = np.array([0, nl // 3, (2 * nl) // 3, nl - 1])
    want, want_abs, _ = oracle.bltc(x, y, z, q, 0.8, 8, leaf, leaf, oracle.KERNEL_YUKAWA, 0.5,
                                    batches=pick, with_abs=True)
    idx = batch_targets(ot, pick)
    assert_close_abs(want[idx], got64[idx], want_abs[idx], FP64_REL2, FP64_ELEM, "8e6 fp64 sampled")

    rng = np.random.default_rng(20031839)
    tidx = np.sort(rng.choice(n, 10000, replace=False))
    ref = _direct_gpu(gpu, X, tidx, p64)
    e64, emx = oracle.rel_err(ref, got64[tidx]), oracle.rel_err(ref, gotmx[tidx])
    # the treecode's own approximation error at theta 0.8, n 8 (Sec. IV: 5-6 digits)
    assert 1e-9 < e64 < 1e-4 and abs(emx - e64) <= 2e-6, (e64, emx)


def test_uniform_2_56e8_sampled(gpu):
    import torch
    n = 256_000_000
    x, y, z, q = system("cube", n, 20031836 + 5)
    X = dev(x, y, z, q)
    p = b.params(10, 0.8, 2000, 2000, b.BLTC_KERNEL_COULOMB, 0.0, b.BLTC_PRECISION_MIXED)
    phi = _solve(gpu, X, p)
    assert np.all(np.isfinite(phi))
    rng = np.random.default_rng(20031841)
    # oracle direct sum on 64 targets (CPU, all host cores)
    t64 = np.sort(rng.choice(n, 64, replace=False))
    ref_cpu = oracle.direct_sum([x[t64], y[t64], z[t64]], [x, y, z], q)
    e_cpu = oracle.rel_err(ref_cpu, phi[t64])
    # GPU FP64 direct sum on 2048 targets, checked itself against the oracle on the 64
    t2k = np.sort(rng.choice(n, 2048, replace=False))
    t2k[:64] = t64
    t2k = np.sort(t2k)
    ref_gpu = _direct_gpu(gpu, X, t2k, b.params(10, 0.8, 2000, precision=b.BLTC_PRECISION_FP64))
    pos = np.searchsorted(t2k, t64)
    assert oracle.rel_err(ref_cpu, ref_gpu[pos]) < 1e-12
    e_gpu = oracle.rel_err(ref_gpu, phi[t2k])
    assert e_cpu < 1e-5 and e_gpu < 1e-5, (e_cpu, e_gpu)
    # tree and lists bit-exact with the oracle at full size, and the mixed treecode within
    # the mixed bar of the FP64 treecode on sampled batches (the FP64 solve of the whole system
    # would take minutes at this size)
    st = b.bltc_tree_build(gpu.h, *X, 2000)
    try:
        ot = oracle.Tree(x, y, z, 2000)
        gt = b.bltc_tree_export(gpu.h, st)
        for k in ("perm", "begin", "count", "parent", "n_children", "children"):
            assert np.array_equal(getattr(ot, k), gt[k].astype(getattr(ot, k).dtype)), k
        for k in ("lo", "hi", "center", "radius"):
            assert np.array_equal(getattr(ot, k).view(np.int64), gt[k].view(np.int64)), k
        del gt
        p64 = b.params(10, 0.8, 2000, 2000, precision=b.BLTC_PRECISION_FP64)
        L = b.bltc_lists_build(gpu.h, st, st, p64)
        got = b.bltc_lists_export(gpu.h, L)
        want = oracle.lists(ot, ot, 0.8, 10)
        for k in want:
            assert np.array_equal(want[k], got[k]), k
        del got, want
        nl = len(ot.leaves)
        pick = np.sort(np.random.default_rng(20031843).choice(nl, 6, replace=False)).astype(np.int32)
        S = b.bltc_lists_select(gpu.h, L, pick)
        b.bltc_modified_charges(gpu.h, st, S, p64)
        phi64 = torch.empty_like(X[0])
        b.bltc_evaluate(gpu.h, S, st, st, p64, phi64)
        torch.cuda.synchronize()
        b.bltc_lists_destroy(S)
        b.bltc_lists_destroy(L)
        idx = batch_targets(ot, pick)
        got64 = host(phi64)[idx]
        assert oracle.rel_err(got64, phi[idx]) <= MIXED_REL2
        # against the oracle's direct sum on 32 of those targets: the treecode's own error
        sub = idx[::max(1, len(idx) // 32)][:32]
        ref_sub = oracle.direct_sum([x[sub], y[sub], z[sub]], [x, y, z], q)
        assert oracle.rel_err(ref_sub, host(phi64)[sub]) < 1e-5
    finally:
        b.bltc_tree_destroy(st)
    # determinism of a repeated solve
    del X
    torch.cuda.empty_cache()
    X = dev(x, y, z, q)
    assert np.array_equal(_solve(gpu, X, p), phi)
