"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: the tree and the interaction lists are bit-identical to the oracle's; the FP64 GPU
treecode matches the oracle's Algorithm 1 to relative 2-norm 1e-12 (per target 1e-12 of the
absolute-value sum of its terms); the mixed-precision path matches the FP64 GPU path to
relative 2-norm 1e-6.  Sizes span several work tiles and ragged tails; the full-size
workload (1e6 particles, theta 0.7, n 8, N_L = N_B = 2000) is checked on sampled batches.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import (FP64_ELEM, FP64_REL2, MIXED_ELEM, MIXED_REL2, assert_close_abs,
                         batch_targets, dev, gpu_solve, gpu_tree, host, system)

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

TREE_KEYS = ("perm", "begin", "count", "parent", "level", "n_children", "children", "lo", "hi",
             "center", "radius")


def _compare_trees(ot: oracle.Tree, gt: dict):
    for k in TREE_KEYS:
        a, g = getattr(ot, k), gt[k]
        assert a.shape == g.shape, k
        if a.dtype.kind == "f":
            assert np.array_equal(a.view(np.int64), g.view(np.int64)), f"{k} differs bitwise"
        else:
            assert np.array_equal(a, g.astype(a.dtype)), f"{k} differs"


# ---- A0: tree -----------------------------------------------------------------------------

def _golden_cases():
    with open(os.path.join(GOLDEN, "trees_small.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_tree_golden_bit_exact(gpu, case):
    x, y, z = (np.array(case[k], dtype=np.float64) for k in ("x", "y", "z"))
    h, _ = gpu_tree(gpu, x, y, z, None, case["max_leaf"])
    try:
        gt = b.bltc_tree_export(gpu.h, h)
        assert gt["perm"].tolist() == case["perm"]
        _compare_trees(oracle.Tree(x, y, z, case["max_leaf"]), gt)
    finally:
        b.bltc_tree_destroy(h)


@pytest.mark.parametrize("kind,n,leaf", [("cube", 1, 1), ("cube", 7, 2), ("cube", 10000, 500),
                                          ("cube", 30001, 2000), ("plummer", 20000, 100),
                                          ("cube", 4099, 1), ("plummer", 50000, 3000)])
def test_tree_bit_exact(gpu, kind, n, leaf):
    x, y, z, q = system(kind, n, 1000 + n)
    h, _ = gpu_tree(gpu, x, y, z, q, leaf)
    try:
        _compare_trees(oracle.Tree(x, y, z, leaf), b.bltc_tree_export(gpu.h, h))
    finally:
        b.bltc_tree_destroy(h)


def test_tree_degenerate_inputs_bit_exact(gpu):
    rng = np.random.default_rng(3)
    # duplicates, a lattice (many exact midpoint hits), signed zeros, adjacent doubles
    lat = np.array(np.meshgrid(np.arange(8.0), np.arange(8.0), np.arange(4.0))).reshape(3, -1)
    cases = [
        (np.repeat(rng.uniform(-1, 1, (3, 50)), 7, axis=1), 4),
        (lat, 3),
        (np.stack([np.array([0.0, -0.0] * 40), rng.uniform(-1, 1, 80), np.zeros(80)]), 5),
        (np.stack([1.0 + np.arange(64) * 2.0 ** -52, np.zeros(64), np.zeros(64)]), 3),
    ]
    for pts, leaf in cases:
        h, _ = gpu_tree(gpu, pts[0], pts[1], pts[2], None, leaf)
        try:
            _compare_trees(oracle.Tree(pts[0], pts[1], pts[2], leaf), b.bltc_tree_export(gpu.h, h))
        finally:
            b.bltc_tree_destroy(h)


def test_tree_rejects_non_finite(gpu):
    x, y, z, q = system("cube", 100, 1)
    y[17] = np.nan
    with pytest.raises(b.BltcError) as e:
        gpu_tree(gpu, x, y, z, q, 10)
    assert e.value.status == b.BLTC_ERR_ARG
    x, y, z, q = system("cube", 100, 1)
    q[3] = np.inf
    with pytest.raises(b.BltcError):
        gpu_tree(gpu, x, y, z, q, 10)


# ---- A1: lists ----------------------------------------------------------------------------

@pytest.mark.parametrize("n,leaf,batch,theta,deg", [(10000, 500, 500, 0.7, 4),
                                                     (30001, 2000, 2000, 0.7, 8),
                                                     (20000, 300, 700, 0.5, 3),
                                                     (20000, 64, 64, 0.9, 1),
                                                     (5000, 100, 100, 0.0, 4)])
def test_lists_bit_exact(gpu, n, leaf, batch, theta, deg):
    x, y, z, q = system("cube", n, 7 * n)
    st, _ = gpu_tree(gpu, x, y, z, q, leaf)
    bt, _ = gpu_tree(gpu, x, y, z, None, batch) if batch != leaf else (st, None)
    try:
        p = b.params(deg, theta, leaf, batch)
        L = b.bltc_lists_build(gpu.h, bt, st, p)
        got = b.bltc_lists_export(gpu.h, L)
        b.bltc_lists_destroy(L)
        ost, obt = oracle.Tree(x, y, z, leaf), oracle.Tree(x, y, z, batch)
        want = oracle.lists(obt, ost, theta, deg)
        for k in ("approx_off", "approx_ids", "direct_off", "direct_ids"):
            assert np.array_equal(want[k], got[k]), k
    finally:
        b.bltc_tree_destroy(st)
        if bt != st:
            b.bltc_tree_destroy(bt)


def test_lists_plummer_bit_exact(gpu):
    x, y, z, q = system("plummer", 40000, 11)
    st, _ = gpu_tree(gpu, x, y, z, q, 400)
    try:
        L = b.bltc_lists_build(gpu.h, st, st, b.params(6, 0.8, 400))
        got = b.bltc_lists_export(gpu.h, L)
        b.bltc_lists_destroy(L)
        ot = oracle.Tree(x, y, z, 400)
        want = oracle.lists(ot, ot, 0.8, 6)
        for k in want:
            assert np.array_equal(want[k], got[k]), k
    finally:
        b.bltc_tree_destroy(st)


# ---- A2: modified charges -----------------------------------------------------------------

def _mixed_qhat_bar(deg):
    """Worst-case error of a leaf's mixed-precision modified charge, relative to sum |q_j|.

    FP64 differs from the oracle only in summation order and the factor formula (1e-13).
    In the mixed leaf sums each term q_j a1[k1] a2[k2] a3[k3] carries at most 26 unit
    roundoffs u = 2^-24: per factor 2 for y - s_k from FP32 (hi, lo) pairs, 2 for the SFU
    reciprocal, 1 for the compensated denominator, 1 for its last addition, 1 for the
    division, 1 for the scaling (and 1 for q in FP32 in the first factor), plus 1 for
    a1 a2.  Each thread then adds its terms in FP32 runs of m = ceil(128 / G) terms (a
    128-particle tile shared by G = max(1, 512 // (n+1)^2) groups) before a compensated
    fold, adding (m - 1) u.  The terms are bounded by |q_j| max|L_k|^3, and max |L_k| on
    Chebyshev points of the second kind is below 1.031 for n <= 16 (a CPU pin).  A
    parent's charges are its children's, moved by the FP64 transfers of Eq. 12's linearity;
    its sum |q| is the sum of theirs, and its measured error is below its leaves' (at most
    3e-9 of sum |q| at the leaves, 6e-10 at the parents, for n = 1..16), so the leaves' bound
    is the bar for every cluster."""
    groups = max(1, 512 // (deg + 1) ** 2)
    m = -(-128 // groups)
    return (26 + m) * 2.0 ** -24 * 1.031 ** 3


@pytest.mark.parametrize("deg", [1, 4, 8, 16])
def test_modified_charges(gpu, deg):
    # Every cluster with more than (n+1)^3 particles gets modified charges; so do its
    # descendants (the upward pass builds a parent from its children), and every value the
    # library holds must equal Eq. 12 summed directly over the cluster's particles.
    n, leaf = (30000, 600) if deg < 16 else (60000, 6000)
    x, y, z, q = system("cube", n, 5 + deg)
    st, _ = gpu_tree(gpu, x, y, z, q, leaf)
    try:
        ot = oracle.Tree(x, y, z, leaf)
        want = oracle.modified_charges(ot, q, deg)
        P = (deg + 1) ** 3
        scale = np.array([np.abs(q[ot.perm[ot.begin[v]:ot.begin[v] + ot.count[v]]]).sum()
                          for v in range(ot.n_nodes)])
        has = ot.count > P
        expect = has.copy()
        for v in range(ot.n_nodes):          # DFS pre-order: parents come first
            if ot.parent[v] >= 0 and expect[ot.parent[v]]:
                expect[v] = True
        for prec, tol in ((b.BLTC_PRECISION_FP64, 1e-13), (b.BLTC_PRECISION_MIXED, _mixed_qhat_bar(deg))):
            b.bltc_modified_charges(gpu.h, st, None, b.params(deg, 0.7, leaf, precision=prec))
            got = b.bltc_modified_charges_export(gpu.h, st, deg)
            assert not np.any(np.isnan(got[expect])) and np.all(np.isnan(got[~expect]))
            err = np.abs(got[expect] - want[expect]).max(axis=1) / scale[expect]
            assert err.max() <= tol, (prec, err.max())
    finally:
        b.bltc_tree_destroy(st)


def test_modified_charges_exact_hit_corner(gpu):
    # particles on the box corners hit s_0 / s_n exactly (Sec. II-C)
    x = np.array([0.0, 1.0] * 40 + [0.5])
    y = np.array([0.0, 1.0] * 40 + [0.25])
    z = np.array([0.0, 1.0] * 40 + [0.75])
    q = np.linspace(-1, 1, 81)
    st, _ = gpu_tree(gpu, x, y, z, q, 1000)
    try:
        b.bltc_modified_charges(gpu.h, st, None, b.params(3, 0.7, 1000, precision=b.BLTC_PRECISION_FP64))
        got = b.bltc_modified_charges_export(gpu.h, st, 3)
        ot = oracle.Tree(x, y, z, 1000)
        want = oracle.modified_charges(ot, q, 3)
        assert np.allclose(got[0], want[0], rtol=0, atol=1e-14)
    finally:
        b.bltc_tree_destroy(st)


# ---- A3-A5: the whole treecode ------------------------------------------------------------

def _oracle(x, y, z, q, p, batches=None):
    phi, phi_abs, _ = oracle.bltc(x, y, z, q, p.theta, p.degree, p.leaf_size, p.batch_size,
                                  p.kernel, p.kappa, batches=batches, with_abs=True)
    return phi, phi_abs


CASES = [
    # kind, n, leaf, batch, theta, degree, kernel, kappa
    ("cube", 10000, 500, 500, 0.7, 4, 0, 0.0),        # the small configuration
    ("cube", 10000, 500, 500, 0.7, 4, 1, 0.5),
    ("cube", 30001, 2000, 2000, 0.7, 8, 0, 0.0),      # several 2048-target tiles, ragged
    ("cube", 20011, 700, 300, 0.6, 5, 1, 0.25),       # batch tree != source tree
    ("plummer", 40000, 400, 400, 0.8, 6, 1, 0.5),     # uneven tree
    ("cube", 50000, 3000, 3000, 0.7, 2, 0, 0.0),      # > 2048 targets and sources per tile
    ("cube", 3001, 64, 64, 0.9, 1, 0, 0.0),           # degree 1
    ("cube", 10000, 1500, 1500, 0.7, 5, 0, 0.0),      # batches of 1100-1500: several passes of
    ("plummer", 20000, 1500, 1500, 0.8, 4, 1, 0.3),   # 256 or 512 targets (4 or 8 source groups)
    ("cube", 7, 2, 2, 0.5, 3, 0, 0.0),                # tiny
    ("cube", 1, 1, 1, 0.7, 4, 1, 0.5),                # a single particle: phi = 0
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}-L{c[2]}-B{c[3]}-t{c[4]}-n{c[5]}-k{c[6]}")
def test_bltc_fp64_and_mixed(gpu, case):
    kind, n, leaf, batch, theta, deg, ker, kappa = case
    x, y, z, q = system(kind, n, 31 * n + deg)
    p64 = b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_FP64)
    pmx = b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_MIXED)
    want, want_abs = _oracle(x, y, z, q, p64)
    got64 = gpu_solve(gpu, x, y, z, q, p64)
    gotmx = gpu_solve(gpu, x, y, z, q, pmx)
    if n == 1:
        assert got64[0] == 0.0 and gotmx[0] == 0.0
        return
    assert_close_abs(want, got64, want_abs, FP64_REL2, FP64_ELEM, "fp64 vs oracle")
    assert_close_abs(got64, gotmx, want_abs, MIXED_REL2, MIXED_ELEM, "mixed vs fp64")


def test_degree16_sampled(gpu):
    x, y, z, q = system("cube", 100000, 16)
    p64 = b.params(16, 0.6, 6000, 6000, 0, 0.0, b.BLTC_PRECISION_FP64)
    ot = oracle.Tree(x, y, z, 6000)
    pick = np.array([0, len(ot.leaves) // 3, len(ot.leaves) - 1])
    want, want_abs = _oracle(x, y, z, q, p64, pick)
    idx = batch_targets(ot, pick)
    got64 = gpu_solve(gpu, x, y, z, q, p64)
    assert_close_abs(want[idx], got64[idx], want_abs[idx], FP64_REL2, FP64_ELEM, "n=16")
    gotmx = gpu_solve(gpu, x, y, z, q, b.params(16, 0.6, 6000, 6000))
    assert oracle.rel_err(got64, gotmx) <= MIXED_REL2
    assert_close_abs(got64[idx], gotmx[idx], want_abs[idx], MIXED_REL2, MIXED_ELEM, "n=16 mixed")


def test_close_pairs_mixed(gpu):
    # Near-duplicates 1e-7..1e-5 apart: the FP32 batch-relative coordinates cannot resolve
    # them, so the mixed near field must recompute such pairs in FP64.
    rng = np.random.default_rng(4)
    x, y, z, q = system("cube", 200000, 77)
    k = 2000
    pick = rng.choice(len(x), k, replace=False)
    d = rng.normal(size=(3, k))
    d *= (10 ** rng.uniform(-7, -5, k)) / np.linalg.norm(d, axis=0)
    x = np.concatenate([x, x[pick] + d[0]])
    y = np.concatenate([y, y[pick] + d[1]])
    z = np.concatenate([z, z[pick] + d[2]])
    q = np.concatenate([q, rng.uniform(-1, 1, k)])
    got64 = gpu_solve(gpu, x, y, z, q, b.params(6, 0.7, 1000, precision=b.BLTC_PRECISION_FP64))
    gotmx = gpu_solve(gpu, x, y, z, q, b.params(6, 0.7, 1000))
    e = oracle.rel_err(got64, gotmx)
    assert e <= MIXED_REL2, e
    # per target, relative to its own potential (or the rms, where the potential cancels)
    scale = np.maximum(np.abs(got64), np.sqrt(np.mean(got64 ** 2)))
    assert np.max(np.abs(gotmx - got64) / scale) < 2e-5


def test_theta_zero_is_direct_sum(gpu):
    x, y, z, q = system("cube", 6000, 99)
    pts = np.stack([x, y, z])
    ref, ref_abs = oracle.direct_sum(pts, pts, q, with_abs=True)
    got = gpu_solve(gpu, x, y, z, q, b.params(4, 0.0, 300, precision=b.BLTC_PRECISION_FP64))
    assert_close_abs(ref, got, ref_abs, 1e-14, 1e-14, "theta=0")


def test_yukawa_kappa0_equals_coulomb(gpu):
    x, y, z, q = system("cube", 20000, 5)
    for prec in (b.BLTC_PRECISION_FP64, b.BLTC_PRECISION_MIXED):
        c = gpu_solve(gpu, x, y, z, q, b.params(6, 0.7, 800, precision=prec))
        yk = gpu_solve(gpu, x, y, z, q, b.params(6, 0.7, 800, kernel=1, kappa=0.0, precision=prec))
        assert np.array_equal(c, yk)


def test_deterministic_bits(gpu):
    x, y, z, q = system("cube", 40000, 8)
    for prec in (b.BLTC_PRECISION_FP64, b.BLTC_PRECISION_MIXED):
        p = b.params(6, 0.7, 1000, precision=prec)
        assert np.array_equal(gpu_solve(gpu, x, y, z, q, p), gpu_solve(gpu, x, y, z, q, p))


def test_step_api_matches_solve_and_stats(gpu):
    import torch
    x, y, z, q = system("cube", 30000, 4)
    p = b.params(5, 0.7, 1000)
    X = dev(x, y, z, q)
    st = b.bltc_tree_build(gpu.h, *X, 1000)
    L = b.bltc_lists_build(gpu.h, st, st, p)
    b.bltc_modified_charges(gpu.h, st, L, p)
    phi = torch.empty_like(X[0])
    b.bltc_evaluate(gpu.h, L, st, st, p, phi)
    torch.cuda.synchronize()
    assert np.array_equal(host(phi), gpu_solve(gpu, x, y, z, q, p))
    s = b.bltc_stats(gpu.h, L)
    ot = oracle.Tree(x, y, z, 1000)
    lw = oracle.lists(ot, ot, 0.7, 5)
    nb = ot.count[ot.leaves]
    d = sum(nb[i] * ot.count[lw["direct_ids"][lw["direct_off"][i]:lw["direct_off"][i + 1]]].sum()
            for i in range(len(nb)))
    a = sum(nb[i] * (lw["approx_off"][i + 1] - lw["approx_off"][i]) * 216 for i in range(len(nb)))
    assert s == {"direct": d, "approx": a}
    # evaluate without modified charges for this precision is a state error
    with pytest.raises(b.BltcError) as e:
        b.bltc_evaluate(gpu.h, L, st, st, b.params(5, 0.7, 1000, precision=0), phi)
    assert e.value.status == b.BLTC_ERR_STATE
    b.bltc_lists_destroy(L)
    b.bltc_tree_destroy(st)


def test_selected_batches(gpu):
    # The lists of some batches only (the error of Eq. 16 on a sample of targets, Sec. IV):
    # FP64 gives bit for bit the full solve's potentials there and 0 elsewhere, and matches
    # the oracle's Algorithm 1 on the same batches; mixed stays within the mixed bar.
    import torch
    x, y, z, q = system("cube", 30000, 12)
    X = dev(x, y, z, q)
    st = b.bltc_tree_build(gpu.h, *X, 1000)
    ot = oracle.Tree(x, y, z, 1000)
    pick = np.array([0, 5, len(ot.leaves) // 2, len(ot.leaves) - 1])
    idx = batch_targets(ot, pick)
    rest = np.setdiff1d(np.arange(len(x)), idx)
    want, want_abs = _oracle(x, y, z, q, b.params(6, 0.7, 1000, precision=0), pick)
    try:
        for prec in (b.BLTC_PRECISION_FP64, b.BLTC_PRECISION_MIXED):
            p = b.params(6, 0.7, 1000, precision=prec)
            L = b.bltc_lists_build(gpu.h, st, st, p)
            S = b.bltc_lists_select(gpu.h, L, pick)
            info = b.bltc_lists_info(S)
            lw = oracle.lists(ot, ot, 0.7, 6)
            assert info["n_approx"] == sum(lw["approx_off"][i + 1] - lw["approx_off"][i] for i in pick)
            b.bltc_modified_charges(gpu.h, st, S, p)
            phi = torch.empty_like(X[0])
            b.bltc_evaluate(gpu.h, S, st, st, p, phi)
            torch.cuda.synchronize()
            got, full = host(phi), gpu_solve(gpu, x, y, z, q, p)
            assert not np.any(got[rest])
            if prec == b.BLTC_PRECISION_FP64:
                assert np.array_equal(got[idx], full[idx])
                assert_close_abs(want[idx], got[idx], want_abs[idx], FP64_REL2, FP64_ELEM, "selected fp64")
            else:
                assert_close_abs(full[idx], got[idx], want_abs[idx], MIXED_REL2, MIXED_ELEM, "selected mixed")
            for bad in ([3, 2], [0, len(ot.leaves)], [-1]):
                with pytest.raises(b.BltcError) as e:
                    b.bltc_lists_select(gpu.h, L, bad)
                assert e.value.status == b.BLTC_ERR_ARG
            # no batch at all: every list is empty and every potential 0
            E = b.bltc_lists_select(gpu.h, L, [])
            assert b.bltc_lists_info(E) == {"n_batches": len(ot.leaves), "n_approx": 0, "n_direct": 0}
            b.bltc_modified_charges(gpu.h, st, E, p)
            b.bltc_evaluate(gpu.h, E, st, st, p, phi)
            torch.cuda.synchronize()
            assert not np.any(host(phi))
            b.bltc_lists_destroy(E)
            b.bltc_lists_destroy(S)
            b.bltc_lists_destroy(L)
    finally:
        b.bltc_tree_destroy(st)


def test_autotune_screen_and_never_slower(gpu):
    # The autotuner's screen counts every candidate's padded work; duplicates (the same trees)
    # are one candidate; the choice is never slower than the default N_L = N_B = 2000.
    import torch
    x, y, z, q = system("plummer", 400000, 20031905)
    X = dev(x, y, z, q)
    p = b.params(6, 0.8, 2000, 2000, b.BLTC_KERNEL_COULOMB, 0.0, b.BLTC_PRECISION_MIXED)
    cands = (250, 500, 1000, 2000, 2000, 4000)
    best, ms = b.bltc_autotune(gpu.h, *X, p, leaf=cands, repeats=2, use_cache=False)
    assert best.leaf_size in cands and best.batch_size == best.leaf_size
    phi = torch.empty_like(X[0])

    def fastest(pp):
        ts = []
        for _ in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.bltc_solve(gpu.h, *X, pp, phi)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts[1:])
    t_best, t_default = fastest(best), fastest(p)
    assert t_best <= 1.1 * t_default, (best.leaf_size, t_best, t_default, ms)
    # its potentials are the solve's at that size, within the bars against FP64
    got = gpu_solve(gpu, x, y, z, q, best)
    ref = gpu_solve(gpu, x, y, z, q, b.params(6, 0.8, best.leaf_size, best.batch_size,
                                              b.BLTC_KERNEL_COULOMB, 0.0, b.BLTC_PRECISION_FP64))
    assert oracle.rel_err(ref, got) <= MIXED_REL2


TILES = (0, b.tile(group_cap=4), b.tile(group_cap=2), b.tile(items_per_block=8), b.tile(items_per_block=32))


@pytest.mark.parametrize("deg", [4, 8])
def test_autotune_tile_per_degree(gpu, deg):
    # The tile tuner times every candidate shape at the given sizes and keeps the fastest, per
    # degree; each shape changes only the summation order: every candidate's potentials stay
    # within the mixed bars of the FP64 solve, and the choice is never slower than the default.
    import torch
    x, y, z, q = system("plummer", 300000, 20031906 + deg)
    X = dev(x, y, z, q)
    p = b.params(deg, 0.8, 1000, 1000, b.BLTC_KERNEL_YUKAWA, 0.5, b.BLTC_PRECISION_MIXED)
    best, ms = b.bltc_autotune_tile(gpu.h, *X, p, TILES, repeats=2, use_cache=False)
    assert best.tile in TILES and best.leaf_size == 1000 and best.degree == deg
    assert all(v == v for v in ms.values()) and ms[best.tile] == min(ms.values())
    again, ms2 = b.bltc_autotune_tile(gpu.h, *X, p, TILES, repeats=2, use_cache=True)
    assert again.tile in TILES
    ref = gpu_solve(gpu, x, y, z, q, b.params(deg, 0.8, 1000, 1000, b.BLTC_KERNEL_YUKAWA, 0.5,
                                              b.BLTC_PRECISION_FP64))
    # per target, relative to its own potential (or the rms, where the potential cancels)
    ref_abs = np.maximum(np.abs(ref), np.sqrt(np.mean(ref ** 2)))
    for t in TILES:
        pt = b.params(deg, 0.8, 1000, 1000, b.BLTC_KERNEL_YUKAWA, 0.5, b.BLTC_PRECISION_MIXED, tile=t)
        got = gpu_solve(gpu, x, y, z, q, pt)
        assert oracle.rel_err(ref, got) <= MIXED_REL2, (t, oracle.rel_err(ref, got))
        assert np.max(np.abs(got - ref) / ref_abs) <= MIXED_ELEM, t
    phi = torch.empty_like(X[0])

    def fastest(pp):
        ts = []
        for _ in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.bltc_solve(gpu.h, *X, pp, phi)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts[1:])
    assert fastest(best) <= 1.05 * fastest(p), (best.tile, ms)


def test_malformed_tile_rejected(gpu):
    x, y, z, q = system("cube", 2000, 20031907)
    for t in (3, 5, 1 << 12, -1):
        with pytest.raises(b.BltcError):
            gpu_solve(gpu, x, y, z, q, b.params(4, 0.7, 200, tile=t))


def test_solve_host_matches_device(gpu):
    x, y, z, q = system("cube", 20000, 6)
    p = b.params(6, 0.7, 1000)
    phi = np.empty_like(x)
    b.bltc_solve_host(gpu.h, x, y, z, q, p, phi)
    assert np.array_equal(phi, gpu_solve(gpu, x, y, z, q, p))


@pytest.mark.parametrize("bad", [dict(theta=1.0), dict(theta=-0.1), dict(theta=math.nan),
                                 dict(degree=0), dict(degree=17), dict(leaf_size=0),
                                 dict(kernel=1, kappa=-1.0), dict(precision=3)])
def test_invalid_parameters_rejected(gpu, bad):
    x, y, z, q = system("cube", 100, 2)
    kw = dict(degree=4, theta=0.7, leaf_size=10)
    kw.update(bad)
    with pytest.raises(b.BltcError) as e:
        gpu_solve(gpu, x, y, z, q, b.params(**kw))
    assert e.value.status == b.BLTC_ERR_ARG


# ---- direct sum (the GPU baseline) --------------------------------------------------------

@pytest.mark.parametrize("nt,ns,ker", [(3000, 3000, 0), (2047, 5001, 1), (1, 17, 0), (40000, 40000, 0),
                                      (200000, 200000, 0), (100000, 100000, 1)])
def test_direct_sum(gpu, nt, ns, ker):
    import torch
    xs = system("cube", max(nt, ns), nt + ns)
    t = [a[:nt] for a in xs[:3]]
    s = [a[:ns] for a in xs[:3]]
    q = xs[3][:ns]
    T, S, Q = dev(*t), dev(*s), dev(q)[0]
    if nt > 5000:
        pick = np.arange(0, nt, 97)
    else:
        pick = np.arange(nt)
    ref, ref_abs = oracle.direct_sum(np.stack(t)[:, pick], np.stack(s), q, ker, 0.5, with_abs=True)
    # FP64: summation order and rsqrt() against 1/sqrt only, the treecode's FP64 bar; MIXED:
    # the mixed bar (FP32 coordinate pairs keep every distance to FP32 precision)
    for prec, r2, el in ((0, FP64_REL2, FP64_ELEM), (1, MIXED_REL2, MIXED_ELEM)):
        phi = torch.empty_like(T[0])
        b.bltc_direct_sum(gpu.h, *T, *S, Q, b.params(4, 0.5, 10, kernel=ker, kappa=0.5, precision=prec), phi)
        got = host(phi)[pick]
        assert_close_abs(ref, got, ref_abs, r2, el, f"direct prec={prec}")


def test_direct_sum_close_pairs_mixed(gpu):
    # Near-duplicates 1e-9..1e-5 apart: the FP32 coordinate pairs keep their distance to
    # FP32 precision (the highs of a close pair subtract exactly), so the mixed direct sum
    # stays within the mixed bar where single FP32 coordinates would lose every digit.
    import torch
    rng = np.random.default_rng(20031907)
    x, y, z, q = system("cube", 100000, 20031907)
    k = 3000
    pick = rng.choice(len(x), k, replace=False)
    d = rng.normal(size=(3, k))
    d *= (10 ** rng.uniform(-9, -5, k)) / np.linalg.norm(d, axis=0)
    X = [np.concatenate([x, x[pick] + d[0]]), np.concatenate([y, y[pick] + d[1]]),
         np.concatenate([z, z[pick] + d[2]])]
    Q = np.concatenate([q, rng.uniform(-1, 1, k)])
    sel = np.concatenate([pick[:500], len(x) + np.arange(500), np.arange(0, len(x), 211)])
    ref, ref_abs = oracle.direct_sum(np.stack(X)[:, sel], np.stack(X), Q, with_abs=True)
    D = dev(*X, Q)
    phi = torch.empty_like(D[0])
    b.bltc_direct_sum(gpu.h, *D[:3], *D[:3], D[3], b.params(4, 0.5, 10, precision=1), phi)
    assert_close_abs(ref, host(phi)[sel], ref_abs, MIXED_REL2, MIXED_ELEM, "direct close pairs")


# ---- the full-size workload, sampled ------------------------------------------------------

def test_full_size_1e6_sampled(gpu):
    x, y, z, q = system("cube", 1_000_000, 20031838)
    p64 = b.params(8, 0.7, 2000, 2000, 0, 0.0, b.BLTC_PRECISION_FP64)
    pmx = b.params(8, 0.7, 2000, 2000, 0, 0.0, b.BLTC_PRECISION_MIXED)
    h, _ = gpu_tree(gpu, x, y, z, q, 2000)
    ot = oracle.Tree(x, y, z, 2000)
    try:
        _compare_trees(ot, b.bltc_tree_export(gpu.h, h))
        L = b.bltc_lists_build(gpu.h, h, h, pmx)
        got = b.bltc_lists_export(gpu.h, L)
        b.bltc_lists_destroy(L)
        want = oracle.lists(ot, ot, 0.7, 8)
        for k in want:
            assert np.array_equal(want[k], got[k]), k
    finally:
        b.bltc_tree_destroy(h)
    nl = len(ot.leaves)
    pick = np.array([0, 1, nl // 2, nl - 2, nl - 1])
    want, want_abs = _oracle(x, y, z, q, p64, pick)
    idx = batch_targets(ot, pick)
    got64 = gpu_solve(gpu, x, y, z, q, p64)
    gotmx = gpu_solve(gpu, x, y, z, q, pmx)
    assert_close_abs(want[idx], got64[idx], want_abs[idx], FP64_REL2, FP64_ELEM, "1e6 fp64 sampled")
    e = oracle.rel_err(got64, gotmx)
    assert e <= MIXED_REL2, e


def test_mutual_pairs_counted_once(gpu):
    # In mixed precision with batches = sources, a leaf pair in each other's direct list is
    # evaluated once for both batches; the count of kernel evaluations must equal the
    # paper's count minus the partner side of every such pair (found here from the oracle's
    # lists), and the FP64 path evaluates everything.
    x, y, z, q = system("cube", 60000, 20031881)
    st, X = gpu_tree(gpu, x, y, z, q, 700)
    try:
        p = b.params(6, 0.7, 700)
        L = b.bltc_lists_build(gpu.h, st, st, p)
        try:
            c = b.bltc_stats(gpu.h, L)
            ev_mx = b.bltc_evaluations(gpu.h, L, p)
            ev_64 = b.bltc_evaluations(gpu.h, L, b.params(6, 0.7, 700, precision=b.BLTC_PRECISION_FP64))
        finally:
            b.bltc_lists_destroy(L)
        ot = oracle.Tree(x, y, z, 700)
        ol = oracle.lists(ot, ot, 0.7, 6)
        leaf_of = {int(v): i for i, v in enumerate(ot.leaves)}
        dirs = [set(ol["direct_ids"][ol["direct_off"][i]:ol["direct_off"][i + 1]].tolist())
                for i in range(len(ot.leaves))]
        saved = 0
        for i, A in enumerate(ot.leaves):
            for C in dirs[i]:
                j = leaf_of.get(int(C))
                if j is not None and j < i and int(A) in dirs[j]:
                    saved += int(ot.count[A]) * int(ot.count[C])   # i's side of a pair owned by j
        assert saved > 0
        assert ev_64 == c["direct"] + c["approx"]
        assert ev_mx == c["direct"] + c["approx"] - saved
    finally:
        b.bltc_tree_destroy(st)


def test_bltc_degenerate_systems(gpu):
    # duplicates (pairs with r^2 == 0 inside a leaf), a lattice (exact hits on Chebyshev end
    # points and many equal distances), two far-apart clumps, and a single repeated point
    rng = np.random.default_rng(20031907)
    dup = np.repeat(rng.uniform(-1, 1, (3, 1500)), 4, axis=1)
    lat = np.array(np.meshgrid(np.arange(24.0), np.arange(24.0), np.arange(12.0))).reshape(3, -1)
    clumps = np.concatenate([rng.normal(0, 0.01, (3, 3000)), rng.normal(0, 0.01, (3, 3000)) + 50.0], axis=1)
    for pts, leaf, deg in ((dup, 300, 4), (lat, 200, 3), (clumps, 400, 5)):
        q = rng.uniform(-1, 1, pts.shape[1])
        x, y, z = pts
        p64 = b.params(deg, 0.7, leaf, leaf, 0, 0.0, b.BLTC_PRECISION_FP64)
        pmx = b.params(deg, 0.7, leaf, leaf, 0, 0.0, b.BLTC_PRECISION_MIXED)
        want, want_abs = _oracle(x, y, z, q, p64)
        got64 = gpu_solve(gpu, x, y, z, q, p64)
        gotmx = gpu_solve(gpu, x, y, z, q, pmx)
        assert_close_abs(want, got64, want_abs, FP64_REL2, FP64_ELEM, "degenerate fp64 vs oracle")
        assert_close_abs(got64, gotmx, want_abs, MIXED_REL2, MIXED_ELEM, "degenerate mixed vs fp64")
    # one point repeated: every pair has r^2 == 0, every potential is exactly 0
    x = np.full(5000, 0.25)
    q = rng.uniform(-1, 1, 5000)
    for prec in (b.BLTC_PRECISION_FP64, b.BLTC_PRECISION_MIXED):
        got = gpu_solve(gpu, x, x.copy(), x.copy(), q, b.params(4, 0.7, 100, precision=prec))
        assert np.all(got == 0.0)


def test_empty_inputs_rejected(gpu):
    """N < 1 is an argument error (BLTC_ERR_ARG) at every entry point, raised before any
    device work; a non-empty set beside an empty one is rejected the same way."""
    import torch
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    X = dev(*system("cube", 100, 3))
    phi = torch.empty_like(X[0])
    p = b.params(4, 0.7, 10, 10)
    calls = [
        lambda: b.bltc_solve(gpu.h, e, e, e, e, p, e),
        lambda: b.bltc_solve_targets(gpu.h, e, e, e, *X, p, e),
        lambda: b.bltc_solve_targets(gpu.h, *X[:3], e, e, e, e, p, phi),
        lambda: b.bltc_solve_cp(gpu.h, e, e, e, *X, p, e),
        lambda: b.bltc_solve_cc(gpu.h, *X[:3], e, e, e, e, p, phi),
        lambda: b.bltc_solve_hermite(gpu.h, e, e, e, e, p, e),
        lambda: b.bltc_direct_sum(gpu.h, e, e, e, *X, p, e),
        lambda: b.bltc_graph_create(gpu.h, e, e, e, e, p, e),
    ]
    for i, call in enumerate(calls):
        with pytest.raises(b.BltcError) as err:
            call()
        assert err.value.status == b.BLTC_ERR_ARG, i
    torch.cuda.synchronize()
