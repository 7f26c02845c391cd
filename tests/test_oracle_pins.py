"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these checks re-types the oracle's own formulas: they use closed forms, hand-derived
trees (tests/golden/trees_small.json), invariants of interpolation (partition of unity,
moment reproduction, exactness for polynomial kernels), special cases that reduce to the
direct sum, and brute-force coverage on small inputs.  A dropped term, a wrong sign or index,
or a transposed operand anywhere in the oracle fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2003_01836_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# Direct sum, Eq. 1-2
# ---------------------------------------------------------------------------------------

def _direct(pts, q, kernel=oracle.KERNEL_COULOMB, kappa=0.0):
    pts = np.asarray(pts, dtype=np.float64).T
    return oracle.direct_sum(pts, pts, np.asarray(q, dtype=np.float64), kernel, kappa)


def test_direct_two_charges_closed_form():
    # phi at each of two charges is the other charge over their distance (Eq. 1-2).
    phi = _direct([[0.0, 0.0, 0.0], [0.0, 0.0, 0.5]], [0.75, -0.25])
    assert phi[0] == -0.5 and phi[1] == 1.5
    kappa = 0.5
    phi = _direct([[0.0, 0.0, 0.0], [0.0, 0.5, 0.0]], [0.75, -0.25], oracle.KERNEL_YUKAWA, kappa)
    assert phi[0] == pytest.approx(-0.25 * math.exp(-kappa * 0.5) / 0.5, rel=1e-15)
    assert phi[1] == pytest.approx(0.75 * math.exp(-kappa * 0.5) / 0.5, rel=1e-15)


def test_direct_pythagorean_triangle_exact():
    # Distances 5, 12, 13 are integers, so every potential is an exact rational.
    pts = [[0, 0, 0], [3, 4, 0], [3, 4, 12]]
    q = [1.0, 2.0, 3.0]
    phi = _direct(pts, q)
    want = [Fraction(2, 5) + Fraction(3, 13), Fraction(1, 5) + Fraction(3, 12),
            Fraction(1, 13) + Fraction(2, 12)]
    for p, w in zip(phi, want):
        assert abs(Fraction(p) - w) <= Fraction(1, 2 ** 50)


def test_direct_cube_corners_symmetric():
    # Eight unit charges on the corners of a cube of side a: by symmetry every corner sees
    # 3 neighbours at a, 3 at a*sqrt2 and 1 at a*sqrt3.
    a = 0.75
    pts = [[a * i, a * j, a * k] for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    phi = _direct(pts, [1.0] * 8)
    want = 3 / a + 3 / (a * math.sqrt(2)) + 1 / (a * math.sqrt(3))
    np.testing.assert_allclose(phi, want, rtol=2e-16 * 8)


def test_direct_self_pairs_skipped():
    # Targets are the sources: the r = 0 pair is skipped, also for duplicated particles.
    assert _direct([[0.1, 0.2, 0.3]], [1.0])[0] == 0.0
    phi = _direct([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [0.5, 0.5, 1.0]], [1.0, 2.0, 4.0])
    assert phi[0] == 8.0 and phi[1] == 8.0 and phi[2] == 6.0


def test_direct_yukawa_kappa0_is_coulomb_bitwise():
    x, y, z, q = inputs.uniform_cube(300, 11)
    pts = np.stack([x, y, z])
    c = oracle.direct_sum(pts, pts, q, oracle.KERNEL_COULOMB)
    yk = oracle.direct_sum(pts, pts, q, oracle.KERNEL_YUKAWA, 0.0)
    assert np.array_equal(c, yk)


# ---------------------------------------------------------------------------------------
# Trees, Sec. II-D and Sec. III-A
# ---------------------------------------------------------------------------------------

def _golden_trees():
    with open(os.path.join(GOLDEN, "trees_small.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_trees(), ids=lambda c: c["name"])
def test_tree_hand_derived(case):
    t = oracle.Tree(case["x"], case["y"], case["z"], case["max_leaf"])
    assert t.perm.tolist() == case["perm"]
    assert t.n_nodes == len(case["nodes"])
    for i, nd in enumerate(case["nodes"]):
        assert t.begin[i] == nd["begin"] and t.count[i] == nd["count"]
        assert t.parent[i] == nd["parent"] and t.level[i] == nd["level"]
        assert t.n_children[i] == len(nd["children"])
        assert t.children[i, :len(nd["children"])].tolist() == nd["children"]
        assert (t.children[i, len(nd["children"]):] == -1).all()
        assert t.lo[i].tolist() == nd["lo"] and t.hi[i].tolist() == nd["hi"]
        assert t.center[i].tolist() == nd["center"]
        assert t.radius[i] == math.sqrt(nd["radius_sq"])


def test_tree_signed_zero_box():
    t = oracle.Tree([0.0, -0.0, 1.0], [1.0, 0.0, 0.5], [1.0, 0.0, 0.5], 3)
    assert math.copysign(1.0, t.lo[0, 0]) == -1.0 and t.lo[0, 0] == 0.0


def check_tree_invariants(t, x, y, z, max_leaf):
    n = len(x)
    assert sorted(t.perm.tolist()) == list(range(n))
    assert t.begin[0] == 0 and t.count[0] == n and t.parent[0] == -1
    coords = np.stack([x, y, z], axis=1)
    sub = np.ones(t.n_nodes, np.int64)
    for v in range(t.n_nodes - 1, -1, -1):
        ch = t.children[v, :t.n_children[v]]
        sub[v] = 1 + sub[ch].sum()
    for v in range(t.n_nodes):
        b, c = t.begin[v], t.count[v]
        pts = coords[t.perm[b:b + c]]
        assert (t.lo[v] == pts.min(axis=0)).all() and (t.hi[v] == pts.max(axis=0)).all()
        ch = t.children[v, :t.n_children[v]]
        if len(ch) == 0:
            continue
        assert len(ch) >= 2
        # children partition the parent's range, in order, and are DFS pre-order numbered
        assert t.begin[ch[0]] == b and ch[0] == v + 1
        for a, bb in zip(ch[:-1], ch[1:]):
            assert t.begin[bb] == t.begin[a] + t.count[a] and bb == a + sub[a]
        assert t.begin[ch[-1]] + t.count[ch[-1]] == b + c
        assert (t.parent[ch] == v).all() and (t.level[ch] == t.level[v] + 1).all()
        assert c > max_leaf
        # every child's particles lie on one side of every split midpoint
        mid = 0.5 * (t.lo[v] + t.hi[v])
        L = t.hi[v] - t.lo[v]
        split = L * 1.4142135623730951 >= L.max()
        for k in ch:
            kp = coords[t.perm[t.begin[k]:t.begin[k] + t.count[k]]]
            for d in range(3):
                if split[d]:
                    side = kp[:, d] < mid[d]
                    assert side.all() or (~side).all()
    # stable partitions of the identity leave every leaf's segment in increasing order
    for v in range(t.n_nodes):
        if t.n_children[v] == 0:
            seg = t.perm[t.begin[v]:t.begin[v] + t.count[v]]
            assert (np.diff(seg) > 0).all()


@pytest.mark.parametrize("kind,n,leaf", [("cube", 5000, 100), ("plummer", 6000, 64),
                                          ("cube", 3000, 1)])
def test_tree_invariants(kind, n, leaf):
    x, y, z, _ = inputs.system(kind, n, 123)
    t = oracle.Tree(x, y, z, leaf)
    check_tree_invariants(t, x, y, z, leaf)
    leaves = t.leaves
    assert (t.count[leaves] <= leaf).all() or kind == "plummer"
    assert t.count[leaves].sum() == n


def test_tree_scale_by_two_identical():
    x, y, z, _ = inputs.uniform_cube(4000, 9)
    a = oracle.Tree(x, y, z, 150)
    b = oracle.Tree(2 * x, 2 * y, 2 * z, 150)
    for k in ("perm", "begin", "count", "parent", "level", "n_children", "children"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    for k in ("lo", "hi", "center", "radius"):
        assert np.array_equal(2 * getattr(a, k), getattr(b, k))


# ---------------------------------------------------------------------------------------
# Barycentric Lagrange interpolation, Sec. II-A and II-C
# ---------------------------------------------------------------------------------------

def test_cheb_points_closed_form():
    s, w = oracle.cheb(4, -1.0, 1.0)
    np.testing.assert_allclose(s, [1, math.sqrt(0.5), 0, -math.sqrt(0.5), -1], atol=1e-16)
    assert s[0] == 1.0 and s[4] == -1.0
    assert w.tolist() == [0.5, -1.0, 1.0, -1.0, 0.5]
    s, w = oracle.cheb(3, 2.0, 6.0)          # [2, 6]: points 6, 5, 3, 2
    np.testing.assert_allclose(s, [6, 5, 3, 2], rtol=1e-15)
    assert s[0] == 6.0 and s[3] == 2.0
    assert w.tolist() == [0.5, -1.0, 1.0, -0.5]


@pytest.mark.parametrize("n", [1, 2, 5, 8, 13])
def test_cheb_weights_match_definition(n):
    # Eq. 4 defines w_k = 1 / prod_{j != k} (s_k - s_j); Eq. 7 is that up to a common factor.
    s, w = oracle.cheb(n, -1.0, 1.0)
    true_w = np.array([1.0 / np.prod([s[k] - s[j] for j in range(n + 1) if j != k])
                       for k in range(n + 1)])
    ratio = true_w / w
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-12)


@pytest.mark.parametrize("n", [1, 4, 8, 13])
def test_lagrange_kronecker_at_nodes(n):
    lo, hi = -0.3, 0.7
    s, _ = oracle.cheb(n, lo, hi)
    for k in range(n + 1):
        a = oracle.lagrange(n, lo, hi, s[k])
        e = np.zeros(n + 1)
        e[k] = 1.0
        assert a.tolist() == e.tolist()      # exact hit, Eq. 5 enforced (Sec. II-C)


@pytest.mark.parametrize("n", [1, 3, 8, 13])
def test_lagrange_reproduces_polynomials(n):
    # sum_k L_k(y) p(s_k) = p(y) for deg p <= n; partition of unity is m = 0.
    lo, hi = -1.25, 0.5
    s, _ = oracle.cheb(n, lo, hi)
    rng = np.random.default_rng(n)
    for yv in rng.uniform(lo, hi, 20):
        a = oracle.lagrange(n, lo, hi, yv)
        for m in range(n + 1):
            assert abs(a @ (s ** m) - yv ** m) <= 1e-12 * max(1.0, abs(yv) ** m)
        # degree n+1 is generally not reproduced (the rule is not trivially exact)
    yv = 0.1234
    a = oracle.lagrange(n, lo, hi, yv)
    assert abs(a @ (s ** (n + 1)) - yv ** (n + 1)) > 1e-10


def test_lagrange_factors_stay_below_1_031():
    # On Chebyshev points of the second kind no Lagrange factor exceeds 1.031 in magnitude for
    # n <= 16 (it reaches 1 at its own node); the mixed modified-charge bar of the GPU tests
    # bounds each term by |q| max|L|^3 with this constant.
    ys = np.linspace(-1.0, 1.0, 8001)
    for n in (1, 2, 4, 8, 12, 16):
        m = max(np.abs(oracle.lagrange(n, -1.0, 1.0, yv)).max() for yv in ys)
        assert 1.0 <= m < 1.031, (n, m)


def test_lagrange_matches_scipy_barycentric():
    scipy_interp = pytest.importorskip("scipy.interpolate")
    n, lo, hi = 9, 0.2, 1.7
    s, _ = oracle.cheb(n, lo, hi)
    f = np.cos(3 * s) + s ** 2
    P = scipy_interp.BarycentricInterpolator(s, f)
    for yv in np.linspace(lo, hi, 37):
        assert oracle.lagrange(n, lo, hi, yv) @ f == pytest.approx(float(P(yv)), abs=1e-12)


def test_lagrange_zero_extent_is_e0():
    a = oracle.lagrange(6, 0.25, 0.25, 0.25)
    assert a.tolist() == [1.0] + [0.0] * 6


# ---------------------------------------------------------------------------------------
# Modified charges, Eq. 12
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 5, 8])
def test_modified_charges_moments(n):
    # qhat reproduces every moment sum_j q_j y1^a y2^b y3^c with a, b, c <= n.
    x, y, z, q = inputs.uniform_cube(3000, 21)
    t = oracle.Tree(x, y, z, 400)
    qh = oracle.modified_charges(t, q, n)
    n1 = n + 1
    for v in [0] + list(range(1, t.n_nodes, max(1, t.n_nodes // 6))):
        idx = t.perm[t.begin[v]:t.begin[v] + t.count[v]]
        s = [oracle.cheb(n, t.lo[v, d], t.hi[v, d])[0] for d in range(3)]
        Q = qh[v].reshape(n1, n1, n1)
        assert Q.sum() == pytest.approx(q[idx].sum(), abs=1e-12 * np.abs(q[idx]).sum())
        for (a, b, c) in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (n, 0, 0), (0, n, n), (n, n, n),
                          (1, 2 % n1, 0)]:
            lhs = np.einsum("ijk,i,j,k->", Q, s[0] ** a, s[1] ** b, s[2] ** c)
            rhs = np.sum(q[idx] * x[idx] ** a * y[idx] ** b * z[idx] ** c)
            scale = np.sum(np.abs(q[idx]))
            assert abs(lhs - rhs) <= 1e-11 * scale, (v, a, b, c)


def test_modified_charges_single_corner_particle():
    # A lone particle at a box corner takes the exact-hit path: qhat = q at that corner.
    x = np.array([0.0, 1.0, 0.25])
    y = np.array([0.0, 1.0, 0.5])
    z = np.array([0.0, 1.0, 0.75])
    q = np.array([2.0, 0.0, 0.0])
    t = oracle.Tree(x, y, z, 8)
    qh = oracle.modified_charges(t, q, 3).reshape(4, 4, 4)
    expect = np.zeros((4, 4, 4))
    expect[3, 3, 3] = 2.0     # s_n = lo on every axis
    assert np.array_equal(qh, expect)


# ---------------------------------------------------------------------------------------
# Treecode, Algorithm 1 + Eq. 11, 13
# ---------------------------------------------------------------------------------------

def _system(n, seed=20031837):
    return inputs.uniform_cube(n, seed)


def test_lists_cover_every_pair_exactly_once():
    x, y, z, _ = _system(6000, 77)
    for theta, n in [(0.7, 4), (0.5, 2), (0.9, 6)]:
        st = oracle.Tree(x, y, z, 200)
        bt = oracle.Tree(x, y, z, 150)
        L = oracle.lists(bt, st, theta, n)
        N = len(x)
        for b_i, B in enumerate(bt.leaves):
            cover = np.zeros(N, np.int64)
            for key in ("approx", "direct"):
                ids = L[key + "_ids"][L[key + "_off"][b_i]:L[key + "_off"][b_i + 1]]
                for C in ids:
                    cover[st.begin[C]:st.begin[C] + st.count[C]] += 1
            assert (cover == 1).all(), (theta, n, b_i)
        P = (n + 1) ** 3
        app = L["approx_ids"]
        assert (st.count[app] > P).all()
        assert len(app) > 0


def test_theta_zero_equals_direct_sum():
    x, y, z, q = _system(4000)
    phi, _, _ = oracle.bltc(x, y, z, q, 0.0, 4, 300, 300)
    ref = oracle.direct_sum(np.stack([x, y, z]), np.stack([x, y, z]), q)
    assert oracle.rel_err(ref, phi) < 1e-14


def test_size_check_routes_everything_direct():
    # With (n+1)^3 >= every cluster size no cluster is approximated (Eq. 13, 2nd condition).
    x, y, z, q = _system(3000)
    phi, _, _ = oracle.bltc(x, y, z, q, 0.9, 13, 100, 100)  # (14)^3 = 2744 < 3000 only at root
    ref = oracle.direct_sum(np.stack([x, y, z]), np.stack([x, y, z]), q)
    assert oracle.rel_err(ref, phi) < 1e-14


def test_yukawa_kappa0_equals_coulomb_bitwise():
    x, y, z, q = _system(3000)
    a, _, _ = oracle.bltc(x, y, z, q, 0.7, 4, 200, 200, oracle.KERNEL_COULOMB)
    b, _, _ = oracle.bltc(x, y, z, q, 0.7, 4, 200, 200, oracle.KERNEL_YUKAWA, 0.0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_polynomial_kernel_is_exact(n):
    # G(x, y) of degree n in every source coordinate is interpolated exactly (Eq. 8), so the
    # treecode equals the direct sum for any theta.
    x, y, z, q = _system(4000, 3)
    phi, _, _ = oracle.bltc(x, y, z, q, 0.7, n, 150, 150, oracle.KERNEL_POLY)
    pts = np.stack([x, y, z])
    ref, ref_abs = oracle.direct_sum(pts, pts, q, oracle.KERNEL_POLY, 0.0, n, with_abs=True)
    assert np.max(np.abs(phi - ref) / ref_abs) < 1e-12
    # and the approximation is actually used
    st = oracle.Tree(x, y, z, 150)
    assert len(oracle.lists(st, st, 0.7, n)["approx_ids"]) > 0


_SAMPLED = {}


def _sampled_system():
    # Sec. IV samples the error at a subset of targets for large N; here three batches of a
    # 2e5-particle cube with N_L = N_B = 2000, large enough that clusters of (n+1)^3 = 2744
    # points (n = 13) still pass the size check of Eq. 13.
    if not _SAMPLED:
        x, y, z, q = inputs.uniform_cube(200000, 5)
        bt = oracle.Tree(x, y, z, 2000)
        pick = np.array([0, len(bt.leaves) // 2, len(bt.leaves) - 1])
        idx = np.concatenate([bt.perm[bt.begin[bt.leaves[b]]:
                                      bt.begin[bt.leaves[b]] + bt.count[bt.leaves[b]]]
                              for b in pick])
        pts = np.stack([x, y, z])
        _SAMPLED.update(x=x, y=y, z=z, q=q, pick=pick, idx=idx,
                        ref=oracle.direct_sum(pts[:, idx], pts, q))
    return _SAMPLED


def _sampled_err(theta, n, kernel=oracle.KERNEL_COULOMB, kappa=0.0, ref=None):
    S = _sampled_system()
    phi, _, _ = oracle.bltc(S["x"], S["y"], S["z"], S["q"], theta, n, 2000, 2000, kernel, kappa,
                            batches=S["pick"])
    return oracle.rel_err(S["ref"] if ref is None else ref, phi[S["idx"]])


def test_error_decays_with_degree():
    # Sec. IV (Fig. 5): for fixed theta the error falls towards machine precision as n grows,
    # and a smaller theta is more accurate at the same n.
    table = {th: [_sampled_err(th, n) for n in (1, 3, 5, 7, 9, 11, 13)] for th in (0.5, 0.7, 0.9)}
    for th, errs in table.items():
        assert all(b < a for a, b in zip(errs, errs[1:])), (th, errs)
        assert errs[0] > 1e-3
    for i in range(7):
        assert table[0.5][i] < table[0.7][i] < table[0.9][i]
    assert table[0.5][-1] < 1e-12


def test_paper_accuracy_band():
    # theta = 0.8, n = 8 gives 5-6 digit accuracy in the paper (Sec. IV, weak and strong
    # scaling: errors 3e-6 .. 1.5e-5 with N_L = N_B = 4000); same broad band here.
    S = _sampled_system()
    assert 1e-8 < _sampled_err(0.8, 8) < 1e-4
    pts = np.stack([S["x"], S["y"], S["z"]])
    ref = oracle.direct_sum(pts[:, S["idx"]], pts, S["q"], oracle.KERNEL_YUKAWA, 0.5)
    assert 1e-8 < _sampled_err(0.8, 8, oracle.KERNEL_YUKAWA, 0.5, ref) < 1e-4


def test_small_n_degenerates_to_direct_sum():
    # With N = 1e4 and N_L = 500 the leaves hold ~156 particles: for n >= 5 every candidate
    # fails the size check (n+1)^3 < N_C at theta = 0.5, so Algorithm 1 is the direct sum.
    x, y, z, q = _system(10000)
    pts = np.stack([x, y, z])
    ref = oracle.direct_sum(pts, pts, q)
    phi, _, _ = oracle.bltc(x, y, z, q, 0.5, 5, 500, 500)
    assert oracle.rel_err(ref, phi) < 1e-14
    phi, _, _ = oracle.bltc(x, y, z, q, 0.7, 4, 500, 500)
    assert 1e-8 < oracle.rel_err(ref, phi) < 1e-4


def test_batch_subset_matches_full_run():
    x, y, z, q = _system(5000)
    full, _, _ = oracle.bltc(x, y, z, q, 0.7, 4, 300, 300)
    bt = oracle.Tree(x, y, z, 300)
    pick = np.array([0, 3, len(bt.leaves) - 1])
    sub, _, _ = oracle.bltc(x, y, z, q, 0.7, 4, 300, 300, batches=pick)
    for b in pick:
        B = bt.leaves[b]
        idx = bt.perm[bt.begin[B]:bt.begin[B] + bt.count[B]]
        assert np.array_equal(sub[idx], full[idx])


# ---------------------------------------------------------------------------------------
# Distinct target and source sets (Sec. II: only target and source positions enter)
# ---------------------------------------------------------------------------------------

def _targets_and_sources(nt, ns, seed=20031851):
    """Sources in [-1, 1]^3; targets in a larger, shifted box (some far from every source,
    some inside the source cloud) plus every 50th source position exactly (r^2 == 0 pairs)."""
    sx, sy, sz, q = inputs.uniform_cube(ns, seed)
    tx, ty, tz, _ = inputs.uniform_cube(nt, seed + 1)
    tx, ty, tz = 1.5 * tx + 0.75, 1.5 * ty, 1.5 * tz - 0.25
    tx = np.concatenate([tx, sx[::50]])
    ty = np.concatenate([ty, sy[::50]])
    tz = np.concatenate([tz, sz[::50]])
    return (tx, ty, tz), (sx, sy, sz), q


def test_ts_same_sets_equal_bltc_bitwise():
    x, y, z, q = _system(3000)
    a, _, _ = oracle.bltc(x, y, z, q, 0.7, 4, 200, 150)
    b, _, _ = oracle.bltc_ts((x, y, z), (x, y, z), q, 0.7, 4, 200, 150)
    assert np.array_equal(a, b)


def test_ts_theta_zero_equals_direct_sum():
    T, S, q = _targets_and_sources(2500, 4000)
    phi, _, _ = oracle.bltc_ts(T, S, q, 0.0, 4, 300, 170)
    ref = oracle.direct_sum(np.stack(T), np.stack(S), q)
    assert oracle.rel_err(ref, phi) < 1e-14


@pytest.mark.parametrize("n", [2, 4])
def test_ts_polynomial_kernel_is_exact(n):
    T, S, q = _targets_and_sources(3000, 5000, 20031853)
    phi, _, _ = oracle.bltc_ts(T, S, q, 0.7, n, 150, 220, oracle.KERNEL_POLY)
    ref, ref_abs = oracle.direct_sum(np.stack(T), np.stack(S), q, oracle.KERNEL_POLY, 0.0, n,
                                     with_abs=True)
    assert np.max(np.abs(phi - ref) / ref_abs) < 1e-12
    bt, st = oracle.Tree(*T, 220), oracle.Tree(*S, 150)
    assert len(oracle.lists(bt, st, 0.7, n)["approx_ids"]) > 0


def test_ts_lists_cover_every_pair_exactly_once():
    T, S, _ = _targets_and_sources(2000, 6000, 20031855)
    st, bt = oracle.Tree(*S, 200), oracle.Tree(*T, 130)
    for theta, n in [(0.7, 4), (0.9, 2)]:
        L = oracle.lists(bt, st, theta, n)
        for b_i in range(len(bt.leaves)):
            cover = np.zeros(len(S[0]), np.int64)
            for key in ("approx", "direct"):
                for C in L[key + "_ids"][L[key + "_off"][b_i]:L[key + "_off"][b_i + 1]]:
                    cover[st.begin[C]:st.begin[C] + st.count[C]] += 1
            assert (cover == 1).all(), (theta, n, b_i)
        assert len(L["approx_ids"]) > 0


def test_ts_error_band_and_decay():
    # the approximation error for separate sets behaves as for targets = sources (Sec. IV)
    T, S, q = _targets_and_sources(3000, 20000, 20031857)
    ref = oracle.direct_sum(np.stack(T), np.stack(S), q)
    errs = [oracle.rel_err(ref, oracle.bltc_ts(T, S, q, 0.7, n, 300, 300)[0]) for n in (1, 3, 5, 7)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert 1e-9 < errs[2] < 1e-4 and errs[0] > 1e-4, errs


# ---------------------------------------------------------------------------------------
# A kernel outside Eq. 2: softened Coulomb 1/sqrt(r^2 + eps^2) (smooth, non-oscillatory)
# ---------------------------------------------------------------------------------------

def test_soft_kernel_closed_form():
    eps = 0.3
    # charges 0.75 at the origin and -0.25 at distance 0.5 (a 3-4-5 triangle scaled)
    phi = _direct([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]], [0.75, -0.25], oracle.KERNEL_SOFT, eps)
    d = math.sqrt(0.25 + eps * eps)
    assert phi[0] == pytest.approx(-0.25 / d, rel=1e-15)
    assert phi[1] == pytest.approx(0.75 / d, rel=1e-15)


def test_soft_kernel_eps0_is_coulomb_bitwise():
    x, y, z, q = _system(3000)
    pts = np.stack([x, y, z])
    a = oracle.direct_sum(pts, pts, q, oracle.KERNEL_COULOMB)
    b = oracle.direct_sum(pts, pts, q, oracle.KERNEL_SOFT, 0.0)
    assert np.array_equal(a, b)


def test_soft_kernel_treecode():
    # theta = 0 is the direct sum; the approximation error falls with n for a smooth kernel
    x, y, z, q = _system(6000, 20031861)
    pts = np.stack([x, y, z])
    ref = oracle.direct_sum(pts, pts, q, oracle.KERNEL_SOFT, 0.05)
    phi, _, _ = oracle.bltc(x, y, z, q, 0.0, 4, 300, 300, oracle.KERNEL_SOFT, 0.05)
    assert oracle.rel_err(ref, phi) < 1e-14
    errs = [oracle.rel_err(ref, oracle.bltc(x, y, z, q, 0.7, n, 300, 300, oracle.KERNEL_SOFT, 0.05)[0])
            for n in (1, 3, 5)]
    assert errs[0] > errs[1] > errs[2] and 1e-9 < errs[2] < 1e-4, errs


# ---------------------------------------------------------------------------------------
# Cluster-particle variant (future work of Sec. V): targets interpolated, sources exact
# ---------------------------------------------------------------------------------------

def test_cp_theta_zero_equals_direct_sum():
    T, S, q = _targets_and_sources(2500, 4000, 20031863)
    phi, _ = oracle.bltc_cp(T, S, q, 0.0, 4, 300, 170)
    ref = oracle.direct_sum(np.stack(T), np.stack(S), q)
    assert oracle.rel_err(ref, phi) < 1e-14


@pytest.mark.parametrize("n", [2, 4])
def test_cp_polynomial_kernel_is_exact(n):
    # G(x, y) of degree n in every TARGET coordinate is reproduced by the interpolant of the
    # target cluster's point potentials, whatever theta
    T, S, q = _targets_and_sources(4000, 3000, 20031865)
    phi, phi_abs = oracle.bltc_cp(T, S, q, 0.7, n, 220, 150, oracle.KERNEL_POLY, with_abs=True)
    ref, ref_abs = oracle.direct_sum(np.stack(T), np.stack(S), q, oracle.KERNEL_POLY, 0.0, n,
                                     with_abs=True)
    assert np.max(np.abs(phi - ref) / ref_abs) < 1e-12
    # the approximation is used: some target cluster is approximated for some batch
    tt, st = oracle.Tree(*T, 220), oracle.Tree(*S, 150)
    assert len(oracle.lists(st, tt, 0.7, n)["approx_ids"]) > 0


def test_cp_same_particles_and_error_decay():
    x, y, z, q = _system(20000, 20031867)
    pts = np.stack([x, y, z])
    ref = oracle.direct_sum(pts, pts, q)
    errs = [oracle.rel_err(ref, oracle.bltc_cp((x, y, z), (x, y, z), q, 0.7, n, 400, 400)[0])
            for n in (1, 3, 5, 7)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert 1e-9 < errs[2] < 1e-4 and errs[0] > 1e-4, errs


def test_cp_lists_cover_every_pair_once():
    # every (target, source batch) pair is in exactly one list entry: an approximated target
    # cluster holding the target, or a direct one
    T, S, _ = _targets_and_sources(3000, 2500, 20031869)
    tt, st = oracle.Tree(*T, 200), oracle.Tree(*S, 130)
    L = oracle.lists(st, tt, 0.7, 4)
    for b in range(len(st.leaves)):
        cover = np.zeros(len(T[0]), np.int64)
        for key in ("approx", "direct"):
            for C in L[key + "_ids"][L[key + "_off"][b]:L[key + "_off"][b + 1]]:
                cover[tt.begin[C]:tt.begin[C] + tt.count[C]] += 1
        assert (cover == 1).all(), b


# ---------------------------------------------------------------------------------------
# Cluster-cluster variant (dual tree traversal, future work of Sec. V)
# ---------------------------------------------------------------------------------------

def test_cc_theta_zero_equals_direct_sum():
    T, S, q = _targets_and_sources(2500, 4000, 20031871)
    phi, _ = oracle.bltc_cc(T, S, q, 0.0, 4, 300, 170)
    ref = oracle.direct_sum(np.stack(T), np.stack(S), q)
    assert oracle.rel_err(ref, phi) < 1e-14


@pytest.mark.parametrize("n", [2, 4])
def test_cc_polynomial_kernel_is_exact(n):
    # a kernel of degree n in every target AND source coordinate is reproduced by both
    # interpolations (CC, CP and PC terms), whatever theta
    x, y, z, q = _system(12000, 20031873)
    T = S = (x, y, z)
    phi, _ = oracle.bltc_cc(T, S, q, 0.7, n, 300, 300, oracle.KERNEL_POLY)
    ref, ref_abs = oracle.direct_sum(np.stack(T), np.stack(S), q, oracle.KERNEL_POLY, 0.0, n,
                                     with_abs=True)
    assert np.max(np.abs(phi - ref) / ref_abs) < 1e-12
    L = oracle.dual_lists(oracle.Tree(x, y, z, 300), oracle.Tree(x, y, z, 300), 0.7, n)
    assert len(L["cc"][0]) > 0 and len(L["pp"][0]) > 0
    # and with separate sets of very different density, the mixed kinds CP and PC appear
    T2, S2, q2 = _targets_and_sources(6000, 1500, 20031874)
    phi2, _ = oracle.bltc_cc(T2, S2, q2, 0.7, n, 40, 400, oracle.KERNEL_POLY)
    ref2, ref2_abs = oracle.direct_sum(np.stack(T2), np.stack(S2), q2, oracle.KERNEL_POLY, 0.0, n,
                                       with_abs=True)
    assert np.max(np.abs(phi2 - ref2) / ref2_abs) < 1e-12
    L2 = oracle.dual_lists(oracle.Tree(*T2, 400), oracle.Tree(*S2, 40), 0.7, n)
    assert len(L2["cp"][0]) + len(L2["pc"][0]) > 0


def test_cc_lists_cover_every_pair_once():
    # every (target, source) pair lies in exactly one interaction (brute force)
    T, S, _ = _targets_and_sources(1200, 1500, 20031875)
    tt, st = oracle.Tree(*T, 60), oracle.Tree(*S, 80)
    L = oracle.dual_lists(tt, st, 0.7, 2)
    cover = np.zeros((len(T[0]), len(S[0])), np.int64)
    for name in ("cc", "cp", "pc", "pp"):
        for a, c in zip(*L[name]):
            cover[np.ix_(tt.perm[tt.begin[a]:tt.begin[a] + tt.count[a]],
                         st.perm[st.begin[c]:st.begin[c] + st.count[c]])] += 1
    assert (cover == 1).all()
    assert all(len(L[k][0]) > 0 for k in ("cc", "pp"))


def test_cc_error_decay_and_band():
    x, y, z, q = _system(20000, 20031877)
    pts = np.stack([x, y, z])
    ref = oracle.direct_sum(pts, pts, q)
    errs = [oracle.rel_err(ref, oracle.bltc_cc((x, y, z), (x, y, z), q, 0.7, n, 400, 400)[0])
            for n in (1, 3, 5, 7)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert 1e-9 < errs[2] < 1e-4 and errs[0] > 1e-4, errs


# ---------------------------------------------------------------------------------------
# Barycentric Hermite treecode (future work of Sec. V)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 3, 6])
def test_hermite_basis_reproduces_degree_2n_plus_1(n):
    rng = np.random.default_rng(n)
    lo, hi = -0.3, 1.7
    s, _ = oracle.cheb(n, lo, hi)
    for deg, exact in ((2 * n + 1, True), (2 * n + 2, False)):
        c = rng.normal(size=deg + 1)
        p = np.polynomial.Polynomial(c)
        dp = p.deriv()
        errs = []
        for yv in rng.uniform(lo, hi, 25):
            h, k = oracle.hermite_factors(n, lo, hi, yv)
            errs.append(abs(np.dot(p(s), h) + np.dot(dp(s), k) - p(yv)) / np.sum(np.abs(c)))
        assert (max(errs) < 1e-12) == exact, (deg, max(errs))
    # at a node: H = e_m, K = 0 (the exact-hit rule)
    h, k = oracle.hermite_factors(n, lo, hi, s[n // 2])
    assert np.array_equal(h, np.eye(n + 1)[n // 2]) and not np.any(k)


@pytest.mark.parametrize("kernel,kappa", [(oracle.KERNEL_COULOMB, 0.0), (oracle.KERNEL_YUKAWA, 0.7),
                                          (oracle.KERNEL_SOFT, 0.2)])
def test_kernel_derivatives_match_finite_differences(kernel, kappa):
    # D^a G from central differences of G itself in the source coordinates
    x = np.array([0.3, -0.2, 0.5])
    y0 = np.array([-0.4, 0.35, -0.15])
    G = lambda yy: oracle.kernel_derivatives(kernel, kappa, 0, x, yy)[0]
    hstep = 1e-3
    got = oracle.kernel_derivatives(kernel, kappa, 0, x, y0)
    for a in range(8):
        dims = [l for l in range(3) if (a >> (2 - l)) & 1]
        tot = 0.0
        for signs in np.ndindex(*([2] * len(dims))):
            yy = y0.copy()
            sgn = 1.0
            for l, sbit in zip(dims, signs):
                yy[l] += hstep if sbit else -hstep
                sgn *= 1.0 if sbit else -1.0
            tot += sgn * G(yy)
        fd = tot / (2 * hstep) ** len(dims)
        assert abs(fd - got[a]) <= 1e-5 * max(1.0, abs(got[a])), (a, fd, got[a])


def test_hermite_treecode_theta0_polynomial_and_decay():
    x, y, z, q = _system(8000, 20031879)
    pts = np.stack([x, y, z])
    ref = oracle.direct_sum(pts, pts, q)
    phi, _ = oracle.bltc_hermite(x, y, z, q, 0.0, 3, 300, 300)
    assert oracle.rel_err(ref, phi) < 1e-14
    # a kernel of degree 2n+1 in every source coordinate is reproduced exactly
    n = 2
    phi, _ = oracle.bltc_hermite(x, y, z, q, 0.7, n, 300, 300, oracle.KERNEL_POLY)
    refp, refp_abs = oracle.direct_sum(pts, pts, q, oracle.KERNEL_POLY, 0.0, 2 * n + 1, with_abs=True)
    assert np.max(np.abs(phi - refp) / refp_abs) < 1e-12
    # the approximation is used: some cluster has more than 8 (n+1)^3 particles and passes
    st = oracle.Tree(x, y, z, 300)
    L = oracle.lists(st, st, 0.7, 2 * n + 1)    # (2n+2)^3 = 8 (n+1)^3 points: the same test
    assert len(L["approx_ids"]) > 0
    # the error falls with n; Hermite at n is more accurate than Lagrange at n
    x2, y2, z2, q2 = _system(20000, 20031881)
    p2 = np.stack([x2, y2, z2])
    ref2 = oracle.direct_sum(p2, p2, q2)
    eh = [oracle.rel_err(ref2, oracle.bltc_hermite(x2, y2, z2, q2, 0.7, n, 200, 200)[0]) for n in (1, 2, 3)]
    assert eh[0] > eh[1] > eh[2], eh
    el = oracle.rel_err(ref2, oracle.bltc(x2, y2, z2, q2, 0.7, 3, 200, 200)[0])
    assert eh[2] < el, (eh, el)


def test_hermite_factors_n1_are_the_cubic_hermite_basis():
    # n = 1 on [0, 1]: points s_0 = 1, s_1 = 0 and the textbook cubic Hermite basis
    # H_0 = (3 - 2y) y^2, K_0 = (y - 1) y^2, H_1 = (1 + 2y)(1 - y)^2, K_1 = y (1 - y)^2
    for yv in (0.25, 0.5, 0.875):
        h, k = oracle.hermite_factors(1, 0.0, 1.0, yv)
        want_h = [(3 - 2 * yv) * yv * yv, (1 + 2 * yv) * (1 - yv) ** 2]
        want_k = [(yv - 1) * yv * yv, yv * (1 - yv) ** 2]
        assert np.allclose(h, want_h, rtol=0, atol=1e-15), (yv, h, want_h)
        assert np.allclose(k, want_k, rtol=0, atol=1e-15), (yv, k, want_k)


# ---------------------------------------------------------------------------------------
# Absolute-value sums sum_j |G(x_i, y_j) q_j| over the terms each path adds (the scale of
# every per-target parity bar of the GPU tests)
# ---------------------------------------------------------------------------------------

def test_direct_abs_sum_closed_forms():
    # two charges of opposite sign at distance 0.5: each sees |q_other| / d (Eq. 1-2)
    pts = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.5]]).T
    q = np.array([0.75, -0.25])
    phi, phi_abs = oracle.direct_sum(pts, pts, q, with_abs=True)
    assert phi.tolist() == [-0.5, 1.5] and phi_abs.tolist() == [0.5, 1.5]
    kappa = 0.5
    _, phi_abs = oracle.direct_sum(pts, pts, q, oracle.KERNEL_YUKAWA, kappa, with_abs=True)
    e = math.exp(-kappa * 0.5) / 0.5
    assert phi_abs[0] == pytest.approx(0.25 * e, rel=1e-15)
    assert phi_abs[1] == pytest.approx(0.75 * e, rel=1e-15)
    # 5-12-13 triangle with charges of both signs: exact rationals
    pts = np.array([[0, 0, 0], [3, 4, 0], [3, 4, 12]], dtype=np.float64).T
    phi, phi_abs = oracle.direct_sum(pts, pts, np.array([1.0, -2.0, 3.0]), with_abs=True)
    want = [Fraction(2, 5) + Fraction(3, 13), Fraction(1, 5) + Fraction(3, 12),
            Fraction(1, 13) + Fraction(2, 12)]
    want_phi = [-Fraction(2, 5) + Fraction(3, 13), Fraction(1, 5) + Fraction(3, 12),
                Fraction(1, 13) - Fraction(2, 12)]
    for p, pa, w, wp in zip(phi, phi_abs, want, want_phi):
        assert abs(Fraction(pa) - w) <= Fraction(1, 2 ** 50)
        assert abs(Fraction(p) - wp) <= Fraction(1, 2 ** 50)
    # cube corners with checkerboard charges: every corner has 3 neighbours of the other
    # sign at a, 3 of its own sign at a sqrt2 and 1 of the other sign at a sqrt3
    a = 0.75
    pts = np.array([[a * i, a * j, a * k] for i in (0, 1) for j in (0, 1) for k in (0, 1)]).T
    q = np.array([(-1.0) ** (i + j + k) for i in (0, 1) for j in (0, 1) for k in (0, 1)])
    phi, phi_abs = oracle.direct_sum(pts, pts, q, with_abs=True)
    np.testing.assert_allclose(phi_abs, 3 / a + 3 / (a * math.sqrt(2)) + 1 / (a * math.sqrt(3)),
                               rtol=2e-16 * 8)
    np.testing.assert_allclose(phi * q, -3 / a + 3 / (a * math.sqrt(2)) - 1 / (a * math.sqrt(3)),
                               rtol=2e-16 * 16)


def test_abs_sums_at_theta_zero_equal_the_direct_sums():
    # theta = 0: every path is the direct sum (no cluster passes the MAC), so the absolute
    # sums hold the same positive terms in another order; with positive charges every term
    # is positive and the absolute sum is the potential itself, bit for bit
    x, y, z, q = _system(3000, 20031893)
    pts = np.stack([x, y, z])
    _, ref_abs = oracle.direct_sum(pts, pts, q, with_abs=True)
    got = {"bltc": oracle.bltc(x, y, z, q, 0.0, 4, 200, 200, with_abs=True)[1],
           "ts": oracle.bltc_ts((x, y, z), (x, y, z), q, 0.0, 4, 200, 150, with_abs=True)[1],
           "cp": oracle.bltc_cp((x, y, z), (x, y, z), q, 0.0, 4, 200, 150, with_abs=True)[1],
           "cc": oracle.bltc_cc((x, y, z), (x, y, z), q, 0.0, 4, 200, 150, with_abs=True)[1],
           "hermite": oracle.bltc_hermite(x, y, z, q, 0.0, 2, 200, 200, with_abs=True)[1]}
    # two orders of a sum of 3000 positive terms differ by at most 2 * 3000 * 2^-53 relative
    for name, pa in got.items():
        assert np.max(np.abs(pa - ref_abs) / ref_abs) < 1e-12, name
    qp = np.abs(q)
    phi, phi_abs = oracle.direct_sum(pts, pts, qp, with_abs=True)
    assert np.array_equal(phi, phi_abs)
    phi, phi_abs, _ = oracle.bltc(x, y, z, qp, 0.0, 4, 200, 200, with_abs=True)
    assert np.array_equal(phi, phi_abs)


def _corner_clusters(per_corner, seed=20031895, degree=1):
    """Four clusters in opposite corners of [-1, 1]^3, each with `per_corner` particles on
    each of its (degree+1)^3 interpolation points and one charge sign per point.  The boxes
    are the minimal ones; at degree 1 their Chebyshev points are the box corners (s_0 = hi,
    s_1 = lo), at degree 2 also the box midpoints (cos(pi/2) + 1 rounds to 1, so s_1 =
    lo + (hi - lo)/2, exact for these boxes of width 1/4).  Every particle is an exact hit
    (Sec. II-C): a modified charge is the sum of the charges at its point, one sign, and
    each far-field term G(x, s_k) qhat_k equals the direct terms of those particles,
    absolute values included."""
    rng = np.random.default_rng(seed)
    X, Q = [], []
    for c in ((-1, -1, -1), (1, 1, 1), (-1, 1, -1), (1, -1, 1)):
        lo = [0.75 if ci > 0 else -1.0 for ci in c]
        hi = [1.0 if ci > 0 else -0.75 for ci in c]
        axes = [[lo[d], hi[d]] if degree == 1 else [lo[d], lo[d] + 0.125, hi[d]]
                for d in range(3)]
        for point in np.ndindex(*([degree + 1] * 3)):
            sign = 1.0 if rng.random() < 0.5 else -1.0
            for _ in range(per_corner):
                X.append([axes[d][point[d]] for d in range(3)])
                Q.append(sign * rng.uniform(0.25, 1.0))
    order = rng.permutation(len(Q))
    X = np.array(X)[order]
    return X[:, 0].copy(), X[:, 1].copy(), X[:, 2].copy(), np.array(Q)[order]


def _assert_matches_direct(phi, phi_abs, ref, ref_abs, what):
    # sums of at most a few hundred terms in another order and grouping
    assert np.max(np.abs(phi - ref) / ref_abs) < 1e-13, what
    assert np.max(np.abs(phi_abs - ref_abs) / ref_abs) < 1e-13, what


def test_abs_sums_of_exact_far_fields_equal_the_direct_sums():
    # with the particles on their clusters' interpolation points the far fields are exact,
    # so every path's potential AND absolute sum equal the direct sum's, while clusters are
    # approximated (theta 0.5 passes every pair of the four clusters)
    x, y, z, q = _corner_clusters(2)
    pts = np.stack([x, y, z])
    ref, ref_abs = oracle.direct_sum(pts, pts, q, with_abs=True)
    st = oracle.Tree(x, y, z, 16)
    assert len(st.leaves) == 4 and len(oracle.lists(st, st, 0.5, 1)["approx_ids"]) == 12
    phi, phi_abs, _ = oracle.bltc(x, y, z, q, 0.5, 1, 16, 16, with_abs=True)
    _assert_matches_direct(phi, phi_abs, ref, ref_abs, "bltc")
    phi, phi_abs = oracle.bltc_cp((x, y, z), (x, y, z), q, 0.5, 1, 16, 16, with_abs=True)
    _assert_matches_direct(phi, phi_abs, ref, ref_abs, "cp")
    phi, phi_abs = oracle.bltc_cc((x, y, z), (x, y, z), q, 0.5, 1, 16, 16, with_abs=True)
    _assert_matches_direct(phi, phi_abs, ref, ref_abs, "cc")
    assert len(oracle.dual_lists(st, st, 0.5, 1)["cc"][0]) > 0
    # distinct targets scattered through the cube: the batches near a cluster sum it
    # directly, the far ones approximate it
    tx, ty, tz, _ = inputs.uniform_cube(400, 20031897)
    tp = np.stack([tx, ty, tz])
    ref, ref_abs = oracle.direct_sum(tp, pts, q, with_abs=True)
    phi, phi_abs, _ = oracle.bltc_ts((tx, ty, tz), (x, y, z), q, 0.5, 1, 16, 25, with_abs=True)
    _assert_matches_direct(phi, phi_abs, ref, ref_abs, "ts")
    L = oracle.lists(oracle.Tree(tx, ty, tz, 25), st, 0.5, 1)
    assert len(L["approx_ids"]) > 0 and len(L["direct_ids"]) > 0
    # Hermite: the size test is 8 (n+1)^3 = 64 < N_C; at a node H = e_m and K = 0, so only
    # the value charges are nonzero and the far field is again the direct sum term by term
    x, y, z, q = _corner_clusters(9, 20031899)
    pts = np.stack([x, y, z])
    ref, ref_abs = oracle.direct_sum(pts, pts, q, with_abs=True)
    st = oracle.Tree(x, y, z, 72)
    assert len(oracle.lists(st, st, 0.5, 3)["approx_ids"]) == 12
    phi, phi_abs = oracle.bltc_hermite(x, y, z, q, 0.5, 1, 72, 72, with_abs=True)
    _assert_matches_direct(phi, phi_abs, ref, ref_abs, "hermite")


def _lagrange_basis(nodes, x):
    """L_k(x) = prod_{m != k} (x - s_m) / (s_k - s_m): Eq. 4's definition, term by term."""
    out = np.ones(len(nodes))
    for k in range(len(nodes)):
        for m in range(len(nodes)):
            if m != k:
                out[k] *= (x - nodes[m]) / (nodes[k] - nodes[m])
    return out


def test_abs_sums_of_interpolated_targets():
    # Targets far from four on-grid source clusters, a kernel of degree n = 2 in every
    # coordinate (non-negative for even n): the cluster-particle and cluster-cluster
    # variants interpolate the point potentials of the one target cluster exactly, and
    # their absolute sums are sum_k |L_k1(x) L_k2(x) L_k3(x)| psi(t_k) with
    # psi(t) = sum_j G(t, y_j) |q_j| at the target box's Chebyshev points t_k.  The
    # Lagrange factors here come from Eq. 4's product form, psi from the direct sum.
    n = 2
    sx, sy, sz, q = _corner_clusters(2, 20031901, degree=n)
    tx, ty, tz, _ = inputs.uniform_cube(300, 20031903)
    tx, ty, tz = 3.15 + 0.15 * tx, 0.15 * ty, 0.15 * tz
    T, S = (tx, ty, tz), (sx, sy, sz)
    ref, ref_abs = oracle.direct_sum(np.stack(T), np.stack(S), q, oracle.KERNEL_POLY, 0.0, n,
                                     with_abs=True)
    grids = [oracle.cheb(n, a.min(), a.max())[0] for a in T]
    g = np.array([[u, v, w] for u in grids[0] for v in grids[1] for w in grids[2]]).T
    psi = oracle.direct_sum(g, np.stack(S), np.abs(q), oracle.KERNEL_POLY, 0.0, n)
    want_abs = np.array([np.sum(np.abs(np.einsum("a,b,c->abc", *[_lagrange_basis(grids[d], p[d])
                                                                 for d in range(3)])).ravel() * psi)
                         for p in zip(tx, ty, tz)])
    assert np.all(want_abs > ref_abs * (1 + 1e-6))      # some factors are negative off the nodes
    tt, st = oracle.Tree(tx, ty, tz, 50), oracle.Tree(sx, sy, sz, 54)
    assert len(oracle.lists(st, tt, 0.5, n)["approx_ids"]) == 4
    assert len(oracle.dual_lists(tt, st, 0.5, n)["cc"][0]) > 0
    for name, fn in (("cp", oracle.bltc_cp), ("cc", oracle.bltc_cc)):
        lb = (50, 54) if name == "cp" else (54, 50)
        phi, phi_abs = fn(T, S, q, 0.5, n, *lb, oracle.KERNEL_POLY, with_abs=True)
        assert np.max(np.abs(phi - ref) / ref_abs) < 1e-13, name
        assert np.max(np.abs(phi_abs - want_abs) / want_abs) < 1e-13, name
    # the treecode approximates the source clusters (exactly, on their nodes) instead
    phi, phi_abs, _ = oracle.bltc_ts(T, S, q, 0.5, n, 54, 50, oracle.KERNEL_POLY, with_abs=True)
    _assert_matches_direct(phi, phi_abs, ref, ref_abs, "ts")
    # 20 far targets form one leaf too small to interpolate ((n+1)^3 = 27 points): the
    # dual traversal pairs it with the source clusters as particle-cluster (PC) terms,
    # exact on the source nodes, absolute values included
    T20 = tuple(a[:20].copy() for a in T)
    ref, ref_abs = oracle.direct_sum(np.stack(T20), np.stack(S), q, oracle.KERNEL_POLY, 0.0, n,
                                     with_abs=True)
    assert len(oracle.dual_lists(oracle.Tree(*T20, 50), st, 0.5, n)["pc"][0]) == 4
    phi, phi_abs = oracle.bltc_cc(T20, S, q, 0.5, n, 54, 50, oracle.KERNEL_POLY, with_abs=True)
    _assert_matches_direct(phi, phi_abs, ref, ref_abs, "cc particle-cluster")
