"""The cluster-cluster variant (dual tree traversal, future work of Sec. V): the GPU's four
interaction lists equal the oracle's (as sets of (target node, source node) pairs, bit-exact
decisions), and bltc_solve_cc matches the oracle's algorithm (FP64 1e-12, mixed 1e-6)."""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import (FP64_ELEM, FP64_REL2, MIXED_ELEM, MIXED_REL2, assert_close_abs, dev, gpu_tree,
                         host, system)

pytestmark = pytest.mark.gpu


def _pairs(t, s):
    return sorted(zip(t.tolist(), s.tolist()))


@pytest.mark.parametrize("same", [True, False])
def test_dual_lists_bit_exact(gpu, same):
    x, y, z, q = system("plummer", 20000, 20031911)
    if same:
        tx, ty, tz = x, y, z
    else:
        tx, ty, tz, _ = system("cube", 9000, 20031912)
    st, _ = gpu_tree(gpu, x, y, z, q, 300)
    tt, _ = gpu_tree(gpu, tx, ty, tz, None, 200)
    try:
        for theta, deg in ((0.7, 4), (0.5, 2), (0.9, 6)):
            got = b.bltc_dual_lists(gpu.h, tt, st, b.params(deg, theta, 300, 200))
            want = oracle.dual_lists(oracle.Tree(tx, ty, tz, 200), oracle.Tree(x, y, z, 300), theta, deg)
            for k in ("cc", "cp", "pc", "pp"):
                assert _pairs(*got[k]) == _pairs(*want[k]), (theta, deg, k)
    finally:
        b.bltc_tree_destroy(st)
        b.bltc_tree_destroy(tt)


def _solve(gpu, T, S, q, p, shared=False):
    import torch
    if shared:
        X = dev(*S, q)
        Td, Sd = X[:3], X
    else:
        Td, Sd = dev(*T), dev(*S, q)
    phi = torch.empty_like(Td[0])
    b.bltc_solve_cc(gpu.h, *Td, *Sd, p, phi)
    torch.cuda.synchronize()
    return host(phi)


CASES = [
    # targets, sources, leaf (sources), batch (targets), theta, n, kernel, kappa, shared arrays
    (("cube", 20000), ("cube", 20000), 500, 500, 0.7, 4, 0, 0.0, True),
    (("plummer", 30000), ("plummer", 30000), 800, 800, 0.8, 6, 1, 0.5, True),
    (("cube", 12011), ("plummer", 9001), 400, 700, 0.6, 5, 0, 0.0, False),
    (("cube", 6000), ("cube", 1500), 40, 400, 0.7, 3, 0, 0.0, False),     # CP and PC terms
    (("cube", 3), ("cube", 30000), 2000, 1, 0.7, 8, 0, 0.0, False),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0][0]}{c[0][1]}-{c[1][0]}{c[1][1]}-n{c[5]}-k{c[6]}")
def test_cc_fp64_and_mixed(gpu, case):
    (tk, tn), (sk, sn), leaf, batch, theta, deg, ker, kappa, shared = case
    sx, sy, sz, q = system(sk, sn, 20031913 + sn)
    if shared:
        tx, ty, tz = sx, sy, sz
    else:
        tx, ty, tz, _ = system(tk, tn, 20031914 + tn)
    T, S = (tx, ty, tz), (sx, sy, sz)
    want, want_abs = oracle.bltc_cc(T, S, q, theta, deg, leaf, batch, ker, kappa, with_abs=True)
    p64 = b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_FP64)
    pmx = b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_MIXED)
    got64 = _solve(gpu, T, S, q, p64, shared)
    gotmx = _solve(gpu, T, S, q, pmx, shared)
    assert_close_abs(want, got64, want_abs, FP64_REL2, FP64_ELEM, "cc fp64 vs oracle")
    assert_close_abs(got64, gotmx, want_abs, MIXED_REL2, MIXED_ELEM, "cc mixed vs fp64")
