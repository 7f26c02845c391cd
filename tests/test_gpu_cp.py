"""The cluster-particle variant (future work of Sec. V): targets interpolated, sources summed
exactly.  bltc_solve_cp against the oracle's cluster-particle Algorithm (FP64 within 1e-12
of the absolute sum per target and in the relative 2-norm; mixed within 1e-6 of FP64)."""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import (FP64_ELEM, FP64_REL2, MIXED_ELEM, MIXED_REL2, assert_close_abs, dev, host,
                         system)

pytestmark = pytest.mark.gpu


def _solve(gpu, T, S, q, p):
    import torch
    Td, Sd = dev(*T), dev(*S, q)
    phi = torch.empty_like(Td[0])
    b.bltc_solve_cp(gpu.h, *Td, *Sd, p, phi)
    torch.cuda.synchronize()
    return host(phi)


CASES = [
    # targets (kind, n), sources (kind, n), leaf (targets), batch (sources), theta, n, kernel, kappa
    (("cube", 10000), ("cube", 10000), 500, 500, 0.7, 4, 0, 0.0),
    (("plummer", 30000), ("plummer", 30000), 1000, 800, 0.8, 6, 1, 0.5),
    (("cube", 20011), ("plummer", 7001), 700, 300, 0.6, 5, 0, 0.0),
    (("cube", 3), ("cube", 50000), 1, 2000, 0.7, 8, 0, 0.0),          # three targets
    (("cube", 40000), ("cube", 5), 3000, 1, 0.7, 2, 1, 1.0),          # five sources
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0][0]}{c[0][1]}-{c[1][0]}{c[1][1]}-n{c[5]}-k{c[6]}")
def test_cp_fp64_and_mixed(gpu, case):
    (tk, tn), (sk, sn), leaf, batch, theta, deg, ker, kappa = case
    tx, ty, tz, _ = system(tk, tn, 20031901 + tn)
    if (tk, tn) == (sk, sn):
        sx, sy, sz, q = system(tk, tn, 20031901 + tn)            # targets = sources
    else:
        sx, sy, sz, q = system(sk, sn, 20031902 + sn)
    T, S = (tx, ty, tz), (sx, sy, sz)
    want, want_abs = oracle.bltc_cp(T, S, q, theta, deg, leaf, batch, ker, kappa, with_abs=True)
    got64 = _solve(gpu, T, S, q, b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_FP64))
    gotmx = _solve(gpu, T, S, q, b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_MIXED))
    assert_close_abs(want, got64, want_abs, FP64_REL2, FP64_ELEM, "cp fp64 vs oracle")
    assert_close_abs(got64, gotmx, want_abs, MIXED_REL2, MIXED_ELEM, "cp mixed vs fp64")


def test_cp_theta0_and_determinism(gpu):
    x, y, z, q = system("cube", 8000, 20031905)
    T = S = (x, y, z)
    got = _solve(gpu, T, S, q, b.params(5, 0.0, 400, 300, precision=b.BLTC_PRECISION_FP64))
    ref = oracle.direct_sum(np.stack(T), np.stack(S), q)
    assert oracle.rel_err(ref, got) < 1e-13
    p = b.params(6, 0.7, 400, 400)
    assert np.array_equal(_solve(gpu, T, S, q, p), _solve(gpu, T, S, q, p))


def test_cp_shared_tree_for_same_particles(gpu):
    # targets and sources passed as the same device arrays with leaf = batch share one tree,
    # so the near half's mutual leaf pairs are evaluated once; results as for separate trees
    import torch
    x, y, z, q = system("plummer", 25000, 20031909)
    X = dev(x, y, z, q)
    want, want_abs = oracle.bltc_cp((x, y, z), (x, y, z), q, 0.7, 6, 700, 700, with_abs=True)
    out = {}
    for prec in (b.BLTC_PRECISION_FP64, b.BLTC_PRECISION_MIXED):
        phi = torch.empty_like(X[0])
        b.bltc_solve_cp(gpu.h, *X[:3], *X, b.params(6, 0.7, 700, 700, precision=prec), phi)
        torch.cuda.synchronize()
        out[prec] = host(phi)
    assert_close_abs(want, out[b.BLTC_PRECISION_FP64], want_abs, FP64_REL2, FP64_ELEM, "cp shared fp64")
    assert_close_abs(out[b.BLTC_PRECISION_FP64], out[b.BLTC_PRECISION_MIXED], want_abs, MIXED_REL2,
                     MIXED_ELEM, "cp shared mixed")
