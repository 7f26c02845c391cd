"""Distinct target and source sets (Sec. II: the treecode needs only target and source
positions): bltc_solve_targets against the oracle's Algorithm 1 for separate sets, FP64
within 1e-12 and mixed within 1e-6 of the FP64 path, with N_t != N_s and N_B != N_L."""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import (FP64_ELEM, FP64_REL2, MIXED_ELEM, MIXED_REL2, assert_close_abs, dev,
                         gpu_solve, host, system)

pytestmark = pytest.mark.gpu


def _sets(kind_s, ns, nt, seed, coincident=50):
    """Sources of the given kind; targets uniform in a larger shifted box, plus every
    `coincident`-th source position exactly (pairs with r^2 == 0 are skipped)."""
    sx, sy, sz, q = system(kind_s, ns, seed)
    tx, ty, tz, _ = system("cube", nt, seed + 1)
    tx, ty, tz = 1.5 * tx + 0.75, 1.5 * ty, 1.5 * tz - 0.25
    if coincident:
        tx = np.concatenate([tx, sx[::coincident]])
        ty = np.concatenate([ty, sy[::coincident]])
        tz = np.concatenate([tz, sz[::coincident]])
    return (tx, ty, tz), (sx, sy, sz), q


def _solve(gpu, T, S, q, p):
    import torch
    Td, Sd = dev(*T), dev(*S, q)
    phi = torch.empty_like(Td[0])
    b.bltc_solve_targets(gpu.h, *Td, *Sd, p, phi)
    torch.cuda.synchronize()
    return host(phi)


CASES = [
    # source kind, ns, nt, leaf, batch, theta, degree, kernel, kappa
    ("cube", 4000, 2500, 300, 170, 0.7, 4, 0, 0.0),
    ("plummer", 30000, 12000, 1000, 600, 0.8, 6, 1, 0.5),
    ("cube", 50000, 3, 2000, 1, 0.7, 8, 0, 0.0),          # three targets, one per batch
    ("cube", 5, 40000, 1, 3000, 0.7, 2, 0, 0.0),          # five sources: all direct
    ("cube", 1, 1000, 1, 100, 0.5, 3, 1, 1.0),            # one source
    ("cube", 60001, 20011, 2000, 2000, 0.7, 8, 0, 0.0),   # several target tiles, ragged
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}-t{c[2]}-L{c[3]}-B{c[4]}-n{c[6]}-k{c[7]}")
def test_targets_fp64_and_mixed(gpu, case):
    kind, ns, nt, leaf, batch, theta, deg, ker, kappa = case
    T, S, q = _sets(kind, ns, nt, 20031870 + ns + nt,
                    coincident=50 if ns >= 50 and nt >= 100 else 0)
    p64 = b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_FP64)
    pmx = b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_MIXED)
    want, want_abs, _ = oracle.bltc_ts(T, S, q, theta, deg, leaf, batch, ker, kappa, with_abs=True)
    got64 = _solve(gpu, T, S, q, p64)
    gotmx = _solve(gpu, T, S, q, pmx)
    assert_close_abs(want, got64, want_abs, FP64_REL2, FP64_ELEM, "fp64 vs oracle")
    assert_close_abs(got64, gotmx, want_abs, MIXED_REL2, MIXED_ELEM, "mixed vs fp64")


def test_targets_equal_sources_matches_solve_bitwise(gpu):
    x, y, z, q = system("plummer", 20000, 20031877)
    for prec in (b.BLTC_PRECISION_FP64, b.BLTC_PRECISION_MIXED):
        p = b.params(6, 0.7, 700, 400, b.BLTC_KERNEL_YUKAWA, 0.3, prec)
        assert np.array_equal(_solve(gpu, (x, y, z), (x, y, z), q, p), gpu_solve(gpu, x, y, z, q, p))


def test_targets_theta0_is_direct_sum(gpu):
    T, S, q = _sets("cube", 8000, 5000, 20031879)
    got = _solve(gpu, T, S, q, b.params(5, 0.0, 400, 300, precision=b.BLTC_PRECISION_FP64))
    ref = oracle.direct_sum(np.stack(T), np.stack(S), q)
    assert oracle.rel_err(ref, got) < 1e-13
