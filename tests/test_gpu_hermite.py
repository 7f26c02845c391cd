"""The barycentric Hermite treecode (future work of Sec. V) on the GPU: bltc_solve_hermite
matches the oracle's algorithm element by element (FP64, 1e-12 of the absolute-value sum),
including clusters with exact hits, ragged batches, batch != leaf and systems where no
cluster passes the size test 8 (n+1)^3 < N_C; the mixed-precision path is within the mixed
bar (1e-6) of the FP64 path; unsupported arguments are rejected."""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import FP64_ELEM, FP64_REL2, MIXED_ELEM, MIXED_REL2, assert_close_abs, dev, host, system

pytestmark = pytest.mark.gpu


def _solve(gpu, x, y, z, q, p):
    import torch
    X = dev(x, y, z, q)
    phi = torch.empty_like(X[0])
    b.bltc_solve_hermite(gpu.h, *X, p, phi)
    torch.cuda.synchronize()
    return host(phi)


CASES = [
    # kind, N, leaf, batch, theta, n, kernel, kappa
    ("cube", 20000, 300, 300, 0.7, 1, 0, 0.0),
    ("cube", 30011, 700, 700, 0.7, 2, 0, 0.0),
    ("plummer", 40000, 1000, 1000, 0.8, 3, 1, 0.5),
    ("cube", 25000, 1200, 400, 0.6, 3, 0, 0.0),          # batch != leaf
    ("plummer", 60000, 5000, 5000, 0.9, 7, 0, 0.0),      # largest degree (8 P = 4096)
    ("cube", 900, 200, 200, 0.7, 3, 0, 0.0),             # no cluster passes the size test
    ("cube", 1, 10, 10, 0.7, 2, 0, 0.0),                 # one particle
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}-n{c[5]}-k{c[6]}-b{c[3]}")
def test_hermite_fp64_vs_oracle(gpu, case):
    kind, n, leaf, batch, theta, deg, ker, kappa = case
    x, y, z, q = system(kind, n, 20031930 + n)
    want, want_abs = oracle.bltc_hermite(x, y, z, q, theta, deg, leaf, batch, ker, kappa, with_abs=True)
    got = _solve(gpu, x, y, z, q, b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_FP64))
    if n == 1:
        assert got[0] == 0.0
        return
    assert_close_abs(want, got, np.maximum(want_abs, 1e-300), FP64_REL2, FP64_ELEM, "hermite fp64 vs oracle")


def test_hermite_exact_hits(gpu):
    """Particles on the Chebyshev points of the root box (lattice of the points of Eq. 6 on
    [0,1]^3 at n = 2): the exact-hit rule H = e_m, K = 0 applies in every dimension."""
    n = 2
    t = 0.5 * (np.cos(np.pi * np.arange(n + 1) / n) + 1.0)
    rng = np.random.default_rng(20031931)
    x, y, z, q = system("cube", 12000, 20031932)
    g = np.array(np.meshgrid(t, t, t, indexing="ij")).reshape(3, -1)
    x = np.concatenate([x, g[0]])
    y = np.concatenate([y, g[1]])
    z = np.concatenate([z, g[2]])
    q = np.concatenate([q, rng.uniform(-1, 1, g.shape[1])])
    want, want_abs = oracle.bltc_hermite(x, y, z, q, 0.7, n, 200, 200, with_abs=True)
    got = _solve(gpu, x, y, z, q, b.params(n, 0.7, 200, 200, 0, 0.0, b.BLTC_PRECISION_FP64))
    assert_close_abs(want, got, want_abs, FP64_REL2, FP64_ELEM, "hermite exact hits")


def test_hermite_is_more_accurate_than_the_treecode_at_equal_degree(gpu):
    """Degree 2n+1 reproduction: at the same n and theta the Hermite far field is closer to
    the direct sum than the Lagrange far field of Eq. 12."""
    x, y, z, q = system("cube", 40000, 20031933)
    p64 = b.params(3, 0.7, 600, 600, 0, 0.0, b.BLTC_PRECISION_FP64)
    X = dev(x, y, z, q)
    import torch
    ref = torch.empty_like(X[0])
    b.bltc_direct_sum(gpu.h, *X[:3], *X, p64, ref)
    torch.cuda.synchronize()
    ref = host(ref)
    herm = _solve(gpu, x, y, z, q, p64)
    lag = torch.empty_like(X[0])
    b.bltc_solve(gpu.h, *X, p64, lag)
    torch.cuda.synchronize()
    assert oracle.rel_err(ref, herm) < oracle.rel_err(ref, host(lag))


MIXED_CASES = [
    # kind, N, leaf, batch, theta, n, kernel, kappa
    ("cube", 30011, 700, 700, 0.7, 2, 0, 0.0),
    ("plummer", 40000, 1000, 1000, 0.8, 3, 1, 0.5),
    ("cube", 25000, 1200, 400, 0.6, 4, 0, 0.0),          # batch != leaf (no mutual pairs)
    ("plummer", 60000, 5000, 5000, 0.9, 7, 1, 0.3),      # largest degree, Yukawa
]


@pytest.mark.parametrize("case", MIXED_CASES, ids=lambda c: f"{c[0]}{c[1]}-n{c[5]}-k{c[6]}-b{c[3]}")
def test_hermite_mixed_vs_fp64(gpu, case):
    kind, n, leaf, batch, theta, deg, ker, kappa = case
    x, y, z, q = system(kind, n, 20031935 + n)
    _, want_abs = oracle.bltc_hermite(x, y, z, q, theta, deg, leaf, batch, ker, kappa, with_abs=True)
    got64 = _solve(gpu, x, y, z, q, b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_FP64))
    gotmx = _solve(gpu, x, y, z, q, b.params(deg, theta, leaf, batch, ker, kappa, b.BLTC_PRECISION_MIXED))
    assert_close_abs(got64, gotmx, want_abs, MIXED_REL2, MIXED_ELEM, "hermite mixed vs fp64")


@pytest.mark.parametrize("bad", ["precision", "degree", "kernel"])
def test_hermite_rejects(gpu, bad):
    x, y, z, q = system("cube", 2000, 20031934)
    p = b.params(3, 0.7, 200, 200, 0, 0.0, b.BLTC_PRECISION_FP64)
    if bad == "precision":
        p.precision = 7
    elif bad == "degree":
        p.degree = 8
    else:
        p.kernel = b.BLTC_KERNEL_USER_BASE
    with pytest.raises(b.BltcError):
        _solve(gpu, x, y, z, q, p)
