"""A solve with fixed positions replayed as one CUDA graph (bltc_graph_*): a launch gives the
bits bltc_solve gives for the same positions and the charges currently in the bound tensor,
for new charges too, for FP64 and mixed, Coulomb, Yukawa and a registered kernel, batch != leaf;
the FP64 replay matches the oracle; a launch runs the captured kernels and nothing else."""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import FP64_ELEM, FP64_REL2, assert_close_abs, dev, host, system

pytestmark = pytest.mark.gpu

SOFT = """
__device__ float bltc_user_g32(float r2, float r, float eps) { return rsqrtf(r2 + eps * eps); }
__device__ double bltc_user_g64(double r2, double r, double eps) { return 1.0 / sqrt(r2 + eps * eps); }
"""


def _solve(gpu, X, q, p):
    import torch
    phi = torch.empty_like(X[0])
    b.bltc_solve(gpu.h, *X, q, p, phi)
    torch.cuda.synchronize()
    return host(phi)


CASES = [
    # kind, N, leaf, batch, theta, n, kernel, kappa, precision
    ("cube", 30000, 800, 800, 0.7, 6, 0, 0.0, b.BLTC_PRECISION_MIXED),
    ("plummer", 40000, 1000, 1000, 0.8, 8, 1, 0.5, b.BLTC_PRECISION_MIXED),
    ("cube", 25011, 1200, 500, 0.6, 5, 0, 0.0, b.BLTC_PRECISION_MIXED),
    ("cube", 20000, 700, 700, 0.7, 4, 0, 0.0, b.BLTC_PRECISION_FP64),
    ("plummer", 15000, 400, 600, 0.8, 3, 1, 0.5, b.BLTC_PRECISION_FP64),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}-b{c[3]}-n{c[5]}-k{c[6]}-p{c[8]}")
def test_graph_replays_give_solve_bits(gpu, case):
    import torch
    kind, n, leaf, batch, theta, deg, ker, kappa, prec = case
    x, y, z, q0 = system(kind, n, 20031940 + n)
    q1 = np.random.default_rng(n).uniform(-1.0, 1.0, n)
    X = dev(x, y, z)
    p = b.params(deg, theta, leaf, batch, ker, kappa, prec)
    qd = dev(q0)[0]
    g = b.Graph(gpu, *X, qd, p)
    try:
        first = host(g.phi).copy()                      # the solve run at creation
        want0 = _solve(gpu, X, dev(q0)[0], p)
        assert np.array_equal(first, want0)
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(host(g.phi), want0)
        qd.copy_(torch.from_numpy(q1))                   # new charges, same positions
        g.launch()
        torch.cuda.synchronize()
        got1 = host(g.phi).copy()
        assert np.array_equal(got1, _solve(gpu, X, dev(q1)[0], p))
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(host(g.phi), got1)
        if prec == b.BLTC_PRECISION_FP64:
            want, want_abs, _ = oracle.bltc(x, y, z, q1, theta, deg, leaf, batch, ker, kappa, with_abs=True)
            assert_close_abs(want, got1, want_abs, FP64_REL2, FP64_ELEM, "graph fp64 vs oracle")
    finally:
        g.close()


def test_graph_launch_runs_the_captured_kernels(gpu):
    import torch
    x, y, z, q = system("cube", 20000, 20031941)
    X = dev(x, y, z, q)
    g = b.Graph(gpu, *X, b.params(6, 0.7, 700, 700))
    try:
        k = g.kernels
        assert k >= 4                                    # gather, leaf sums, reduce, sweep, finalize
        c0 = b.bltc_context_launch_count(gpu.h)
        for _ in range(3):
            g.launch()
        torch.cuda.synchronize()
        assert b.bltc_context_launch_count(gpu.h) - c0 == 3 * k
    finally:
        g.close()


def test_graph_with_registered_kernel(gpu):
    import torch
    st, log = b.bltc_kernel_check(SOFT, 103)
    if st == b.BLTC_ERR_STATE:
        pytest.skip("NVRTC not available: " + log)
    kid = b.bltc_kernel_register(gpu.h, SOFT)
    x, y, z, q = system("plummer", 20000, 20031942)
    X = dev(x, y, z)
    qd = dev(q)[0]
    p = b.params(6, 0.7, 600, 600, kid, 0.05, b.BLTC_PRECISION_MIXED)
    g = b.Graph(gpu, *X, qd, p)
    try:
        qd.mul_(-0.5)
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(host(g.phi), _solve(gpu, X, dev(-0.5 * q)[0], p))
    finally:
        g.close()


def test_graph_single_particle_and_errors(gpu):
    import torch
    X = dev(np.array([0.25]), np.array([-0.5]), np.array([0.125]), np.array([0.75]))
    g = b.Graph(gpu, *X, b.params(4, 0.7, 10, 10))
    try:
        g.launch()
        torch.cuda.synchronize()
        assert host(g.phi)[0] == 0.0
        other = b.Context(0)
        try:
            with pytest.raises(b.BltcError):
                b.bltc_graph_launch(other.h, g.h)
        finally:
            other.close()
    finally:
        g.close()
    x, y, z, q = system("cube", 1000, 20031943)
    X = dev(x, y, z, q)
    with pytest.raises(b.BltcError):
        b.Graph(gpu, *X, b.params(4, 1.5, 100, 100))      # theta >= 1 is rejected
