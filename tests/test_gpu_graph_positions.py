"""The whole solve as one CUDA graph, sized on the device (bltc_graph_create_positions): every
launch reads the positions and charges now in the bound tensors and gives the bits bltc_solve
gives for them, for FP64 and mixed, Coulomb and Yukawa, batch != leaf; positions that outgrow the
capacities are solved on the host-driven path and the graph is rebuilt; non-finite positions are
reported; the FP64 graph matches the oracle."""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from gpu_helpers import FP64_ELEM, FP64_REL2, assert_close_abs, dev, host, system

pytestmark = pytest.mark.gpu


def _solve(gpu, x, y, z, q, p):
    import torch
    X = dev(x, y, z, q)
    phi = torch.empty_like(X[0])
    b.bltc_solve(gpu.h, *X, p, phi)
    torch.cuda.synchronize()
    return host(phi)


def _load(X, x, y, z, q):
    import torch
    for t, a in zip(X, (x, y, z, q)):
        t.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)))


CASES = [
    # kind, N, leaf, batch, theta, n, kernel, kappa, precision
    ("cube", 30000, 800, 800, 0.7, 6, 0, 0.0, b.BLTC_PRECISION_MIXED),
    ("plummer", 40000, 1000, 1000, 0.8, 8, 1, 0.5, b.BLTC_PRECISION_MIXED),
    ("cube", 25011, 1200, 500, 0.6, 5, 0, 0.0, b.BLTC_PRECISION_MIXED),
    ("cube", 20000, 700, 700, 0.7, 4, 0, 0.0, b.BLTC_PRECISION_FP64),
    ("plummer", 15000, 400, 600, 0.8, 3, 1, 0.5, b.BLTC_PRECISION_FP64),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}-b{c[3]}-n{c[5]}-k{c[6]}-p{c[8]}")
def test_positions_graph_gives_solve_bits(gpu, case):
    import torch
    kind, n, leaf, batch, theta, deg, ker, kappa, prec = case
    x, y, z, q = system(kind, n, 20031950 + n)
    p = b.params(deg, theta, leaf, batch, ker, kappa, prec)
    X = dev(x, y, z, q)
    g = b.Graph(gpu, *X[:3], X[3], p, positions=True)
    try:
        want = _solve(gpu, x, y, z, q, p)
        assert np.array_equal(host(g.phi), want)           # the solve run at creation
        g.launch()
        assert np.array_equal(host(g.phi), want)
        # moved particles and new charges: a small displacement of every particle
        rng = np.random.default_rng(n)
        x1, y1, z1 = (a + 1e-3 * rng.standard_normal(n) for a in (x, y, z))
        q1 = rng.uniform(-1.0, 1.0, n)
        _load(X, x1, y1, z1, q1)
        g.launch()
        got1 = host(g.phi).copy()
        assert np.array_equal(got1, _solve(gpu, x1, y1, z1, q1, p))
        g.launch()
        assert np.array_equal(host(g.phi), got1)
        # another draw of the same distribution
        x2, y2, z2, q2 = system(kind, n, 20031960 + n)
        _load(X, x2, y2, z2, q2)
        g.launch()
        torch.cuda.synchronize()
        got2 = host(g.phi).copy()
        assert np.array_equal(got2, _solve(gpu, x2, y2, z2, q2, p))
        info = g.info
        assert info["launches"] == 4 and info["kernels"] > 0
        if prec == b.BLTC_PRECISION_FP64:
            ref, ref_abs, _ = oracle.bltc(x2, y2, z2, q2, theta, deg, leaf, batch, ker, kappa, with_abs=True)
            assert_close_abs(ref, got2, ref_abs, FP64_REL2, FP64_ELEM, "positions graph fp64 vs oracle")
    finally:
        g.close()


def test_positions_graph_outgrown_capacities_are_redone(gpu):
    # capacities from a uniform cube with no headroom; a Plummer sphere of the same size needs a
    # deeper tree with more nodes and levels: the launch is redone on the host-driven path and the
    # graph rebuilt, and the next launches run the new graph
    import torch
    n = 30000
    p = b.params(6, 0.7, 500, 500)
    x, y, z, q = system("cube", n, 20031970)
    X = dev(x, y, z, q)
    g = b.Graph(gpu, *X[:3], X[3], p, positions=True, headroom=1.0)
    try:
        assert g.info["captures"] == 1
        xp, yp, zp, qp = system("plummer", n, 20031971)
        _load(X, xp, yp, zp, qp)
        g.launch()
        want = _solve(gpu, xp, yp, zp, qp, p)
        assert np.array_equal(host(g.phi), want)
        info = g.info
        assert info["redone"] == 1 and info["captures"] == 2
        c0 = b.bltc_context_launch_count(gpu.h)
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(host(g.phi), want)
        assert g.info["redone"] == 1
        assert b.bltc_context_launch_count(gpu.h) - c0 == g.kernels
        # back to the cube: correct whether or not it fits the Plummer sphere's capacities
        _load(X, x, y, z, q)
        g.launch()
        assert np.array_equal(host(g.phi), _solve(gpu, x, y, z, q, p))
        assert g.info["redone"] in (1, 2)
    finally:
        g.close()


def test_positions_graph_reports_non_finite_positions(gpu):
    n = 5000
    p = b.params(4, 0.7, 300, 300)
    x, y, z, q = system("cube", n, 20031972)
    X = dev(x, y, z, q)
    g = b.Graph(gpu, *X[:3], X[3], p, positions=True)
    try:
        bad = x.copy()
        bad[17] = np.nan
        _load(X, bad, y, z, q)
        with pytest.raises(b.BltcError):
            g.launch()
        _load(X, x, y, z, q)
        g.launch()
        assert np.array_equal(host(g.phi), _solve(gpu, x, y, z, q, p))
    finally:
        g.close()


def test_positions_graph_single_particle_and_headroom(gpu):
    X = dev(np.array([0.25]), np.array([-0.5]), np.array([0.125]), np.array([0.75]))
    g = b.Graph(gpu, *X[:3], X[3], b.params(4, 0.7, 10, 10), positions=True)
    try:
        g.launch()
        assert host(g.phi)[0] == 0.0
    finally:
        g.close()
    x, y, z, q = system("cube", 1000, 20031973)
    X = dev(x, y, z, q)
    with pytest.raises(b.BltcError):
        b.Graph(gpu, *X[:3], X[3], b.params(4, 0.7, 100, 100), positions=True, headroom=0.5)


SOFT = """
__device__ float bltc_user_g32(float r2, float r, float eps) { return rsqrtf(r2 + eps * eps); }
__device__ double bltc_user_g64(double r2, double r, double eps) { return 1.0 / sqrt(r2 + eps * eps); }
"""


def test_positions_graph_with_registered_kernel(gpu):
    # a kernel compiled at run time is launched inside the capture like the built-in ones
    st, log = b.bltc_kernel_check(SOFT, 103)
    if st == b.BLTC_ERR_STATE:
        pytest.skip("NVRTC not available: " + log)
    kid = b.bltc_kernel_register(gpu.h, SOFT)
    x, y, z, q = system("plummer", 20000, 20031974)
    p = b.params(6, 0.7, 600, 600, kid, 0.05, b.BLTC_PRECISION_MIXED)
    X = dev(x, y, z, q)
    g = b.Graph(gpu, *X[:3], X[3], p, positions=True)
    try:
        x1, y1, z1, q1 = system("plummer", 20000, 20031975)
        _load(X, x1, y1, z1, q1)
        g.launch()
        assert np.array_equal(host(g.phi), _solve(gpu, x1, y1, z1, q1, p))
    finally:
        g.close()
