"""User kernels: a hook for any smooth, non-oscillatory radial G (the treecode needs only
kernel evaluations).  CPU: the run-time compilation of the sweeps with a user's G succeeds,
and a broken source is rejected with the compiler's message.  GPU: a registered softened
Coulomb kernel 1/sqrt(r^2 + eps^2) matches the oracle's Algorithm 1 with that kernel (FP64
1e-12, mixed 1e-6 of the FP64 path), for targets = sources and for separate sets."""
import numpy as np
import pytest

import oracle
import paper_2003_01836_gb300 as b
from paper_2003_01836_gb300 import inputs

SOFT = """
__device__ float bltc_user_g32(float r2, float r, float eps) { return rsqrtf(r2 + eps * eps); }
__device__ double bltc_user_g64(double r2, double r, double eps) { return 1.0 / sqrt(r2 + eps * eps); }
"""


def _check(src):
    if not b.library_built():
        pytest.skip("libbltc.so not built")
    st, log = b.bltc_kernel_check(src, 103)
    if st == b.BLTC_ERR_STATE:
        pytest.skip("NVRTC not available: " + log)
    return st, log


def test_user_kernel_compiles_for_sm103():
    st, log = _check(SOFT)
    assert st == b.BLTC_OK, log


def test_user_kernel_compile_error_is_reported():
    st, log = _check("__device__ float bltc_user_g32(float r2, float r, float e) { return r2 * undefined_name; }\n")
    assert st == b.BLTC_ERR_ARG
    assert "undefined_name" in log


# ---- GPU ------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def soft(gpu):
    return b.bltc_kernel_register(gpu.h, SOFT)


@pytest.mark.gpu
@pytest.mark.parametrize("case", [("cube", 20000, 700, 700, 0.7, 6, 0.05),
                                  ("plummer", 30000, 1000, 1000, 0.8, 8, 0.2),
                                  ("cube", 12001, 500, 300, 0.6, 4, 0.01)])
def test_soft_kernel_matches_oracle(gpu, soft, case):
    from gpu_helpers import FP64_ELEM, FP64_REL2, MIXED_ELEM, MIXED_REL2, assert_close_abs, gpu_solve
    kind, n, leaf, batch, theta, deg, eps = case
    x, y, z, q = inputs.system(kind, n, 20031890 + n)
    p64 = b.params(deg, theta, leaf, batch, soft, eps, b.BLTC_PRECISION_FP64)
    pmx = b.params(deg, theta, leaf, batch, soft, eps, b.BLTC_PRECISION_MIXED)
    want, want_abs, _ = oracle.bltc(x, y, z, q, theta, deg, leaf, batch, oracle.KERNEL_SOFT, eps,
                                    with_abs=True)
    got64 = gpu_solve(gpu, x, y, z, q, p64)
    gotmx = gpu_solve(gpu, x, y, z, q, pmx)
    assert_close_abs(want, got64, want_abs, FP64_REL2, FP64_ELEM, "user fp64 vs oracle")
    assert_close_abs(got64, gotmx, want_abs, MIXED_REL2, MIXED_ELEM, "user mixed vs fp64")


@pytest.mark.gpu
def test_soft_kernel_separate_sets(gpu, soft):
    import torch
    from gpu_helpers import FP64_ELEM, FP64_REL2, assert_close_abs, dev, host
    sx, sy, sz, q = inputs.system("cube", 15000, 20031895)
    tx, ty, tz, _ = inputs.system("plummer", 7000, 20031896)
    p = b.params(6, 0.7, 800, 400, soft, 0.1, b.BLTC_PRECISION_FP64)
    T, S = dev(tx, ty, tz), dev(sx, sy, sz, q)
    phi = torch.empty_like(T[0])
    b.bltc_solve_targets(gpu.h, *T, *S, p, phi)
    torch.cuda.synchronize()
    want, want_abs, _ = oracle.bltc_ts((tx, ty, tz), (sx, sy, sz), q, 0.7, 6, 800, 400,
                                       oracle.KERNEL_SOFT, 0.1, with_abs=True)
    assert_close_abs(want, host(phi), want_abs, FP64_REL2, FP64_ELEM, "user fp64 separate sets")


@pytest.mark.gpu
def test_user_kernel_ids_are_checked(gpu, soft):
    from gpu_helpers import dev
    import torch
    x, y, z, q = inputs.system("cube", 2000, 3)
    X = dev(x, y, z, q)
    phi = torch.empty_like(X[0])
    with pytest.raises(b.BltcError) as e:          # an id no one registered
        b.bltc_solve(gpu.h, *X, b.params(4, 0.7, 200, kernel=soft + 7), phi)
    assert e.value.status == b.BLTC_ERR_ARG
    with pytest.raises(b.BltcError) as e:          # the direct sum takes built-in kernels only
        b.bltc_direct_sum(gpu.h, *X[:3], *X, b.params(4, 0.7, 200, kernel=soft), phi)
    assert e.value.status == b.BLTC_ERR_ARG
