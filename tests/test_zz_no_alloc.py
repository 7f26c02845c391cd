"""bltc_direct_sum_noalloc, the direct sum for callers that cannot allocate device memory
(their device heap belongs to another allocator).  It must give what bltc_direct_sum gives,
within the direct-sum tolerances of the parity tests, on two calls in a row (the fixed
scratch array keeps the previous call's contents, which must not leak into the next).

This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process (the gpu fixture builds the
library and opens the context)."""
import ctypes

import numpy as np
import pytest

import paper_2003_01836_gb300 as b
from gpu_helpers import dev, host, system

pytestmark = pytest.mark.gpu


def _call_noalloc(ctx, T, S, Q, p, phi):
    import torch
    lib = b.lib()
    b.bltc_context_set_stream(ctx, torch.cuda.current_stream().cuda_stream)
    st = lib.bltc_direct_sum_noalloc(ctx, T[0].data_ptr(), T[1].data_ptr(), T[2].data_ptr(),
                                     T[0].numel(), S[0].data_ptr(), S[1].data_ptr(),
                                     S[2].data_ptr(), Q.data_ptr(), S[0].numel(),
                                     ctypes.byref(p), phi.data_ptr())
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("prec,rel", [(b.BLTC_PRECISION_FP64, 1e-14), (b.BLTC_PRECISION_MIXED, 1e-6)])
def test_noalloc_matches_direct_sum_twice(gpu, prec, rel):
    import torch
    for call, (nt, ns, ker, seed) in enumerate([(30000, 50000, 0, 11), (7001, 9000, 1, 12)]):
        xs = system("cube", max(nt, ns), seed)
        T, S, Q = dev(*(a[:nt] for a in xs[:3])), dev(*(a[:ns] for a in xs[:3])), dev(xs[3][:ns])[0]
        p = b.params(4, 0.5, 10, kernel=ker, kappa=0.5, precision=prec)
        want = torch.empty_like(T[0])
        b.bltc_direct_sum(gpu.h, *T, *S, Q, p, want)
        got = torch.full_like(T[0], np.nan)
        assert _call_noalloc(gpu.h, T, S, Q, p, got) == b.BLTC_OK, b.bltc_last_error(gpu.h)
        w, g = host(want), host(got)
        assert np.all(np.isfinite(g)), f"call {call}"
        e = np.sqrt(np.sum((g - w) ** 2) / np.sum(w ** 2))
        assert e <= rel, (call, e)


def test_noalloc_rejects_too_many_targets(gpu):
    import torch
    nt = (1 << 23) + 1
    T = [torch.zeros(nt, dtype=torch.float64, device="cuda") for _ in range(3)]
    S = [torch.zeros(4, dtype=torch.float64, device="cuda") for _ in range(3)]
    Q = torch.ones(4, dtype=torch.float64, device="cuda")
    phi = torch.empty(nt, dtype=torch.float64, device="cuda")
    assert _call_noalloc(gpu.h, T, S, Q, b.params(4, 0.5, 10), phi) == b.BLTC_ERR_ARG
    assert "8388608" in b.bltc_last_error(gpu.h)
