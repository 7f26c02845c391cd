"""Helpers shared by the GPU parity tests (device copies, oracle subsets, tolerances)."""
import numpy as np

import oracle
import paper_2003_01836_gb300 as b
from paper_2003_01836_gb300 import inputs

# Tolerances of the parity tests:
#   FP64 GPU path vs FP64 oracle: relative 2-norm <= 1e-12, and per target
#   |phi_gpu - phi_oracle| <= 1e-12 * sum_j |G_ij q_j| (the absolute-value sum of the same terms).
#   MIXED vs FP64 GPU path: relative 2-norm <= 1e-6, per target <= 2e-5 * the same absolute sum.
FP64_REL2 = 1e-12
FP64_ELEM = 1e-12
MIXED_REL2 = 1e-6
MIXED_ELEM = 2e-5


def dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda() for a in arrays]


def host(t):
    return t.detach().cpu().numpy()


def system(kind, n, seed):
    return inputs.system(kind, n, seed)


def gpu_tree(ctx, x, y, z, q, leaf):
    X = dev(x, y, z) + (dev(q) if q is not None else [None])
    return b.bltc_tree_build(ctx.h, X[0], X[1], X[2], X[3], leaf), X


def gpu_solve(ctx, x, y, z, q, p):
    import torch
    X = dev(x, y, z, q)
    phi = torch.empty_like(X[0])
    b.bltc_solve(ctx.h, *X, p, phi)
    torch.cuda.synchronize()
    return host(phi)


def batch_targets(tree: oracle.Tree, batches):
    return np.concatenate([tree.perm[tree.begin[tree.leaves[i]]:
                                     tree.begin[tree.leaves[i]] + tree.count[tree.leaves[i]]]
                           for i in batches])


def assert_close_abs(ref, got, ref_abs, rel2, elem, what=""):
    e2 = oracle.rel_err(ref, got)
    assert e2 <= rel2, f"{what}: relative 2-norm {e2:.3e} > {rel2:.1e}"
    worst = np.max(np.abs(got - ref) / ref_abs)
    assert worst <= elem, f"{what}: worst per-target error {worst:.3e} > {elem:.1e}"
    return e2
