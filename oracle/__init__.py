"""FP64 CPU oracle of the barycentric Lagrange treecode (test infrastructure only).

This package is the plain, slow reference that the CUDA library is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and reference legs
may import it.
It shares no code with ``paper_2003_01836_gb300``; the two meet only through the seeded input
arrays of ``paper_2003_01836_gb300.inputs``, which hold none of the method's arithmetic.

The C source (``bltc_oracle.c``) cites the paper passage each function follows:
Eq. 1-2 (direct sum, kernels), Eq. 4-7 (barycentric Lagrange interpolation at Chebyshev
points of the second kind), Sec. II-C (exact hits), Eq. 12 (modified charges), Eq. 13 (MAC)
and Algorithm 1 (the treecode, for targets = sources and for separate sets), the
cluster-particle variant named as future work in Sec. V, plus Eq. 16 (relative 2-norm error)
here in Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bltc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KERNEL_COULOMB = 0
KERNEL_YUKAWA = 1
KERNEL_POLY = 2
KERNEL_SOFT = 3          # 1/sqrt(r^2 + eps^2), eps passed as kappa
MAX_DEGREE = 32

_f64 = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bltc_oracle.h")))
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # BLTC_ORACLE_LIB lets the mutation tests load a deliberately broken copy.
        lib = ctypes.CDLL(os.environ.get("BLTC_ORACLE_LIB") or build())
        c = ctypes
        lib.oracle_direct_sum.argtypes = [_f64, _f64, _f64, c.c_int64, _f64, _f64, _f64, _f64,
                                          c.c_int64, c.c_int32, c.c_double, c.c_int32,
                                          c.c_int32, _f64, c.c_void_p]
        lib.oracle_direct_sum.restype = c.c_int
        lib.oracle_tree_build.argtypes = [_f64, _f64, _f64, c.c_int64, c.c_int32,
                                          c.POINTER(c.c_void_p)]
        lib.oracle_tree_build.restype = c.c_int
        lib.oracle_tree_free.argtypes = [c.c_void_p]
        lib.oracle_tree_num_nodes.argtypes = [c.c_void_p]
        lib.oracle_tree_num_nodes.restype = c.c_int64
        lib.oracle_tree_export.argtypes = [c.c_void_p, _i64, _i64, _i64, _i32, _i32, _i32, _i32,
                                           _f64, _f64, _f64, _f64]
        lib.oracle_num_leaves.argtypes = [c.c_void_p]
        lib.oracle_num_leaves.restype = c.c_int64
        lib.oracle_leaves.argtypes = [c.c_void_p, _i64]
        lib.oracle_cheb.argtypes = [c.c_int32, c.c_double, c.c_double, _f64, _f64]
        lib.oracle_lagrange.argtypes = [c.c_int32, c.c_double, c.c_double, c.c_double, _f64]
        lib.oracle_modified_charges.argtypes = [c.c_void_p, _f64, _f64, _f64, _f64, c.c_int32,
                                                c.c_int32, _f64]
        lib.oracle_modified_charges.restype = c.c_int
        lib.oracle_lists.argtypes = [c.c_void_p, c.c_void_p, c.c_double, c.c_int32,
                                     c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p,
                                     c.POINTER(c.c_int64), c.POINTER(c.c_int64)]
        lib.oracle_lists.restype = c.c_int
        lib.oracle_bltc.argtypes = [_f64, _f64, _f64, _f64, c.c_int64, c.c_double, c.c_int32,
                                    c.c_int32, c.c_int32, c.c_int32, c.c_double, c.c_int32,
                                    c.c_void_p, c.c_int64, _f64, c.c_void_p, _f64]
        lib.oracle_bltc.restype = c.c_int
        lib.oracle_bltc_ts.argtypes = [_f64, _f64, _f64, c.c_int64, _f64, _f64, _f64, _f64,
                                       c.c_int64, c.c_double, c.c_int32, c.c_int32, c.c_int32,
                                       c.c_int32, c.c_double, c.c_int32, c.c_void_p, c.c_int64,
                                       _f64, c.c_void_p, _f64]
        lib.oracle_bltc_ts.restype = c.c_int
        lib.oracle_bltc_prepare.argtypes = [_f64, _f64, _f64, c.c_int64, _f64, _f64, _f64, _f64,
                                            c.c_int64, c.c_double, c.c_int32, c.c_int32, c.c_int32,
                                            c.c_int32, c.c_double, c.c_int32, c.POINTER(c.c_void_p),
                                            _f64]
        lib.oracle_bltc_prepare.restype = c.c_int
        lib.oracle_bltc_num_batches.argtypes = [c.c_void_p]
        lib.oracle_bltc_num_batches.restype = c.c_int64
        lib.oracle_bltc_evaluate.argtypes = [c.c_void_p, c.c_void_p, c.c_int64, c.c_int32, _f64,
                                             c.c_void_p, c.POINTER(c.c_double)]
        lib.oracle_bltc_evaluate.restype = c.c_int
        lib.oracle_bltc_release.argtypes = [c.c_void_p]
        lib.oracle_bltc_release.restype = None
        lib.oracle_bltc_cp.argtypes = [_f64, _f64, _f64, c.c_int64, _f64, _f64, _f64, _f64,
                                       c.c_int64, c.c_double, c.c_int32, c.c_int32, c.c_int32,
                                       c.c_int32, c.c_double, c.c_int32, _f64, c.c_void_p]
        lib.oracle_bltc_cp.restype = c.c_int
        lib.oracle_hermite_factors.argtypes = [c.c_int32, c.c_double, c.c_double, c.c_double, _f64, _f64]
        lib.oracle_hermite_factors.restype = None
        lib.oracle_kernel_dG.argtypes = [c.c_int32, c.c_double, c.c_int32, _f64, _f64, _f64]
        lib.oracle_kernel_dG.restype = c.c_int
        lib.oracle_bltc_hermite.argtypes = [_f64, _f64, _f64, _f64, c.c_int64, c.c_double, c.c_int32,
                                            c.c_int32, c.c_int32, c.c_int32, c.c_double, c.c_int32,
                                            _f64, c.c_void_p]
        lib.oracle_bltc_hermite.restype = c.c_int
        lib.oracle_bltc_cc.argtypes = lib.oracle_bltc_cp.argtypes
        lib.oracle_bltc_cc.restype = c.c_int
        lib.oracle_dual_lists_export.argtypes = [c.c_void_p, c.c_void_p, c.c_double, c.c_int32,
                                                 c.c_void_p, c.c_void_p, c.c_void_p]
        lib.oracle_dual_lists_export.restype = c.c_int
        lib.oracle_max_threads.restype = c.c_int
        _lib = lib
        return lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def direct_sum(targets, sources, q, kernel=KERNEL_COULOMB, kappa=0.0, degree=0, threads=0,
               with_abs=False):
    """Eq. 1: phi(x_i) = sum_j G(x_i, y_j) q_j (pairs with r^2 == 0 skipped).

    ``targets`` and ``sources`` are (3, n) arrays (x, y, z rows)."""
    lib = _load()
    tx, ty, tz = (_c(targets[d]) for d in range(3))
    sx, sy, sz = (_c(sources[d]) for d in range(3))
    sq = _c(q)
    phi = np.empty(tx.shape[0])
    phi_abs = np.empty(tx.shape[0]) if with_abs else None
    rc = lib.oracle_direct_sum(tx, ty, tz, tx.shape[0], sx, sy, sz, sq, sx.shape[0], kernel,
                               float(kappa), degree, threads, phi,
                               phi_abs.ctypes.data if with_abs else None)
    if rc:
        raise ValueError(f"oracle_direct_sum failed ({rc})")
    return (phi, phi_abs) if with_abs else phi


class Tree:
    """A tree of clusters (Sec. II-D) as plain numpy arrays, nodes in DFS pre-order."""

    def __init__(self, x, y, z, max_leaf):
        lib = _load()
        self.x, self.y, self.z = _c(x), _c(y), _c(z)
        h = ctypes.c_void_p()
        rc = lib.oracle_tree_build(self.x, self.y, self.z, self.x.shape[0], int(max_leaf),
                                   ctypes.byref(h))
        if rc:
            raise ValueError(f"oracle_tree_build failed ({rc})")
        self._h = h
        m = lib.oracle_tree_num_nodes(h)
        n = self.x.shape[0]
        self.n_nodes = int(m)
        self.perm = np.empty(n, np.int64)
        self.begin = np.empty(m, np.int64)
        self.count = np.empty(m, np.int64)
        self.parent = np.empty(m, np.int32)
        self.level = np.empty(m, np.int32)
        self.n_children = np.empty(m, np.int32)
        self.children = np.empty((m, 8), np.int32)
        self.lo = np.empty((m, 3))
        self.hi = np.empty((m, 3))
        self.center = np.empty((m, 3))
        self.radius = np.empty(m)
        lib.oracle_tree_export(h, self.perm, self.begin, self.count, self.parent, self.level,
                               self.n_children, self.children, self.lo, self.hi, self.center,
                               self.radius)
        nl = lib.oracle_num_leaves(h)
        self.leaves = np.empty(nl, np.int64)
        lib.oracle_leaves(h, self.leaves)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_tree_free(h)
            self._h = None

    def as_dict(self):
        return {k: getattr(self, k) for k in ("perm", "begin", "count", "parent", "level",
                                              "n_children", "children", "lo", "hi", "center",
                                              "radius")}


def cheb(degree, lo, hi):
    """Eq. 6-7: Chebyshev points of the 2nd kind on [lo, hi] and barycentric weights."""
    s = np.empty(degree + 1)
    w = np.empty(degree + 1)
    _load().oracle_cheb(degree, float(lo), float(hi), s, w)
    return s, w


def lagrange(degree, lo, hi, y):
    """Eq. 4 with the Sec. II-C exact-hit rule: the vector L_k(y), k = 0..n."""
    a = np.empty(degree + 1)
    _load().oracle_lagrange(degree, float(lo), float(hi), float(y), a)
    return a


def modified_charges(tree: Tree, q, degree, threads=0):
    """Eq. 12 for every node of ``tree``: array (n_nodes, (n+1)^3), k = (k1, k2, k3) C-order."""
    n1 = degree + 1
    out = np.empty(tree.n_nodes * n1 ** 3)
    rc = _load().oracle_modified_charges(tree._h, tree.x, tree.y, tree.z, _c(q), degree,
                                         threads, out)
    if rc:
        raise ValueError(f"oracle_modified_charges failed ({rc})")
    return out.reshape(tree.n_nodes, n1 ** 3)


def lists(batches: Tree, sources: Tree, theta, degree):
    """Algorithm 1's walk of the source tree for every batch (leaves of ``batches`` in DFS
    order), recording the approximation and direct lists as CSR arrays of node ids."""
    lib = _load()
    na, nd = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.oracle_lists(batches._h, sources._h, float(theta), degree, None, None, None, None,
                          ctypes.byref(na), ctypes.byref(nd))
    if rc:
        raise ValueError(f"oracle_lists failed ({rc})")
    nb = batches.leaves.shape[0]
    ao = np.empty(nb + 1, np.int64)
    ai = np.empty(max(na.value, 1), np.int64)
    do = np.empty(nb + 1, np.int64)
    di = np.empty(max(nd.value, 1), np.int64)
    rc = lib.oracle_lists(batches._h, sources._h, float(theta), degree, ao.ctypes.data,
                          ai.ctypes.data, do.ctypes.data, di.ctypes.data, ctypes.byref(na),
                          ctypes.byref(nd))
    if rc:
        raise ValueError(f"oracle_lists failed ({rc})")
    return {"approx_off": ao, "approx_ids": ai[:na.value], "direct_off": do,
            "direct_ids": di[:nd.value]}


def bltc(x, y, z, q, theta, degree, leaf_size, batch_size, kernel=KERNEL_COULOMB, kappa=0.0,
         threads=0, batches=None, with_abs=False):
    """Algorithm 1 end to end, targets = sources.  Returns (phi, phi_abs or None, timings).

    ``batches`` optionally restricts evaluation to those batch indices (leaves of the batch
    tree in DFS order); the other targets' potentials are returned as 0."""
    lib = _load()
    x, y, z, q = _c(x), _c(y), _c(z), _c(q)
    n = x.shape[0]
    phi = np.empty(n)
    phi_abs = np.empty(n) if with_abs else None
    tm = np.zeros(3)
    sub = None if batches is None else _c(batches, np.int64)
    rc = lib.oracle_bltc(x, y, z, q, n, float(theta), int(degree), int(leaf_size),
                         int(batch_size), int(kernel), float(kappa), int(threads),
                         None if sub is None else sub.ctypes.data,
                         0 if sub is None else sub.shape[0], phi,
                         None if phi_abs is None else phi_abs.ctypes.data, tm)
    if rc:
        raise ValueError(f"oracle_bltc failed ({rc})")
    return phi, phi_abs, {"setup": tm[0], "precompute": tm[1], "compute": tm[2]}


class Prepared:
    """Algorithm 1's setup for targets = sources (trees and modified charges), kept for
    evaluations of all or some batches: ``evaluate(batches=None, threads=0, with_abs=False)``
    returns (phi, phi_abs or None, seconds).  ``timings`` holds the setup's two phases."""

    def __init__(self, x, y, z, q, theta, degree, leaf_size, batch_size, kernel=KERNEL_COULOMB,
                 kappa=0.0, threads=0):
        lib = _load()
        self._arrays = [_c(x), _c(y), _c(z), _c(q)]     # read by every evaluation
        x, y, z, q = self._arrays
        self.n = x.shape[0]
        tm = np.zeros(2)
        h = ctypes.c_void_p()
        rc = lib.oracle_bltc_prepare(x, y, z, self.n, x, y, z, q, self.n, float(theta), int(degree),
                                     int(leaf_size), int(batch_size), int(kernel), float(kappa),
                                     int(threads), ctypes.byref(h), tm)
        if rc:
            raise ValueError(f"oracle_bltc_prepare failed ({rc})")
        self._h = h.value
        self.timings = {"setup": tm[0], "precompute": tm[1]}
        self.n_batches = int(lib.oracle_bltc_num_batches(self._h))

    def evaluate(self, batches=None, threads=0, with_abs=False):
        phi = np.empty(self.n)
        phi_abs = np.empty(self.n) if with_abs else None
        sub = None if batches is None else _c(batches, np.int64)
        sec = ctypes.c_double()
        rc = _load().oracle_bltc_evaluate(self._h, None if sub is None else sub.ctypes.data,
                                          0 if sub is None else sub.shape[0], int(threads), phi,
                                          None if phi_abs is None else phi_abs.ctypes.data,
                                          ctypes.byref(sec))
        if rc:
            raise ValueError(f"oracle_bltc_evaluate failed ({rc})")
        return phi, phi_abs, sec.value

    def close(self):
        if getattr(self, "_h", None):
            _load().oracle_bltc_release(self._h)
            self._h = None

    def __del__(self):
        self.close()


def bltc_ts(targets, sources, q, theta, degree, leaf_size, batch_size,
            kernel=KERNEL_COULOMB, kappa=0.0, threads=0, batches=None, with_abs=False):
    """Algorithm 1 for distinct target and source sets: ``targets`` = (tx, ty, tz),
    ``sources`` = (sx, sy, sz) with charges ``q``.  Source tree with ``leaf_size``, target
    batch tree with ``batch_size``.  Returns (phi[nt], phi_abs or None, timings)."""
    lib = _load()
    tx, ty, tz = (_c(a) for a in targets)
    sx, sy, sz = (_c(a) for a in sources)
    q = _c(q)
    nt, ns = tx.shape[0], sx.shape[0]
    phi = np.empty(nt)
    phi_abs = np.empty(nt) if with_abs else None
    tm = np.zeros(3)
    sub = None if batches is None else _c(batches, np.int64)
    rc = lib.oracle_bltc_ts(tx, ty, tz, nt, sx, sy, sz, q, ns, float(theta), int(degree),
                            int(leaf_size), int(batch_size), int(kernel), float(kappa),
                            int(threads), None if sub is None else sub.ctypes.data,
                            0 if sub is None else sub.shape[0], phi,
                            None if phi_abs is None else phi_abs.ctypes.data, tm)
    if rc:
        raise ValueError(f"oracle_bltc_ts failed ({rc})")
    return phi, phi_abs, {"setup": tm[0], "precompute": tm[1], "compute": tm[2]}


def bltc_cp(targets, sources, q, theta, degree, leaf_size, batch_size,
            kernel=KERNEL_COULOMB, kappa=0.0, threads=0, with_abs=False):
    """Cluster-particle variant: targets in clusters of ``leaf_size`` (interpolated),
    sources in batches of ``batch_size`` (summed exactly).  Returns (phi, phi_abs or None)."""
    lib = _load()
    tx, ty, tz = (_c(a) for a in targets)
    sx, sy, sz = (_c(a) for a in sources)
    q = _c(q)
    phi = np.empty(tx.shape[0])
    phi_abs = np.empty(tx.shape[0]) if with_abs else None
    rc = lib.oracle_bltc_cp(tx, ty, tz, tx.shape[0], sx, sy, sz, q, sx.shape[0], float(theta),
                            int(degree), int(leaf_size), int(batch_size), int(kernel),
                            float(kappa), int(threads), phi,
                            None if phi_abs is None else phi_abs.ctypes.data)
    if rc:
        raise ValueError(f"oracle_bltc_cp failed ({rc})")
    return phi, phi_abs


def bltc_cc(targets, sources, q, theta, degree, leaf_size, batch_size,
            kernel=KERNEL_COULOMB, kappa=0.0, threads=0, with_abs=False):
    """Cluster-cluster variant (dual tree traversal): sources in a tree with ``leaf_size``,
    targets in a tree with ``batch_size``.  Returns (phi, phi_abs or None)."""
    lib = _load()
    tx, ty, tz = (_c(a) for a in targets)
    sx, sy, sz = (_c(a) for a in sources)
    q = _c(q)
    phi = np.empty(tx.shape[0])
    phi_abs = np.empty(tx.shape[0]) if with_abs else None
    rc = lib.oracle_bltc_cc(tx, ty, tz, tx.shape[0], sx, sy, sz, q, sx.shape[0], float(theta),
                            int(degree), int(leaf_size), int(batch_size), int(kernel),
                            float(kappa), int(threads), phi,
                            None if phi_abs is None else phi_abs.ctypes.data)
    if rc:
        raise ValueError(f"oracle_bltc_cc failed ({rc})")
    return phi, phi_abs


def dual_lists(targets: Tree, sources: Tree, theta, degree):
    """The dual traversal's interaction lists: {"cc", "cp", "pc", "pp"} -> (target ids,
    source ids), each in traversal order."""
    lib = _load()
    counts = np.zeros(4, np.int64)
    lib.oracle_dual_lists_export(targets._h, sources._h, float(theta), int(degree),
                                 counts.ctypes.data, None, None)
    tot = int(counts.sum())
    t = np.empty(max(tot, 1), np.int64)
    s = np.empty(max(tot, 1), np.int64)
    rc = lib.oracle_dual_lists_export(targets._h, sources._h, float(theta), int(degree),
                                      counts.ctypes.data, t.ctypes.data, s.ctypes.data)
    if rc:
        raise ValueError(f"oracle_dual_lists_export failed ({rc})")
    out, o = {}, 0
    for name, n in zip(("cc", "cp", "pc", "pp"), counts):
        out[name] = (t[o:o + n].copy(), s[o:o + n].copy())
        o += int(n)
    return out


def hermite_factors(degree, lo, hi, y):
    """The 1-D Hermite basis on the Chebyshev points of [lo, hi]: (H_k(y), K_k(y)), k = 0..n."""
    h = np.empty(degree + 1)
    k = np.empty(degree + 1)
    _load().oracle_hermite_factors(int(degree), float(lo), float(hi), float(y), h, k)
    return h, k


def kernel_derivatives(kernel, kappa, kdeg, x, y):
    """D^a G(x, y) for a in {0,1}^3 (index a1*4 + a2*2 + a3); None when r^2 == 0."""
    out = np.empty(8)
    ok = _load().oracle_kernel_dG(int(kernel), float(kappa), int(kdeg), _c(np.asarray(x, float)),
                                  _c(np.asarray(y, float)), out)
    return out if ok else None


def bltc_hermite(x, y, z, q, theta, degree, leaf_size, batch_size, kernel=KERNEL_COULOMB,
                 kappa=0.0, threads=0, with_abs=False):
    """The barycentric Hermite treecode (targets = sources).  Returns (phi, phi_abs or None)."""
    lib = _load()
    x, y, z, q = _c(x), _c(y), _c(z), _c(q)
    phi = np.empty(x.shape[0])
    phi_abs = np.empty(x.shape[0]) if with_abs else None
    rc = lib.oracle_bltc_hermite(x, y, z, q, x.shape[0], float(theta), int(degree), int(leaf_size),
                                 int(batch_size), int(kernel), float(kappa), int(threads), phi,
                                 None if phi_abs is None else phi_abs.ctypes.data)
    if rc:
        raise ValueError(f"oracle_bltc_hermite failed ({rc})")
    return phi, phi_abs


def rel_err(reference, approx):
    """Eq. 16: relative 2-norm error of ``approx`` against ``reference``."""
    reference = np.asarray(reference, dtype=np.float64)
    approx = np.asarray(approx, dtype=np.float64)
    return float(np.sqrt(np.sum((reference - approx) ** 2) / np.sum(reference ** 2)))
