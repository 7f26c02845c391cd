"""GB300-native barycentric Lagrange treecode (BLTC), Python binding of include/bltc.h.

The functions below carry the C ABI's names and only marshal arguments: torch tensors become
device pointers, torch's current CUDA stream becomes the context's stream, and a non-zero
status becomes a ``BltcError``.  Every step of the treecode runs in the CUDA library
``_build/libbltc.so`` (built by ``build.build()``); there is no CPU path, and importing a
function that needs the library raises if it has not been built.

The paper: Vaughn, Wilson and Krasny, "A GPU-Accelerated Barycentric Lagrange Treecode"
(2020) -- Eq. 1-2 (potentials), Eq. 4-8 (barycentric Lagrange interpolation), Eq. 11-13
(approximation, modified charges, MAC), Algorithm 1 (the treecode).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbltc.so")

BLTC_OK = 0
BLTC_ERR_ARG = -1
BLTC_ERR_OOM = -2
BLTC_ERR_CUDA = -3
BLTC_ERR_TIMEOUT = -4
BLTC_ERR_STATE = -5
BLTC_ERR_CANCELLED = -6
BLTC_KERNEL_COULOMB = 0
BLTC_KERNEL_YUKAWA = 1
BLTC_PRECISION_FP64 = 0
BLTC_PRECISION_MIXED = 1
BLTC_MAX_DEGREE = 16
BLTC_KERNEL_USER_BASE = 16

_STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_TIMEOUT",
           -5: "ERR_STATE", -6: "ERR_CANCELLED"}


class BltcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class bltc_params(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("theta", ctypes.c_double), ("kappa", ctypes.c_double)]


def params(degree=8, theta=0.7, leaf_size=2000, batch_size=None, kernel=BLTC_KERNEL_COULOMB,
           kappa=0.0, precision=BLTC_PRECISION_MIXED, tile=0) -> bltc_params:
    """Treecode parameters (theta, n, N_L, N_B of Algorithm 1) plus kernel, precision and the
    sweep's tile shape (0: the defaults; see tile())."""
    return bltc_params(int(degree), int(leaf_size),
                       int(leaf_size if batch_size is None else batch_size), int(kernel),
                       int(precision), int(tile), float(theta), float(kappa))


def tile(group_cap=0, items_per_block=0):
    """bltc_params.tile from its fields: the cap on a batch's source groups (0: 8; else 1, 2, 4
    or 8) and the persistent sweep's work items per resident block (0: 16; else 1..255)."""
    return int(group_cap) | (int(items_per_block) << 4)


class bltc_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("setup_workers", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("linger_us", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("slice_us", ctypes.c_int32),
                ("setup_blocks", ctypes.c_int32), ("slices_in_flight", ctypes.c_int32)]


class bltc_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("bytes_reserved", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_ready", ctypes.c_double),
                ("t_done", ctypes.c_double), ("t_swept", ctypes.c_double),
                ("t_copy", ctypes.c_double)]


class bltc_server_counters(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "submitted", "completed", "failed", "cancelled", "queued", "sweep_launches", "max_batch",
        "budget_bytes", "reserved_bytes", "peak_reserved_bytes", "live_bytes", "peak_live_bytes")]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_void_p)

_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_pp = ctypes.POINTER(ctypes.c_void_p)
_P = ctypes.POINTER(bltc_params)

_SIGNATURES = {
    "bltc_version": ([], ctypes.c_int),
    "bltc_context_create": ([ctypes.c_int, _vp, _pp], ctypes.c_int),
    "bltc_context_destroy": ([_vp], None),
    "bltc_context_set_stream": ([_vp, _vp], ctypes.c_int),
    "bltc_context_set_allocator": ([_vp, ALLOC_FN, FREE_FN, _vp], ctypes.c_int),
    "bltc_synchronize": ([_vp], ctypes.c_int),
    "bltc_last_error": ([_vp], ctypes.c_char_p),
    "bltc_device_sm_count": ([_vp], ctypes.c_int),
    "bltc_context_launch_count": ([_vp], ctypes.c_int64),
    "bltc_context_set_timing": ([_vp, ctypes.c_int], ctypes.c_int),
    "bltc_last_timings": ([_vp, _vp], ctypes.c_int),
    "bltc_tree_build": ([_vp, _vp, _vp, _vp, _vp, _i64, _i32, _pp], ctypes.c_int),
    "bltc_tree_destroy": ([_vp], None),
    "bltc_tree_info": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "bltc_tree_export": ([_vp] * 13, ctypes.c_int),
    "bltc_lists_build": ([_vp, _vp, _vp, _P, _pp], ctypes.c_int),
    "bltc_lists_select": ([_vp, _vp, _vp, _i64, _pp], ctypes.c_int),
    "bltc_lists_destroy": ([_vp], None),
    "bltc_lists_info": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "bltc_lists_export": ([_vp] * 6, ctypes.c_int),
    "bltc_stats": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "bltc_evaluations": ([_vp, _vp, _P, _vp], ctypes.c_int),
    "bltc_modified_charges": ([_vp, _vp, _vp, _P], ctypes.c_int),
    "bltc_modified_charges_export": ([_vp, _vp, _vp], ctypes.c_int),
    "bltc_evaluate": ([_vp, _vp, _vp, _vp, _P, _vp], ctypes.c_int),
    "bltc_solve": ([_vp, _vp, _vp, _vp, _vp, _i64, _P, _vp], ctypes.c_int),
    "bltc_solve_host": ([_vp, _vp, _vp, _vp, _vp, _i64, _P, _vp], ctypes.c_int),
    "bltc_solve_cp": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _P, _vp], ctypes.c_int),
    "bltc_solve_cc": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _P, _vp], ctypes.c_int),
    "bltc_solve_hermite": ([_vp, _vp, _vp, _vp, _vp, _i64, _P, _vp], ctypes.c_int),
    "bltc_graph_create": ([_vp, _vp, _vp, _vp, _vp, _i64, _P, _vp, _pp], ctypes.c_int),
    "bltc_graph_launch": ([_vp, _vp], ctypes.c_int),
    "bltc_graph_kernels": ([_vp], _i64),
    "bltc_graph_destroy": ([_vp], None),
    "bltc_graph_create_positions": ([_vp, _vp, _vp, _vp, _vp, _i64, _P, _vp, ctypes.c_double, _pp],
                                    ctypes.c_int),
    "bltc_graph_info": ([_vp, _vp], ctypes.c_int),
    "bltc_autotune_tile": ([_vp, _vp, _vp, _vp, _vp, _i64, _P, _vp, _i32, _i32, _i32, _P, _vp],
                           ctypes.c_int),
    "bltc_dual_lists": ([_vp, _vp, _vp, _P, _vp, _vp, _vp], ctypes.c_int),
    "bltc_solve_targets": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _P, _vp],
                           ctypes.c_int),
    "bltc_direct_sum": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _P, _vp],
                        ctypes.c_int),
    "bltc_direct_sum_noalloc": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _P, _vp],
                                ctypes.c_int),
    "bltc_autotune": ([_vp, _vp, _vp, _vp, _vp, _i64, _P, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                       ctypes.c_int32, _P, _vp], ctypes.c_int),
    "bltc_kernel_register": ([_vp, ctypes.c_char_p, ctypes.POINTER(_i32)], ctypes.c_int),
    "bltc_kernel_check": ([ctypes.c_char_p, _i32, ctypes.c_char_p, _i64], ctypes.c_int),
    "bltc_server_create": ([ctypes.POINTER(bltc_server_config), _pp], ctypes.c_int),
    "bltc_server_submit": ([_vp, _vp, _vp, _vp, _vp, _i64, _P, _vp, ctypes.POINTER(ctypes.c_uint64)],
                           ctypes.c_int),
    "bltc_server_wait": ([_vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(bltc_request_info)],
                         ctypes.c_int),
    "bltc_server_cancel": ([_vp, ctypes.c_uint64], ctypes.c_int),
    "bltc_server_stats": ([_vp, ctypes.POINTER(bltc_server_counters)], ctypes.c_int),
    "bltc_server_last_error": ([_vp, ctypes.c_char_p, _i64], _i64),
    "bltc_server_destroy": ([_vp], None),
}


def library_built() -> bool:
    return os.path.exists(LIB_PATH)


def lib():
    """The loaded libbltc.so.  Raises if it was not built: there is no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libbltc.so is not built ({LIB_PATH}); run "
                                   "paper_2003_01836_gb300.build.build() first")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
        return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _ptr(t):
    """Device (or host) address of a contiguous float64 tensor/array, checked."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if t.dtype != np.float64 or not t.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a contiguous float64 array")
        return t.ctypes.data
    if t.dtype.is_floating_point and t.dtype.itemsize != 8:
        raise TypeError("expected float64 tensors")
    if not t.is_contiguous():
        raise TypeError("expected contiguous tensors")
    return t.data_ptr()


def _check(ctx, status):
    if status != BLTC_OK:
        msg = lib().bltc_last_error(ctx).decode() if ctx else ""
        raise BltcError(status, msg)


def _stream(ctx):
    import torch
    lib().bltc_context_set_stream(ctx, torch.cuda.current_stream().cuda_stream)


# ---- torch's caching allocator as the library's device allocator ---------------------

class _TorchAllocator:
    def __init__(self, device):
        import torch
        self.device = device
        self.torch = torch

        def alloc(size, stream, user):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(size), self.device,
                                                               int(stream or 0))
            except Exception:   # reported to the library as NULL -> BLTC_ERR_OOM
                return None

        def free(ptr, size, stream, user):
            self.torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


# ---- the C ABI, same names -------------------------------------------------------------

def bltc_version() -> int:
    return lib().bltc_version()


def bltc_context_create(device=0, stream=None):
    h = ctypes.c_void_p()
    st = lib().bltc_context_create(int(device), stream, ctypes.byref(h))
    if st != BLTC_OK:
        raise BltcError(st, "context creation failed")
    return h.value


def bltc_context_destroy(ctx):
    lib().bltc_context_destroy(ctx)


def bltc_context_set_stream(ctx, stream):
    _check(ctx, lib().bltc_context_set_stream(ctx, stream))


def bltc_context_set_allocator(ctx, alloc_fn, free_fn, user=None):
    _check(ctx, lib().bltc_context_set_allocator(ctx, alloc_fn, free_fn, user))


def bltc_synchronize(ctx):
    _check(ctx, lib().bltc_synchronize(ctx))


def bltc_last_error(ctx) -> str:
    return lib().bltc_last_error(ctx).decode()


def bltc_device_sm_count(ctx) -> int:
    return lib().bltc_device_sm_count(ctx)


def bltc_context_launch_count(ctx) -> int:
    return lib().bltc_context_launch_count(ctx)


def bltc_context_set_timing(ctx, enable=True):
    _check(ctx, lib().bltc_context_set_timing(ctx, 1 if enable else 0))


PHASES = ("trees", "lists", "modified_charges", "plan", "sweep", "finalize", "total")


def bltc_last_timings(ctx):
    ms = (ctypes.c_float * 7)()
    _check(ctx, lib().bltc_last_timings(ctx, ctypes.addressof(ms)))
    return {k: float(v) for k, v in zip(PHASES, ms)}


def bltc_tree_build(ctx, x, y, z, q, max_leaf):
    _stream(ctx)
    h = ctypes.c_void_p()
    _check(ctx, lib().bltc_tree_build(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(q), x.numel(),
                                      int(max_leaf), ctypes.byref(h)))
    return h.value


def bltc_tree_destroy(tree):
    lib().bltc_tree_destroy(tree)


def bltc_tree_info(tree):
    v = [ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()]
    _check(None, lib().bltc_tree_info(tree, *[ctypes.byref(a) for a in v]))
    return {"n_particles": v[0].value, "n_nodes": v[1].value, "n_leaves": v[2].value,
            "n_levels": v[3].value}


_TREE_FIELDS = ("perm", "begin", "count", "parent", "level", "n_children", "children", "lo", "hi",
                "center", "radius")


def bltc_tree_export(ctx, tree, want=_TREE_FIELDS):
    """The tree's arrays on the host (those named in `want`)."""
    info = bltc_tree_info(tree)
    n, m = info["n_particles"], info["n_nodes"]
    make = {"perm": lambda: np.empty(n, np.int64), "begin": lambda: np.empty(m, np.int64),
            "count": lambda: np.empty(m, np.int64), "parent": lambda: np.empty(m, np.int32),
            "level": lambda: np.empty(m, np.int32), "n_children": lambda: np.empty(m, np.int32),
            "children": lambda: np.empty((m, 8), np.int32), "lo": lambda: np.empty((m, 3)),
            "hi": lambda: np.empty((m, 3)), "center": lambda: np.empty((m, 3)),
            "radius": lambda: np.empty(m)}
    out = {k: make[k]() for k in _TREE_FIELDS if k in want}
    _check(ctx, lib().bltc_tree_export(ctx, tree, *[out[k].ctypes.data if k in out else None
                                                    for k in _TREE_FIELDS]))
    return out


def bltc_lists_build(ctx, batches, sources, p: bltc_params):
    _stream(ctx)
    h = ctypes.c_void_p()
    _check(ctx, lib().bltc_lists_build(ctx, batches, sources, ctypes.byref(p), ctypes.byref(h)))
    return h.value


def bltc_lists_select(ctx, lists, batches):
    """The lists of the given batches only (others empty: their targets get phi = 0)."""
    sel = np.ascontiguousarray(batches, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(ctx, lib().bltc_lists_select(ctx, lists, sel.ctypes.data, sel.shape[0], ctypes.byref(h)))
    return h.value


def bltc_lists_destroy(lists):
    lib().bltc_lists_destroy(lists)


def bltc_lists_info(lists):
    v = [ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()]
    _check(None, lib().bltc_lists_info(lists, *[ctypes.byref(a) for a in v]))
    return {"n_batches": v[0].value, "n_approx": v[1].value, "n_direct": v[2].value}


def bltc_lists_export(ctx, lists):
    info = bltc_lists_info(lists)
    nb = info["n_batches"]
    out = {"approx_off": np.empty(nb + 1, np.int64),
           "approx_ids": np.empty(max(1, info["n_approx"]), np.int64),
           "direct_off": np.empty(nb + 1, np.int64),
           "direct_ids": np.empty(max(1, info["n_direct"]), np.int64)}
    _check(ctx, lib().bltc_lists_export(ctx, lists, out["approx_off"].ctypes.data,
                                        out["approx_ids"].ctypes.data,
                                        out["direct_off"].ctypes.data,
                                        out["direct_ids"].ctypes.data))
    out["approx_ids"] = out["approx_ids"][:info["n_approx"]]
    out["direct_ids"] = out["direct_ids"][:info["n_direct"]]
    return out


def bltc_stats(ctx, lists):
    _stream(ctx)
    d, a = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, lib().bltc_stats(ctx, lists, ctypes.byref(d), ctypes.byref(a)))
    return {"direct": d.value, "approx": a.value}


def bltc_evaluations(ctx, lists, p: bltc_params):
    """Kernel evaluations of bltc_evaluate for these lists and parameters."""
    _stream(ctx)
    n = ctypes.c_int64()
    _check(ctx, lib().bltc_evaluations(ctx, lists, ctypes.byref(p), ctypes.byref(n)))
    return n.value


def bltc_modified_charges(ctx, sources, lists, p: bltc_params):
    _stream(ctx)
    _check(ctx, lib().bltc_modified_charges(ctx, sources, lists, ctypes.byref(p)))


def bltc_modified_charges_export(ctx, sources, degree):
    m = bltc_tree_info(sources)["n_nodes"]
    P = (degree + 1) ** 3
    out = np.empty(m * P)
    _check(ctx, lib().bltc_modified_charges_export(ctx, sources, out.ctypes.data))
    return out.reshape(m, P)


def bltc_evaluate(ctx, lists, batches, sources, p: bltc_params, phi):
    _stream(ctx)
    _check(ctx, lib().bltc_evaluate(ctx, lists, batches, sources, ctypes.byref(p), _ptr(phi)))


def bltc_solve(ctx, x, y, z, q, p: bltc_params, phi):
    _stream(ctx)
    _check(ctx, lib().bltc_solve(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(q), x.numel(),
                                 ctypes.byref(p), _ptr(phi)))


def bltc_solve_targets(ctx, tx, ty, tz, sx, sy, sz, sq, p: bltc_params, phi):
    """Distinct target (tx, ty, tz) and source (sx, sy, sz, sq) sets; device tensors."""
    _stream(ctx)
    _check(ctx, lib().bltc_solve_targets(ctx, _ptr(tx), _ptr(ty), _ptr(tz), tx.numel(), _ptr(sx),
                                         _ptr(sy), _ptr(sz), _ptr(sq), sx.numel(), ctypes.byref(p),
                                         _ptr(phi)))


def bltc_solve_cp(ctx, tx, ty, tz, sx, sy, sz, sq, p: bltc_params, phi):
    """Cluster-particle variant: targets interpolated (leaf_size), sources exact (batch_size)."""
    _stream(ctx)
    _check(ctx, lib().bltc_solve_cp(ctx, _ptr(tx), _ptr(ty), _ptr(tz), tx.numel(), _ptr(sx), _ptr(sy),
                                    _ptr(sz), _ptr(sq), sx.numel(), ctypes.byref(p), _ptr(phi)))


def bltc_solve_cc(ctx, tx, ty, tz, sx, sy, sz, sq, p: bltc_params, phi):
    """Cluster-cluster variant: sources in clusters of leaf_size, targets of batch_size."""
    _stream(ctx)
    _check(ctx, lib().bltc_solve_cc(ctx, _ptr(tx), _ptr(ty), _ptr(tz), tx.numel(), _ptr(sx), _ptr(sy),
                                    _ptr(sz), _ptr(sq), sx.numel(), ctypes.byref(p), _ptr(phi)))


def bltc_dual_lists(ctx, targets, sources, p: bltc_params):
    """The dual traversal's lists: {"cc", "cp", "pc", "pp"} -> (target ids, source ids)."""
    counts = np.zeros(4, np.int64)
    _check(ctx, lib().bltc_dual_lists(ctx, targets, sources, ctypes.byref(p), counts.ctypes.data,
                                      None, None))
    tot = int(counts.sum())
    t = np.empty(max(tot, 1), np.int64)
    s = np.empty(max(tot, 1), np.int64)
    _check(ctx, lib().bltc_dual_lists(ctx, targets, sources, ctypes.byref(p), counts.ctypes.data,
                                      t.ctypes.data, s.ctypes.data))
    out, o = {}, 0
    for name, n in zip(("cc", "cp", "pc", "pp"), counts):
        out[name] = (t[o:o + n].copy(), s[o:o + n].copy())
        o += int(n)
    return out


def bltc_solve_hermite(ctx, x, y, z, q, p: bltc_params, phi):
    """The barycentric Hermite treecode (FP64 or mixed, degree <= 7); device tensors."""
    _stream(ctx)
    _check(ctx, lib().bltc_solve_hermite(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(q), x.numel(),
                                         ctypes.byref(p), _ptr(phi)))


def bltc_graph_create(ctx, x, y, z, q, p: bltc_params, phi):
    """Capture a solve with fixed positions; q and phi (device tensors) are bound to the graph."""
    _stream(ctx)
    h = ctypes.c_void_p()
    _check(ctx, lib().bltc_graph_create(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(q), x.numel(),
                                        ctypes.byref(p), _ptr(phi), ctypes.byref(h)))
    return h.value


def bltc_graph_create_positions(ctx, x, y, z, q, p: bltc_params, phi, headroom=0.0):
    """Capture the whole solve sized on the device; x, y, z, q and phi (device tensors) are bound
    to the graph and read (written) at every launch."""
    _stream(ctx)
    h = ctypes.c_void_p()
    _check(ctx, lib().bltc_graph_create_positions(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(q), x.numel(),
                                                  ctypes.byref(p), _ptr(phi), float(headroom),
                                                  ctypes.byref(h)))
    return h.value


def bltc_graph_info(graph):
    """{kernels, launches, redone, captures} of a graph."""
    out = (ctypes.c_int64 * 4)()
    if lib().bltc_graph_info(graph, out) != BLTC_OK:
        raise BltcError(BLTC_ERR_ARG, "graph_info: NULL graph")
    return {"kernels": out[0], "launches": out[1], "redone": out[2], "captures": out[3]}


def bltc_graph_launch(ctx, graph):
    """Replay: reads the charges now in the bound q, overwrites the bound phi."""
    _stream(ctx)
    _check(ctx, lib().bltc_graph_launch(ctx, graph))


def bltc_graph_kernels(graph):
    return int(lib().bltc_graph_kernels(graph))


def bltc_graph_destroy(graph):
    lib().bltc_graph_destroy(graph)


def bltc_solve_host(ctx, x, y, z, q, p: bltc_params, phi):
    """Host buffers (numpy arrays or CPU tensors, pinned recommended)."""
    _stream(ctx)
    n = x.shape[0]
    _check(ctx, lib().bltc_solve_host(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(q), n,
                                      ctypes.byref(p), _ptr(phi)))


def bltc_kernel_register(ctx, source: str) -> int:
    """Compiles the sweeps for a user kernel (CUDA source defining bltc_user_g32 and
    bltc_user_g64) and returns its id for ``params.kernel`` in this context."""
    kid = _i32()
    _check(ctx, lib().bltc_kernel_register(ctx, source.encode(), ctypes.byref(kid)))
    return kid.value


def bltc_kernel_check(source: str, arch: int = 103):
    """Compiles a user kernel for sm_<arch> without a device: (status, compiler log)."""
    buf = ctypes.create_string_buffer(1 << 16)
    st = lib().bltc_kernel_check(source.encode(), int(arch), buf, len(buf))
    return st, buf.value.decode(errors="replace")


def bltc_direct_sum(ctx, tx, ty, tz, sx, sy, sz, sq, p: bltc_params, phi):
    _stream(ctx)
    _check(ctx, lib().bltc_direct_sum(ctx, _ptr(tx), _ptr(ty), _ptr(tz), tx.numel(), _ptr(sx),
                                      _ptr(sy), _ptr(sz), _ptr(sq), sx.numel(), ctypes.byref(p),
                                      _ptr(phi)))


def bltc_autotune(ctx, x, y, z, q, p: bltc_params, leaf=(500, 1000, 2000, 3000, 4000),
                  batch=None, repeats=2, use_cache=True):
    """Returns (best params, {(leaf, batch): fastest ms}) for the device system x, y, z, q."""
    _stream(ctx)
    L = np.ascontiguousarray(leaf, dtype=np.int32)
    B = None if batch is None else np.ascontiguousarray(batch, dtype=np.int32)
    ms = np.full(len(L), np.nan, dtype=np.float32)
    best = bltc_params()
    _check(ctx, lib().bltc_autotune(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(q), x.numel(),
                                    ctypes.byref(p), L.ctypes.data,
                                    None if B is None else B.ctypes.data, len(L), int(repeats),
                                    1 if use_cache else 0, ctypes.byref(best), ms.ctypes.data))
    keys = [(int(l), int(bb)) for l, bb in zip(L, L if B is None else B)]
    return best, {k: float(v) for k, v in zip(keys, ms)}


def bltc_autotune_tile(ctx, x, y, z, q, p: bltc_params, tiles, repeats=1, use_cache=True):
    """Returns (params with the fastest tile, {tile: fastest ms}) at p's leaf and batch sizes."""
    _stream(ctx)
    T = np.ascontiguousarray(tiles, dtype=np.int32)
    ms = np.full(len(T), np.nan, dtype=np.float32)
    best = bltc_params()
    _check(ctx, lib().bltc_autotune_tile(ctx, _ptr(x), _ptr(y), _ptr(z), _ptr(q), x.numel(),
                                         ctypes.byref(p), T.ctypes.data, len(T), int(repeats),
                                         1 if use_cache else 0, ctypes.byref(best), ms.ctypes.data))
    return best, {int(t): float(v) for t, v in zip(T, ms)}


# ---- serving -------------------------------------------------------------------------

def bltc_server_create(device=0, setup_workers=2, max_batch=32, hbm_budget_bytes=0, linger_us=0,
                       slice_us=15000, setup_blocks=0, slices_in_flight=0):
    cfg = bltc_server_config(int(device), int(setup_workers), int(max_batch), int(linger_us),
                             int(hbm_budget_bytes), int(slice_us), int(setup_blocks),
                             int(slices_in_flight))
    h = ctypes.c_void_p()
    st = lib().bltc_server_create(ctypes.byref(cfg), ctypes.byref(h))
    if st != BLTC_OK:
        raise BltcError(st, "server creation failed")
    return h.value


def bltc_server_submit(server, x, y, z, q, p: bltc_params, phi):
    """Host arrays (contiguous float64); they must stay alive until bltc_server_wait returns."""
    t = ctypes.c_uint64()
    st = lib().bltc_server_submit(server, _ptr(x), _ptr(y), _ptr(z), _ptr(q), x.shape[0],
                                  ctypes.byref(p), _ptr(phi), ctypes.byref(t))
    if st != BLTC_OK:
        raise BltcError(st, "submit rejected")
    return t.value


def bltc_server_wait(server, ticket, timeout_s=-1.0):
    """Returns (status, info dict); status TIMEOUT leaves the ticket valid."""
    info = bltc_request_info()
    st = lib().bltc_server_wait(server, ticket, float(timeout_s), ctypes.byref(info))
    return st, {k: getattr(info, k) for k, _ in bltc_request_info._fields_}


def bltc_server_cancel(server, ticket):
    st = lib().bltc_server_cancel(server, ticket)
    if st != BLTC_OK:
        raise BltcError(st, "cancel refused")


def bltc_server_stats(server):
    c = bltc_server_counters()
    st = lib().bltc_server_stats(server, ctypes.byref(c))
    if st != BLTC_OK:
        raise BltcError(st, "stats failed")
    return {k: getattr(c, k) for k, _ in bltc_server_counters._fields_}


def bltc_server_last_error(server):
    """Message of the most recently failed request ('' if none)."""
    buf = ctypes.create_string_buffer(1024)
    lib().bltc_server_last_error(server, buf, len(buf))
    return buf.value.decode(errors="replace")


def bltc_server_destroy(server):
    lib().bltc_server_destroy(server)


class Server:
    """Owns a serving runtime; keeps each request's host arrays alive until it is waited."""

    def __init__(self, device=0, setup_workers=2, max_batch=32, hbm_budget_bytes=0, linger_us=0,
                 slice_us=15000, setup_blocks=0, slices_in_flight=0):
        self.h = bltc_server_create(device, setup_workers, max_batch, hbm_budget_bytes, linger_us,
                                    slice_us, setup_blocks, slices_in_flight)
        self._keep = {}

    def submit(self, x, y, z, q, p, phi=None):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, q)]
        if phi is None:
            phi = np.empty(arrs[0].shape[0])
        t = bltc_server_submit(self.h, *arrs, p, phi)
        self._keep[t] = (arrs, phi)
        return t

    def wait(self, ticket, timeout_s=-1.0):
        st, info = bltc_server_wait(self.h, ticket, timeout_s)
        if st == BLTC_ERR_TIMEOUT:
            return st, None, info
        arrs, phi = self._keep.pop(ticket)
        return st, phi, info

    def cancel(self, ticket):
        bltc_server_cancel(self.h, ticket)

    def stats(self):
        return bltc_server_stats(self.h)

    def last_error(self):
        return bltc_server_last_error(self.h)

    def close(self):
        if self.h:
            bltc_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bltc_direct_sum_noalloc(ctx, tx, ty, tz, sx, sy, sz, sq, p: bltc_params, phi):
    """bltc_direct_sum without any device allocation (fixed 64 MiB library scratch; calls
    on one device must not overlap on the GPU; at most 8,388,608 targets)."""
    _stream(ctx)
    _check(ctx, lib().bltc_direct_sum_noalloc(ctx, _ptr(tx), _ptr(ty), _ptr(tz), tx.numel(),
                                              _ptr(sx), _ptr(sy), _ptr(sz), _ptr(sq), sx.numel(),
                                              ctypes.byref(p), _ptr(phi)))


# ---- convenience owner of a context ----------------------------------------------------

class Graph:
    """A solve with fixed positions, replayed as one CUDA graph (bltc_graph_*).  The charges
    tensor ``q`` and the output ``phi`` are bound: write new charges into ``q`` (in place), call
    ``launch()``, read ``phi``."""

    def __init__(self, ctx, x, y, z, q, p, phi=None, positions=False, headroom=0.0):
        """``positions=True``: the whole solve sized on the device, so the positions tensors
        ``x, y, z`` are bound too and may change (in place) between launches."""
        import torch
        self.ctx = ctx
        self.x, self.y, self.z, self.q = x, y, z, q
        self.phi = torch.empty_like(x) if phi is None else phi
        if positions:
            self.h = bltc_graph_create_positions(ctx.h, x, y, z, q, p, self.phi, headroom)
        else:
            self.h = bltc_graph_create(ctx.h, x, y, z, q, p, self.phi)

    @property
    def kernels(self):
        return bltc_graph_kernels(self.h)

    @property
    def info(self):
        return bltc_graph_info(self.h)

    def launch(self):
        bltc_graph_launch(self.ctx.h, self.h)
        return self.phi

    def close(self):
        if self.h:
            bltc_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Owns a bltc context on ``device``; by default the library allocates its working
    memory through torch's caching allocator."""

    def __init__(self, device=0, torch_allocator=True):
        import torch
        self.device = device
        self.h = bltc_context_create(device, torch.cuda.current_stream(device).cuda_stream)
        self._alloc = None
        if torch_allocator:
            self._alloc = _TorchAllocator(device)
            bltc_context_set_allocator(self.h, self._alloc.alloc, self._alloc.free)

    def close(self):
        if self.h:
            bltc_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def sm_count(self):
        return bltc_device_sm_count(self.h)

    def solve(self, x, y, z, q, p, phi=None):
        import torch
        if phi is None:
            phi = torch.empty_like(x)
        bltc_solve(self.h, x, y, z, q, p, phi)
        return phi

    def direct_sum(self, targets, sources, q, p, phi=None):
        import torch
        if phi is None:
            phi = torch.empty_like(targets[0])
        bltc_direct_sum(self.h, targets[0], targets[1], targets[2], sources[0], sources[1],
                        sources[2], q, p, phi)
        return phi
