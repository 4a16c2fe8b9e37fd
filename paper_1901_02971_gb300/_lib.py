"""ctypes binding of the spaND C ABI (``include/spand.h``).

Argument marshalling only: every step of the method runs inside
``libspand.so`` (host analysis in C++, factorization / apply / PCG in CUDA
kernels for sm_103a).  There is no Python or CPU fallback: if the library is
missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspand.so")

SPAND_OK = 0
SPAND_ERR_INVALID_ARG = 1
SPAND_ERR_NOT_SPD = 2
SPAND_ERR_NO_CONVERGENCE = 3
SPAND_ERR_CUDA = 4
SPAND_ERR_OOM = 5
SPAND_ERR_STATE = 6
SPAND_ERR_TIMEOUT = 7
SPAND_FP64 = 0
SPAND_FP32 = 1
SPAND_TF32 = 2
SPAND_BF16 = 3
SPAND_COLOURED = 0
SPAND_SIMULTANEOUS = 1
SPAND_CPQR = 0
SPAND_RANDOMIZED = 1
SPAND_ORTHS = 0
SPAND_INS = 1
SPAND_IN = 2

# every function declared in include/spand.h
EXPORTS = ["spand_default_opts", "spand_analyze", "spand_analyze_batch", "spand_factorize", "spand_solve", "spand_apply",
           "spand_apply_noalloc", "spand_sampled_outer", "spand_sketch_gaussian",
           "spand_get_tree", "spand_get_step", "spand_get_ranks", "spand_get_stats",
           "spand_get_phase_times", "spand_set_profiling", "spand_get_kernel_profile",
           "spand_reset_kernel_profile", "spand_get_launch_count", "spand_set_apply_wait", "spand_set_apply_shape",
           "spand_destroy",
           "spand_error_string",
           "spand_last_error"]
KERNEL_FAMILIES = ["potrf", "trsm", "schur", "cpqr", "copy", "apply", "pcg"]


class Opts(C.Structure):
    _fields_ = [("levels", C.c_int32), ("eps", C.c_double), ("skip", C.c_int32),
                ("precision", C.c_int32), ("maxit", C.c_int32), ("tol", C.c_double),
                ("sparsify_order", C.c_int32), ("compression", C.c_int32), ("sketch_seed", C.c_uint64),
                ("variant", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("vals", C.c_void_p),
                ("coords", C.c_void_p), ("dim", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("t_analyze_s", C.c_double), ("t_factor_s", C.c_double), ("t_solve_s", C.c_double),
                ("n_cg", C.c_int32), ("relres", C.c_double), ("size_top", C.c_int64),
                ("mem_f", C.c_int64), ("factor_flops", C.c_double), ("apply_bytes", C.c_double),
                ("fail_step", C.c_int32), ("fail_cluster", C.c_int32), ("device_bytes", C.c_int64),
                ("apply_ctas_per_sm", C.c_int32)]


class SpandError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spaND error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libspand.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1901_02971_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    i32p = C.POINTER(C.c_int32)
    L.spand_default_opts.argtypes = [C.POINTER(Opts)]
    L.spand_default_opts.restype = None
    L.spand_analyze.argtypes = [C.c_int64, P, P, P, P, C.c_int32, C.POINTER(Opts), C.POINTER(C.c_void_p)]
    L.spand_analyze_batch.argtypes = [C.c_int32, C.POINTER(Problem), C.POINTER(Opts), C.POINTER(C.c_void_p)]
    L.spand_factorize.argtypes = [C.c_void_p, P, P]
    L.spand_solve.argtypes = [C.c_void_p, P, P, i32p, C.POINTER(C.c_double), P]
    L.spand_apply.argtypes = [C.c_void_p, P, P, P]
    L.spand_apply_noalloc.argtypes = [C.c_void_p, P, P, P]
    L.spand_sampled_outer.argtypes = [C.c_void_p, P, P, P, P]
    L.spand_sketch_gaussian.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P]
    L.spand_get_tree.argtypes = [C.c_void_p, P, P, P, i32p, i32p]
    L.spand_get_step.argtypes = [C.c_void_p, C.c_int32] + [P] * 10
    L.spand_get_ranks.argtypes = [C.c_void_p, C.c_int32, P, P]
    L.spand_get_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
    L.spand_get_phase_times.argtypes = [C.c_void_p, P]
    L.spand_set_profiling.argtypes = [C.c_void_p, C.c_int32]
    L.spand_get_kernel_profile.argtypes = [C.c_void_p, C.c_int32, P]
    L.spand_reset_kernel_profile.argtypes = [C.c_void_p]
    L.spand_get_launch_count.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
    L.spand_set_apply_wait.argtypes = [C.c_void_p, C.c_uint32, C.c_int32]
    L.spand_set_apply_shape.argtypes = [C.c_void_p, C.c_int32]
    L.spand_destroy.argtypes = [C.c_void_p]
    L.spand_destroy.restype = None
    L.spand_error_string.argtypes = [C.c_int]
    L.spand_error_string.restype = C.c_char_p
    L.spand_last_error.argtypes = []
    L.spand_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("spand_default_opts", "spand_destroy", "spand_error_string", "spand_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != SPAND_OK:
        raise SpandError(rc, lib().spand_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().spand_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def spand_analyze(rowptr, colind, vals, coords=None, opts: Optional[Opts] = None) -> int:
    """Returns an opaque handle (int)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    n = rowptr.size - 1
    cptr, dim = None, 0
    if coords is not None:
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        dim = coords.shape[1] if coords.ndim == 2 else 1
        cptr = _ptr(coords)
    opts = opts or default_opts()
    h = C.c_void_p()
    _check(lib().spand_analyze(n, _ptr(rowptr), _ptr(colind), _ptr(vals), cptr, dim, C.byref(opts), C.byref(h)))
    return h.value


def spand_analyze_batch(problems, opts_list) -> list:
    """problems: list of (rowptr, colind, vals, coords-or-None); opts_list: one
    Opts per problem.  Returns the list of handles (ints), analyzed on parallel
    host threads inside the library."""
    k = len(problems)
    if len(opts_list) != k:
        raise ValueError("one Opts per problem")
    keep = []
    P = (Problem * max(k, 1))()
    for i, (rowptr, colind, vals, coords) in enumerate(problems):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colind = np.ascontiguousarray(colind, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        dim = 0
        if coords is not None:
            coords = np.ascontiguousarray(coords, dtype=np.float64)
            dim = coords.shape[1] if coords.ndim == 2 else 1
        keep += [rowptr, colind, vals, coords]
        P[i] = Problem(rowptr.size - 1, rowptr.ctypes.data, colind.ctypes.data, vals.ctypes.data,
                       coords.ctypes.data if coords is not None else None, dim)
    O = (Opts * max(k, 1))(*opts_list)
    H = (C.c_void_p * max(k, 1))()
    _check(lib().spand_analyze_batch(k, P, O, H))
    return [H[i] for i in range(k)]


def spand_factorize(h: int, vals_ptr: Optional[int] = None, stream: int = 0):
    """vals_ptr: None (values given to analyze) or the address of float64[nnz]
    (host or device)."""
    _check(lib().spand_factorize(h, vals_ptr, stream or None))


def spand_solve(h: int, b_ptr: int, x_ptr: int, stream: int = 0, check: bool = True):
    """b_ptr / x_ptr: addresses of float64[n] (host or device).  Returns
    (rc, iterations, relative residual)."""
    it = C.c_int32(0)
    rr = C.c_double(0.0)
    rc = lib().spand_solve(h, b_ptr, x_ptr, C.byref(it), C.byref(rr), stream or None)
    if check and rc not in (SPAND_OK,):
        _check(rc)
    return rc, it.value, rr.value


def spand_apply(h: int, r_ptr: int, z_ptr: int, stream: int = 0):
    _check(lib().spand_apply(h, r_ptr, z_ptr, stream or None))


def spand_apply_noalloc(h: int, r_ptr: int, z_ptr: int, stream: int = 0):
    """z = M M^T r on device vectors without allocating device memory (fixed
    work array inside the library; see include/spand.h)."""
    _check(lib().spand_apply_noalloc(h, r_ptr, z_ptr, stream or None))


def spand_sampled_outer(h: int, lam_ptr: int, x_ptr: int, out_ptr: int, stream: int = 0):
    """out[e] = -lam[i] x[j] on A's stored pattern (device pointers)."""
    _check(lib().spand_sampled_outer(h, lam_ptr, x_ptr, out_ptr, stream or None))


def spand_sketch_gaussian(seed: int, step: int, cluster: int, m: int, ell: int, out_ptr: int, stream: int = 0):
    """Gaussian test matrix (m x ell, column-major, device float64) of the
    randomized compression, drawn on the device from its counter."""
    _check(lib().spand_sketch_gaussian(seed, step, cluster, m, ell, out_ptr, stream or None))


def spand_get_tree(h: int) -> dict:
    """perm, cluster_ptr, keys (3 per cluster) and the number of steps."""
    nc = C.c_int32(0)
    ns = C.c_int32(0)
    _check(lib().spand_get_tree(h, None, None, None, C.byref(nc), C.byref(ns)))
    cptr = np.zeros(nc.value + 1, dtype=np.int32)
    keys = np.zeros(3 * nc.value, dtype=np.int32)
    _check(lib().spand_get_tree(h, None, _ptr(cptr), _ptr(keys), C.byref(nc), None))
    perm = np.zeros(int(cptr[-1]), dtype=np.int32)
    _check(lib().spand_get_tree(h, _ptr(perm), None, None, C.byref(nc), None))
    return {"perm": perm, "cluster_ptr": cptr, "keys": keys, "n_steps": ns.value}


def spand_get_step(h: int, t: int) -> dict:
    counts = np.zeros(5, dtype=np.int32)
    nul = [None] * 9
    _check(lib().spand_get_step(h, t, _ptr(counts), *nul))
    n, nch, nadj, nadjf, _ = (int(v) for v in counts)
    out = {
        "keys": np.zeros(3 * n, np.int32), "child_ptr": np.zeros(n + 1, np.int32),
        "child_idx": np.zeros(nch, np.int32), "elim": np.zeros(n, np.int32), "colour": np.zeros(n, np.int32),
        "adj_ptr": np.zeros(n + 1, np.int32), "adj_idx": np.zeros(nadj, np.int32),
        "adjf_ptr": np.zeros(n + 1, np.int32), "adjf_idx": np.zeros(nadjf, np.int32),
    }
    order = ["keys", "child_ptr", "child_idx", "elim", "colour", "adj_ptr", "adj_idx", "adjf_ptr", "adjf_idx"]
    _check(lib().spand_get_step(h, t, _ptr(counts), *[_ptr(out[k]) for k in order]))
    return out


def spand_get_ranks(h: int, t: int):
    n = spand_get_step(h, t)["elim"].size
    before = np.zeros(n, np.int32)
    after = np.zeros(n, np.int32)
    _check(lib().spand_get_ranks(h, t, _ptr(before), _ptr(after)))
    return before, after


def spand_get_stats(h: int) -> Stats:
    s = Stats()
    _check(lib().spand_get_stats(h, C.byref(s)))
    return s


def spand_get_phase_times(h: int) -> np.ndarray:
    out = np.zeros(6, dtype=np.float64)
    _check(lib().spand_get_phase_times(h, _ptr(out)))
    return out


def spand_set_profiling(h: int, on: bool):
    _check(lib().spand_set_profiling(h, 1 if on else 0))


def spand_get_kernel_profile(h: int) -> dict:
    """family -> dict(launches, ms, flops, bytes)."""
    out = {}
    buf = np.zeros(4)
    for i, name in enumerate(KERNEL_FAMILIES):
        _check(lib().spand_get_kernel_profile(h, i, _ptr(buf)))
        out[name] = {"launches": int(buf[0]), "ms": float(buf[1]), "flops": float(buf[2]), "bytes": float(buf[3])}
    return out


def spand_reset_kernel_profile(h: int):
    _check(lib().spand_reset_kernel_profile(h))


def spand_get_launch_count(h: int) -> int:
    v = C.c_int64(0)
    _check(lib().spand_get_launch_count(h, C.byref(v)))
    return v.value


def spand_set_apply_wait(h: int, polls: int = 0, unreachable: bool = False):
    """Failure-path knob: bound the apply's grid-barrier waits by `polls`
    polls (0 = default); `unreachable` makes every wait run out."""
    _check(lib().spand_set_apply_wait(h, polls, 1 if unreachable else 0))


def spand_set_apply_shape(h: int, ctas_per_sm: int = 0):
    """CTAs per SM of the preconditioner apply (1..4), or 0: autotuned."""
    _check(lib().spand_set_apply_shape(h, ctas_per_sm))


def spand_destroy(h: int):
    if h:
        lib().spand_destroy(h)


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    relres: float
    rc: int
