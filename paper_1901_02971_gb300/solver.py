"""Convenience wrapper over the C ABI (argument marshalling only)."""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import _lib as L


def _addr(a):
    """Address of a contiguous float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data
    assert str(a.dtype) == "torch.float64" and a.is_contiguous()
    return a.data_ptr()


PRECISIONS = {"fp64": L.SPAND_FP64, "fp32": L.SPAND_FP32, "tf32": L.SPAND_TF32, "bf16": L.SPAND_BF16}
ORDERS = {"coloured": L.SPAND_COLOURED, "simultaneous": L.SPAND_SIMULTANEOUS}
COMPRESSIONS = {"cpqr": L.SPAND_CPQR, "randomized": L.SPAND_RANDOMIZED}
VARIANTS = {"OrthS": L.SPAND_ORTHS, "InS": L.SPAND_INS, "In": L.SPAND_IN}


class Solver:
    """analyze -> factorize -> solve on one CSR matrix.

    Parameters follow ``spand_opts``: levels (L of Algorithm 3), eps, skip,
    precision ("fp64", "fp32", or "tf32" / "bf16": FP32 factors whose Schur
    GEMMs run on the tensor cores with TF32 / BF16 operands), maxit, tol,
    sparsify_order ("coloured", or "simultaneous": every interface of a level
    compressed from the same scaled matrix, one launch per level),
    compression ("cpqr", or "randomized": a Gaussian-sketch range finder in
    place of the column-pivoted QR, sketches keyed by sketch_seed), variant
    ("OrthS", or the interpolative "InS" / "In" of Sec. 2.6.2, with / without
    the block scaling).
    """

    def __init__(self, rowptr, colind, vals, coords=None, levels: int = 8, eps: float = 1e-2, skip: int = 0,
                 precision: str = "fp64", maxit: int = 500, tol: float = 1e-10, sparsify_order: str = "coloured",
                 compression: str = "cpqr", sketch_seed: int = 0, variant: str = "OrthS"):
        prec = PRECISIONS[precision]
        order = ORDERS[sparsify_order]
        self.opts = L.default_opts(levels=levels, eps=eps, skip=skip, precision=prec, maxit=maxit, tol=tol,
                                   sparsify_order=order, compression=COMPRESSIONS[compression],
                                   sketch_seed=int(sketch_seed), variant=VARIANTS[variant])
        self.n = int(np.asarray(rowptr).size - 1)
        self.nnz = int(np.asarray(rowptr)[-1])
        self.h = L.spand_analyze(rowptr, colind, vals, coords, self.opts)

    @classmethod
    def from_problem(cls, prob, use_coords: bool = True, **kw):
        return cls(prob.rowptr, prob.colind, prob.vals, prob.coords if use_coords else None, **kw)

    def factorize(self, vals=None, stream: int = 0):
        L.spand_factorize(self.h, None if vals is None else _addr(vals), stream)
        return self

    def solve(self, b, x=None, stream: int = 0, check: bool = True):
        """b: float64 numpy array (host) or torch CUDA tensor; returns (x, iters, relres)."""
        if x is None:
            x = np.empty(self.n) if isinstance(b, np.ndarray) else b.new_empty(b.shape)
        if stream == 0 and not isinstance(b, np.ndarray):
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        rc, it, rr = L.spand_solve(self.h, _addr(b), _addr(x), stream, check=check)
        return x, it, rr

    def apply(self, r, z=None, stream: int = 0):
        if z is None:
            z = r.new_empty(r.shape)
        L.spand_apply(self.h, _addr(r), _addr(z), stream)
        return z

    def tree(self) -> dict:
        return L.spand_get_tree(self.h)

    def step(self, t: int) -> dict:
        return L.spand_get_step(self.h, t)

    def ranks(self, t: int):
        return L.spand_get_ranks(self.h, t)

    def stats(self):
        return L.spand_get_stats(self.h)

    def phase_times(self):
        return L.spand_get_phase_times(self.h)

    def set_profiling(self, on: bool = True):
        L.spand_set_profiling(self.h, on)

    def kernel_profile(self) -> dict:
        return L.spand_get_kernel_profile(self.h)

    def reset_kernel_profile(self):
        L.spand_reset_kernel_profile(self.h)

    def launch_count(self) -> int:
        return L.spand_get_launch_count(self.h)

    def close(self):
        if self.h:
            L.spand_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @classmethod
    def batch(cls, problems, opts_list) -> list:
        """Solvers for k independent problems, analyzed together
        (spand_analyze_batch, parallel host threads).  problems: objects with
        rowptr, colind, vals and coords (or None); opts_list: one dict of
        Solver keyword arguments per problem."""
        opts = []
        for kw in opts_list:
            prec = PRECISIONS[kw.get("precision", "fp64")]
            opts.append(L.default_opts(levels=kw.get("levels", 8), eps=kw.get("eps", 1e-2), skip=kw.get("skip", 0),
                                       precision=prec, maxit=kw.get("maxit", 500), tol=kw.get("tol", 1e-10),
                                       sparsify_order=ORDERS[kw.get("sparsify_order", "coloured")],
                                       compression=COMPRESSIONS[kw.get("compression", "cpqr")],
                                       sketch_seed=int(kw.get("sketch_seed", 0)),
                                       variant=VARIANTS[kw.get("variant", "OrthS")]))
        hs = L.spand_analyze_batch([(p.rowptr, p.colind, p.vals, p.coords) for p in problems], opts)
        out = []
        for p, o, h in zip(problems, opts, hs):
            s = cls.__new__(cls)
            s.opts, s.n, s.nnz, s.h = o, int(p.rowptr.size - 1), int(p.rowptr[-1]), h
            out.append(s)
        return out


def _each_on_own_stream(solvers, fn):
    """Runs fn(index, solver, stream) for every solver at once, one host thread
    and one CUDA stream per solver (independent handles share nothing; the
    library releases the GIL inside every call)."""
    import concurrent.futures as cf
    import torch
    dev = torch.cuda.current_device()
    streams = [torch.cuda.Stream() for _ in solvers]

    def run(i):
        torch.cuda.set_device(dev)
        with torch.cuda.stream(streams[i]):
            return fn(i, solvers[i], streams[i].cuda_stream)

    with cf.ThreadPoolExecutor(max_workers=max(1, len(solvers))) as ex:
        res = list(ex.map(run, range(len(solvers))))
    for st in streams:
        st.synchronize()
    return res


def factorize_all(solvers, vals_list=None):
    """Factorizes independent solvers concurrently (one stream each)."""
    _each_on_own_stream(solvers, lambda i, s, st: s.factorize(None if vals_list is None else vals_list[i], stream=st))
    return solvers


def solve_all(solvers, bs, xs=None):
    """Solves independent systems concurrently; returns [(x, iters, relres)]."""
    return _each_on_own_stream(solvers, lambda i, s, st: s.solve(bs[i], None if xs is None else xs[i], stream=st))
