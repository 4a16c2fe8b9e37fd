"""GB300-native sparsified nested dissection (spaND) preconditioned CG.

The work happens in ``libspand.so`` behind the C ABI of ``include/spand.h``:
host-side analysis (Algorithm 3), level-by-level factorization on the GPU
(Algorithm 2, OrthS) and PCG with the z = M M^T r preconditioner (Sec. 2.8).
This package only marshals arguments (``_lib``) and offers the ``Solver``
convenience wrapper; ``inputs`` holds seeded synthetic problem generators.
"""
from __future__ import annotations

from ._lib import (SPAND_FP32, SPAND_FP64, SpandError, default_opts, lib, spand_analyze, spand_apply,
                   spand_destroy, spand_factorize, spand_get_phase_times, spand_get_ranks, spand_get_stats,
                   spand_get_step, spand_get_tree, spand_solve)
from .solver import Solver, factorize_all, solve_all

__all__ = ["Solver", "factorize_all", "solve_all", "SpandError", "SPAND_FP32", "SPAND_FP64", "default_opts", "lib", "spand_analyze",
           "spand_apply", "spand_destroy", "spand_factorize", "spand_get_phase_times", "spand_get_ranks",
           "spand_get_stats", "spand_get_step", "spand_get_tree", "spand_solve"]
