"""The C ABI loads, exports every declared symbol, and rejects bad input on
the host (no GPU needed for these checks)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1901_02971_gb300 import _lib as L
from paper_1901_02971_gb300 import inputs as I

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "spand.h")


def declared():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(spand_[a-z_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert declared() == sorted(L.EXPORTS)


def test_every_symbol_exported(spand_lib):
    for name in declared():
        assert hasattr(spand_lib, name), name


def test_error_strings(spand_lib):
    for code in range(8):
        assert spand_lib.spand_error_string(code)


def _analyze_rc(rowptr, colind, vals, levels=3):
    o = L.default_opts(levels=levels)
    h = C.c_void_p()
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colind = np.ascontiguousarray(colind, np.int32)
    vals = np.ascontiguousarray(vals, np.float64)
    rc = L.lib().spand_analyze(rowptr.size - 1, rowptr.ctypes.data, colind.ctypes.data, vals.ctypes.data, None, 0,
                               C.byref(o), C.byref(h))
    if h.value:
        L.spand_destroy(h.value)
    return rc


def test_malformed_csr_rejected(spand_lib):
    p = I.laplacian_2d(4)
    assert _analyze_rc(p.rowptr, p.colind, p.vals) == L.SPAND_OK
    # non-symmetric pattern: drop one off-diagonal entry of row 0
    rp, ci, va = p.rowptr.copy(), p.colind.copy(), p.vals.copy()
    k = int(rp[0]) + 1
    ci2 = np.delete(ci, k)
    va2 = np.delete(va, k)
    rp2 = rp.copy()
    rp2[1:] -= 1
    assert _analyze_rc(rp2, ci2, va2) == L.SPAND_ERR_INVALID_ARG
    # unsorted columns in a row
    ci3 = ci.copy()
    ci3[rp[1]], ci3[rp[1] + 1] = ci3[rp[1] + 1], ci3[rp[1]]
    assert _analyze_rc(rp, ci3, va) == L.SPAND_ERR_INVALID_ARG
    # column out of range
    ci4 = ci.copy()
    ci4[-1] = p.n
    assert _analyze_rc(rp, ci4, va) == L.SPAND_ERR_INVALID_ARG
    # bad levels
    assert _analyze_rc(rp, ci, va, levels=0) == L.SPAND_ERR_INVALID_ARG
    assert "levels" in L.lib().spand_last_error().decode()


def test_sparsify_order_option(spand_lib):
    assert L.default_opts().sparsify_order == L.SPAND_COLOURED
    p = I.laplacian_2d(6)
    for order, want in [(L.SPAND_COLOURED, L.SPAND_OK), (L.SPAND_SIMULTANEOUS, L.SPAND_OK), (2, L.SPAND_ERR_INVALID_ARG),
                        (-1, L.SPAND_ERR_INVALID_ARG)]:
        o = L.default_opts(levels=3, sparsify_order=order)
        h = C.c_void_p()
        rc = L.lib().spand_analyze(p.n, p.rowptr.ctypes.data, p.colind.ctypes.data, p.vals.ctypes.data, None, 0,
                                   C.byref(o), C.byref(h))
        if h.value:
            L.spand_destroy(h.value)
        assert rc == want, (order, rc)
    assert "sparsify_order" in L.lib().spand_last_error().decode()


def test_missing_diagonal_rejected(spand_lib):
    rowptr = np.array([0, 1, 2], np.int64)
    colind = np.array([1, 0], np.int32)
    assert _analyze_rc(rowptr, colind, np.ones(2)) == L.SPAND_ERR_INVALID_ARG


def test_solve_before_factorize_is_state_error(spand_lib):
    p = I.laplacian_2d(4)
    h = L.spand_analyze(p.rowptr, p.colind, p.vals, p.coords, L.default_opts(levels=2))
    try:
        b = np.ones(p.n)
        x = np.zeros(p.n)
        rc, _, _ = L.spand_solve(h, b.ctypes.data, x.ctypes.data, check=False)
        assert rc == L.SPAND_ERR_STATE
        with pytest.raises(L.SpandError):
            L.spand_get_ranks(h, 1)
    finally:
        L.spand_destroy(h)


def _tree_arrays(h):
    t = L.spand_get_tree(h)
    return {k: np.asarray(v) for k, v in t.items()}


def test_analyze_batch_matches_single(spand_lib):
    """Batch analysis (parallel host threads) gives, problem by problem, the
    same ordering, clusters and steps as spand_analyze."""
    probs = [I.laplacian_2d(24), I.diffusion_2d(20, 3), I.laplacian_3d(10), I.knn_laplacian(400, 6, 2)]
    levels = [5, 4, 4, 5]
    opts = [L.default_opts(levels=lv) for lv in levels]
    hs = L.spand_analyze_batch([(p.rowptr, p.colind, p.vals, p.coords) for p in probs], opts)
    try:
        for p, lv, h in zip(probs, levels, hs):
            h1 = L.spand_analyze(p.rowptr, p.colind, p.vals, p.coords, L.default_opts(levels=lv))
            try:
                a, b = _tree_arrays(h), _tree_arrays(h1)
                assert a.keys() == b.keys()
                for k in a:
                    assert np.array_equal(a[k], b[k]), k
                for t in range(1, lv + 1):
                    sa, sb = L.spand_get_step(h, t), L.spand_get_step(h1, t)
                    for k in sa:
                        assert np.array_equal(np.asarray(sa[k]), np.asarray(sb[k])), (t, k)
            finally:
                L.spand_destroy(h1)
    finally:
        for h in hs:
            L.spand_destroy(h)


def test_analyze_batch_error_names_problem(spand_lib):
    good = I.laplacian_2d(12)
    bad_colind = good.colind.copy()
    bad_colind[1], bad_colind[2] = bad_colind[2], bad_colind[1]  # unsorted row
    probs = [(good.rowptr, good.colind, good.vals, good.coords), (good.rowptr, bad_colind, good.vals, None),
             (good.rowptr, good.colind, good.vals, None)]
    with pytest.raises(L.SpandError) as e:
        L.spand_analyze_batch(probs, [L.default_opts(levels=3)] * 3)
    assert e.value.code == L.SPAND_ERR_INVALID_ARG
    assert "problem 1" in str(e.value)
    assert L.spand_analyze_batch([], []) == []


def test_batch_and_solver_pass_the_sparsify_order(spand_lib):
    """The Python layer forwards the order to spand_opts (analysis only)."""
    from paper_1901_02971_gb300 import Solver
    ps = [I.laplacian_2d(8), I.laplacian_2d(9)]
    ss = Solver.batch(ps, [{"levels": 3, "sparsify_order": "simultaneous"}, {"levels": 3}])
    try:
        assert ss[0].opts.sparsify_order == L.SPAND_SIMULTANEOUS
        assert ss[1].opts.sparsify_order == L.SPAND_COLOURED
    finally:
        for s in ss:
            s.close()
    s = Solver.from_problem(ps[0], levels=3, sparsify_order="simultaneous")
    try:
        assert s.opts.sparsify_order == L.SPAND_SIMULTANEOUS
    finally:
        s.close()
    with pytest.raises(KeyError):
        Solver.from_problem(ps[0], levels=3, sparsify_order="random")



def test_sketch_argument_checks(spand_lib):
    """Host-side checks of spand_sketch_gaussian (no launch happens)."""
    f = spand_lib.spand_sketch_gaussian
    assert f(1, 0, 0, -1, 4, None, None) == L.SPAND_ERR_INVALID_ARG
    assert f(1, 0, 0, 4, -1, None, None) == L.SPAND_ERR_INVALID_ARG
    assert f(1, -1, 0, 4, 4, None, None) == L.SPAND_ERR_INVALID_ARG
    assert f(1, 0, -1, 4, 4, None, None) == L.SPAND_ERR_INVALID_ARG
    assert f(1, 0, 0, 4, 4, None, None) == L.SPAND_ERR_INVALID_ARG   # null output
    host = np.zeros(16)
    assert f(1, 0, 0, 4, 4, host.ctypes.data, None) == L.SPAND_ERR_INVALID_ARG  # not device memory
    assert f(1, 0, 0, 0, 4, None, None) == L.SPAND_OK                # empty: nothing to do
    assert f(1, 0, 0, 4, 0, None, None) == L.SPAND_OK


def test_apply_wait_knob_argument_checks(spand_lib):
    """The failure-path knob and the launch shape of the apply are host-side
    settings."""
    assert spand_lib.spand_set_apply_wait(None, 16, 1) == L.SPAND_ERR_INVALID_ARG
    assert spand_lib.spand_set_apply_shape(None, 2) == L.SPAND_ERR_INVALID_ARG
    p = I.laplacian_2d(8)
    h = L.spand_analyze(p.rowptr, p.colind, p.vals, p.coords, L.default_opts(levels=3))
    try:
        L.spand_set_apply_wait(h, 16, True)
        L.spand_set_apply_wait(h, 0, False)
        assert spand_lib.spand_set_apply_shape(h, 5) == L.SPAND_ERR_INVALID_ARG
        assert spand_lib.spand_set_apply_shape(h, -1) == L.SPAND_ERR_INVALID_ARG
        L.spand_set_apply_shape(h, 3)
        L.spand_set_apply_shape(h, 0)
    finally:
        L.spand_destroy(h)


def test_compression_option(spand_lib):
    """compression is SPAND_CPQR by default; SPAND_RANDOMIZED is accepted in
    the coloured order only; unknown values are refused."""
    assert L.default_opts().compression == L.SPAND_CPQR and L.default_opts().sketch_seed == 0
    p = I.laplacian_2d(6)
    for comp, order, want in [(L.SPAND_CPQR, L.SPAND_COLOURED, L.SPAND_OK),
                              (L.SPAND_RANDOMIZED, L.SPAND_COLOURED, L.SPAND_OK),
                              (L.SPAND_RANDOMIZED, L.SPAND_SIMULTANEOUS, L.SPAND_ERR_INVALID_ARG),
                              (2, L.SPAND_COLOURED, L.SPAND_ERR_INVALID_ARG)]:
        o = L.default_opts(levels=3, compression=comp, sparsify_order=order, sketch_seed=2 ** 63 + 5)
        h = C.c_void_p()
        rc = L.lib().spand_analyze(p.n, p.rowptr.ctypes.data, p.colind.ctypes.data, p.vals.ctypes.data, None, 0,
                                   C.byref(o), C.byref(h))
        if h.value:
            L.spand_destroy(h.value)
        assert rc == want, (comp, order, rc)


def test_variant_option(spand_lib):
    """variant is SPAND_ORTHS by default; the interpolative SPAND_INS /
    SPAND_IN run in the coloured order with column-pivoted QR only; unknown
    values are refused."""
    assert L.default_opts().variant == L.SPAND_ORTHS
    p = I.laplacian_2d(6)
    for var, order, comp, want in [(L.SPAND_ORTHS, L.SPAND_SIMULTANEOUS, L.SPAND_CPQR, L.SPAND_OK),
                                   (L.SPAND_INS, L.SPAND_COLOURED, L.SPAND_CPQR, L.SPAND_OK),
                                   (L.SPAND_IN, L.SPAND_COLOURED, L.SPAND_CPQR, L.SPAND_OK),
                                   (L.SPAND_INS, L.SPAND_SIMULTANEOUS, L.SPAND_CPQR, L.SPAND_ERR_INVALID_ARG),
                                   (L.SPAND_IN, L.SPAND_COLOURED, L.SPAND_RANDOMIZED, L.SPAND_ERR_INVALID_ARG),
                                   (3, L.SPAND_COLOURED, L.SPAND_CPQR, L.SPAND_ERR_INVALID_ARG),
                                   (-1, L.SPAND_COLOURED, L.SPAND_CPQR, L.SPAND_ERR_INVALID_ARG)]:
        o = L.default_opts(levels=3, variant=var, sparsify_order=order, compression=comp)
        h = C.c_void_p()
        rc = L.lib().spand_analyze(p.n, p.rowptr.ctypes.data, p.colind.ctypes.data, p.vals.ctypes.data, None, 0,
                                   C.byref(o), C.byref(h))
        if h.value:
            L.spand_destroy(h.value)
        assert rc == want, (var, order, comp, rc)
