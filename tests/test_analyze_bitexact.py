"""Host analysis (C++, in libspand.so) against the oracle's independent
implementation of Algorithm 3 and the per-step symbolic structure: every
integer output must match bit for bit."""
import numpy as np
import pytest

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import _lib as L
from paper_1901_02971_gb300 import inputs as I


def _compare(p, levels, geo=True):
    coords = p.coords if geo else None
    ref = O.flat_tree(O.analyze(p.n, p.rowptr, p.colind, coords, levels))
    h = L.spand_analyze(p.rowptr, p.colind, p.vals, coords, L.default_opts(levels=levels))
    try:
        got = L.spand_get_tree(h)
        for k in ("perm", "cluster_ptr", "keys"):
            assert np.array_equal(got[k], ref[k]), k
        assert got["n_steps"] == levels
        for t in range(1, levels + 1):
            gs = L.spand_get_step(h, t)
            rs = ref[f"step{t}"]
            for k in rs:
                assert np.array_equal(gs[k], rs[k]), (t, k)
    finally:
        L.spand_destroy(h)


def _empty():
    """The empty system (n = 0): no clusters, every step empty."""
    return I.Problem("empty", 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros((0, 2)), 2)


def _path_plus_isolated():
    """1 - 0 - 2 and an isolated vertex 3 (the BFS tie-break and unreached-
    vertex case of the oracle pins)."""
    rowptr = np.array([0, 3, 5, 7, 8], np.int64)
    colind = np.array([0, 1, 2, 0, 1, 0, 2, 3], np.int32)
    vals = np.array([3.0, -1, -1, -1, 2, -1, 2, 1])
    return I.Problem("path_iso", 4, rowptr, colind, vals, None, 1)


CASES = [
    ("bfs_path_iso_L2", lambda: _path_plus_isolated(), 2, False),
    ("bfs_path_iso_L3", lambda: _path_plus_isolated(), 3, False),
    ("bfs_grid_4x3_L2", lambda: I._assemble((3, 4), np.ones((3, 4)), "grid_4x3"), 2, False),
    ("lapl2d_8_L3", lambda: I.laplacian_2d(8), 3, True),
    ("lapl2d_64_L8", lambda: I.laplacian_2d(64), 8, True),
    ("lapl2d_37_L6", lambda: I.laplacian_2d(37), 6, True),
    ("lapl2d_5_L7", lambda: I.laplacian_2d(5), 7, True),
    ("lapl3d_16_L6", lambda: I.laplacian_3d(16), 6, True),
    ("diff3d_12_L5", lambda: I.diffusion_3d(12, 2, block=3), 5, True),
    ("diff2d_30_L6_nogeo", lambda: I.diffusion_2d(30, 4), 6, False),
    ("knn_3000_L7", lambda: I.knn_laplacian(3000, 10, 3), 7, False),
    ("empty_L3", lambda: _empty(), 3, True),
    ("lapl2d_1_L1", lambda: I.laplacian_2d(1), 1, True),
    ("lapl2d_2_L3", lambda: I.laplacian_2d(2), 3, True),
    # extruded thin 3D mesh, partitioned with its (x, y) coordinates only
    ("extr_24x20x4_L6", lambda: I.extruded_3d(24, 20, 4, 1), 6, True),
    ("extr_33x17x3_L7", lambda: I.extruded_3d(33, 17, 3, 2), 7, True),
]


@pytest.mark.parametrize("name,gen,levels,geo", CASES, ids=[c[0] for c in CASES])
def test_analyze_bitexact(spand_lib, name, gen, levels, geo):
    _compare(gen(), levels, geo)


@pytest.mark.slow
def test_analyze_bitexact_3d_64(spand_lib):
    """The benchmark workload itself: 7-point Laplacian on 64^3, L = 10."""
    _compare(I.laplacian_3d(64), 10, True)


def test_extruded_partition_keeps_columns_whole(spand_lib):
    """With (x, y) coordinates the separators are vertical: every column of
    cells (same x, y, all z) lies in one cluster."""
    p = I.extruded_3d(40, 28, 5, 3)
    h = L.spand_analyze(p.rowptr, p.colind, p.vals, p.coords, L.default_opts(levels=7))
    try:
        t = L.spand_get_tree(h)
        cl = np.empty(p.n, dtype=np.int64)
        ptr = np.asarray(t["cluster_ptr"])
        for c in range(len(ptr) - 1):
            cl[np.asarray(t["perm"])[ptr[c]:ptr[c + 1]]] = c
        col = cl.reshape(5, 28 * 40)
        assert np.all(col == col[0]), "a column is split between clusters"
    finally:
        L.spand_destroy(h)
