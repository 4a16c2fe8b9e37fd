"""The differentiable coefficient assembly (paper_1901_02971_gb300.autograd.
CoefficientAssembly) against the problem generators: same stored values for
the 5- and 7-point variable-coefficient stencils (harmonic-mean faces,
Dirichlet boundary), and its derivative with respect to one cell
coefficient against central finite differences (no GPU needed)."""
import numpy as np
import pytest
import torch

from paper_1901_02971_gb300 import inputs as I
from paper_1901_02971_gb300.autograd import CoefficientAssembly


def _cells_2d(n, seed, sigma=1.0):
    return np.exp(sigma * I.rng(seed).standard_normal((n, n)))


def test_values_match_generator_2d():
    p = I.diffusion_2d(17, 5)
    asm = CoefficientAssembly((17, 17), p.rowptr, p.colind, device="cpu")
    v = asm(torch.from_numpy(_cells_2d(17, 5))).numpy()
    assert np.abs(v - p.vals).max() <= 1e-15 * np.abs(p.vals).max()


def test_values_match_generator_3d():
    p = I.diffusion_3d(6, 2, block=2)
    u = I.rng(2).uniform(-3, 3, size=(3, 3, 3))
    cell = np.repeat(np.repeat(np.repeat(10.0 ** u, 2, 0), 2, 1), 2, 2)
    asm = CoefficientAssembly((6, 6, 6), p.rowptr, p.colind, device="cpu")
    v = asm(torch.from_numpy(cell)).numpy()
    assert np.abs(v - p.vals).max() <= 1e-15 * np.abs(p.vals).max()


def test_rectangular_grid_and_wrong_pattern():
    cell = I.rng(1).random((5, 9)) + 0.5
    p = I._assemble((5, 9), cell, "r")
    asm = CoefficientAssembly((5, 9), p.rowptr, p.colind, device="cpu")
    assert np.allclose(asm(torch.from_numpy(cell)).numpy(), p.vals, rtol=1e-15, atol=0)
    with pytest.raises(ValueError):
        CoefficientAssembly((9, 5), p.rowptr, p.colind, device="cpu")


@pytest.mark.parametrize("cell_idx", [0, 37, 144])
def test_derivative_matches_finite_differences(cell_idx):
    n = 13
    p = I.diffusion_2d(n, 9)
    a0 = torch.from_numpy(_cells_2d(n, 9)).reshape(-1)
    asm = CoefficientAssembly((n, n), p.rowptr, p.colind, device="cpu")
    w = torch.from_numpy(I.rhs(p.nnz, 4))
    a = a0.clone().requires_grad_(True)
    (asm(a) * w).sum().backward()
    h = 1e-6 * float(a0[cell_idx])
    ap, am = a0.clone(), a0.clone()
    ap[cell_idx] += h
    am[cell_idx] -= h
    fd = float(((asm(ap) - asm(am)) * w).sum()) / (2 * h)
    assert abs(fd - float(a.grad[cell_idx])) <= 1e-7 * max(1.0, abs(fd))
