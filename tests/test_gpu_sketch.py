"""Device side of the counter-based Gaussian sketch (spand_sketch_gaussian,
the test matrix of the randomized compression) against the oracle's own
implementation of the same published generator (Philox4x64-10 + Box-Muller,
`oracle.spand_oracle.sketch_philox`): the same entries up to the rounding of
the transcendental functions (log, cos/sin against cospi/sinpi), for
several keys and shapes, including ragged row blocks (m not a multiple of 4)
and one-entry matrices."""
import numpy as np
import pytest

from oracle import spand_oracle as O
from paper_1901_02971_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,step,cluster,m,ell", [
    (0, 1, 0, 50, 20), (3, 2, 7, 1, 1), (12345678901234, 9, 4095, 1001, 37), (1, 3, 2, 7, 3),
    (2 ** 63 + 5, 1, 1, 4096, 64),
])
def test_device_sketch_matches_oracle(cuda_ok, seed, step, cluster, m, ell):
    import torch
    out = torch.full((ell, m), float("nan"), dtype=torch.float64, device="cuda")  # column-major m x ell
    L.spand_sketch_gaussian(seed, step, cluster, m, ell, out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy().T
    want = O.sketch_philox(seed, step, cluster, m, ell)
    assert np.isfinite(got).all()
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))
