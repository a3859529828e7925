"""GPU parity of the ray casting of analytic primitives (dexel_raycast) against the oracle's
caster: the same correctly rounded operations, so FP64 grids are identical bit for bit; FP32
grids equal the oracle's rounded to float with touching segments joined."""
import numpy as np
import pytest

import oracle
from synth import shapes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["grid64", "grid512", "grid2048", "thin", "empty"])
def test_raycast_matches_oracle(case):
    import torch
    import paper_1804_08968_gb300 as dx
    if case == "grid64":
        prims, nx, ny = shapes.grid64_prims(), 64, 64
    elif case == "grid512":
        prims, nx, ny = shapes.grid512_prims(), 512, 512
    elif case == "grid2048":
        prims, nx, ny = shapes.grid2048_prims(), 768, 768
    elif case == "thin":
        # a non-square grid, nested shells and boxes thinner than a spacing
        prims = [("shell", 0.5, 0.4, 0.5, 0.3 - 0.02 * q, 0.006) for q in range(12)]
        prims += [("box", 0.1, 0.9, 0.2, 0.21, 0.3, 0.7), ("box", 0.45, 0.46, 0.0, 1.0, 0.1, 0.9)]
        nx, ny = 300, 170
    else:
        prims, nx, ny = [], 17, 9
    h = 1.0 / max(nx, ny)
    ref = oracle.raycast(prims, nx, ny, h)
    g = dx.raycast(prims, nx, ny, h)
    off, z = g.to_host()
    assert np.array_equal(off, ref.col_off), case
    assert np.array_equal(z, ref.z), case
    g32 = dx.raycast(prims, nx, ny, h, dtype=torch.float32)
    off, z = g32.to_host()
    r32 = oracle.round_float32(ref)
    assert np.array_equal(off, r32.col_off), case
    assert np.array_equal(z, r32.z), case
