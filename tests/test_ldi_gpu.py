"""GPU parity of the three-view layered depth image: ray casting along x and y
(dexel_raycast_axis) bit for bit against the oracle, and the offset of the three views
(dexel_offset_ldi) against the oracle's offset of each view (FP64 1e-10)."""
import numpy as np
import pytest

import oracle
from synth import shapes

pytestmark = pytest.mark.gpu


def _cmp(off, z, ref, what, tol=1e-10):
    assert np.array_equal(np.asarray(off, np.int64), np.asarray(ref.col_off, np.int64)), what
    if ref.z.size:
        assert np.max(np.abs(np.asarray(z, np.float64) - ref.z)) <= tol, what


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_raycast_axis(axis):
    import paper_1804_08968_gb300 as dx
    prims = shapes.grid512_prims(120, seed=12)
    n, m = 256, 200
    g = dx.raycast(prims, n, m, 1 / 256, axis=axis)
    off, z = g.to_host()
    ref = oracle.raycast_axis(prims, axis, n, m, 1 / 256)
    assert np.array_equal(off, ref.col_off) and np.array_equal(z, ref.z)


@pytest.mark.parametrize("op", ["dilate", "close"])
def test_offset_ldi(op):
    import paper_1804_08968_gb300 as dx
    prims = shapes.grid512_prims(40, seed=14)
    n = 160 if op == "dilate" else 96
    h = 1.0 / n
    views = [dx.raycast(prims, n, n, h, axis=a) for a in (2, 0, 1)]
    ctx = dx.Context(0)
    k = 6.0 if op == "dilate" else 3.0
    outs = ctx.offset_ldi(dx.DILATE if op == "dilate" else dx.CLOSE, views, k)
    for a, v, o in zip((2, 0, 1), views, outs):
        host = oracle.raycast_axis(prims, a, n, n, h)
        ref = oracle.dilate(host, k) if op == "dilate" else oracle.close(host, k)
        off, z = o.to_host()
        _cmp(off, z, ref, f"ldi {op} view along axis {a}")
