"""GPU parity of the Boolean operations and the thick shell (dexel_boolean, dexel_shell)
against the oracle.  The Boolean kernels do no arithmetic on heights, so their results must
equal the oracle's bit for bit in both precisions; the shell carries the offsets' tolerances
(FP64 1e-10, FP32 endpoints 4e-6)."""
import numpy as np
import pytest

import oracle
from synth import shapes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dx():
    import torch  # noqa: F401
    import paper_1804_08968_gb300 as m
    return m


def _dev(dx, g, f32):
    import torch
    return dx.Grid.from_synth(g, dtype=torch.float32 if f32 else torch.float64)


def _exact(off, z, ref, what):
    assert np.array_equal(np.asarray(off, np.int64), np.asarray(ref.col_off, np.int64)), what
    assert np.array_equal(np.asarray(z, np.float64).reshape(-1, 2),
                          np.asarray(ref.z, np.float64).reshape(-1, 2)), what


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_boolean_random(dx, seed, f32):
    rng = np.random.default_rng(500 + seed)
    nx, ny = int(rng.integers(1, 60)), int(rng.integers(1, 60))
    a = shapes.random_grid(rng, nx, ny, 7, fill=0.7, point_frac=0.1, h=1 / 32,
                           dtype=np.float32 if f32 else np.float64)
    b = shapes.random_grid(rng, nx, ny, 7, fill=0.7, point_frac=0.1, h=1 / 32,
                           dtype=np.float32 if f32 else np.float64)
    da, db = _dev(dx, a, f32), _dev(dx, b, f32)
    for op, ref in ((dx.UNION, oracle.union(a, b)), (dx.INTERSECT, oracle.intersection(a, b)),
                    (dx.DIFFERENCE, oracle.difference(a, b)), (dx.DIFFERENCE, None)):
        if ref is None:  # b minus a as well
            ref = oracle.difference(b, a)
            out = dx.boolean(op, db, da)
        else:
            out = dx.boolean(op, da, db)
        off, z = out.to_host()
        _exact(off, z, ref, f"boolean op={op} seed={seed} f32={f32}")


def test_boolean_shapes_and_edges(dx):
    """Boxes and spheres ray-cast at 256 x 256; empty grids; a 1 x 1 grid; size mismatch."""
    a = shapes.raycast(shapes.grid512_prims(60, seed=3), 256)
    b = shapes.raycast(shapes.grid512_prims(60, seed=4), 256)
    da, db = _dev(dx, a, False), _dev(dx, b, False)
    for op, fn in ((dx.UNION, oracle.union), (dx.INTERSECT, oracle.intersection),
                   (dx.DIFFERENCE, oracle.difference)):
        off, z = dx.boolean(op, da, db).to_host()
        _exact(off, z, fn(a, b), f"shapes op={op}")
    e = shapes.from_columns(256, 256, 1 / 256, {})
    de = _dev(dx, e, False)
    off, z = dx.boolean(dx.UNION, de, de).to_host()
    assert off[-1] == 0
    off, z = dx.boolean(dx.DIFFERENCE, da, de).to_host()
    _exact(off, z, oracle.difference(a, e), "minus empty")
    one_a = shapes.from_columns(1, 1, 0.5, {(0, 0): [(0.1, 0.4), (0.6, 0.6)]})
    one_b = shapes.from_columns(1, 1, 0.5, {(0, 0): [(0.3, 0.7)]})
    for op, fn in ((dx.UNION, oracle.union), (dx.INTERSECT, oracle.intersection),
                   (dx.DIFFERENCE, oracle.difference)):
        off, z = dx.boolean(op, _dev(dx, one_a, False), _dev(dx, one_b, False)).to_host()
        _exact(off, z, fn(one_a, one_b), f"1x1 op={op}")
    small = _dev(dx, shapes.from_columns(4, 4, 0.25, {}), False)
    with pytest.raises(ValueError):
        dx.boolean(dx.UNION, da, small)


@pytest.mark.parametrize("f32", [False, True])
def test_shell(dx, f32):
    """Shell = dilation minus erosion, every column against the oracle's composite."""
    import torch
    rng = np.random.default_rng(77)
    cases = [(shapes.grid64(), 4.0), (shapes.raycast(shapes.grid512_prims(50, seed=8), 96), 3.7),
             (shapes.random_grid(rng, 30, 41, 5, fill=0.8, point_frac=0.05, h=1 / 64), 6.5)]
    for g, k in cases:
        if f32:
            g = shapes.to_float32(g)
        out = dx.shell(_dev(dx, g, f32), k)
        off, z = out.to_host()
        ref = oracle.shell(g, k)
        rc, gc = np.diff(ref.col_off), np.diff(off)
        same = rc == gc
        if f32:
            # a count may differ only where the oracle's gap is below one float ulp
            for c in np.flatnonzero(~same):
                segs = ref.z[ref.col_off[c]:ref.col_off[c + 1]]
                gaps = segs[1:, 0] - segs[:-1, 1]
                assert gaps.size and np.min(gaps / np.maximum(np.abs(segs[1:, 0]), 1.0)) < 2.0 ** -23
        else:
            assert same.all()
        zg = np.asarray(z, np.float64).reshape(-1, 2)[np.repeat(same, gc)]
        zr = np.asarray(ref.z, np.float64).reshape(-1, 2)[np.repeat(same, rc)]
        if zr.size:
            assert np.max(np.abs(zg - zr)) <= (4e-6 if f32 else 1e-10)
