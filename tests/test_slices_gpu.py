"""GPU parity of the 2D slice offsets (dexel_offset_slices: every row a 2D dexel image offset
by a disk, Sec. 3.2) against the oracle, FP64 at 1e-10 and FP32 endpoints at 4e-6, with
counts identical (FP32: except where the oracle's gap is below one float ulp)."""
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


def _cmp(off, z, ref, f32, what):
    rc, gc = np.diff(ref.col_off), np.diff(np.asarray(off, np.int64))
    same = rc == gc
    for c in np.flatnonzero(~same):
        segs = ref.z[ref.col_off[c]:ref.col_off[c + 1]]
        gaps = segs[1:, 0] - segs[:-1, 1]
        if f32:
            scale = np.maximum(np.abs(segs[1:, 0]), 1.0)
            assert gaps.size and np.min(gaps / scale) < 2.0 ** -23, f"{what}: count at {c}"
        else:
            assert gaps.size and np.min(gaps) < 1e-9, f"{what}: count at {c}"
    zg = np.asarray(z, np.float64).reshape(-1, 2)[np.repeat(same, gc)]
    zr = np.asarray(ref.z, np.float64).reshape(-1, 2)[np.repeat(same, rc)]
    if zr.size:
        err = float(np.max(np.abs(zg - zr)))
        assert err <= (4e-6 if f32 else 1e-10), f"{what}: error {err}"


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("seed", range(3))
def test_slices_random(dx, seed, f32):
    import torch
    rng = np.random.default_rng(700 + seed)
    nx, ny = int(rng.integers(1, 160)), int(rng.integers(1, 30))
    g = shapes.random_grid(rng, nx, ny, 6, fill=0.75, point_frac=0.05, h=1 / 128,
                           dtype=np.float32 if f32 else np.float64)
    dg = dx.Grid.from_synth(g, dtype=torch.float32 if f32 else torch.float64)
    for k in (0.0, 1.0, 2.5, 7.0, 40.5, 70.0):
        for op in ("dilate", "erode"):
            out = (dx.dilate_slices if op == "dilate" else dx.erode_slices)(dg, k)
            off, z = out.to_host()
            ref = (oracle.dilate_slices if op == "dilate" else oracle.erode_slices)(g, k)
            _cmp(off, z, ref, f32, f"slices {op} k={k} {nx}x{ny} f32={f32}")


def test_slices_shapes_and_rows(dx):
    """A 512 x 48 strip of the 512^2 workload at k = 32: against the oracle, and each row equal
    to the 3D offset of that row alone (a 1-row grid, where disk and ball coincide)."""
    import torch
    big = shapes.grid512()
    cols = {(i, j): [tuple(s) for s in big.column(i, j + 200)]
            for i in range(512) for j in range(48) if big.column(i, j + 200).size}
    g = shapes.from_columns(512, 48, big.h, cols)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    for op in (dx.DILATE, dx.ERODE):
        out = ctx.slices(op, dg, 32.0)
        off, z = out.to_host()
        ref = (oracle.dilate_slices if op == dx.DILATE else oracle.erode_slices)(g, 32.0)
        _cmp(off, z, ref, False, f"strip op={op}")
        for j in (0, 17, 47):
            c0, c1 = g.col_off[j * 512], g.col_off[(j + 1) * 512]
            row = shapes.DexelGrid(512, 1, g.h, g.col_off[j * 512:(j + 1) * 512 + 1] - c0, g.z[c0:c1])
            r3 = ctx.run(op, dx.Grid.from_synth(row, dtype=torch.float64), 32.0)
            o3, z3 = r3.to_host()
            assert np.array_equal(o3, off[j * 512:(j + 1) * 512 + 1] - off[j * 512])
            assert np.array_equal(z3, z[off[j * 512]:off[(j + 1) * 512]])
