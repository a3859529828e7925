"""GPU parity at the sizes the benchmark times: the 2048 x 2048 grid of 1000 primitives
(nested hollow spheres, thin plates, spheres, boxes, shells; up to 58 segments a column),
offset by k = 64 spacings, in the launch configuration the benchmark uses (one call through
the C ABI, library-owned scratch).  The oracle computes sampled output columns one by one:
2000 random ones, one full row and one full column, compared element by element with the
tolerances of the small-grid tests (FP64 1e-10, FP32 endpoints 4e-6, counts identical except
where the oracle's gap is below the mode's threshold).  These sizes take the paths the small
grids do not reach: the 16384-event pass-1 tiles of the densest windows and the gather
buckets learnt for a 129-column window.
"""
import numpy as np
import pytest

import oracle
from synth import shapes

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 4e-6
GAP64 = 1e-9
K = 64.0


@pytest.fixture(scope="module")
def grids():
    g64 = shapes.grid2048()
    return {"fp64": g64, "fp32": shapes.to_float32(g64)}


def _cols(n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.choice(n * n, 2000, replace=False),
                                     np.arange(n) + 777 * n, np.arange(n) * n + 1301]))


def _check(off, z, ref, cols, f32, what):
    tol = TOL32 if f32 else TOL64
    for t, c in enumerate(cols):
        got = np.asarray(z[off[c]:off[c + 1]], np.float64)
        exp = ref.column(t)
        if got.shape != exp.shape:
            gaps = exp[1:, 0] - exp[:-1, 1]
            if f32:
                scale = np.maximum(np.maximum(np.abs(exp[1:, 0]), np.abs(exp[:-1, 1])), 1.0)
                ok = gaps.size > 0 and np.min(gaps / scale) < 2.0 ** -23
            else:
                ok = gaps.size > 0 and np.min(gaps) < GAP64
            assert ok, f"{what}: count mismatch at column {c}: {got.shape} vs {exp.shape}"
            continue
        if exp.size:
            err = float(np.max(np.abs(got - exp)))
            assert err <= tol, f"{what}: column {c} endpoint error {err}"


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_2048_k64_sampled(grids, mode, op):
    import torch
    import paper_1804_08968_gb300 as dx
    g = grids[mode]
    f32 = mode == "fp32"
    dg = dx.Grid.from_synth(g, dtype=torch.float32 if f32 else torch.float64)
    ctx = dx.Context(0)
    out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, K)
    torch.cuda.synchronize()
    st = ctx.stats()
    off, z = out.to_host()
    del out, dg
    torch.cuda.empty_cache()
    cols = _cols(g.nx, 5 if op == "dilate" else 6)
    if op == "erode":
        cols = cols[::3]  # the erosion oracle is the slower one
    ref = (oracle.dilate if op == "dilate" else oracle.erode)(g, K, cols=cols)
    _check(off, z, ref, cols, f32, f"2048^2 k=64 {op} {mode}")
    assert st[0] == g.nseg and st[3] == off[-1]


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_blocks_of_lines(op, monkeypatch):
    """An offset split into blocks of whole y lines (a small block budget forces ten or so):
    S_mid and the level lists exist for one block at a time, the result is unchanged."""
    import torch
    import paper_1804_08968_gb300 as dx
    monkeypatch.setenv("DEXEL_BLOCK_MB", "1")
    rng = np.random.default_rng(71)
    g = shapes.random_grid(rng, 300, 70, 6, fill=0.75, point_frac=0.05, h=1 / 256)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    for k in (5.5, 12.0, 40.0):
        out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
        off, z = out.to_host()
        assert ctx.stats()[9] > 1, "the offset was not split into blocks"
        ref = (oracle.dilate if op == "dilate" else oracle.erode)(g, k)
        cols = np.arange(g.nx * g.ny)
        _check(off, z, _Full(ref), cols, False, f"blocks {op} k={k}")


class _Full:
    """A full oracle grid seen through the sampled-column interface."""

    def __init__(self, g):
        self.g = g

    def column(self, t):
        return self.g.z[self.g.col_off[t]:self.g.col_off[t + 1]]


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_reach_128(op):
    """k = 128 spacings (reach 128, the lane kernel's widest source masks), on a grid long
    enough in x for full windows; FP64 against the oracle."""
    import torch
    import paper_1804_08968_gb300 as dx
    prims = shapes.grid512_prims(60, seed=13)
    big = shapes.raycast(prims, 320)
    cols = {(i, j): [tuple(s) for s in big.column(i, j + 150)]
            for i in range(320) for j in range(16) if big.column(i, j + 150).size}
    g = shapes.from_columns(320, 16, 1 / 8000, cols)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    k = 128.4
    out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
    off, z = out.to_host()
    ref = (oracle.dilate if op == "dilate" else oracle.erode)(g, k)
    _check(off, z, _Full(ref), np.arange(g.nx * g.ny), False, f"reach 128 {op}")


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
@pytest.mark.parametrize("op", ["close", "open"])
def test_morphology_blocks_reduced(mode, op, monkeypatch):
    """Closing and opening of the 4096^2 workload's kind of shape (spheres, boxes, hollow
    shells) at reduced scale, 384 x 384 at k = 12, every column against the oracle's
    composite (erosion of the dilation, dilation of the erosion), with both stages split into
    blocks of y lines."""
    import torch
    import paper_1804_08968_gb300 as dx
    monkeypatch.setenv("DEXEL_BLOCK_MB", "4")
    g = shapes.raycast(shapes.grid4096_prims(nprim=60, seed=21), 384)
    f32 = mode == "fp32"
    if f32:
        g = shapes.to_float32(g)
    dg = dx.Grid.from_synth(g, dtype=torch.float32 if f32 else torch.float64)
    ctx = dx.Context(0)
    k = 12.0
    out = ctx.run(dx.CLOSE if op == "close" else dx.OPEN, dg, k)
    off, z = out.to_host()
    assert ctx.stats()[9] > 1, "the offsets were not split into blocks"
    ref = oracle.close(g, k) if op == "close" else oracle.open_(g, k)
    _check(off, z, _Full(ref), np.arange(g.nx * g.ny), f32, f"{op} 384^2 k=12 {mode}")


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_gather_collapse(op, monkeypatch):
    """Windows whose level lists hold more intervals than the gather's bucket (kept at 256):
    81 lists of 6-7 intervals a column, united into their runs part way; the result is still
    the oracle's."""
    import torch
    import paper_1804_08968_gb300 as dx
    monkeypatch.setenv("DEXEL_GATHER_BUCKET_MAX", "256")
    rng = np.random.default_rng(91)
    cols = {}
    for i in range(24):
        for j in range(96):
            ph = float(rng.uniform(0.0, 0.01))
            cols[(i, j)] = [(0.2 + q * 0.1 + ph, 0.25 + q * 0.1 + ph) for q in range(6)]
    g = shapes.from_columns(24, 96, 1 / 8192, cols)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    for k in (40.0, 33.3):
        for _ in range(2):  # the second call keeps the 256-interval bucket
            out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
        off, z = out.to_host()
        st = ctx.stats()
        assert st[12] <= 256 and st[11] > 0, st  # columns united part way
        ref = (oracle.dilate if op == "dilate" else oracle.erode)(g, k)
        _check(off, z, _Full(ref), np.arange(g.nx * g.ny), False, f"collapse {op} k={k}")
