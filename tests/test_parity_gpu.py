"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances, in units of the depth extent Z = 1: FP64 endpoints within 1e-10, FP32-endpoint
mode within 4e-6.  Segment counts are identical column by column, with one excuse each:
  * FP64: a column whose oracle result has a gap below 1e-9 Z (two runs the method may
    legitimately join at that resolution);
  * FP32: a column whose oracle result has a gap below one float32 ulp of its ends
    (2^-23 max(|z|, 1)): rounding each end once to float moves a gap by up to one ulp, and
    runs that touch after rounding are merged, so such a gap cannot survive in float32.
Every column whose count matches has its endpoints compared, whatever happens elsewhere.
"""
import math

import numpy as np
import pytest

import oracle
from synth import shapes

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 4e-6


@pytest.fixture(scope="module")
def dx():
    import torch  # noqa: F401
    import paper_1804_08968_gb300 as m
    return m


def _gpu(dx, g, op, k, f32=False):
    import torch
    gg = shapes.to_float32(g) if f32 else g
    dg = dx.Grid.from_synth(gg, dtype=torch.float32 if f32 else torch.float64)
    fn = {"dilate": dx.dilate, "erode": dx.erode, "close": dx.close, "open": dx.open_}[op]
    out = fn(dg, k)
    torch.cuda.synchronize()
    off, z = out.to_host()
    return gg, off, z.astype(np.float64)


def _ref(g, op, k, cols=None):
    if op == "dilate":
        return oracle.dilate(g, k, cols=cols)
    if op == "erode":
        return oracle.erode(g, k, cols=cols)
    if op == "close":
        return oracle.close(g, k)
    return oracle.open_(g, k)


GAP64 = 1e-9


def _excused(ref, c, f32):
    """True when the oracle's column c has a gap below the mode's threshold."""
    segs = ref.z[ref.col_off[c]:ref.col_off[c + 1]]
    if segs.shape[0] < 2:
        return False
    gaps = segs[1:, 0] - segs[:-1, 1]
    if f32:
        scale = np.maximum(np.maximum(np.abs(segs[1:, 0]), np.abs(segs[:-1, 1])), 1.0)
        return bool(np.min(gaps / scale) < 2.0 ** -23)
    return bool(np.min(gaps) < GAP64)


def _compare_full(off, z, ref, f32, what):
    """Counts per column (with the excuse above), then the endpoints of every column whose
    count matches."""
    off = np.asarray(off, np.int64)
    rc = np.diff(ref.col_off)
    gc = np.diff(off)
    bad = np.flatnonzero(rc != gc)
    unexcused = [int(c) for c in bad if not _excused(ref, c, f32)]
    assert not unexcused, f"{what}: count mismatch at columns {unexcused[:8]}"
    same = rc == gc
    if not same.any():
        return
    # segments of the matching columns, in the same order on both sides
    sel_g = np.repeat(same, gc)
    sel_r = np.repeat(same, rc)
    zg = np.asarray(z, np.float64).reshape(-1, 2)[sel_g]
    zr = np.asarray(ref.z, np.float64).reshape(-1, 2)[sel_r]
    assert zg.shape == zr.shape, what
    if zg.size:
        err = float(np.max(np.abs(zg - zr)))
        assert err <= (TOL32 if f32 else TOL64), f"{what}: max endpoint error {err}"


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_random_small(dx, seed, op):
    rng = np.random.default_rng(1000 + seed)
    nx, ny = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    g = shapes.random_grid(rng, nx, ny, 5, fill=0.7, point_frac=0.05, h=1 / 32)
    for k in [0.0, 0.5, 1.0, math.sqrt(2.0), 2.0, 3.7, 7.0, 12.5]:
        gg, off, z = _gpu(dx, g, op, k)
        _compare_full(off, z, _ref(gg, op, k), False, f"{op} seed={seed} k={k} {nx}x{ny}")


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_random_fp32(dx, op):
    rng = np.random.default_rng(77)
    g = shapes.random_grid(rng, 37, 29, 6, fill=0.8, point_frac=0.05, h=1 / 40)
    for k in [1.0, 4.2, 9.0]:
        gg, off, z = _gpu(dx, g, op, k, f32=True)
        _compare_full(off, z, _ref(gg, op, k), True, f"fp32 {op} k={k}")


def test_grid64_dilation(dx):
    """64 x 64, 8 spheres, k = 4, FP64 (the smallest workload)."""
    g = shapes.grid64()
    gg, off, z = _gpu(dx, g, "dilate", 4.0)
    _compare_full(off, z, _ref(gg, "dilate", 4.0), False, "grid64")


@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("k", [2.0, 8.0])
def test_grid512_full(dx, op, k):
    """512 x 512, 200 primitives: every column compared with the oracle."""
    g = shapes.grid512()
    gg, off, z = _gpu(dx, g, op, k)
    _compare_full(off, z, _ref(gg, op, k), False, f"grid512 {op} k={k}")


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_grid512_k32_sampled(dx, op):
    """k = 32 at 512 x 512: 3000 sampled columns plus two full lines against the oracle."""
    g = shapes.grid512()
    k = 32.0
    gg, off, z = _gpu(dx, g, op, k)
    rng = np.random.default_rng(5)
    cols = np.concatenate([rng.choice(512 * 512, 3000, replace=False),
                           np.arange(512) + 200 * 512, np.arange(512) * 512 + 300])
    ref = _ref(gg, op, k, cols=cols)
    for t, c in enumerate(cols):
        got = z[off[c]:off[c + 1]]
        exp = ref.column(t)
        assert got.shape == exp.shape, (op, c, got, exp)
        if exp.size:
            assert np.max(np.abs(got - exp)) <= TOL64


@pytest.mark.parametrize("op", ["close", "open"])
def test_morphology_small(dx, op):
    g = shapes.raycast(shapes.grid512_prims(80, seed=3), 96)
    for k in [2.0, 5.0]:
        gg, off, z = _gpu(dx, g, op, k)
        _compare_full(off, z, _ref(gg, op, k), False, f"{op} k={k}")


def test_edge_cases(dx):
    # empty grid
    g = shapes.from_columns(7, 5, 0.1, {})
    for op in ("dilate", "erode"):
        gg, off, z = _gpu(dx, g, op, 2.0)
        assert off[-1] == 0
    # single column, single segment; a 1 x n and n x 1 grid
    for (nx, ny, i, j) in [(1, 1, 0, 0), (1, 9, 0, 4), (9, 1, 4, 0)]:
        g = shapes.from_columns(nx, ny, 1 / 16, {(i, j): [(0.25, 0.5)]})
        for op in ("dilate", "erode"):
            for k in (0.0, 1.0, 3.0):
                gg, off, z = _gpu(dx, g, op, k)
                _compare_full(off, z, _ref(gg, op, k), False, f"edge {nx}x{ny} {op} {k}")
    # zero-length segments only
    g = shapes.from_columns(6, 6, 1 / 8, {(2, 2): [(0.5, 0.5)], (3, 3): [(0.25, 0.25), (0.5, 0.5)]})
    for k in (0.0, 1.0, 2.5):
        gg, off, z = _gpu(dx, g, "dilate", k)
        _compare_full(off, z, _ref(gg, "dilate", k), False, f"points k={k}")


def test_bad_csr_rejected(dx):
    import torch
    g = shapes.from_columns(4, 4, 0.25, {(1, 1): [(0.2, 0.4), (0.3, 0.6)]})  # overlapping
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    with pytest.raises(dx.DexelError) as e:
        dx.dilate(dg, 1.0)
    assert e.value.code == -2
    assert dx._default_ctx(dg).validate(dg) == -2


def test_output_capacity_retry(dx):
    """A too-small output buffer reports the needed size; the binding retries."""
    import torch
    g = shapes.grid64()
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    out = ctx.run(dx.DILATE, dg, 4.0, capacity=3)
    ref = oracle.dilate(g, 4.0)
    assert out.nseg == ref.nseg


def _stack_column(n, lo, hi, gap_frac):
    """n equal segments in [lo, hi] separated by gaps of gap_frac of the pitch."""
    pitch = (hi - lo) / n
    return [(lo + q * pitch, lo + q * pitch + pitch * (1 - gap_frac)) for q in range(n)]


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_dense_windows_chunked(dx, op):
    """Windows holding more pieces than one staging area (a band of columns with 2500 close
    segments each): the tiled kernel covers such a column in several chunks."""
    cols = {(i, j): _stack_column(2500, 0.1, 0.9, 0.3) for i in range(6, 9) for j in range(0, 16)}
    g = shapes.from_columns(16, 16, 1 / 16, cols)
    for k in (3.0, 6.5):
        gg, off, z = _gpu(dx, g, op, k)
        _compare_full(off, z, _ref(gg, op, k), False, f"dense {op} k={k}")


def _runs_grid(op, n, nx, h, gap):
    """Many disjoint runs in the result: for dilation a 3 x 3 block of columns of n thin
    segments; for erosion every column holds n thick segments, so the dilated complement
    keeps n runs."""
    c = nx // 2
    if op == "dilate":
        cols = {(i, j): _stack_column(n, 0.05, 0.95, gap) for i in range(c - 1, c + 2)
                for j in range(c - 1, c + 2)}
    else:
        cols = {(i, j): _stack_column(n, 0.05, 0.95, 1 - gap) for i in range(nx) for j in range(nx)}
    return shapes.from_columns(nx, nx, h, cols)


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_many_runs_redo(dx, op):
    """Output columns with ~700 disjoint runs, whose windows take several rounds: the union
    outgrows the round bucket, the columns go to the second gather kernel (k_pass2c), and the
    result is still exact."""
    import torch
    g = _runs_grid(op, 700, 8, 1 / 4096, 0.8)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    k = 1.0
    out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
    off, z = out.to_host()
    ref = _ref(g, op, k)
    assert np.diff(ref.col_off).max() > 600
    _compare_full(off, z.astype(np.float64), ref, False, f"runs {op} k={k}")
    assert ctx.stats()[5] > 0  # some columns were redone


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_per_line_sweep_path(dx, op, monkeypatch):
    """The per-line sweep (used when a column's union outgrows every gather bucket, or on
    request) against the oracle, and a case that needs it: 3000 runs in a column."""
    import torch
    monkeypatch.setenv("DEXEL_PASS2", "sweep")
    rng = np.random.default_rng(11)
    g = shapes.random_grid(rng, 23, 31, 6, fill=0.8, point_frac=0.05, h=1 / 32)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    for k in (1.0, 3.7, 9.0):
        out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
        off, z = out.to_host()
        _compare_full(off, z.astype(np.float64), _ref(g, op, k), False, f"sweep {op} k={k}")
    monkeypatch.delenv("DEXEL_PASS2")
    g = _runs_grid(op, 3000, 6, 1 / 32768, 0.8)
    gg, off, z = _gpu(dx, g, op, 1.0)
    ref = _ref(gg, op, 1.0)
    assert np.diff(ref.col_off).max() > 2500
    _compare_full(off, z, ref, False, f"3000 runs {op}")


@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("k", [40.0, 90.5])
def test_wide_reach(dx, op, k):
    """Reaches beyond 31 and 63 spacings (pass-1 source masks of two and four words), on a
    grid long enough in x for the windows to be full; the xy spacing is small against the
    depth (h = 1/4000) so that the results keep their gaps."""
    if op == "dilate":
        prims = shapes.grid512_prims(40, seed=9)
        g = shapes.raycast(prims, 200)
        cols = {(i, j): [tuple(s) for s in g.column(i, j + 88)]
                for i in range(200) for j in range(24) if g.column(i, j + 88).size}
    else:
        # a solid slab with holes of several depths in a few patches of columns
        rng = np.random.default_rng(4)
        holes = [(int(rng.integers(0, 200)), int(rng.integers(0, 24)), int(rng.integers(2, 12)),
                  float(rng.uniform(0.2, 0.7))) for _ in range(10)]
        cols = {}
        for i in range(200):
            for j in range(24):
                zs = [0.1, 0.9]
                for (hi, hj, hr, hz) in holes:
                    if (i - hi) ** 2 + (j - hj) ** 2 <= hr * hr:
                        zs = [0.1, hz, hz + 0.05, 0.9]
                        break
                cols[(i, j)] = [(zs[q], zs[q + 1]) for q in range(0, len(zs), 2)]
    sub = shapes.from_columns(200, 24, 1 / 4000, cols)
    gg, off, z = _gpu(dx, sub, op, k)
    _compare_full(off, z, _ref(gg, op, k), False, f"wide {op} k={k}")


@pytest.mark.parametrize("gw", ["1", "2", "4", "8"])
def test_pass1_lane_groups(dx, gw, monkeypatch):
    """The pass-1 window kernel with every warp-group size (chunked walks of 1 to 8 warps),
    and with a small event room (256 events a tile) that splits tiles into narrower runs of
    columns and hands the densest columns' rows to the sweep."""
    import torch
    rng = np.random.default_rng(31)
    g = shapes.random_grid(rng, 45, 37, 12, fill=0.7, point_frac=0.05, h=1 / 64)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    monkeypatch.setenv("DEXEL_PASS1", "lane")  # also at the short reaches (not the merge)
    for ecap in (None, "256"):
        monkeypatch.setenv("DEXEL_PASS1_GW", gw)
        if ecap:
            monkeypatch.setenv("DEXEL_PASS1_ECAP", ecap)
        ctx = dx.Context(0)
        for op in ("dilate", "erode"):
            for k in (1.0, 4.5, 9.0):
                out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
                off, z = out.to_host()
                _compare_full(off, z.astype(np.float64), _ref(g, op, k), False,
                              f"gw={gw} ecap={ecap} {op} k={k}")
        monkeypatch.delenv("DEXEL_PASS1_ECAP", raising=False)


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_pass1_gather_variant(dx, op, monkeypatch):
    """The per-column pass-1 kernel (DEXEL_PASS1=gather) against the oracle."""
    import torch
    monkeypatch.setenv("DEXEL_PASS1", "gather")
    rng = np.random.default_rng(32)
    g = shapes.random_grid(rng, 29, 41, 8, fill=0.75, point_frac=0.05, h=1 / 48)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    for k in (1.0, 3.7, 12.0):
        out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
        off, z = out.to_host()
        _compare_full(off, z.astype(np.float64), _ref(g, op, k), False, f"gather {op} k={k}")


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_pass1_ring_spill(dx, op, monkeypatch):
    """Ring regions of 16 pieces (DEXEL_PASS1_RING_CAP): lanes of dense columns outgrow them,
    their tiles are walked again straight into the arena, and the result is unchanged."""
    import torch
    monkeypatch.setenv("DEXEL_PASS1", "lane")
    monkeypatch.setenv("DEXEL_PASS1_RING_CAP", "16")
    rng = np.random.default_rng(33)
    g = shapes.random_grid(rng, 41, 35, 12, fill=0.8, point_frac=0.05, h=1 / 64)
    dg = dx.Grid.from_synth(g, dtype=torch.float64)
    ctx = dx.Context(0)
    for k in (2.5, 9.0, 20.0):
        out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
        off, z = out.to_host()
        ref = _ref(g, op, k)
        assert ctx.stats()[4] > 16  # some column has more pieces than a region holds
        _compare_full(off, z.astype(np.float64), ref, False, f"ring 16 {op} k={k}")


@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_levels_exact_reads(dx, op, monkeypatch):
    """Level walks at reach >= 32 reading S_mid itself (DEXEL_LEVELS_EXACT=1, no packed float
    copy) against the oracle, FP64 and FP32 endpoints."""
    import torch
    monkeypatch.setenv("DEXEL_LEVELS_EXACT", "1")
    rng = np.random.default_rng(41)
    g = shapes.random_grid(rng, 90, 80, 4, fill=0.6, point_frac=0.05, h=1 / 512)
    for f32 in (False, True):
        gg = shapes.to_float32(g) if f32 else g
        dg = dx.Grid.from_synth(gg, dtype=torch.float32 if f32 else torch.float64)
        ctx = dx.Context(0)
        for k in (32.0, 40.5):
            out = ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, dg, k)
            off, z = out.to_host()
            _compare_full(off, z.astype(np.float64), _ref(gg, op, k), f32,
                          f"levels exact {op} k={k} f32={f32}")
