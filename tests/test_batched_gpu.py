"""GPU parity of the batched entry point (dexel_offset_batched) against the FP64 oracle.

Shapes of uneven size with their own radius and operation run in one batched call (one
launch per stage over all shapes); every shape's result is compared with the oracle with the
tolerances of the other parity tests.  Later calls with the same shapes replay the recorded
CUDA graph (through the output write); their results must be the same.
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


def _ref(g, op, k, f32=False):
    """The oracle; in FP32 mode the intermediate grid of a closing / opening is stored in
    float32 (rounded and re-merged), as the library stores it."""
    if op == "dilate":
        return oracle.dilate(g, k)
    if op == "erode":
        return oracle.erode(g, k)
    first, second = (oracle.dilate, oracle.erode) if op == "close" else (oracle.erode, oracle.dilate)
    mid = first(g, k)
    if f32:
        mid = shapes.to_float32(mid)
    return second(mid, k)


def _round_f32(ref, erode_last):
    """The FP32 output rule applied to an oracle grid: endpoints rounded once to float32,
    pieces that touch after rounding merged, and (when the last offset is an erosion) pieces
    of zero length after rounding dropped."""
    z32 = ref.z.astype(np.float32).astype(np.float64)
    off = [0]
    out = []
    for c in range(ref.nx * ref.ny):
        col = []
        for a, b in z32[ref.col_off[c]:ref.col_off[c + 1]]:
            if erode_last and not a < b:
                continue
            if col and a <= col[-1][1]:
                col[-1][1] = max(col[-1][1], b)
            else:
                col.append([a, b])
        out.extend(col)
        off.append(len(out))
    return shapes.DexelGrid(ref.nx, ref.ny, ref.h, np.asarray(off, np.int64),
                            np.asarray(out, np.float64).reshape(-1, 2))


def _same(off, z, ref, tol, what):
    assert np.array_equal(off, ref.col_off), what
    if z.size:
        assert np.max(np.abs(z.astype(np.float64) - ref.z)) <= tol, what


def _batch(seed, n, f32):
    rng = np.random.default_rng(seed)
    items = []
    for q in range(n):
        nx, ny = int(rng.integers(1, 48)), int(rng.integers(1, 48))
        g = shapes.random_grid(rng, nx, ny, 6, fill=0.75, point_frac=0.05, h=1 / 40)
        if f32:
            g = shapes.to_float32(g)
        k = float(rng.choice([0.0, 0.7, 1.0, math.sqrt(2.0), 2.5, 4.0, 7.3, 11.0]))
        op = ["dilate", "erode", "close", "open"][q % 4]
        items.append((g, op, k))
    return items


@pytest.mark.parametrize("f32", [False, True])
def test_batched_random_shapes(dx, f32):
    import torch
    items = _batch(5 + f32, 24, f32)
    code = {"dilate": dx.DILATE, "erode": dx.ERODE, "close": dx.CLOSE, "open": dx.OPEN}
    dt = torch.float32 if f32 else torch.float64
    grids = [dx.Grid.from_synth(g, dtype=dt) for g, _, _ in items]
    ctx = dx.Context(0)
    # the second call sizes the closings' and openings' internal grids from the first call's
    # totals and records the sequence through the output write; the third replays that graph
    for rep in range(3):
        outs = ctx.run_batched([code[op] for _, op, _ in items], grids, [k for _, _, k in items])
        for (g, op, k), o in zip(items, outs):
            off, z = o.to_host()
            ref = _ref(g, op, k, f32)
            if f32:
                ref = _round_f32(ref, op in ("erode", "close"))
            _same(off, z, ref, TOL32 if f32 else TOL64, f"{op} k={k} {g.nx}x{g.ny} rep {rep}")


def test_batched_matches_single_calls(dx):
    """Batched results equal the single-shape entry point's on spheres of several sizes."""
    import torch
    rng = np.random.default_rng(3)
    grids, ks, ops = [], [], []
    for q in range(8):
        n = int(rng.integers(24, 96))
        prims = [("sphere", *rng.uniform(0.3, 0.7, 3), float(rng.uniform(0.1, 0.25)))]
        grids.append(dx.Grid.from_synth(shapes.raycast(prims, n), dtype=torch.float64))
        ks.append(float(rng.uniform(1, 12)))
        ops.append([dx.DILATE, dx.ERODE, dx.CLOSE, dx.OPEN][q % 4])
    ctx = dx.Context(0)
    outs = ctx.run_batched(ops, grids, ks)
    for g, k, op, o in zip(grids, ks, ops, outs):
        r = ctx.run(op, g, k)
        a_off, a_z = o.to_host()
        b_off, b_z = r.to_host()
        assert np.array_equal(a_off, b_off)
        if a_z.size:
            assert np.max(np.abs(a_z - b_z)) <= TOL64


def test_batched_capacity_and_bad_shape(dx):
    """A shape whose output buffer is too small reports its need (the binding retries); a
    shape with a malformed CSR fails alone while the others complete."""
    import ctypes
    import torch
    L = dx.lib()
    good = shapes.grid64()
    bad = shapes.from_columns(4, 4, 0.25, {(1, 1): [(0.2, 0.4), (0.3, 0.6)]})
    grids = [dx.Grid.from_synth(good), dx.Grid.from_synth(bad), dx.Grid.from_synth(good)]
    ins = (dx._In * 3)(*[g._in() for g in grids])
    keep = []
    outs = (dx._Out * 3)()
    for q, g in enumerate(grids):
        cap = 8 if q == 2 else 200000
        off = torch.empty(g.nx * g.ny + 1, dtype=torch.int32, device="cuda")
        z = torch.empty((cap, 2), dtype=torch.float64, device="cuda")
        keep.append((off, z))
        outs[q] = dx._Out(off.data_ptr(), z.data_ptr(), cap, 0)
    kk = (ctypes.c_double * 3)(4.0, 1.0, 4.0)
    oo = (ctypes.c_int * 3)(dx.DILATE, dx.DILATE, dx.DILATE)
    dst = torch.zeros(3, dtype=torch.int32, device="cuda")
    ctx = dx.Context(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.dexel_offset_batched(ctx.ptr, 3, ins, kk, oo, 0, outs, None, 0,
                                ctypes.c_void_p(dst.data_ptr()), stream)
    st = dst.cpu().numpy().tolist()
    assert st == [0, -2, -3] and rc != 0
    ref = oracle.dilate(good, 4.0)
    assert outs[0].nseg == ref.nseg and outs[2].nseg == ref.nseg
    off, z = keep[0]
    _same(off.cpu().numpy().astype(np.int64), z[: outs[0].nseg].cpu().numpy(), ref, TOL64, "good shape")


def test_batched_wide_reach(dx):
    """Reaches beyond 31 and 63 spacings in one batch with a small one (pass-1 masks of two
    words, level groups, and the level walk's flat table once a reach passes 63)."""
    import torch
    rng = np.random.default_rng(21)
    items = []
    for n, k, op in ((96, 66.0, "dilate"), (80, 40.0, "erode"), (30, 3.0, "dilate"),
                     (64, 33.5, "close")):
        g = shapes.random_grid(rng, n, n, 4, fill=0.5, point_frac=0.05, h=1 / 4000)
        items.append((g, op, k))
    code = {"dilate": dx.DILATE, "erode": dx.ERODE, "close": dx.CLOSE, "open": dx.OPEN}
    grids = [dx.Grid.from_synth(g, dtype=torch.float64) for g, _, _ in items]
    ctx = dx.Context(0)
    outs = ctx.run_batched([code[op] for _, op, _ in items], grids, [k for _, _, k in items])
    for (g, op, k), o in zip(items, outs):
        off, z = o.to_host()
        _same(off, z, _ref(g, op, k), TOL64, f"{op} k={k} {g.nx}x{g.ny}")


def test_batched_large_shapes_single_path(dx, monkeypatch):
    """Shapes above the batch size limit (here 600 columns) take the single-shape path inside
    the batched call, closings and openings included; every result matches the oracle."""
    import torch
    monkeypatch.setenv("DEXEL_BATCH_MAX_COLS", "600")
    items = _batch(7, 12, False)
    code = {"dilate": dx.DILATE, "erode": dx.ERODE, "close": dx.CLOSE, "open": dx.OPEN}
    grids = [dx.Grid.from_synth(g, dtype=torch.float64) for g, _, _ in items]
    ctx = dx.Context(0)
    outs = ctx.run_batched([code[op] for _, op, _ in items], grids, [k for _, _, k in items])
    big = sum(g.nx * g.ny > 600 for g, _, _ in items)
    assert 0 < big < len(items)
    assert ctx.stats()[5] == big
    for (g, op, k), o in zip(items, outs):
        off, z = o.to_host()
        _same(off, z, _ref(g, op, k), TOL64, f"{op} k={k} {g.nx}x{g.ny}")


def test_batched_large_shapes_stream_ordered(dx, monkeypatch):
    """A second batched call on the same context queues the large dilations and erosions
    stream-ordered (the plans the first call recorded) beside the batch; only the large
    closings and openings take the synchronous single-shape path; every result matches the
    oracle on both calls."""
    import torch
    monkeypatch.setenv("DEXEL_BATCH_MAX_COLS", "600")
    items = _batch(7, 12, False)
    code = {"dilate": dx.DILATE, "erode": dx.ERODE, "close": dx.CLOSE, "open": dx.OPEN}
    grids = [dx.Grid.from_synth(g, dtype=torch.float64) for g, _, _ in items]
    ctx = dx.Context(0)
    big = [op for g, op, _ in items if g.nx * g.ny > 600]
    big_morph = sum(op in ("close", "open") for op in big)
    assert len(big) > big_morph
    for call in range(2):
        outs = ctx.run_batched([code[op] for _, op, _ in items], grids, [k for _, _, k in items])
        assert ctx.stats()[5] == (len(big) if call == 0 else big_morph)
        for (g, op, k), o in zip(items, outs):
            off, z = o.to_host()
            _same(off, z, _ref(g, op, k), TOL64, f"call {call}: {op} k={k} {g.nx}x{g.ny}")
