"""Stream-ordered offsets (dexel_offset_enqueue): no host synchronisation in the call.

A synchronous dexel_dilate / dexel_erode records the counters it reads (its plan); the
stream-ordered call replays the plan with every redo launch made and reports on the device.
The tests check, through the C ABI, that a replayed offset equals the synchronous result bit
for bit (FP64 and FP32 endpoints, dilation and erosion, one block and several blocks of y
lines, twice in a row), that the result words carry the status and size, that data which
needs more than the plan is reported rather than written, and the host-side refusals.
"""
import os

import numpy as np
import pytest

from synth import shapes

pytestmark = pytest.mark.gpu


def _grid(n, seed, nprim=60, dtype="fp64"):
    import torch
    import paper_1804_08968_gb300 as dx
    g = shapes.raycast(shapes.grid512_prims(nprim=nprim, seed=seed), n)
    if dtype == "fp32":
        g = shapes.to_float32(g)
    return dx.Grid.from_synth(g, dtype=torch.float32 if dtype == "fp32" else torch.float64)


def _enqueue(ctx, op, g, k, ws_bytes=None, cap=None):
    import torch
    ws = torch.empty(ws_bytes or ctx.last_required(), dtype=torch.uint8, device="cuda")
    cap = cap if cap is not None else max(4 * g.nseg + g.nx * g.ny, 1024)
    off = torch.full((g.nx * g.ny + 1,), -5, dtype=torch.int32, device="cuda")
    z = torch.full((max(cap, 1), 2), float("nan"), dtype=g.z.dtype, device="cuda")
    res = torch.full((2,), -99, dtype=torch.int64, device="cuda")
    rc = ctx.enqueue(op, g, k, ws, off, z, res)
    torch.cuda.synchronize()
    r = res.cpu().numpy()
    n = int(r[1]) if rc == 0 and r[0] == 0 else 0
    return rc, r, off.cpu().numpy().astype(np.int64), z[:n].cpu().numpy()


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
@pytest.mark.parametrize("op,k", [("dilate", 20.0), ("erode", 20.0), ("dilate", 64.0),
                                  ("dilate", 2.0)])
def test_replay_equals_synchronous(dtype, op, k):
    import paper_1804_08968_gb300 as dx
    g = _grid(256, 5, dtype=dtype)
    code = dx.DILATE if op == "dilate" else dx.ERODE
    ctx = dx.Context(0)
    ref_off, ref_z = ctx.run(code, g, k).to_host()
    for _ in range(2):
        rc, r, off, z = _enqueue(ctx, code, g, k)
        assert rc == 0 and r[0] == 0, (rc, r)
        assert r[1] == ref_z.shape[0]
        assert np.array_equal(off, ref_off)
        assert np.array_equal(z, ref_z)


def test_replay_in_blocks_of_lines(monkeypatch):
    import paper_1804_08968_gb300 as dx
    monkeypatch.setenv("DEXEL_BLOCK_MB", "40")  # (read when the context is created)
    g = _grid(384, 6, nprim=90)
    ctx = dx.Context(0)
    ref_off, ref_z = ctx.run(dx.DILATE, g, 40.0).to_host()
    assert ctx.stats()[9] > 1  # several blocks
    for _ in range(2):
        rc, r, off, z = _enqueue(ctx, dx.DILATE, g, 40.0)
        assert rc == 0 and r[0] == 0, (rc, r)
        assert np.array_equal(off, ref_off) and np.array_equal(z, ref_z)


def test_other_data_same_plan_is_exact_or_reported():
    """A plan replayed on other data of the same size: the result is either exact or the
    result words ask for a synchronous call (nothing written)."""
    import paper_1804_08968_gb300 as dx
    ctx = dx.Context(0)
    g1 = _grid(256, 7, nprim=30)
    ctx.run(dx.DILATE, g1, 24.0)
    ws_bytes = ctx.last_required() * 2
    outcomes = set()
    for seed, nprim in [(8, 30), (9, 120), (10, 5)]:
        g2 = _grid(256, seed, nprim=nprim)
        rc, r, off, z = _enqueue(ctx, dx.DILATE, g2, 24.0, ws_bytes=ws_bytes)
        assert rc == 0
        ref_off, ref_z = dx.Context(0).run(dx.DILATE, g2, 24.0).to_host()
        if r[0] == 0:
            assert np.array_equal(off, ref_off) and np.array_equal(z, ref_z)
        else:
            assert r[0] in (dx.ERR_NO_PLAN, dx.ERR_CAPACITY), r
        outcomes.add(int(r[0]))
    assert 0 in outcomes


def test_output_capacity_and_bad_input_reported_on_device():
    import torch
    import paper_1804_08968_gb300 as dx
    ctx = dx.Context(0)
    g = _grid(128, 11, nprim=25)
    _, ref_z = ctx.run(dx.DILATE, g, 10.0).to_host()
    rc, r, _, _ = _enqueue(ctx, dx.DILATE, g, 10.0, cap=ref_z.shape[0] - 1)
    assert rc == 0 and r[0] == dx.ERR_CAPACITY and r[1] == ref_z.shape[0]
    # a segment with z_in > z_out: the validation's status, no pass over the bad input
    zb = g.z.clone()
    zb[3, 0], zb[3, 1] = zb[3, 1] + 1.0, zb[3, 0]
    bad = dx.Grid(g.nx, g.ny, g.h, g.col_off, zb)
    rc, r, _, _ = _enqueue(ctx, dx.DILATE, bad, 10.0)
    assert rc == 0 and r[0] == dx.ERR_BAD_CSR
    # the context still works
    rc, r, _, z = _enqueue(ctx, dx.DILATE, g, 10.0)
    assert rc == 0 and r[0] == 0 and np.array_equal(z, ref_z)


def test_host_side_refusals():
    import torch
    import paper_1804_08968_gb300 as dx
    ctx = dx.Context(0)
    g = _grid(64, 12, nprim=10)
    # no plan recorded for this offset yet
    rc, _, _, _ = _enqueue(ctx, dx.DILATE, g, 6.0, ws_bytes=1 << 20)
    assert rc == dx.ERR_NO_PLAN
    ctx.run(dx.DILATE, g, 6.0)
    # a workspace below the plan's need: refused before anything is queued
    need = ctx.last_required()
    rc, r, _, _ = _enqueue(ctx, dx.DILATE, g, 6.0, ws_bytes=need // 4)
    assert rc == dx.ERR_CAPACITY and r[0] == -99
    rc, r, _, _ = _enqueue(ctx, dx.DILATE, g, 6.0, ws_bytes=need)
    assert rc == 0 and r[0] == 0
