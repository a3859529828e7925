"""The allocation-free entry point (dexel_offset_noalloc) against dexel_dilate / dexel_erode.

dexel_offset_noalloc exists for callers that cannot allocate device memory when they need
an offset (an application whose pool owns the GPU memory, a real-time loop that must not
pay cudaMalloc's synchronisation): its scratch is a static device array inside the library.
The test calls it through the C ABI on two different inputs in a row -- the second call
reuses the array the first one left behind -- and checks each result against the existing
entry point, with the tolerance of the other parity tests (identical segment counts, FP64
endpoints within 1e-10).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from synth import shapes

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _noalloc(dx, grid, k, op):
    import torch
    L = dx.lib()
    L.dexel_offset_noalloc.argtypes = [ctypes.POINTER(dx._In), ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(dx._Out), ctypes.c_void_p]
    L.dexel_offset_noalloc.restype = ctypes.c_int
    cap = max(4 * grid.nseg + grid.nx * grid.ny, 1024)
    off = torch.empty(grid.nx * grid.ny + 1, dtype=torch.int32, device="cuda")
    z = torch.empty((cap, 2), dtype=grid.z.dtype, device="cuda")
    gin = grid._in()
    out = dx._Out(off.data_ptr(), z.data_ptr(), cap, 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.dexel_offset_noalloc(ctypes.byref(gin), float(k), op, grid.mode, ctypes.byref(out), stream)
    torch.cuda.synchronize()
    return rc, off.cpu().numpy().astype(np.int64), z[: out.nseg].cpu().numpy()


def _existing(dx, grid, k, op):
    out = dx.Context(0).run(op, grid, k)
    return out.to_host()


def _same(a_off, a_z, b_off, b_z):
    assert np.array_equal(a_off, b_off)
    assert a_z.shape == b_z.shape
    if a_z.size:
        assert np.max(np.abs(a_z.astype(np.float64) - b_z.astype(np.float64))) <= TOL64


def test_noalloc_matches_existing_entry_point_twice():
    import torch
    import paper_1804_08968_gb300 as dx
    rng = np.random.default_rng(2024)
    cases = [
        (shapes.config1(), 4.0, dx.DILATE),
        (shapes.random_grid(rng, 45, 37, 5, fill=0.8, point_frac=0.05, h=1 / 40), 3.5, dx.ERODE),
    ]
    for g, k, op in cases:  # two calls in a row on different inputs
        grid = dx.Grid.from_synth(g, dtype=torch.float64)
        rc, off, z = _noalloc(dx, grid, k, op)
        assert rc == 0, dx.STATUS.get(rc, rc)
        ref_off, ref_z = _existing(dx, grid, k, op)
        _same(off, z, ref_off, ref_z)


def test_noalloc_rejects_grids_beyond_its_limit():
    import torch
    import paper_1804_08968_gb300 as dx
    g = shapes.from_columns(300, 300, 1 / 300, {(5, 5): [(0.25, 0.5)]})
    grid = dx.Grid.from_synth(g, dtype=torch.float64)
    rc, _, _ = _noalloc(dx, grid, 2.0, dx.DILATE)
    assert rc == -3  # DEXEL_ERR_CAPACITY: more columns than the static scratch serves
