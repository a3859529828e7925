"""The allocation-free entry point (dexel_offset_noalloc).

dexel_offset_noalloc exists for callers that cannot allocate device memory when they need
an offset (an application whose pool owns the GPU memory, a real-time loop that must not
pay cudaMalloc's synchronisation): its scratch is a static device array inside the library.
The tests call it through the C ABI, several times in a row -- every call reuses the array
the last one left behind -- and check each result against the FP64 oracle and against the
existing entry points (dexel_dilate / dexel_erode), with the tolerances of the other parity
tests: identical segment counts, endpoints within 1e-10 (FP64) or 4e-6 (FP32 endpoints).
They also check its limits (a grid beyond the array is refused with nseg = -1 and nothing
written), the output-size retry signal, and that a call allocates no device memory.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synth import shapes

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 4e-6


def _noalloc(dx, grid, k, op, cap=None, fill=None):
    import torch
    L = dx.lib()
    L.dexel_offset_noalloc.argtypes = [ctypes.POINTER(dx._In), ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(dx._Out), ctypes.c_void_p]
    L.dexel_offset_noalloc.restype = ctypes.c_int
    if cap is None:
        cap = max(4 * grid.nseg + grid.nx * grid.ny, 1024)
    off = torch.full((grid.nx * grid.ny + 1,), -7, dtype=torch.int32, device="cuda")
    z = torch.full((max(cap, 1), 2), float("nan") if fill is None else fill, dtype=grid.z.dtype,
                   device="cuda")
    gin = grid._in()
    out = dx._Out(off.data_ptr(), z.data_ptr(), cap, 12345)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.dexel_offset_noalloc(ctypes.byref(gin), float(k), op, grid.mode, ctypes.byref(out), stream)
    torch.cuda.synchronize()
    n = max(int(out.nseg), 0)
    return rc, int(out.nseg), off.cpu().numpy().astype(np.int64), z[:n].cpu().numpy(), z


def _existing(dx, grid, k, op):
    out = dx.Context(0).run(op, grid, k)
    return out.to_host()


def _same(a_off, a_z, b_off, b_z, tol):
    assert np.array_equal(a_off, b_off)
    assert a_z.shape == b_z.shape
    if a_z.size:
        assert np.max(np.abs(a_z.astype(np.float64) - b_z.astype(np.float64))) <= tol


def _oracle(g, k, op, dx):
    return oracle.dilate(g, k) if op == dx.DILATE else oracle.erode(g, k)


def test_noalloc_matches_existing_entry_point_twice():
    import torch
    import paper_1804_08968_gb300 as dx
    rng = np.random.default_rng(2024)
    cases = [
        (shapes.grid64(), 4.0, dx.DILATE),
        (shapes.random_grid(rng, 45, 37, 5, fill=0.8, point_frac=0.05, h=1 / 40), 3.5, dx.ERODE),
    ]
    for g, k, op in cases:  # two calls in a row on different inputs
        grid = dx.Grid.from_synth(g, dtype=torch.float64)
        rc, nseg, off, z, _ = _noalloc(dx, grid, k, op)
        assert rc == 0, dx.STATUS.get(rc, rc)
        assert nseg == off[-1]
        ref_off, ref_z = _existing(dx, grid, k, op)
        _same(off, z, ref_off, ref_z, TOL64)
        ref = _oracle(g, k, op, dx)
        _same(off, z, ref.col_off, ref.z, TOL64)


def test_noalloc_fp32_endpoints():
    """FP32 endpoints with FP64 decisions, against the oracle on the same float32 input."""
    import torch
    import paper_1804_08968_gb300 as dx
    rng = np.random.default_rng(2025)
    g = shapes.random_grid(rng, 33, 29, 6, fill=0.8, point_frac=0.05, h=1 / 40, dtype=np.float32)
    grid = dx.Grid.from_synth(g, dtype=torch.float32)
    for k, op in ((4.2, dx.DILATE), (2.5, dx.ERODE)):
        rc, _, off, z, _ = _noalloc(dx, grid, k, op)
        assert rc == 0, dx.STATUS.get(rc, rc)
        ref_off, ref_z = _existing(dx, grid, k, op)
        _same(off, z, ref_off, ref_z, TOL32)
        ref = _oracle(g, k, op, dx)
        _same(off, z, ref.col_off, ref.z, TOL32)


def test_noalloc_largest_advertised_grid():
    """256 x 256 columns at k = 32, the edge of the documented envelope, must succeed."""
    import torch
    import paper_1804_08968_gb300 as dx
    g = shapes.raycast(shapes.grid64_prims(), 256)
    grid = dx.Grid.from_synth(g, dtype=torch.float64)
    rc, nseg, off, z, _ = _noalloc(dx, grid, 32.0, dx.DILATE)
    assert rc == 0, dx.STATUS.get(rc, rc)
    ref_off, ref_z = _existing(dx, grid, 32.0, dx.DILATE)
    _same(off, z, ref_off, ref_z, TOL64)
    rng = np.random.default_rng(8)
    cols = rng.choice(256 * 256, 300, replace=False)
    ref = oracle.dilate(g, 32.0, cols=cols)
    for t, c in enumerate(cols):
        got = z[off[c]:off[c + 1]]
        exp = ref.column(t)
        assert got.shape == exp.shape
        if exp.size:
            assert np.max(np.abs(got - exp)) <= TOL64


def test_noalloc_limits_and_retry_signals():
    import torch
    import paper_1804_08968_gb300 as dx
    # more columns than the static scratch serves: refused, nseg = -1, nothing written
    g = shapes.from_columns(300, 300, 1 / 300, {(5, 5): [(0.25, 0.5)]})
    grid = dx.Grid.from_synth(g, dtype=torch.float64)
    rc, nseg, off, _, zt = _noalloc(dx, grid, 2.0, dx.DILATE)
    assert rc == -3 and nseg == -1
    assert (off == -7).all() and torch.isnan(zt).all()
    # data needing more scratch than the array holds (dense stacks of segments): refused the
    # same way, with no partial CSR
    cols = {(i, j): [(0.1 + q * 0.0025 + 0.0002 * ((i + 3 * j) % 7),
                      0.1 + q * 0.0025 + 0.0002 * ((i + 3 * j) % 7) + 0.001) for q in range(300)]
            for i in range(64) for j in range(64)}
    g = shapes.from_columns(64, 64, 1 / 64, cols)
    grid = dx.Grid.from_synth(g, dtype=torch.float64)
    rc, nseg, off, _, zt = _noalloc(dx, grid, 16.0, dx.DILATE)
    assert rc == -3 and nseg == -1
    assert (off == -7).all() and torch.isnan(zt).all()
    # an output buffer that is too small: nseg is the size needed, z untouched; a retry with
    # that size succeeds
    g = shapes.grid64()
    grid = dx.Grid.from_synth(g, dtype=torch.float64)
    rc, nseg, _, _, zt = _noalloc(dx, grid, 4.0, dx.DILATE, cap=3)
    assert rc == -3 and nseg > 3
    assert torch.isnan(zt).all()
    rc, nseg2, off, z, _ = _noalloc(dx, grid, 4.0, dx.DILATE, cap=nseg)
    assert rc == 0 and nseg2 == nseg
    ref = oracle.dilate(g, 4.0)
    _same(off, z, ref.col_off, ref.z, TOL64)


def test_noalloc_allocates_nothing():
    """Across calls neither torch's allocator nor the device's free memory changes."""
    import torch
    import paper_1804_08968_gb300 as dx
    g = shapes.grid64()
    grid = dx.Grid.from_synth(g, dtype=torch.float64)
    L = dx.lib()
    L.dexel_offset_noalloc.argtypes = [ctypes.POINTER(dx._In), ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(dx._Out), ctypes.c_void_p]
    L.dexel_offset_noalloc.restype = ctypes.c_int
    cap = 4 * grid.nseg + 4096
    off = torch.empty(grid.nx * grid.ny + 1, dtype=torch.int32, device="cuda")
    z = torch.empty((cap, 2), dtype=torch.float64, device="cuda")
    gin = grid._in()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        out = dx._Out(off.data_ptr(), z.data_ptr(), cap, 0)
        rc = L.dexel_offset_noalloc(ctypes.byref(gin), 4.0, dx.DILATE, dx.FP64, ctypes.byref(out), stream)
        torch.cuda.synchronize()
        assert rc == 0
        return int(out.nseg)

    n0 = call()  # the first call may load the library's module on this device
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert call() == n0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
