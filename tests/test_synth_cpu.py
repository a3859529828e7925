"""Host-side checks of the seeded input generator and of the parity comparison helper."""
import numpy as np
import pytest

from synth import shapes


@pytest.mark.parametrize("which", ["grid64", "grid512_small", "grid2048_crop"])
def test_compiled_raycast_matches_numpy(which):
    """The compiled ray caster gives the numpy one's grid bit for bit."""
    if which == "grid64":
        prims, n = shapes.grid64_prims(), 64
    elif which == "grid512_small":
        prims, n = shapes.grid512_prims(120, seed=5), 256
    else:
        prims, n = shapes.grid2048_prims()[:200], 160
    a = shapes.raycast(prims, n)
    b = shapes.raycast_numpy(prims, n)
    assert np.array_equal(a.col_off, b.col_off)
    assert np.array_equal(a.z, b.z)


def test_raycast_sphere_closed_form():
    """A lone sphere: every column inside its disk holds cz -+ sqrt(R^2 - d^2)."""
    n, R, cz = 40, 0.3, 0.5
    g = shapes.raycast([("sphere", 0.5, 0.5, cz, R)], n)
    h = 1.0 / n
    for j in range(n):
        for i in range(n):
            d2 = ((i + 0.5) * h - 0.5) ** 2 + ((j + 0.5) * h - 0.5) ** 2
            col = g.column(i, j)
            if d2 < R * R:
                s = np.sqrt(R * R - d2)
                assert col.shape == (1, 2)
                assert abs(col[0, 0] - (cz - s)) < 1e-15 and abs(col[0, 1] - (cz + s)) < 1e-15
            else:
                assert col.shape == (0, 2)


def test_compare_full_checks_every_matching_column():
    """An excused count mismatch in one column does not switch off the endpoint check of the
    others (FP32 mode), and an unexcused one fails."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "parity_gpu", os.path.join(os.path.dirname(os.path.abspath(__file__)), "test_parity_gpu.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    _compare_full = mod._compare_full
    ref = shapes.from_columns(3, 1, 0.1, {(0, 0): [(0.1, 0.2), (0.2 + 2e-9, 0.3)],
                                          (1, 0): [(0.4, 0.5)], (2, 0): [(0.1, 0.9)]})
    # the GPU merged column 0's two runs (gap below one float ulp): excused
    got = shapes.from_columns(3, 1, 0.1, {(0, 0): [(0.1, 0.3)], (1, 0): [(0.4, 0.5)],
                                          (2, 0): [(0.1, 0.9)]})
    _compare_full(got.col_off, got.z, ref, True, "ok")
    bad = shapes.from_columns(3, 1, 0.1, {(0, 0): [(0.1, 0.3)], (1, 0): [(0.4, 0.5 + 1e-4)],
                                          (2, 0): [(0.1, 0.9)]})
    with pytest.raises(AssertionError):
        _compare_full(bad.col_off, bad.z, ref, True, "planted endpoint error")
    # in FP64 a gap of 2e-9 is not below the 1e-9 threshold: the merge is not excused
    with pytest.raises(AssertionError):
        _compare_full(got.col_off, got.z, ref, False, "planted merge")


def test_float32_rounding_merge_matches_sorting_union():
    """The linear re-merge after rounding gives the sort-and-union result."""
    rng = np.random.default_rng(3)
    g = shapes.random_grid(rng, 30, 20, 8, fill=0.8, point_frac=0.1, h=1 / 32)
    # squeeze some gaps below float resolution so that rounding makes segments touch
    z = g.z.copy()
    for c in range(g.nx * g.ny):
        s0, s1 = g.col_off[c], g.col_off[c + 1]
        for s in range(s0 + 1, s1):
            if rng.random() < 0.3 and z[s - 1, 1] + 1e-9 < z[s, 1]:
                z[s, 0] = z[s - 1, 1] + 1e-9
    g2 = shapes.DexelGrid(g.nx, g.ny, g.h, g.col_off, z)
    a = shapes.to_float32(g2)
    b = shapes.to_float32_sorting(g2)
    assert np.array_equal(a.col_off, b.col_off)
    assert np.array_equal(a.z, b.z)
    assert a.nseg < g2.nseg  # some segments did merge
