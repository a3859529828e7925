"""Pins of the oracle's ray casting of analytic primitives (CPU): closed forms of a sphere and
a box, a hollow sphere as the difference of two spheres (the Boolean oracle), agreement with
the seeded input generator's own ray caster (another implementation), and the volume of a
sphere approached as the grid is refined."""
import math

import numpy as np
import pytest

import oracle
from synth import shapes


def test_sphere_closed_form():
    n, R, c = 33, 0.31, (0.52, 0.47, 0.5)
    g = oracle.raycast([("sphere", *c, R)], n, n, 1 / n)
    for j in range(n):
        for i in range(n):
            x, y = (i + 0.5) / n, (j + 0.5) / n
            d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2
            col = g.column(i, j)
            if d2 < R * R:
                s = math.sqrt(R * R - d2)
                assert col.shape == (1, 2)
                assert abs(col[0, 0] - (c[2] - s)) <= 1e-15 and abs(col[0, 1] - (c[2] + s)) <= 1e-15
            else:
                assert col.shape == (0, 2)


def test_box_closed_form_and_non_square_grid():
    g = oracle.raycast([("box", 0.2, 0.55, 0.3, 0.9, 0.1, 0.4)], 20, 10, 1 / 20)
    for j in range(10):
        for i in range(20):
            x, y = (i + 0.5) / 20, (j + 0.5) / 20
            want = [[0.1, 0.4]] if (0.2 < x < 0.55 and 0.3 < y < 0.9) else []
            assert g.column(i, j).tolist() == want, (i, j)


def test_shell_is_the_difference_of_two_spheres():
    n = 40
    c, R, t = (0.5, 0.5, 0.5), 0.3, 0.07
    sh = oracle.raycast([("shell", *c, R, t)], n, n, 1 / n)
    outer = oracle.raycast([("sphere", *c, R)], n, n, 1 / n)
    inner = oracle.raycast([("sphere", *c, R - t)], n, n, 1 / n)
    d = oracle.difference(outer, inner)
    assert np.array_equal(sh.col_off, d.col_off) and np.array_equal(sh.z, d.z)


@pytest.mark.parametrize("which", ["grid64", "grid512", "grid2048_part"])
def test_matches_the_input_generator(which):
    if which == "grid64":
        prims, n = shapes.grid64_prims(), 64
    elif which == "grid512":
        prims, n = shapes.grid512_prims(100, seed=2), 200
    else:
        prims, n = shapes.grid2048_prims()[:150], 128
    a = oracle.raycast(prims, n, n, 1.0 / n)
    b = shapes.raycast(prims, n)
    assert np.array_equal(a.col_off, b.col_off) and np.array_equal(a.z, b.z)


def test_sphere_volume_converges():
    R = 0.3
    errs = []
    for n in (32, 64, 128):
        g = oracle.raycast([("sphere", 0.5, 0.5, 0.5, R)], n, n, 1 / n)
        vol = float(np.sum(g.z[:, 1] - g.z[:, 0])) / (n * n)
        errs.append(abs(vol - 4.0 / 3.0 * math.pi * R ** 3))
    assert errs[2] < errs[0] and errs[2] < 1e-4
