"""Pins of the oracle's three views of a solid (ray casting along x, y and z: a layered depth
image, Sec. 5) -- CPU only."""
import numpy as np

import oracle


def _inside(col, w):
    return bool(np.any((col[:, 0] <= w) & (w <= col[:, 1]))) if col.size else False


def test_centred_sphere_views_coincide():
    n = 40
    s = [("sphere", 0.5, 0.5, 0.5, 0.33)]
    g = [oracle.raycast_axis(s, a, n, n, 1 / n) for a in (2, 0, 1)]
    for q in (1, 2):
        assert np.array_equal(g[0].col_off, g[q].col_off) and np.array_equal(g[0].z, g[q].z)


def test_box_views_closed_form():
    b = [("box", 0.1, 0.3, 0.2, 0.7, 0.4, 0.95)]
    n = 20
    gx = oracle.raycast_axis(b, 0, n, n, 1 / n)  # columns over (y, z), heights x
    gy = oracle.raycast_axis(b, 1, n, n, 1 / n)  # columns over (z, x), heights y
    for j in range(n):
        for i in range(n):
            u, v = (i + 0.5) / n, (j + 0.5) / n
            wx = [[0.1, 0.3]] if (0.2 < u < 0.7 and 0.4 < v < 0.95) else []
            wy = [[0.2, 0.7]] if (0.4 < u < 0.95 and 0.1 < v < 0.3) else []
            assert gx.column(i, j).tolist() == wx and gy.column(i, j).tolist() == wy


def test_views_agree_at_lattice_points():
    """A lattice point ((i+1/2)h, (j+1/2)h, (l+1/2)h) is a ray sample of all three views; away
    from the surfaces its membership is the same in each."""
    from synth import shapes
    prims = shapes.grid512_prims(30, seed=11)
    n = 48
    h = 1 / n
    gz, gx, gy = (oracle.raycast_axis(prims, a, n, n, h) for a in (2, 0, 1))
    rng = np.random.default_rng(5)
    for _ in range(3000):
        i, j, l = (int(x) for x in rng.integers(0, n, 3))
        x, y, z = (i + 0.5) * h, (j + 0.5) * h, (l + 0.5) * h
        a = _inside(gz.column(i, j), z)
        b = _inside(gx.column(j, l), x)
        c = _inside(gy.column(l, i), y)
        ends = np.concatenate([gz.column(i, j).ravel() - z, gx.column(j, l).ravel() - x,
                               gy.column(l, i).ravel() - y])
        if ends.size and np.min(np.abs(ends)) < 1e-12:
            continue
        assert a == b == c, (i, j, l)
