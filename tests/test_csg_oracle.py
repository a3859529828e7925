"""Pins of the oracle's Boolean operations and thick shell (CPU, no GPU).

The oracle (oracle/oracle.c) computes union, intersection and difference of two dexel grids
from point membership of each column's elementary intervals, and the shell as the dilation
minus the erosion (Sec. 4 "3D Printing", teaser figure).  These tests pin it to things other
than itself: closed forms of overlapping boxes and concentric spheres, the additivity of
length (|A u B| + |A n B| = |A| + |B|), set identities, point membership sampled at random
heights, and, for the shell, the golden capsule and the relations between shell, dilation
and erosion.
"""
import numpy as np
import pytest

import oracle
from synth import shapes


def _len(g):
    """Total length of every column's segments."""
    z = np.asarray(g.z, np.float64).reshape(-1, 2)
    col = np.repeat(np.arange(g.nx * g.ny), np.diff(g.col_off))
    return np.bincount(col, weights=z[:, 1] - z[:, 0], minlength=g.nx * g.ny)


def _drop_points(g):
    z = np.asarray(g.z, np.float64).reshape(-1, 2)
    keep = z[:, 1] > z[:, 0]
    col = np.repeat(np.arange(g.nx * g.ny), np.diff(g.col_off))[keep]
    off = np.zeros(g.nx * g.ny + 1, np.int64)
    np.cumsum(np.bincount(col, minlength=g.nx * g.ny), out=off[1:])
    return shapes.DexelGrid(g.nx, g.ny, g.h, off, z[keep])


def _same(a, b):
    assert np.array_equal(np.asarray(a.col_off), np.asarray(b.col_off))
    assert np.array_equal(np.asarray(a.z, np.float64).reshape(-1, 2),
                          np.asarray(b.z, np.float64).reshape(-1, 2))


def _inside(z, x):
    return bool(np.any((z[:, 0] <= x) & (x <= z[:, 1])))


def test_boxes_closed_form():
    """Boxes A (z in [0.2, 0.6]) and B (z in [0.4, 0.8]) with overlapping footprints: every
    column's result is one of the literal intervals below."""
    n = 32
    A = [("box", 0.1, 0.6, 0.1, 0.6, 0.2, 0.6)]
    B = [("box", 0.4, 0.9, 0.3, 0.8, 0.4, 0.8)]
    ga, gb = shapes.raycast(A, n), shapes.raycast(B, n)
    u, i, d = oracle.union(ga, gb), oracle.intersection(ga, gb), oracle.difference(ga, gb)
    for jj in range(n):
        for ii in range(n):
            ina = ga.column(ii, jj).shape[0] == 1
            inb = gb.column(ii, jj).shape[0] == 1
            want_u = [[0.2, 0.8]] if ina and inb else ([[0.2, 0.6]] if ina else ([[0.4, 0.8]] if inb else []))
            want_i = [[0.4, 0.6]] if ina and inb else []
            want_d = [[0.2, 0.4]] if ina and inb else ([[0.2, 0.6]] if ina else [])
            for g, want in ((u, want_u), (i, want_i), (d, want_d)):
                got = g.column(ii, jj).tolist()
                assert got == want, (ii, jj, got, want)


def test_concentric_spheres_difference_is_the_shell():
    """sphere(R) minus sphere(R - t) is the ray-cast hollow shell, bit for bit."""
    n = 48
    c, R, t = (0.5, 0.47, 0.5), 0.35, 0.08
    outer = shapes.raycast([("sphere", c[0], c[1], c[2], R)], n)
    inner = shapes.raycast([("sphere", c[0], c[1], c[2], R - t)], n)
    shell = shapes.raycast([("shell", c[0], c[1], c[2], R, t)], n)
    _same(oracle.difference(outer, inner), shell)
    # and the union of the shell with the inner sphere is the outer sphere again
    _same(oracle.union(shell, inner), outer)


@pytest.mark.parametrize("seed", range(4))
def test_length_additivity_and_identities(seed):
    rng = np.random.default_rng(300 + seed)
    a = shapes.random_grid(rng, 9, 7, 6, fill=0.8, point_frac=0.1, h=1 / 8)
    b = shapes.random_grid(rng, 9, 7, 6, fill=0.8, point_frac=0.1, h=1 / 8)
    u, i, d = oracle.union(a, b), oracle.intersection(a, b), oracle.difference(a, b)
    la, lb = _len(a), _len(b)
    assert np.allclose(_len(u) + _len(i), la + lb, atol=1e-12)
    assert np.allclose(_len(d), la - _len(i), atol=1e-12)
    # commutativity; identities with the empty grid and with itself
    _same(u, oracle.union(b, a))
    _same(i, oracle.intersection(b, a))
    empty = shapes.from_columns(9, 7, 1 / 8, {})
    _same(oracle.union(a, empty), a)
    _same(oracle.difference(a, empty), _drop_points(a))
    _same(oracle.intersection(a, a), _drop_points(a))
    assert oracle.difference(a, a).nseg == 0
    assert oracle.intersection(a, empty).nseg == 0


@pytest.mark.parametrize("seed", range(3))
def test_point_membership(seed):
    """At random heights (away from every endpoint) a result holds z exactly when the
    Boolean of the inputs' memberships says so."""
    rng = np.random.default_rng(400 + seed)
    a = shapes.random_grid(rng, 6, 5, 5, fill=0.9, point_frac=0.05, h=1 / 8)
    b = shapes.random_grid(rng, 6, 5, 5, fill=0.9, point_frac=0.05, h=1 / 8)
    res = {"u": oracle.union(a, b), "i": oracle.intersection(a, b), "d": oracle.difference(a, b)}
    for c in range(a.nx * a.ny):
        za = np.asarray(a.z[a.col_off[c]:a.col_off[c + 1]], np.float64)
        zb = np.asarray(b.z[b.col_off[c]:b.col_off[c + 1]], np.float64)
        ends = np.concatenate([za.ravel(), zb.ravel()])
        for x in rng.uniform(-0.1, 1.1, 200):
            if ends.size and np.min(np.abs(ends - x)) < 1e-9:
                continue
            ia, ib = _inside(za, x), _inside(zb, x)
            for key, want in (("u", ia or ib), ("i", ia and ib), ("d", ia and not ib)):
                g = res[key]
                zr = np.asarray(g.z[g.col_off[c]:g.col_off[c + 1]], np.float64)
                assert _inside(zr, x) == want, (key, c, x)


def test_union_keeps_isolated_points():
    a = shapes.from_columns(1, 1, 0.1, {(0, 0): [(0.5, 0.5)]})
    b = shapes.from_columns(1, 1, 0.1, {(0, 0): [(0.1, 0.2)]})
    assert oracle.union(a, b).z.tolist() == [[0.1, 0.2], [0.5, 0.5]]
    assert oracle.intersection(a, b).nseg == 0


def test_shell_of_a_lone_segment_is_the_capsule():
    """A segment too thin to survive the erosion: its shell is its dilation, the golden
    capsule (hand-derived Pythagorean radii)."""
    from helpers import read_golden as rg
    g = shapes.from_columns(24, 20, 1 / 64, {(10, 10): [(0.25, 0.5)]})
    s = oracle.shell(g, 5.0)
    for i, j, segs in rg("capsule_k5.txt"):
        assert [tuple(x) for x in s.column(i, j).tolist()] == [tuple(x) for x in segs], (i, j)


def test_shell_relations():
    """shell u E = D and |shell| = |D| - |E| (the erosion lies inside the dilation)."""
    g = shapes.raycast(shapes.grid512_prims(40, seed=7), 64)
    k = 3.0
    d, e = oracle.dilate(g, k), oracle.erode(g, k)
    s = oracle.shell(g, k)
    assert np.allclose(_len(s), _len(d) - _len(e), atol=1e-12)
    _same(oracle.union(s, e), d)
    assert np.allclose(_len(oracle.intersection(s, e)), 0.0)
