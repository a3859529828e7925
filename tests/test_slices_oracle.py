"""Pins of the oracle's 2D slice offsets (Sec. 3.2: a 2D dexel image -- parallel segments on
a regular grid -- offset by a disk), every row of a grid an independent image (CPU)."""
import math

import numpy as np
import pytest

import oracle
from helpers import read_golden
from synth import shapes


def test_lone_segment_slice_is_the_capsule_row():
    """In 2D a lone segment becomes a stadium: on the segment's row the 3D capsule's row
    (hand-derived Pythagorean radii, dj = 0), every other row empty."""
    g = shapes.from_columns(24, 20, 1 / 64, {(10, 10): [(0.25, 0.5)]})
    d = oracle.dilate_slices(g, 5.0)
    gold = {(i, j): segs for i, j, segs in read_golden("capsule_k5.txt")}
    for j in range(20):
        for i in range(24):
            got = [tuple(x) for x in d.column(i, j).tolist()]
            if j != 10:
                assert got == [], (i, j)
            elif (i, j) in gold:
                assert got == [tuple(x) for x in gold[(i, j)]], (i, j)
    # the reach along the row: |di| <= 5
    assert [i for i in range(24) if d.column(i, 10).size] == list(range(5, 16))


@pytest.mark.parametrize("seed", range(3))
def test_disk_membership_brute_force(seed):
    """A point (x_i, z) of a row is in the 2D dilation iff some segment of the same row lies
    within distance r of it (and in the 2D erosion iff the disk around it lies in the shape's
    row); checked at random heights."""
    rng = np.random.default_rng(600 + seed)
    g = shapes.random_grid(rng, 11, 4, 4, fill=0.8, point_frac=0.1, h=1 / 16)
    k = float(rng.uniform(1.0, 4.5))
    h, r = g.h, k * g.h
    d, e = oracle.dilate_slices(g, k), oracle.erode_slices(g, k)
    for j in range(g.ny):
        for i in range(g.nx):
            zd = d.column(i, j)
            ze = e.column(i, j)
            for zq in rng.uniform(-0.3, 1.3, 60):
                near = False
                for ii in range(g.nx):
                    for a, b in g.column(ii, j):
                        dz = 0.0 if a <= zq <= b else min(abs(zq - a), abs(zq - b))
                        if (ii - i) ** 2 * h * h + dz * dz <= r * r:
                            near = True
                ind = bool(np.any((zd[:, 0] <= zq) & (zq <= zd[:, 1]))) if zd.size else False
                if ind != near:
                    # only a height on the result's boundary may disagree (rounding)
                    ends = zd.ravel()
                    assert ends.size and np.min(np.abs(ends - zq)) < 1e-9, (i, j, zq)
                # erosion: the whole disk inside the row's shape (in-grid columns only)
                inside = True
                for ii in range(g.nx):
                    dx2 = (ii - i) ** 2 * h * h
                    if dx2 > r * r:
                        continue
                    w = math.sqrt(r * r - dx2)
                    col = g.column(ii, j)
                    if not any(a <= zq - w and zq + w <= b for a, b in col):
                        inside = False
                ine = bool(np.any((ze[:, 0] <= zq) & (zq <= ze[:, 1]))) if ze.size else False
                if ine != inside:
                    ends = ze.ravel()
                    assert ends.size and np.min(np.abs(ends - zq)) < 1e-9, ("erode", i, j, zq)


def test_slices_are_independent_rows():
    """A row offset alone (a 1-row grid, where disk and ball coincide) equals the same row
    of the slices result; and the slices result never exceeds the 3D one."""
    rng = np.random.default_rng(7)
    g = shapes.random_grid(rng, 30, 9, 5, fill=0.8, point_frac=0.05, h=1 / 32)
    k = 3.3
    sl = oracle.dilate_slices(g, k)
    full = oracle.dilate(g, k)
    for j in range(g.ny):
        row = shapes.DexelGrid(g.nx, 1, g.h, g.col_off[j * g.nx:(j + 1) * g.nx + 1] - g.col_off[j * g.nx],
                               g.z[g.col_off[j * g.nx]:g.col_off[(j + 1) * g.nx]])
        one = oracle.dilate(row, k)
        for i in range(g.nx):
            assert np.array_equal(one.column(i, 0), sl.column(i, j))
            for a, b in sl.column(i, j):
                fz = full.column(i, j)
                assert np.any((fz[:, 0] <= a) & (b <= fz[:, 1]))


def test_slice_duality():
    """2D erosion is the complement of the 2D dilation of the complement."""
    rng = np.random.default_rng(8)
    g = shapes.random_grid(rng, 17, 5, 4, fill=0.9, point_frac=0.0, h=1 / 16)
    k = 2.5
    e = oracle.erode_slices(g, k)
    dc = oracle.dilate_slices(oracle.complement(g), k)
    back = oracle.complement(dc)
    for c in range(g.nx * g.ny):
        a = e.z[e.col_off[c]:e.col_off[c + 1]]
        b = back.z[back.col_off[c]:back.col_off[c + 1]]
        b = b[b[:, 1] > b[:, 0]] if b.size else b
        assert np.allclose(a, b, atol=1e-12), c
