"""Pins for the FP64 oracle (CPU only): it is checked against facts fixed by the paper's
definitions and by mathematics, not against itself.

* closed forms with exact (Pythagorean) radii: lone segment -> capsule, box -> rounded box
  (golden files written by hand under tests/golden/);
* point membership against the distance definition of dilation (Sec. 3.1, Eq. of D_r) and
  against the ball-inclusion definition of erosion, on tiny random grids (brute force);
* erosion/dilation duality (Sec. 3.1 "Erosion"), monotonicity in r, union commuting with
  dilation, extensivity, closing idempotence, k = 0 identity;
* a ray-cast sphere of radius R dilated by r lies inside the ray-cast sphere R + r and
  converges to it under refinement.
"""
import math

import numpy as np
import pytest

import oracle
from synth import shapes
from tests.helpers import columns_of, csr_union, included, read_golden

KS = [0.0, 0.5, 1.0, math.sqrt(2.0), 2.0, 3.7]


def _grid_single(nx, ny, h, i, j, segs):
    return shapes.from_columns(nx, ny, h, {(i, j): segs})


@pytest.mark.parametrize("erode", [False])
def test_capsule_golden(erode):
    g = _grid_single(24, 20, 1 / 64, 10, 10, [(0.25, 0.5)])
    out = oracle.dilate(g, 5.0)
    for i, j, segs in read_golden("capsule_k5.txt"):
        got = out.column(i, j)
        assert len(got) == len(segs), (i, j, got, segs)
        for (a, b), (ea, eb) in zip(got, segs):
            assert a == ea and b == eb, (i, j, a, b, ea, eb)


def test_capsule_reach_count():
    # the ball of radius 5 (closed) meets exactly the columns with di^2+dj^2 <= 25: 81 of them
    g = _grid_single(24, 20, 1 / 64, 10, 10, [(0.25, 0.5)])
    out = oracle.dilate(g, 5.0)
    assert int(np.count_nonzero(np.diff(out.col_off))) == 81


def test_rounded_box_golden():
    cols = {(i, j): [(0.25, 0.75)] for i in range(10, 21) for j in range(12, 16)}
    g = shapes.from_columns(48, 40, 1 / 128, cols)
    out = oracle.dilate(g, 13.0)
    for i, j, segs in read_golden("box_k13.txt"):
        got = out.column(i, j)
        assert len(got) == len(segs), (i, j, got, segs)
        for (a, b), (ea, eb) in zip(got, segs):
            assert a == ea and b == eb, (i, j, a, b, ea, eb)


def _dist2_col(zq, segs):
    """Squared distance from height zq to the union of segments of one column (inf if none)."""
    best = math.inf
    for a, b in segs:
        d = 0.0 if a <= zq <= b else min(abs(zq - a), abs(zq - b))
        best = min(best, d * d)
    return best


def _inside_depth(zq, segs):
    """Distance from zq to the complement of the column's shape (0 if zq is outside)."""
    for a, b in segs:
        if a <= zq <= b:
            return min(zq - a, b - zq)
    return 0.0


def _probe_points(rng, cols_out, extra=40):
    pts = list(rng.uniform(-0.3, 1.3, extra))
    for segs in cols_out:
        for a, b in segs:
            for e in (a, b):
                if np.isfinite(e):
                    pts += [e - 1e-7, e + 1e-7]
    return pts


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("k", KS)
def test_dilation_membership_brute_force(seed, k):
    """z is in D(c) iff some input point is within distance r (Sec. 3.1 Eq. of D_r)."""
    rng = np.random.default_rng(100 + seed)
    nx, ny = 6, 5
    g = shapes.random_grid(rng, nx, ny, 3, fill=0.6, point_frac=0.15, h=0.05)
    r = k * g.h
    out = oracle.dilate(g, k)
    incols = [[tuple(s) for s in g.column(i, j)] for j in range(ny) for i in range(nx)]
    for j in range(ny):
        for i in range(nx):
            segs_out = [tuple(s) for s in out.column(i, j)]
            for zq in _probe_points(rng, [segs_out], 30):
                d2 = math.inf
                for jj in range(ny):
                    for ii in range(nx):
                        n = (i - ii) ** 2 + (j - jj) ** 2
                        d2 = min(d2, n * g.h * g.h + _dist2_col(zq, incols[jj * nx + ii]))
                member = any(a <= zq <= b for a, b in segs_out)
                if d2 <= r * r - 1e-12:
                    assert member, (i, j, zq, d2, r * r, segs_out)
                elif d2 >= r * r + 1e-12:
                    assert not member, (i, j, zq, d2, r * r, segs_out)


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("k", KS)
def test_erosion_membership_brute_force(seed, k):
    """z is in E(c) iff the ball around (c, z), restricted to the grid's columns, lies in S."""
    rng = np.random.default_rng(200 + seed)
    nx, ny = 5, 6
    g = shapes.random_grid(rng, nx, ny, 3, fill=0.95, h=0.02)
    r = k * g.h
    out = oracle.erode(g, k)
    incols = [[tuple(s) for s in g.column(i, j)] for j in range(ny) for i in range(nx)]
    for j in range(ny):
        for i in range(nx):
            segs_out = [tuple(s) for s in out.column(i, j)]
            for zq in _probe_points(rng, [segs_out] + [incols[j * nx + i]], 30):
                # margin: min over reached columns of (depth^2 + n h^2) - r^2
                margin = math.inf
                for jj in range(ny):
                    for ii in range(nx):
                        n = (i - ii) ** 2 + (j - jj) ** 2
                        if n * g.h * g.h > r * r:
                            continue
                        dep = _inside_depth(zq, incols[jj * nx + ii])
                        margin = min(margin, n * g.h * g.h + dep * dep - r * r)
                        if dep == 0.0:
                            margin = min(margin, -1.0)
                member = any(a <= zq <= b for a, b in segs_out)
                if margin >= 1e-12:
                    assert member, (i, j, zq, margin, segs_out)
                elif margin <= -1e-12:
                    assert not member, (i, j, zq, margin, segs_out)


@pytest.mark.parametrize("seed", [3, 4, 5])
@pytest.mark.parametrize("k", [0.0, 1.0, 2.5, 4.0])
def test_duality(seed, k):
    """Direct erosion equals complement(dilation(complement)) (Sec. 3.1 "Erosion")."""
    rng = np.random.default_rng(seed)
    g = shapes.random_grid(rng, 13, 9, 4, fill=0.8, point_frac=0.1, h=1 / 16)
    e = oracle.erode(g, k)
    d = oracle.complement(oracle.dilate(oracle.complement(g), k))
    assert np.array_equal(e.col_off, d.col_off)
    assert np.array_equal(e.z, d.z)


@pytest.mark.parametrize("seed", [6, 7])
def test_monotone_in_radius(seed):
    rng = np.random.default_rng(seed)
    g = shapes.random_grid(rng, 12, 10, 3, fill=0.7, h=1 / 20)
    prev_d = prev_e = None
    for k in [0.0, 0.7, 1.5, 2.0, 3.2]:
        d = columns_of(*(lambda x: (x.col_off, x.z))(oracle.dilate(g, k)))
        e = columns_of(*(lambda x: (x.col_off, x.z))(oracle.erode(g, k)))
        if prev_d is not None:
            assert included(prev_d, d)
            assert included(e, prev_e)
        prev_d, prev_e = d, e


@pytest.mark.parametrize("seed", [8, 9])
@pytest.mark.parametrize("k", [1.0, 2.2])
def test_union_commutes(seed, k):
    rng = np.random.default_rng(seed)
    a = shapes.random_grid(rng, 10, 11, 2, fill=0.5, h=1 / 16)
    b = shapes.random_grid(rng, 10, 11, 2, fill=0.5, h=1 / 16)
    lhs = oracle.dilate(csr_union(a, b), k)
    rhs = csr_union(oracle.dilate(a, k), oracle.dilate(b, k))
    assert np.array_equal(lhs.col_off, rhs.col_off)
    assert np.array_equal(lhs.z, rhs.z)


@pytest.mark.parametrize("seed", [10, 11])
@pytest.mark.parametrize("k", [1.0, 2.0, 3.0])
def test_extensive_and_closing(seed, k):
    rng = np.random.default_rng(seed)
    g = shapes.random_grid(rng, 12, 12, 3, fill=0.8, h=1 / 24)
    S = columns_of(g.col_off, g.z)
    D = oracle.dilate(g, k)
    E = oracle.erode(g, k)
    C = oracle.erode(D, k)
    O = oracle.dilate(E, k)
    assert included(S, columns_of(D.col_off, D.z))
    assert included(columns_of(E.col_off, E.z), S)
    assert included(S, columns_of(C.col_off, C.z), tol=1e-12)
    assert included(columns_of(O.col_off, O.z), S, tol=1e-12)
    # closing is idempotent (a closure operator); compare up to rounding of (b + w) - w
    CC = oracle.close(C, k)
    assert np.array_equal(CC.col_off, C.col_off)
    assert np.max(np.abs(CC.z - C.z), initial=0.0) <= 1e-12


def test_k0_identity():
    rng = np.random.default_rng(12)
    g = shapes.random_grid(rng, 9, 7, 4, fill=0.8, point_frac=0.2, h=1 / 16)
    d = oracle.dilate(g, 0.0)
    assert np.array_equal(d.col_off, g.col_off) and np.array_equal(d.z, g.z)
    e = oracle.erode(g, 0.0)
    keep = g.z[:, 0] < g.z[:, 1]
    assert np.array_equal(e.z, g.z[keep])


@pytest.mark.parametrize("n", [32, 64, 128])
def test_sphere_inside_offset_sphere(n):
    """Ray-cast sphere R dilated by r lies in the ray-cast sphere R + r, columnwise."""
    R, r = 0.25, 0.125
    k = r * n
    g = shapes.raycast([("sphere", 0.5, 0.5, 0.5, R)], n)
    big = shapes.raycast([("sphere", 0.5, 0.5, 0.5, R + r)], n)
    d = oracle.dilate(g, k)
    assert included(columns_of(d.col_off, d.z), columns_of(big.col_off, big.z), tol=1e-12)


def test_sphere_converges():
    """Away from the silhouette the top endpoint error shrinks under refinement."""
    R, r = 0.25, 0.125
    errs = []
    for n in (16, 32, 64):
        k = r * n
        g = shapes.raycast([("sphere", 0.5, 0.5, 0.5, R)], n)
        big = shapes.raycast([("sphere", 0.5, 0.5, 0.5, R + r)], n)
        d = oracle.dilate(g, k)
        h = 1.0 / n
        worst = 0.0
        for j in range(n):
            for i in range(n):
                x, y = (i + 0.5) * h, (j + 0.5) * h
                if (x - 0.5) ** 2 + (y - 0.5) ** 2 > (R * 0.9) ** 2:
                    continue
                got = d.column(i, j)
                ref = big.column(i, j)
                assert len(got) == 1 and len(ref) == 1
                worst = max(worst, abs(got[0][1] - ref[0][1]), abs(got[0][0] - ref[0][0]))
        errs.append(worst)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1.0 / 64


def test_sampled_columns_match_full():
    rng = np.random.default_rng(13)
    g = shapes.random_grid(rng, 17, 15, 4, fill=0.7, h=1 / 32)
    full = oracle.dilate(g, 2.5)
    cols = rng.choice(17 * 15, 40, replace=False)
    part = oracle.dilate(g, 2.5, cols=cols)
    for t, c in enumerate(cols):
        assert np.array_equal(part.column(t), full.z[full.col_off[c]:full.col_off[c + 1]])


def test_non_square_orientation():
    """Columns are row-major (c = j*nx + i): on a 4 x 9 grid a point segment at (1, 6)
    reaches (1, 2) (offset (0,-4), n = 16, w = 3h) and (1, 3) (n = 9, w = 4h) for k = 5,
    but not (1, 0) (n = 36)."""
    g = _grid_single(4, 9, 1 / 64, 1, 6, [(0.5, 0.5)])
    out = oracle.dilate(g, 5.0)
    assert tuple(out.column(1, 2)[0]) == (0.5 - 3 / 64, 0.5 + 3 / 64)
    assert tuple(out.column(1, 3)[0]) == (0.5 - 4 / 64, 0.5 + 4 / 64)
    assert tuple(out.column(1, 6)[0]) == (0.5 - 5 / 64, 0.5 + 5 / 64)
    assert len(out.column(1, 0)) == 0
    assert int(np.count_nonzero(np.diff(out.col_off))) == sum(
        1 for i in range(4) for j in range(9) if (i - 1) ** 2 + (j - 6) ** 2 <= 25)
