"""Shared test utilities: CSR comparison, inclusion and golden-file reading.

These helpers compare results; they hold none of the offset arithmetic.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p = line.split()
            i, j, cnt = int(p[0]), int(p[1]), int(p[2])
            segs = [(float(p[3 + 2 * t]), float(p[4 + 2 * t])) for t in range(cnt)]
            rows.append((i, j, segs))
    return rows


def columns_of(off, z):
    return [np.asarray(z[off[c]:off[c + 1]], np.float64) for c in range(len(off) - 1)]


def assert_same_csr(off_a, z_a, off_b, z_b, atol, gap_exempt=None, what=""):
    """Identical per-column counts and endpoints within atol.

    ``gap_exempt``: columns whose count may differ because the reference has a gap below the
    stated threshold there (checked by the caller).
    """
    off_a = np.asarray(off_a, np.int64)
    off_b = np.asarray(off_b, np.int64)
    assert off_a.shape == off_b.shape, what
    ca = np.diff(off_a)
    cb = np.diff(off_b)
    bad = np.flatnonzero(ca != cb)
    if gap_exempt is not None and bad.size:
        bad = np.array([c for c in bad if c not in gap_exempt], np.int64)
    assert bad.size == 0, f"{what}: count mismatch at columns {bad[:10]} ({ca[bad[:10]]} vs {cb[bad[:10]]})"
    same = ca == cb
    if z_a.shape[0] and same.all():
        d = np.abs(np.asarray(z_a, np.float64) - np.asarray(z_b, np.float64))
        d = np.where(np.isinf(z_a) & (np.asarray(z_a) == np.asarray(z_b)), 0.0, d)
        assert np.nanmax(d) <= atol, f"{what}: max endpoint error {np.nanmax(d)} > {atol}"


def included(cols_a, cols_b, tol=0.0):
    """Every segment of a lies within one segment of b (per column), up to tol."""
    for ca, cb in zip(cols_a, cols_b):
        for a, b in ca:
            ok = False
            for c, d in cb:
                if c <= a + tol and b <= d + tol:
                    ok = True
                    break
            if not ok:
                return False
    return True


def csr_union(grid_a, grid_b):
    """Closed union of two grids (CSG in dexel space)."""
    from synth.shapes import DexelGrid, union_merge
    n = grid_a.nx * grid_a.ny
    col = np.concatenate([np.repeat(np.arange(n), np.diff(grid_a.col_off)),
                          np.repeat(np.arange(n), np.diff(grid_b.col_off))]).astype(np.int64)
    z = np.concatenate([np.asarray(grid_a.z, np.float64).reshape(-1, 2),
                        np.asarray(grid_b.z, np.float64).reshape(-1, 2)])
    off, zz = union_merge(col, z[:, 0], z[:, 1], n)
    return DexelGrid(grid_a.nx, grid_a.ny, grid_a.h, off, zz)
