"""Seeded synthetic dexel shapes: analytic ray casting of primitives into CSR dexel grids.

A dexel grid (Sec. 3.1, "Dexel Representation") stores, for every cell (i, j) of a regular
N x N grid over [0,1]^2, the sorted list of disjoint segments [z_in, z_out] where the vertical
ray through the cell centre ((i+1/2)h, (j+1/2)h) is inside the solid.  Columns are numbered
row-major: col = j * nx + i.

This module only BUILDS inputs.  It holds none of the offset method's arithmetic (no dilation,
erosion, distance or power computation); both the oracle tests and the GPU tests draw their
inputs from it.  Everything is numpy float64; the float32 variant rounds the endpoints and
re-merges segments that the rounding made touch, so that the result is again a valid grid
(strictly positive gaps between consecutive segments of a column).

The paper's test models are not available; the shapes below (spheres, axis-aligned boxes,
hollow spherical shells, thin plates, nested concentric shells) stand in for its mechanical
and organic models (Sec. 4).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np


@dataclasses.dataclass
class DexelGrid:
    """CSR dexel grid. ``col_off`` has nx*ny+1 entries, ``z`` has shape (nseg, 2)."""

    nx: int
    ny: int
    h: float
    col_off: np.ndarray  # int64, nx*ny+1
    z: np.ndarray  # float64 or float32, (nseg, 2)

    @property
    def nseg(self) -> int:
        return int(self.col_off[-1])

    def column(self, i: int, j: int) -> np.ndarray:
        c = j * self.nx + i
        return self.z[self.col_off[c]:self.col_off[c + 1]]

    def segs_per_col(self) -> np.ndarray:
        return np.diff(self.col_off)

    def stats(self) -> dict:
        s = self.segs_per_col()
        return {"nx": self.nx, "ny": self.ny, "nseg": self.nseg,
                "mean_segs_per_col": float(s.mean()) if s.size else 0.0,
                "max_segs_per_col": int(s.max()) if s.size else 0}


# ----------------------------------------------------------------------------------------------
# primitives: tuples (kind, params...) in world units over [0,1]^3
#   ("sphere", cx, cy, cz, R)
#   ("box", x0, x1, y0, y1, z0, z1)
#   ("shell", cx, cy, cz, R, t)      hollow sphere: outer radius R, inner radius R - t
# ----------------------------------------------------------------------------------------------

def _footprint(prim):
    kind = prim[0]
    if kind in ("sphere", "shell"):
        _, cx, cy, _, R = prim[:5]
        return cx - R, cx + R, cy - R, cy + R
    if kind == "box":
        _, x0, x1, y0, y1 = prim[:5]
        return x0, x1, y0, y1
    raise ValueError(kind)


def _cast(prim, xs, ys):
    """Ray-cast one primitive at column centres (xs, ys) (same-shape arrays).

    Returns (mask_list) as a list of (sel, a, b) with sel a boolean mask over the inputs.
    Tangent rays (zero-length chords) are excluded by strict inequalities.
    """
    kind = prim[0]
    out = []
    if kind == "sphere":
        _, cx, cy, cz, R = prim
        d2 = (xs - cx) ** 2 + (ys - cy) ** 2
        sel = d2 < R * R
        s = np.sqrt(np.maximum(R * R - d2, 0.0))
        out.append((sel, cz - s, cz + s))
    elif kind == "shell":
        _, cx, cy, cz, R, t = prim
        Ri = R - t
        d2 = (xs - cx) ** 2 + (ys - cy) ** 2
        so = np.sqrt(np.maximum(R * R - d2, 0.0))
        si = np.sqrt(np.maximum(Ri * Ri - d2, 0.0))
        outer = d2 < R * R
        inner = d2 < Ri * Ri
        out.append((outer & ~inner, cz - so, cz + so))
        out.append((outer & inner, cz - so, cz - si))
        out.append((outer & inner, cz + si, cz + so))
    elif kind == "box":
        _, x0, x1, y0, y1, z0, z1 = prim
        sel = (xs > x0) & (xs < x1) & (ys > y0) & (ys < y1)
        out.append((sel, np.full(xs.shape, z0), np.full(xs.shape, z1)))
    else:
        raise ValueError(kind)
    return out


def union_merge(col: np.ndarray, a: np.ndarray, b: np.ndarray, ncols: int):
    """Per-column closed union of intervals (touching or overlapping intervals merge).

    Returns (col_off int64[ncols+1], z float64[(m,2)]).
    """
    if col.size == 0:
        return np.zeros(ncols + 1, np.int64), np.zeros((0, 2), np.float64)
    order = np.lexsort((b, a, col))
    col = col[order]
    a = a[order]
    b = b[order]
    # segmented (per column) running max of b by pointer doubling
    run = b.copy()
    shift = 1
    while shift < run.size:
        same = col[shift:] == col[:-shift]
        if not same.any():
            break
        cand = np.where(same, np.maximum(run[shift:], run[:-shift]), run[shift:])
        run[shift:] = cand
        shift *= 2
    new = np.ones(a.size, bool)
    same_col = col[1:] == col[:-1]
    new[1:] = ~same_col | (a[1:] > run[:-1])
    starts = np.flatnonzero(new)
    za = a[starts]
    zb = np.maximum.reduceat(b, starts)
    counts = np.bincount(col[starts], minlength=ncols)
    off = np.zeros(ncols + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    return off, np.stack([za, zb], axis=1)


_HERE = os.path.dirname(os.path.abspath(__file__))
_RC_SRC = os.path.join(_HERE, "raycast.c")
_RC_LIB = os.path.join(_HERE, "libraycast.so")
_rc = None
_KIND = {"sphere": 0, "box": 1, "shell": 2}


def build(force: bool = False) -> str:
    """Compile raycast.c (the compiled twin of ``raycast_numpy``) into libraycast.so."""
    if force or not os.path.exists(_RC_LIB) or os.path.getmtime(_RC_LIB) < os.path.getmtime(_RC_SRC):
        tmp = _RC_LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-pthread", _RC_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _RC_LIB)
    return _RC_LIB


def _rclib():
    global _rc
    if _rc is None:
        build()
        L = ctypes.CDLL(_RC_LIB)
        P = ctypes.c_void_p
        L.rc_count.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, ctypes.c_int]
        L.rc_fill.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, ctypes.c_int]
        _rc = L
    return _rc


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def raycast(prims, n: int) -> DexelGrid:
    """Ray-cast a union of primitives on an n x n grid over [0,1]^2 (h = 1/n), in C over
    the host's threads; bit-identical to ``raycast_numpy``."""
    L = _rclib()
    kind = np.array([_KIND[p[0]] for p in prims], np.int32)
    prm = np.zeros((max(len(prims), 1), 8), np.float64)
    for q, p in enumerate(prims):
        prm[q, : len(p) - 1] = p[1:]
    counts = np.zeros(n * n, np.int64)
    th = _threads()
    if L.rc_count(n, prm.ctypes.data, kind.ctypes.data, len(prims), counts.ctypes.data, th) != 0:
        raise MemoryError("ray cast (count)")
    off = np.zeros(n * n + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    z = np.zeros((int(off[-1]), 2), np.float64)
    if z.size and L.rc_fill(n, prm.ctypes.data, kind.ctypes.data, len(prims), off.ctypes.data,
                            z.ctypes.data, th) != 0:
        raise MemoryError("ray cast (fill)")
    return DexelGrid(n, n, 1.0 / n, off, z)


def raycast_numpy(prims, n: int, row_block: int = 256) -> DexelGrid:
    """Ray-cast a union of primitives on an n x n grid over [0,1]^2 (h = 1/n)."""
    h = 1.0 / n
    fps = np.array([_footprint(p) for p in prims], dtype=np.float64).reshape(-1, 4)
    offs = [np.zeros(1, np.int64)]
    zs = []
    base = 0
    for j0 in range(0, n, row_block):
        j1 = min(n, j0 + row_block)
        cols, za, zb = [], [], []
        ylo = (j0 + 0.5) * h
        yhi = (j1 - 0.5) * h
        for p, (x0, x1, y0, y1) in zip(prims, fps):
            if y1 < ylo or y0 > yhi:
                continue
            i_lo = max(0, int(math.floor(x0 / h - 0.5)))
            i_hi = min(n - 1, int(math.ceil(x1 / h - 0.5)))
            jj_lo = max(j0, int(math.floor(y0 / h - 0.5)))
            jj_hi = min(j1 - 1, int(math.ceil(y1 / h - 0.5)))
            if i_lo > i_hi or jj_lo > jj_hi:
                continue
            ii = np.arange(i_lo, i_hi + 1)
            jj = np.arange(jj_lo, jj_hi + 1)
            I, J = np.meshgrid(ii, jj)
            xs = (I + 0.5) * h
            ys = (J + 0.5) * h
            for sel, a, b in _cast(p, xs, ys):
                if not sel.any():
                    continue
                cols.append(((J[sel] - j0) * n + I[sel]).astype(np.int64))
                za.append(a[sel])
                zb.append(b[sel])
        ncols = (j1 - j0) * n
        if cols:
            off, z = union_merge(np.concatenate(cols), np.concatenate(za), np.concatenate(zb), ncols)
        else:
            off, z = np.zeros(ncols + 1, np.int64), np.zeros((0, 2))
        offs.append(off[1:] + base)
        zs.append(z)
        base += int(off[-1])
    col_off = np.concatenate(offs)
    z = np.concatenate(zs) if zs else np.zeros((0, 2))
    return DexelGrid(n, n, h, col_off, z)


def from_columns(nx: int, ny: int, h: float, columns: dict, dtype=np.float64) -> DexelGrid:
    """Build a grid from {(i, j): [(a, b), ...]} (segments given sorted and disjoint)."""
    counts = np.zeros(nx * ny, np.int64)
    for (i, j), segs in columns.items():
        counts[j * nx + i] = len(segs)
    off = np.zeros(nx * ny + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    z = np.zeros((int(off[-1]), 2), dtype)
    for (i, j), segs in columns.items():
        c = j * nx + i
        if segs:
            z[off[c]:off[c + 1]] = np.asarray(segs, dtype)
    return DexelGrid(nx, ny, h, off, z)


def to_float32(g: DexelGrid) -> DexelGrid:
    """Round endpoints to float32 and re-merge segments that now touch or overlap.

    Rounding to nearest is monotone, so every column stays sorted; a segment joins the one
    before it (same column) exactly when its rounded start is at or below that one's rounded
    end, and the joined run ends at the rounded end of its last segment (ends stay ordered).
    """
    z32 = np.asarray(g.z, np.float64).reshape(-1, 2).astype(np.float32)
    n = g.nx * g.ny
    cnt = np.diff(g.col_off)
    if z32.shape[0] == 0:
        return DexelGrid(g.nx, g.ny, g.h, np.zeros(n + 1, np.int64), np.zeros((0, 2), np.float32))
    col = np.repeat(np.arange(n, dtype=np.int64), cnt)
    new = np.ones(z32.shape[0], bool)
    new[1:] = (col[1:] != col[:-1]) | (z32[1:, 0] > z32[:-1, 1])
    starts = np.flatnonzero(new)
    ends = np.append(starts[1:], z32.shape[0]) - 1
    za = z32[starts, 0]
    zb = z32[ends, 1]
    counts = np.bincount(col[starts], minlength=n)
    off = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    return DexelGrid(g.nx, g.ny, g.h, off, np.stack([za, zb], axis=1).astype(np.float32))


def to_float32_sorting(g: DexelGrid) -> DexelGrid:
    """The same rounding and re-merge through a full per-column sort and closed union."""
    z32 = g.z.astype(np.float32)
    col = np.repeat(np.arange(g.nx * g.ny, dtype=np.int64), np.diff(g.col_off))
    off, z = union_merge(col, z32[:, 0].astype(np.float64), z32[:, 1].astype(np.float64), g.nx * g.ny)
    return DexelGrid(g.nx, g.ny, g.h, off, z.astype(np.float32))


def random_grid(rng: np.random.Generator, nx: int, ny: int, max_segs: int, fill: float = 0.7,
                zlo: float = 0.0, zhi: float = 1.0, point_frac: float = 0.0,
                dtype=np.float64, h: float | None = None) -> DexelGrid:
    """Random valid CSR: each column gets U{0..max_segs} sorted disjoint segments with gaps > 0.

    A column is empty with probability 1 - fill.  ``point_frac`` of the segments are made
    zero-length (a == b), which the dexel representation allows (a tangent sample).
    """
    counts = np.where(rng.random(nx * ny) < fill, rng.integers(1, max_segs + 1, nx * ny), 0)
    off = np.zeros(nx * ny + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    zs = np.zeros((int(off[-1]), 2), np.float64)
    for c in np.flatnonzero(counts):
        m = int(counts[c])
        while True:
            pts = np.sort(rng.uniform(zlo, zhi, 2 * m))
            if np.all(np.diff(pts)[1::2] > 0) if m > 1 else True:
                break
        seg = pts.reshape(m, 2)
        if point_frac > 0:
            pm = rng.random(m) < point_frac
            seg[pm, 1] = seg[pm, 0]
        zs[off[c]:off[c + 1]] = seg
    g = DexelGrid(nx, ny, 1.0 / max(nx, ny) if h is None else h, off, zs)
    return to_float32(g) if dtype == np.float32 else g


# ----------------------------------------------------------------------------------------------
# the five workloads (seeded)
# ----------------------------------------------------------------------------------------------

def _u(rng, lo, hi, size=None):
    return rng.uniform(lo, hi, size)


def _sphere(rng, rlo, rhi, clo=0.2, chi=0.8):
    R = _u(rng, rlo, rhi)
    c = _u(rng, clo, chi, 3)
    c[2] = min(max(c[2], R), 1 - R)
    return ("sphere", c[0], c[1], c[2], R)


def _box(rng, slo, shi, lo=0.05, hi=0.95):
    s = _u(rng, slo, shi, 3)
    p = _u(rng, lo, hi - s)
    return ("box", p[0], p[0] + s[0], p[1], p[1] + s[1], p[2], p[2] + s[2])


def _shell(rng, rlo, rhi, tlo, thi, clo=0.15, chi=0.85):
    R = _u(rng, rlo, rhi)
    t = min(_u(rng, tlo, thi), 0.9 * R)
    c = _u(rng, clo, chi, 3)
    c[2] = min(max(c[2], R), 1 - R)
    return ("shell", c[0], c[1], c[2], R, t)


def grid64_prims():
    """64 x 64, union of 8 spheres, centres U[0.2,0.8]^3, radii U[0.05,0.2], seed 0."""
    rng = np.random.default_rng(0)
    prims = []
    for _ in range(8):
        c = rng.uniform(0.2, 0.8, 3)
        R = rng.uniform(0.05, 0.2)
        prims.append(("sphere", c[0], c[1], c[2], R))
    return prims


def grid64() -> DexelGrid:
    return raycast(grid64_prims(), 64)


def grid512_prims(nprim: int = 200, seed: int = 1):
    """512 x 512: 1/3 spheres, 1/3 boxes (sides U[0.02,0.3]), 1/3 hollow shells (t U[0.005,0.03])."""
    rng = np.random.default_rng(seed)
    prims = []
    for q in range(nprim):
        kind = q % 3
        if kind == 0:
            prims.append(_sphere(rng, 0.02, 0.12, 0.1, 0.9))
        elif kind == 1:
            prims.append(_box(rng, 0.02, 0.3))
        else:
            prims.append(_shell(rng, 0.04, 0.15, 0.005, 0.03, 0.1, 0.9))
    return prims


def capped(prims, n, max_segs):
    """Drop primitives (last first) until no column holds more than max_segs segments."""
    prims = list(prims)
    while True:
        g = raycast(prims, n)
        if g.stats()["max_segs_per_col"] <= max_segs:
            return g, prims
        prims.pop()


def grid512() -> DexelGrid:
    g, _ = capped(grid512_prims(), 512, 16)
    return g


def grid2048_prims(r_world: float = 64.0 / 2048.0, seed: int = 2):
    """2048 x 2048, 1000 primitives: spheres, boxes, thin plates (one side U[0.2,0.9] r) and
    groups of nested concentric hollow spheres (up to 32 shells -> up to 64 segments/column)."""
    rng = np.random.default_rng(seed)
    prims = []
    # 4 nested groups of concentric shells (shell + gap ~ 0.009, thickness 0.004)
    for g in range(4):
        nsh = int(rng.integers(16, 33))
        c = rng.uniform(0.35, 0.65, 3)
        Rout = 0.009 * nsh + 0.01
        c[2] = min(max(c[2], Rout), 1 - Rout)
        c[0] = 0.25 + 0.5 * (g % 2) + rng.uniform(-0.05, 0.05)
        c[1] = 0.25 + 0.5 * (g // 2) + rng.uniform(-0.05, 0.05)
        for s in range(nsh):
            R = Rout - 0.009 * s
            prims.append(("shell", c[0], c[1], c[2], R, 0.004))
    while len(prims) < 1000:
        kind = len(prims) % 4
        if kind == 0:
            prims.append(_sphere(rng, 0.01, 0.06, 0.05, 0.95))
        elif kind == 1:
            prims.append(_box(rng, 0.01, 0.12))
        elif kind == 2:
            # thin plate: one side thinner than the radius
            s = rng.uniform(0.05, 0.25, 3)
            ax = int(rng.integers(0, 3))
            s[ax] = rng.uniform(0.2, 0.9) * r_world
            p = rng.uniform(0.03, 0.97 - s)
            prims.append(("box", p[0], p[0] + s[0], p[1], p[1] + s[1], p[2], p[2] + s[2]))
        else:
            prims.append(_shell(rng, 0.02, 0.07, 0.004, 0.02, 0.05, 0.95))
    return prims


def grid2048() -> DexelGrid:
    return raycast(grid2048_prims(), 2048)


def batch256_shapes(nshapes: int = 256, seed: int = 3):
    """256 shapes, N log-uniform in [32, 1024], U{4..400} spheres/boxes each, k ~ U[1,48]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nshapes):
        n = int(round(math.exp(rng.uniform(math.log(32), math.log(1024)))))
        m = int(rng.integers(4, 401))
        k = float(rng.uniform(1.0, 48.0))
        prims = []
        for q in range(m):
            if q % 2 == 0:
                prims.append(_sphere(rng, 0.02, 0.15, 0.1, 0.9))
            else:
                prims.append(_box(rng, 0.02, 0.2))
        out.append((n, k, prims))
    return out


def grid4096_prims(seed: int = 4, nprim: int = 550):
    """4096 x 4096, mixed spheres/boxes/shells: 61.6 M segments, at most 15 per column."""
    rng = np.random.default_rng(seed)
    prims = []
    for q in range(nprim):
        kind = q % 3
        if kind == 0:
            prims.append(_sphere(rng, 0.01, 0.08, 0.05, 0.95))
        elif kind == 1:
            prims.append(_box(rng, 0.01, 0.15))
        else:
            prims.append(_shell(rng, 0.02, 0.08, 0.004, 0.02, 0.05, 0.95))
    return prims


def grid4096() -> DexelGrid:
    return raycast(grid4096_prims(), 4096)
